"""Python surface of the full-order MPM step (Algorithm 1): argument marshalling only.

All computation runs in libmpmrom.so (csrc/mpm.cu).  Tensors are torch
tensors (device memory or pinned host memory) or numpy arrays (host memory);
only their data pointers cross the C ABI.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _abi


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, torch.Tensor):
        assert a.is_contiguous() and a.dtype in (torch.float32, torch.int32), "contiguous float32/int32 expected"
        return C.c_void_p(a.data_ptr())
    assert isinstance(a, np.ndarray) and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.c_void_p)


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class MPM:
    """One context of the C ABI: a batch of MPM instances sharing grid and material law."""

    def __init__(self, *, dim, n_grid, dx, dt, gravity, bc, bc_width, material, transfer, rho, p_vol,
                 E, nu, inst_offsets, polar_eft=0, plastic_compression=2.5e-2, plastic_stretch=7.5e-3):
        L = _abi.lib()
        self._E = np.ascontiguousarray(np.atleast_1d(E), np.float32)
        self._nu = np.ascontiguousarray(np.atleast_1d(nu), np.float32)
        self._offs = np.ascontiguousarray(inst_offsets, np.int64)
        g = (C.c_float * 3)(*[float(v) for v in gravity])
        self.cfg = _abi.MpmConfig(dim, n_grid, dx, dt, g, bc, bc_width, material, transfer, rho, p_vol,
                                  len(self._E), self._E.ctypes.data_as(C.POINTER(C.c_float)),
                                  self._nu.ctypes.data_as(C.POINTER(C.c_float)),
                                  self._offs.ctypes.data_as(C.POINTER(C.c_int64)), int(polar_eft),
                                  float(plastic_compression), float(plastic_stretch))
        h = C.c_void_p()
        _abi.check(L.mpm_init(C.byref(self.cfg), C.byref(h)))
        self._h = h
        self.dim = dim
        self.n_grid = n_grid
        self.P = int(self._offs[-1])
        self.n_inst = len(self._E)

    @classmethod
    def from_scene(cls, sc, polar_eft=0):
        """Context for a synth.scenes.Scene (configuration and kinematic groups; no state)."""
        ctx = cls(dim=sc.dim, n_grid=sc.n_grid, dx=sc.dx, dt=sc.dt, gravity=sc.gravity, bc=sc.bc,
                  bc_width=sc.bc_width, material=sc.material, transfer=sc.transfer, rho=sc.rho,
                  p_vol=sc.p_vol, E=sc.E, nu=sc.nu, inst_offsets=sc.inst_offsets, polar_eft=polar_eft,
                  plastic_compression=sc.theta_c, plastic_stretch=sc.theta_s)
        if getattr(sc, "kin_group", None) is not None:
            ctx.set_kinematic(sc.kin_group, sc.kin_vel)
        return ctx

    def set_kinematic(self, group, velocities, stream=None):
        """Kinematic (Dirichlet) groups: group id per particle (-1 free), prescribed velocity per
        group (n_groups, dim).  group=None removes them."""
        if group is None:
            _abi.check(_abi.lib().mpm_set_kinematic(self._h, None, 0, None, _stream(stream)))
            return
        g = np.ascontiguousarray(group, np.int32)
        v = np.ascontiguousarray(velocities, np.float32).reshape(-1, self.dim)
        _abi.check(_abi.lib().mpm_set_kinematic(self._h, g.ctypes.data_as(C.c_void_p), int(len(v)),
                                                v.ctypes.data_as(C.c_void_p), _stream(stream)))

    def close(self):
        if getattr(self, "_h", None):
            _abi.lib().mpm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, x, v, F, C_=None, stream=None):
        _abi.check(_abi.lib().mpm_set_state(self._h, _ptr(x), _ptr(v), _ptr(F), _ptr(C_), _stream(stream)))

    def get_state(self, x=None, v=None, F=None, C_=None, stream=None):
        _abi.check(_abi.lib().mpm_get_state(self._h, _ptr(x), _ptr(v), _ptr(F), _ptr(C_), _stream(stream)))

    def step(self, n_steps=1, stream=None):
        _abi.check(_abi.lib().mpm_step(self._h, int(n_steps), _stream(stream)))

    def step_profiled(self, n_steps=1, flush=None, stream=None):
        """Steps with CUDA events around every kernel, all steps enqueued before one final
        synchronisation; `flush` (a CUDA tensor) is overwritten between steps, outside the timed
        intervals.  Returns (n_steps, 4) ms [fused, scan, permute, whole step]."""
        out = (C.c_float * (4 * n_steps))()
        fb = None if flush is None else C.c_void_p(flush.data_ptr())
        nb = 0 if flush is None else flush.numel() * flush.element_size()
        _abi.check(_abi.lib().mpm_step_profiled(self._h, int(n_steps), fb, nb, out, _stream(stream)))
        return np.frombuffer(out, np.float32).reshape(n_steps, 4).copy()

    def step_timed(self, n_steps, flush=None, stream=None):
        """mpm_step_timed: n_steps steps with events at step boundaries only; returns (n_steps,) ms."""
        out = (C.c_float * max(1, n_steps))()
        fb = None if flush is None else C.c_void_p(flush.data_ptr())
        nb = 0 if flush is None else flush.numel() * flush.element_size()
        _abi.check(_abi.lib().mpm_step_timed(self._h, int(n_steps), fb, nb, out, _stream(stream)))
        return np.frombuffer(out, np.float32)[:n_steps].copy()

    def status(self, clear=True, stream=None):
        w = C.c_uint32()
        _abi.check(_abi.lib().mpm_status_word(self._h, C.byref(w), int(clear), _stream(stream)))
        return w.value

    def num_block_keys(self):
        return int(_abi.lib().mpm_num_block_keys(self._h))

    def debug_bins(self, stream=None):
        ck = np.empty(self.P, np.int32)
        bk = np.empty(self.P, np.int32)
        off = np.empty(self.num_block_keys() + 1, np.int32)
        _abi.check(_abi.lib().mpm_debug_bins(self._h, _ptr(ck), _ptr(bk), _ptr(off), _stream(stream)))
        return ck, bk, off

    def debug_grid(self, stream=None):
        N = self.n_inst * self.n_grid ** self.dim
        m = np.empty(N, np.float32)
        p = np.empty((N, self.dim), np.float32)
        v = np.empty((N, self.dim), np.float32)
        _abi.check(_abi.lib().mpm_debug_grid(self._h, _ptr(m), _ptr(p), _ptr(v), _stream(stream)))
        shp = (self.n_inst,) + (self.n_grid,) * self.dim
        return m.reshape(shp), p.reshape(shp + (self.dim,)), v.reshape(shp + (self.dim,))

    # convenience for tests and benchmarks -------------------------------------------------
    def load_numpy(self, x, v, F, C_=None):
        """Loads float64/float32 numpy state (copied to float32 host arrays)."""
        f = lambda a: None if a is None else np.ascontiguousarray(a, np.float32)
        self._host = [f(x), f(v), f(F), f(C_)]
        self.set_state(*self._host)
        torch.cuda.synchronize()

    def read_numpy(self):
        d = self.dim
        x = np.empty((self.P, d), np.float32)
        v = np.empty((self.P, d), np.float32)
        F = np.empty((self.P, d, d), np.float32)
        Cm = np.empty((self.P, d, d), np.float32)
        self.get_state(x, v, F, Cm)
        torch.cuda.synchronize()
        return x, v, F, Cm


def step_noalloc(scene_cfg, x, v, F, C_=None, n_steps=1, stream=None):
    """mpm_step_noalloc through the C ABI: steps the state held in the caller's CUDA tensors
    x (P, d), v (P, d), F (P, d, d), C (P, d, d) in place, using only the library's fixed
    device scratch (no allocation).  `scene_cfg` is an MPM context's configuration source:
    a synth.scenes.Scene.  Returns the status bits raised during the call.

    The kernels write these tensors in place and the C entry point cannot see their lengths, so
    every one must be a contiguous float32 CUDA tensor on the current device holding exactly
    P*d (x, v) or P*d*d (F, C) elements, P = inst_offsets[-1]; anything else raises ValueError
    before the call."""
    sc = scene_cfg
    P, d = int(np.asarray(sc.inst_offsets)[-1]), int(sc.dim)
    dev = torch.cuda.current_device()
    for name, t, n in (("x", x, P * d), ("v", v, P * d), ("F", F, P * d * d), ("C", C_, P * d * d)):
        if t is None and name == "C":
            continue
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.device.index != dev:
            raise ValueError(f"step_noalloc: {name} must be a CUDA tensor on the current device")
        if t.dtype != torch.float32 or not t.is_contiguous() or t.numel() != n:
            raise ValueError(f"step_noalloc: {name} must be contiguous float32 with {n} elements")
    E = np.ascontiguousarray(np.atleast_1d(sc.E), np.float32)
    nu = np.ascontiguousarray(np.atleast_1d(sc.nu), np.float32)
    offs = np.ascontiguousarray(sc.inst_offsets, np.int64)
    g = (C.c_float * 3)(*[float(a) for a in sc.gravity])
    cfg = _abi.MpmConfig(sc.dim, sc.n_grid, sc.dx, sc.dt, g, sc.bc, sc.bc_width, sc.material, sc.transfer, sc.rho,
                         sc.p_vol, len(E), E.ctypes.data_as(C.POINTER(C.c_float)),
                         nu.ctypes.data_as(C.POINTER(C.c_float)), offs.ctypes.data_as(C.POINTER(C.c_int64)), 0,
                         float(sc.theta_c), float(sc.theta_s))
    w = C.c_uint32()
    _abi.check(_abi.lib().mpm_step_noalloc(C.byref(cfg), _ptr(x), _ptr(v), _ptr(F), _ptr(C_), int(n_steps),
                                           C.byref(w), _stream(stream)))
    return w.value
