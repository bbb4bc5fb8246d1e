"""Python surface of the reduced-order step (Algorithms 2, 3, 5, 6, 7): argument marshalling only.

All computation runs in libmpmrom.so (csrc/rom.cu, csrc/decoder.cu).
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _abi
from .mpm import _ptr, _stream


def _p64(a):
    if a is None:
        return None
    if isinstance(a, torch.Tensor):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


class ROM:
    """One reduced-order instance bound to a decoder and the reference positions X."""

    def __init__(self, decoder, X, *, dim, n_grid, dx, dt, gravity, bc, bc_width, material, transfer, rho,
                 p_vol, E, nu, n_samples, seed, instance=0, gn_iters=3, projection=0, ridge=0.0, affine=0,
                 f_reference=0, quadrature=0, ell=0, newton_iters=0, newton_tol=0.0):
        L = _abi.lib()
        g = (C.c_float * 3)(*[float(v) for v in gravity])
        self.cfg = _abi.RomConfig(dim, n_grid, dx, dt, g, bc, bc_width, material, transfer, rho, p_vol, E, nu,
                                  decoder.r, n_samples, seed, instance, gn_iters, projection, ridge, affine,
                                  f_reference, quadrature, ell, newton_iters, newton_tol)
        self.eulerian = bool(quadrature)
        self.ell = int(ell or 2)
        self._X = np.ascontiguousarray(X, np.float32) if isinstance(X, np.ndarray) else X
        self.P = int(self._X.shape[0])
        self.d, self.r = dim, decoder.r
        self.n_samples = min(int(n_samples), self.P)
        self.decoder = decoder  # keeps the decoder alive
        h = C.c_void_p()
        _abi.check(L.rom_create(C.byref(self.cfg), decoder._h, _ptr(self._X), self.P, C.byref(h)))
        self._h = h

    @classmethod
    def from_scene(cls, decoder, sc, n_samples, seed, instance=0, gn_iters=3, projection=0, X=None, ridge=0.0,
                   affine=0, f_reference=0, quadrature=0, ell=0, newton_iters=0, newton_tol=0.0):
        k = 0
        return cls(decoder, sc.x if X is None else X, dim=sc.dim, n_grid=sc.n_grid, dx=sc.dx, dt=sc.dt,
                   gravity=sc.gravity, bc=sc.bc, bc_width=sc.bc_width, material=sc.material,
                   transfer=sc.transfer, rho=sc.rho, p_vol=sc.p_vol, E=float(sc.E[k]), nu=float(sc.nu[k]),
                   n_samples=n_samples, seed=seed, instance=instance, gn_iters=gn_iters, projection=projection,
                   ridge=ridge, affine=affine, f_reference=f_reference, quadrature=quadrature, ell=ell,
                   newton_iters=newton_iters, newton_tol=newton_tol)

    def close(self):
        if getattr(self, "_h", None):
            _abi.lib().rom_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, xhat, vhat, xhat_prev, step=0, stream=None):
        f = lambda a: np.ascontiguousarray(a, np.float64)
        a, b, c = f(xhat), f(vhat), f(xhat_prev)
        _abi.check(_abi.lib().rom_set_state(self._h, _p64(a), _p64(b), _p64(c), int(step), _stream(stream)))

    def get_state(self, stream=None):
        xh = np.empty(self.r)
        vh = np.empty(self.r)
        xp = np.empty(self.r)
        st = C.c_int64()
        _abi.check(_abi.lib().rom_get_state(self._h, _p64(xh), _p64(vh), _p64(xp), C.c_void_p(C.addressof(st)),
                                            _stream(stream)))
        return xh, vh, xp, st.value

    def fit_initial(self, target, V0, iters=20, stream=None):
        t = np.ascontiguousarray(target, np.float32)
        v = np.ascontiguousarray(np.broadcast_to(V0, (self.P, self.d)), np.float32)
        _abi.check(_abi.lib().rom_fit_initial(self._h, _ptr(t), _ptr(v), int(iters), _stream(stream)))

    def set_reference(self, xhat_ref, stream=None):
        a = np.ascontiguousarray(xhat_ref, np.float64)
        _abi.check(_abi.lib().rom_set_reference(self._h, _p64(a), _stream(stream)))

    def step(self, n_steps=1, stream=None):
        _abi.check(_abi.lib().rom_step(self._h, int(n_steps), _stream(stream)))

    def status(self, clear=True, stream=None):
        w = C.c_uint32()
        _abi.check(_abi.lib().rom_status_word(self._h, C.byref(w), int(clear), _stream(stream)))
        return w.value

    def set_kinematic(self, group, velocities, min_samples=5, stream=None):
        """Kinematic (Dirichlet) boundaries: group id per particle (-1 free), prescribed velocity per
        group; at least min_samples samples per group each step.  group=None removes them."""
        if group is None:
            _abi.check(_abi.lib().rom_set_kinematic(self._h, None, 0, None, 1, _stream(stream)))
            return
        g = np.ascontiguousarray(group, np.int32)
        v = np.ascontiguousarray(velocities, np.float32).reshape(-1, self.d)
        _abi.check(_abi.lib().rom_set_kinematic(self._h, _ptr(g), int(len(v)), _ptr(v), int(min_samples),
                                                _stream(stream)))

    def debug(self, stream=None):
        q = np.empty(self.P, np.int32)
        cnt = np.empty(3, np.int32)
        xa = np.empty((self.P, self.d), np.float32)
        vt = np.empty((self.P, self.d), np.float32)    # at least the sample capacity
        xt = np.empty((self.P, self.d), np.float32)
        _abi.check(_abi.lib().rom_debug(self._h, _ptr(q), _ptr(cnt), _ptr(xa), _ptr(vt), _ptr(xt), _stream(stream)))
        nP, nQ = int(cnt[0]), int(cnt[1])
        vt, xt = vt[:nP].copy(), xt[:nP].copy()
        if self.eulerian:
            return dict(samples=q[:nP].copy(), neigh=q[:0].copy(), n_points=nQ, v_trial=vt, x_trial=xt)
        return dict(samples=q[:nP].copy(), neigh=q[nP:nQ].copy(), x_all=xa, v_trial=vt, x_trial=xt)

    def line_search_picks(self, stream=None):
        """Per Gauss-Newton iteration of the last step, the m of the accepted step 2^-m (-1: none)."""
        picks = np.empty(16, np.int32)
        n = C.c_int32()
        _abi.check(_abi.lib().rom_debug_line_search(self._h, _ptr(picks), C.byref(n), _stream(stream)))
        return picks[:n.value].copy()

    def quadrature_points(self, stream=None):
        """Eulerian quadrature of the last step: dict of x (points), X (reference positions), mass, V0."""
        d, n = self.d, self.cfg.n_grid
        cap = min((n - 3) ** d, 6 ** d * self.n_samples) * self.ell ** d
        x = np.empty((cap, d), np.float32)
        X = np.empty((cap, d), np.float32)
        m = np.empty(cap, np.float32)
        v0 = np.empty(cap, np.float32)
        nq = C.c_int32()
        _abi.check(_abi.lib().rom_debug_quadrature(self._h, C.byref(nq), _ptr(x), _ptr(X), _ptr(m), _ptr(v0),
                                                   _stream(stream)))
        k = nq.value
        return dict(x=x[:k].copy(), X=X[:k].copy(), mass=m[:k].copy(), V0=v0[:k].copy())

    def decode_all(self, out=None, stream=None):
        if out is None:
            out = torch.empty((self.P, self.d), dtype=torch.float32, device="cuda")
        _abi.check(_abi.lib().rom_decode_all(self._h, _ptr(out), _stream(stream)))
        return out


    def decode_points(self, X, out=None, stream=None):
        """g(X; xhat_n) at arbitrary reference positions X (n, d) CUDA tensor (super-resolution)."""
        X = X.contiguous()
        if out is None:
            out = torch.empty((X.shape[0], self.d), dtype=torch.float32, device=X.device)
        _abi.check(_abi.lib().rom_decode_points(self._h, _ptr(X), int(X.shape[0]), _ptr(out), _stream(stream)))
        return out


def metric_accumulate(a, b, acc, stream=None):
    """acc (2,) float64 CUDA tensor += [sum (a - b)^2, sum b^2] (Section 5 error metric)."""
    _abi.check(_abi.lib().metric_accumulate(_ptr(a), _ptr(b), a.numel(), _p64(acc), _stream(stream)))


class RomBatch:
    """Many reduced-order contexts stepped by one CUDA graph launch (rom_batch_create / step).
    The ROM objects must stay alive while the batch exists."""

    def __init__(self, roms):
        self.roms = list(roms)
        arr = (C.c_void_p * len(self.roms))(*[r._h.value for r in self.roms])
        h = C.c_void_p()
        _abi.check(_abi.lib().rom_batch_create(arr, len(self.roms), C.byref(h)))
        self._h = h

    def step(self, n_steps=1, stream=None):
        _abi.check(_abi.lib().rom_batch_step(self._h, int(n_steps), _stream(stream)))

    def close(self):
        if getattr(self, "_h", None):
            _abi.lib().rom_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
