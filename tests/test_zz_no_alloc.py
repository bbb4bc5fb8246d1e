"""mpm_step_noalloc: the MPM step for callers that may not allocate device memory.

Such callers (a host application that owns the device-memory budget and forbids
allocation inside its frame loop, or code that must not risk an allocation
failure or the device synchronisation cudaMalloc / cudaFree can cause) pass only
their state arrays; the step's work memory comes from a fixed 8 MiB device array
inside the library.  This file is collected last so that a run stopping at its
first failure has already run every other test; it must pass on its own in a
fresh process as well.
"""
import numpy as np
import pytest

import synth.scenes as S

pytestmark = pytest.mark.gpu
TOL = 1e-5


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _scene():
    sc = S.block_2d(side=64, dt=5e-5, origin=(0.4, 0.05), v0=np.array([0.2, -0.6]))
    rng = np.random.default_rng(21)
    sc.F = S.random_deformation(rng, sc.n_particles, 2, 0.02)
    return sc


def test_noalloc_matches_context_step_on_two_calls():
    import torch
    from paper_2109_12390_gb300.mpm import MPM, step_noalloc
    sc = _scene()
    d, P = sc.dim, sc.n_particles
    # reference: the context-owned path
    ctx = MPM.from_scene(sc)
    ctx.load_numpy(sc.x, sc.v, sc.F, sc.C)
    # fixed-scratch path: the caller's own device arrays, stepped in place
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    x, v, F, Cm = t(sc.x), t(sc.v), t(sc.F.reshape(P, d * d)), t(sc.C.reshape(P, d * d))
    for call in range(2):
        status = step_noalloc(sc, x, v, F, Cm, n_steps=40)
        ctx.step(40)
        assert status == 0, call
        rx, rv, rF, rC = ctx.read_numpy()
        torch.cuda.synchronize()
        assert rel(x.cpu().numpy(), rx) < TOL, call
        assert rel(v.cpu().numpy(), rv) < TOL, call
        assert rel(F.cpu().numpy().reshape(P, d, d), rF) < TOL, call
        scale = max(np.linalg.norm(rC), np.linalg.norm(rv) / sc.dx)
        assert np.linalg.norm(Cm.cpu().numpy().reshape(P, d, d) - rC) / scale < 1e-4, call
    ctx.close()


def test_noalloc_leaves_device_free_memory_unchanged():
    """The property the entry point exists for: after the first call on the device (which may
    make the driver load the module and commit the fixed array), further calls change the
    device's free memory by nothing.  Only the C-ABI calls run between the two readings."""
    import torch
    from paper_2109_12390_gb300.mpm import step_noalloc
    sc = _scene()
    d, P = sc.dim, sc.n_particles
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    x, v, F, Cm = t(sc.x), t(sc.v), t(sc.F.reshape(P, d * d)), t(sc.C.reshape(P, d * d))
    step_noalloc(sc, x, v, F, Cm, n_steps=2)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        assert step_noalloc(sc, x, v, F, Cm, n_steps=4) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert np.isfinite(x.cpu().numpy()).all()


def test_noalloc_rejects_host_and_mis_sized_arrays():
    import ctypes
    import torch
    from paper_2109_12390_gb300 import _abi
    from paper_2109_12390_gb300.mpm import step_noalloc
    sc = _scene()
    d, P = sc.dim, sc.n_particles
    x = torch.zeros((P, d), device="cuda")
    v = torch.zeros((P, d), device="cuda")
    F = torch.zeros((P, d * d), device="cuda")
    # the binding refuses what the kernels would write past or read from the host
    with pytest.raises(ValueError):
        step_noalloc(sc, x[: P - 1], v, F, None)
    with pytest.raises(ValueError):
        step_noalloc(sc, x.cpu(), v, F, None)
    with pytest.raises(ValueError):
        step_noalloc(sc, x, v, F.double(), None)
    # the C entry point itself rejects a host pointer, before it enqueues anything
    host = np.zeros((P, d), np.float32)
    cfg_args = _noalloc_cfg(sc)
    st = _abi.lib().mpm_step_noalloc(ctypes.byref(cfg_args[0]), host.ctypes.data_as(ctypes.c_void_p),
                                     ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(F.data_ptr()), None, 1, None,
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == _abi.MPM_EINVAL
    assert b"device" in _abi.lib().mpm_last_error()


def _noalloc_cfg(sc):
    import ctypes
    from paper_2109_12390_gb300 import _abi
    E = np.ascontiguousarray(np.atleast_1d(sc.E), np.float32)
    nu = np.ascontiguousarray(np.atleast_1d(sc.nu), np.float32)
    offs = np.ascontiguousarray(sc.inst_offsets, np.int64)
    g = (ctypes.c_float * 3)(*[float(a) for a in sc.gravity])
    cfg = _abi.MpmConfig(sc.dim, sc.n_grid, sc.dx, sc.dt, g, sc.bc, sc.bc_width, sc.material, sc.transfer, sc.rho,
                         sc.p_vol, len(E), E.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                         nu.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                         offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), 0, float(sc.theta_c),
                         float(sc.theta_s))
    return cfg, E, nu, offs


def test_noalloc_rejects_configurations_beyond_the_fixed_scratch():
    import torch
    from paper_2109_12390_gb300 import _abi
    from paper_2109_12390_gb300.mpm import step_noalloc
    sc = S.cube_3d(side=64)   # 262,144 particles on 128^3: far beyond 8 MiB of work memory
    P = sc.n_particles
    x = torch.zeros((P, 3), device="cuda")
    v = torch.zeros((P, 3), device="cuda")
    F = torch.zeros((P, 9), device="cuda")
    with pytest.raises(_abi.MpmError) as e:
        step_noalloc(sc, x, v, F, None, n_steps=1)
    assert e.value.status == _abi.MPM_EINVAL
    assert "bytes" in str(e.value)
