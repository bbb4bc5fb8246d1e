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
