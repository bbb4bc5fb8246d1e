"""GPU parity of the full-order MPM step (Algorithm 1) against the FP64 oracle, through the C ABI.

Tolerance: 1e-5 relative, norm-wise per quantity (|a - b|_2 / |b|_2), for the FP32 kernels
against the FP64 oracle.  Where a quantity amplifies FP32 rounding (C, a velocity gradient that
is small against |v| / dx; stress waves through an impact; clamped singular values of the plastic
law), the bound is derived from the oracle's measured sensitivity (tests/fp32_bounds.py) and
printed next to the error.  Cell keys, block counts and block offsets are bit-exact (the oracle
bins the GPU's own FP32 positions).
"""
import numpy as np
import pytest

import fp32_bounds as FB
import oracle.mpm as OM
import synth.scenes as S

pytestmark = pytest.mark.gpu
TOL = 1e-5


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def _ctx(sc):
    from paper_2109_12390_gb300.mpm import MPM
    ctx = MPM.from_scene(sc)
    ctx.load_numpy(sc.x, sc.v, sc.F, sc.C)
    return ctx


def _compare(ctx, ref, init, steps):
    """x, v, F and C of the GPU run against the FP64 oracle run `ref` of `steps` steps from
    `init`: each within 1e-5 or, where the trajectory amplifies FP32 rounding, within K times the
    oracle's own deviation when its state is rounded to FP32 every step (tests/fp32_bounds.py)."""
    x, v, F, Cm = ctx.read_numpy()
    errs = FB.fom_errors(x, v, F, Cm, ref)
    bounds, sens = FB.fom_bounds(init, ref, steps)
    print("errors", errs, "sensitivities", sens)
    assert all(errs[k] < bounds[k] for k in errs), (errs, bounds)
    return errs


def test_config1_block_200_steps():
    """2D neo-Hookean block, 4096 particles, 128^2, dt = 1e-4, 200 steps (free flight)."""
    sc = S.block_2d()
    ctx = _ctx(sc)
    ctx.step(200)
    assert ctx.status() == 0
    ref = sc.copy()
    OM.step(ref, 200)
    _compare(ctx, ref, sc, 200)


@pytest.mark.parametrize("material", [OM.NEO_HOOKEAN, OM.FIXED_COROTATED])
def test_2d_stressed_block_impact(material):
    """2D MLS block with a random initial deformation, dropped onto the sticky floor (dt = 5e-5)."""
    sc = S.block_2d(side=32, dt=5e-5, origin=(0.4, 0.03), v0=np.array([0.3, -0.8]))
    sc.material = material
    rng = np.random.default_rng(1)
    sc.F = S.random_deformation(rng, sc.n_particles, 2, 0.03)
    ctx = _ctx(sc)
    ctx.step(150)
    assert ctx.status() == 0
    ref = sc.copy()
    OM.step(ref, 150)
    assert ref.x[:, 1].min() < 4.5 / 128  # the block reached the floor band
    _compare(ctx, ref, sc, 150)


@pytest.mark.parametrize("material", [OM.NEO_HOOKEAN, OM.FIXED_COROTATED])
def test_2d_pic_impact_from_rest_shape(material):
    """Literal PIC transfers of Algorithm 1 (exact basis gradients) through an impact, from F = I.

    PIC from a rough random F is ill-conditioned (the FP64 oracle itself moves
    v and F by ~5e-5 for a 1e-7 input perturbation), so the PIC case starts
    from a stress-free shape and builds its stress in the impact."""
    sc = S.block_2d(side=32, dt=5e-5, origin=(0.4, 0.03), v0=np.array([0.3, -0.8]))
    sc.transfer, sc.material = OM.PIC, material
    ctx = _ctx(sc)
    ctx.step(150)
    assert ctx.status() == 0
    ref = sc.copy()
    OM.step(ref, 150)
    assert ref.x[:, 1].min() < 4.5 / 128
    assert np.abs(ref.F - np.eye(2)).max() > 1e-3   # stress did build up
    _compare(ctx, ref, sc, 150)


def test_3d_fixed_corotated_cube_slip_floor():
    """3D MLS fixed-corotated jittered cube (16^3), FP64-refined polar, slip floor impact."""
    sc = S.cube_3d(side=16, bottom=0.03)
    rng = np.random.default_rng(2)
    sc.F = S.random_deformation(rng, sc.n_particles, 3, 0.02)
    ctx = _ctx(sc)
    ctx.step(80)
    assert ctx.status() == 0
    ref = sc.copy()
    OM.step(ref, 80)
    assert ref.x[:, 1].min() < 3.5 / 128
    _compare(ctx, ref, sc, 80)


def test_3d_polar_compensated_fp32_matches_fp64():
    """The compensated-FP32 rotation correction of the polar factor (polar_eft = 1) against the
    FP64 one and the oracle, on the stressed 3D impact: same trajectory to FP32 rounding."""
    from paper_2109_12390_gb300.mpm import MPM
    sc = S.cube_3d(side=16, bottom=0.03)
    rng = np.random.default_rng(2)
    sc.F = S.random_deformation(rng, sc.n_particles, 3, 0.02)
    out = []
    for eft in (0, 1):
        ctx = MPM.from_scene(sc, polar_eft=eft)
        ctx.load_numpy(sc.x, sc.v, sc.F, sc.C)
        ctx.step(80)
        assert ctx.status() == 0
        out.append(ctx.read_numpy())
        if eft:
            ref = sc.copy()
            OM.step(ref, 80)
            _compare(ctx, ref, sc, 80)
    # the two runs differ by FP32 rounding amplified over 80 stressed steps (float atomics
    # alone make two runs of one variant differ at ~1e-6)
    for a, b in zip(out[0][:3], out[1][:3]):   # x, v, F
        assert rel(b, a.astype(np.float64)) < 5e-6


def test_3d_pic_homogeneous_deformation():
    """Literal PIC transfers in 3D (exact basis gradients) on a cube released from a homogeneous
    deformation.  (Through an impact at this dt the FP64 oracle itself diverges under PIC, so the
    impact case is covered by MLS only.)"""
    sc = S.cube_3d(side=12, bottom=0.3, dt=2.5e-5)
    sc.transfer = OM.PIC
    A = np.random.default_rng(1).uniform(-1, 1, (3, 3))
    sc.F[:] = np.eye(3) + 0.02 * A
    ctx = _ctx(sc)
    ctx.step(60)
    assert ctx.status() == 0
    ref = sc.copy()
    OM.step(ref, 60)
    _compare(ctx, ref, sc, 60)


def test_batched_uneven_instances():
    """Several instances with uneven particle counts (one empty) in one context."""
    sc = S.batch_2d(seed=3, n_inst=4, count_range=(500, 3000), origin_y=0.03)
    sc = sc.subset_instances([0, 1, 2, 3])
    # make instance 2 empty
    sizes = np.diff(sc.inst_offsets)
    keep = np.ones(sc.n_particles, bool)
    keep[sc.inst_offsets[2]:sc.inst_offsets[3]] = False
    sizes[2] = 0
    sc.x, sc.v, sc.F, sc.C = sc.x[keep], sc.v[keep], sc.F[keep], sc.C[keep]
    sc.inst_offsets = np.concatenate([[0], np.cumsum(sizes)])
    rng = np.random.default_rng(4)
    for k in range(sc.n_inst):   # one homogeneous initial deformation per instance
        s = slice(sc.inst_offsets[k], sc.inst_offsets[k + 1])
        sc.F[s] = np.eye(2) + 0.01 * rng.uniform(-1, 1, (2, 2))
    ctx = _ctx(sc)
    ctx.step(25)
    assert ctx.status() == 0
    ref = sc.copy()
    OM.step(ref, 25)
    _compare(ctx, ref, sc, 25)


def test_cell_keys_and_block_offsets_bit_exact():
    sc = S.cube_3d(side=12, bottom=0.2)
    rng = np.random.default_rng(5)
    sc.v = rng.uniform(-1, 1, size=sc.v.shape)
    ctx = _ctx(sc)
    ctx.step(7)
    x, _, _, _ = ctx.read_numpy()
    ck, bk, off = ctx.debug_bins()
    ref_ck = OM.cell_keys(x.astype(np.float64), sc.dx, sc.n_grid)
    np.testing.assert_array_equal(ck, ref_ck)
    n, B = sc.n_grid, 4
    base = OM.stencil_base(x.astype(np.float64), sc.dx)
    ref_bk = ((base[:, 0] // B) * (n // B) + base[:, 1] // B) * (n // B) + base[:, 2] // B
    np.testing.assert_array_equal(bk, ref_bk)
    _, ref_off = OM.bin_sort(ref_bk, (n // B) ** 3)
    np.testing.assert_array_equal(off, ref_off)


@pytest.mark.parametrize("dim", [2, 3])
def test_grid_transfer_and_update(dim):
    """Algorithm 1 steps 1-2: grid mass, momentum(+dt f) and updated velocity of a stressed state."""
    if dim == 2:
        sc = S.block_2d(side=24, dt=5e-5, origin=(0.45, 0.01))
    else:
        sc = S.cube_3d(side=10, bottom=0.01)
    rng = np.random.default_rng(6)
    sc.F = S.random_deformation(rng, sc.n_particles, dim, 0.05)
    sc.C = rng.uniform(-3, 3, size=sc.C.shape)
    ctx = _ctx(sc)
    m, p, v = ctx.debug_grid()
    mu, lam = OM.lame(sc.E[0], sc.nu[0])
    rm, rp = OM.p2g(sc.x.astype(np.float32).astype(np.float64), sc.v.astype(np.float32).astype(np.float64),
                    sc.F.astype(np.float32).astype(np.float64), sc.C.astype(np.float32).astype(np.float64),
                    sc.p_mass, sc.p_vol, mu, lam, dx=sc.dx, dt=sc.dt, n_grid=sc.n_grid,
                    material=sc.material, transfer=sc.transfer)
    rv = OM.grid_update(rm, rp, dt=sc.dt, gravity=sc.gravity, bc=sc.bc, bc_width=sc.bc_width)
    assert rel(m[0], rm) < TOL
    assert rel(p[0], rp) < TOL
    assert rel(v[0], rv) < TOL
    # walls: the floor band holds wall nodes that received mass
    assert (rm[(slice(None), slice(0, 3))] > 0).any()


def test_single_particle():
    """One particle.  (At E = 1e4, dt = 1e-4 a lone MLS particle is a stiff one-element
    oscillator with amplification |1 - 4 dt^2 (2 mu + lam) / (rho dx^2)| ~ 7.8 per step: any
    FP32 round-off in F grows to overflow, so the case is run at a soft E.)"""
    sc = S.block_2d(side=1, E=50.0)
    sc.v[:] = (0.5, 0.2)
    ctx = _ctx(sc)
    ctx.step(30)
    ref = sc.copy()
    OM.step(ref, 30)
    _compare(ctx, ref, sc, 30)


def test_out_of_grid_is_reported_not_written():
    sc = S.block_2d(side=4)
    sc.x[0] = (0.001, 0.5)  # stencil leaves the grid on the low side
    ctx = _ctx(sc)
    from paper_2109_12390_gb300 import _abi
    word = ctx.status()
    assert "OUT_OF_GRID" in _abi.status_names(word)
    ctx.step(2)
    x, _, _, _ = ctx.read_numpy()
    assert np.isfinite(x).all()


def test_blow_up_is_reported_not_written():
    """A particle whose speed overflows the grid spacing (|v| = 1e30) drags its neighbours to
    huge, then non-finite, coordinates: the step must flag them and keep every index in range
    (no write outside the grid, binning still consistent), and the context stays usable."""
    from paper_2109_12390_gb300 import _abi
    sc = S.block_2d(side=8)
    sc.v[0] = (1e30, 0.0)
    sc.x[1] = (np.nan, 0.5)
    ctx = _ctx(sc)
    ctx.step(4)
    names = _abi.status_names(ctx.status())
    assert "NONFINITE" in names or "OUT_OF_GRID" in names
    x, _, _, _ = ctx.read_numpy()
    assert x.shape == sc.x.shape
    # a clean state loaded into the same context steps normally
    sc2 = S.block_2d(side=8)
    ctx.load_numpy(sc2.x, sc2.v, sc2.F, sc2.C)
    ctx.step(3)
    ref = sc2.copy()
    OM.step(ref, 3)
    _compare(ctx, ref, sc2, 3)


def _sampled_oracle_step(sc, x0, v0, F0, C0, quad, samples):
    """One oracle step of `samples` from the grid of their neighbourhood `quad` (exact locality of
    the stencils: no other particle reaches the samples' stencil nodes)."""
    mu, lam = OM.lame(sc.E[0], sc.nu[0])
    rm, rp = OM.p2g(x0[quad], v0[quad], F0[quad], C0[quad], sc.p_mass, sc.p_vol, mu, lam, dx=sc.dx, dt=sc.dt,
                    n_grid=sc.n_grid, material=sc.material, transfer=sc.transfer)
    rv = OM.grid_update(rm, rp, dt=sc.dt, gravity=sc.gravity, bc=sc.bc, bc_width=sc.bc_width)
    return OM.g2p(x0[samples], F0[samples], rv, dx=sc.dx, dt=sc.dt, transfer=sc.transfer)


def _check_sampled_step(sc, x0, v0, F0, C0, quad, samples, gpu, ref):
    """x, v, F, C of the samples after one GPU step against the oracle's step on the GPU's own
    FP32 input state; bounds from the step's sensitivity to one FP32 ulp of that state."""
    x1, v1, F1, C1 = gpu
    xs, vs, Fs, Cs = ref
    q = np.sort(quad)

    def step(x_, v_, F_, C_):
        xx, vv, FF, CC = (a.copy() for a in (x0, v0, F0, C0))
        xx[q], vv[q], FF[q], CC[q] = x_, v_, F_, C_
        return np.concatenate([a.ravel() for a in _sampled_oracle_step(sc, xx, vv, FF, CC, q, samples)])

    P = len(samples)
    d = sc.dim
    rng = np.random.default_rng(99)
    base = step(x0[q], v0[q], F0[q], C0[q])
    pert = step(*(FB.perturb(a[q], rng) for a in (x0, v0, F0, C0)))
    parts = np.cumsum([P * d, P * d, P * d * d])
    sens = dict(x=FB.rel(pert[:parts[0]], base[:parts[0]]), v=FB.rel(pert[parts[0]:parts[1]], base[parts[0]:parts[1]]),
                F=FB.rel(pert[parts[1]:parts[2]], base[parts[1]:parts[2]]))
    scale = max(np.linalg.norm(Cs), np.linalg.norm(vs) / sc.dx)
    sens["C"] = float(np.linalg.norm(pert[parts[2]:] - base[parts[2]:]) / scale)
    errs = dict(x=FB.rel(x1[samples], xs), v=FB.rel(v1[samples], vs), F=FB.rel(F1[samples], Fs),
                C=float(np.linalg.norm(C1[samples] - Cs) / scale))
    print("errors", errs, "sensitivities", sens)
    for k in errs:
        assert errs[k] < FB.bound(sens[k]), (k, errs, sens)


def _full_size_sampled(pre_steps, pick, n_sample, seed):
    """262,144-particle cube on 128^3 in the benchmark's launch configuration: after `pre_steps`
    GPU steps, the next step of sampled particles (chosen by `pick` from the GPU's state)
    against the oracle evaluated on their neighbourhood only (exact locality of the stencils)."""
    import oracle.rom as OR
    sc = S.cube_3d()
    ctx = _ctx(sc)
    ctx.step(pre_steps)
    assert ctx.status() == 0
    x0, v0, F0, C0 = [a.astype(np.float64) for a in ctx.read_numpy()]
    m, _, _ = ctx.debug_grid()
    assert float(m.sum(dtype=np.float64)) == pytest.approx(sc.n_particles * sc.p_mass, rel=1e-5)
    ctx.step(1)
    x1, v1, F1, C1 = ctx.read_numpy()
    samples = np.sort(pick(x0, np.random.default_rng(seed), n_sample))
    basis, neigh = OR.neighbourhood(x0, samples, sc.dx, sc.n_grid)
    quad = np.concatenate([samples, neigh])
    ref = _sampled_oracle_step(sc, x0, v0, F0, C0, quad, samples)
    _check_sampled_step(sc, x0, v0, F0, C0, quad, samples, (x1, v1, F1, C1), ref)
    ctx.close()
    return sc, x0, basis


def test_config2_full_size_sampled():
    """Free fall: 64 particles anywhere in the cube after 5 steps, plus global mass conservation."""
    _full_size_sampled(5, lambda x, rng, n: rng.choice(len(x), n, replace=False), 64, 7)


def test_config2_full_size_sampled_after_floor_impact():
    """After 600 GPU steps the cube has hit the slip floor (the low-y band of 3 nodes clamps
    v_y >= 0): 96 particles whose stencils reach that band, so that the floor condition, the
    contact's stress and the affine velocities there are all in the comparison."""
    def pick(x, rng, n):
        # base = floor(y / dx - 0.5) <= 2 reaches a node j < 3 of the slip band
        near = np.flatnonzero(np.floor(x[:, 1] * 128.0 - 0.5) <= 2)
        assert len(near) >= n, len(near)
        return rng.choice(near, n, replace=False)
    sc, x0, basis = _full_size_sampled(600, pick, 96, 8)
    j = (basis // sc.n_grid) % sc.n_grid          # linear node id = (i n + j) n + k
    assert (j < 3).any()


def _plastic_flow(sc, steps):
    """The elastic oracle run from the same state: its F differs from the plastic run's only
    where the return mapping acted."""
    ela = sc.copy()
    ela.material = OM.FIXED_COROTATED
    OM.step(ela, steps)
    return ela


@pytest.mark.parametrize("transfer", [OM.MLS, OM.PIC])
def test_2d_plastic_block_impact(transfer):
    """Plastic fixed-corotated block (singular values clamped to [1 - theta_c, 1 + theta_s] after
    every F update) dropped onto the floor: the return mapping acts on most particles and the
    trajectory matches the FP64 oracle to FP32 tolerance."""
    sc = S.block_2d(side=32, dt=5e-5, origin=(0.4, 0.03), v0=np.array([0.3, -0.8]))
    sc.material, sc.transfer = OM.FIXED_COROTATED_PLASTIC, transfer
    if transfer == OM.MLS:
        sc.F = S.random_deformation(np.random.default_rng(1), sc.n_particles, 2, 0.03)
    ctx = _ctx(sc)
    ctx.step(150)
    assert ctx.status() == 0
    ref = sc.copy()
    OM.step(ref, 150)
    assert ref.x[:, 1].min() < 4.5 / 128
    assert np.abs(ref.F - _plastic_flow(sc, 150).F).max() > 1e-4      # plastic flow did happen
    _compare(ctx, ref, sc, 150)


def test_3d_plastic_cube_slip_floor():
    """3D plastic fixed-corotated cube (FP64-refined polar for the stress, FP32 polar and Jacobi
    eigen-decomposition for the return mapping) through a slip-floor impact."""
    sc = S.cube_3d(side=16, bottom=0.03)
    sc.material = OM.FIXED_COROTATED_PLASTIC
    sc.F = S.random_deformation(np.random.default_rng(2), sc.n_particles, 3, 0.02)
    ctx = _ctx(sc)
    ctx.step(80)
    assert ctx.status() == 0
    ref = sc.copy()
    OM.step(ref, 80)
    assert np.abs(ref.F - _plastic_flow(sc, 80).F).max() > 1e-4
    _compare(ctx, ref, sc, 80)


def test_plastic_material_with_wide_bounds_is_elastic():
    """With bounds no singular value reaches, the plastic material is the elastic one (the return
    mapping leaves F untouched); runs differ only by float-atomic ordering."""
    sc = S.cube_3d(side=12, bottom=0.03)
    sc.F = S.random_deformation(np.random.default_rng(3), sc.n_particles, 3, 0.02)
    out = []
    for mat in (OM.FIXED_COROTATED, OM.FIXED_COROTATED_PLASTIC):
        s2 = sc.copy()
        s2.material = mat
        s2.theta_c, s2.theta_s = 0.9, 10.0
        ctx = _ctx(s2)
        ctx.step(40)
        assert ctx.status() == 0
        out.append(ctx.read_numpy())
    for a, b in zip(out[0][:3], out[1][:3]):
        assert rel(b, a.astype(np.float64)) < 5e-6


def test_kinematic_boundaries_clamped_bar():
    """Kinematic (Dirichlet) groups: the held rows stay, the moving rows translate at their
    velocity exactly, and the whole bar matches the FP64 oracle."""
    sc = S.clamped_bar_2d(side=32)
    ctx = _ctx(sc)
    ctx.step(100)
    assert ctx.status() == 0
    ref = sc.copy()
    OM.step(ref, 100)
    x, v, F, Cm = ctx.read_numpy()
    g = sc.kin_group
    np.testing.assert_array_equal(x[g == 0], sc.x[g == 0].astype(np.float32))
    np.testing.assert_allclose(x[g == 1], ref.x[g == 1], rtol=0, atol=2e-6)
    assert np.all(v[g == 1] == sc.kin_vel[1].astype(np.float32)) and np.all(Cm[g >= 0] == 0)
    # the prescribed rows impose a velocity jump at the boundary whose stress waves carry FP32
    # rounding into the free particles' velocities: bounds derived from the oracle's sensitivity
    _compare(ctx, ref, sc, 100)


def test_state_transfer_paths_agree():
    """mpm_set_state / mpm_get_state with pageable host arrays (staged by copies), page-locked host
    tensors (read and written by the kernels directly over the host link) and CUDA tensors: the
    round trip of a loaded state returns it bit for bit through every pair of paths; after three
    steps the state read through every output path (and through an output view that is not
    16-byte aligned) is bit-identical; states loaded through different paths agree after three
    steps up to the order of the float atomics."""
    import torch
    from paper_2109_12390_gb300.mpm import MPM
    sc = S.cube_3d(seed=5, side=12, n_grid=32)
    P, d = len(sc.x), sc.dim
    host = [np.ascontiguousarray(a, np.float32).reshape(P, -1) for a in (sc.x, sc.v, sc.F, sc.C)]

    def buffers(kind):
        if kind == "pageable":
            return [np.empty_like(a) for a in host]
        return [torch.empty(a.shape, dtype=torch.float32, device="cuda" if kind == "cuda" else "cpu",
                            pin_memory=(kind == "pinned")) for a in host]

    def numpy(bufs):
        return [b if isinstance(b, np.ndarray) else b.cpu().numpy() for b in bufs]

    kinds = ("pageable", "pinned", "cuda")
    stepped = []
    for kin in kinds:
        ctx = MPM.from_scene(sc)
        ins = host if kin == "pageable" else [torch.from_numpy(a).pin_memory() if kin == "pinned"
                                              else torch.from_numpy(a).cuda() for a in host]
        ctx.set_state(*ins)
        for kout in kinds:
            outs = buffers(kout)
            ctx.get_state(*outs)
            torch.cuda.synchronize()
            for a, b in zip(numpy(outs), host):
                np.testing.assert_array_equal(a, b)
        ctx.step(3)
        reads = []
        for kout in kinds:
            outs = buffers(kout)
            ctx.get_state(*outs)
            torch.cuda.synchronize()
            reads.append(numpy(outs))
        buf = torch.empty(P * d + 1, dtype=torch.float32, pin_memory=True)
        ctx.get_state(buf[1:].view(P, d))      # starts 4 bytes into a page-locked buffer
        torch.cuda.synchronize()
        np.testing.assert_array_equal(buf[1:].numpy().reshape(P, d), reads[0][0])
        for r in reads[1:]:
            for a, b in zip(r, reads[0]):
                np.testing.assert_array_equal(a, b)
        assert ctx.status() == 0
        stepped.append(reads[0])
        ctx.close()
    for r in stepped[1:]:
        for a, b in zip(r, stepped[0]):
            np.testing.assert_allclose(a, b, rtol=0, atol=1e-5 * np.abs(b).max())
