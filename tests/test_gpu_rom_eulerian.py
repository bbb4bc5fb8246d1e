"""GPU parity of the reduced-order step with the Eulerian quadrature (Algorithm 4) against the FP64
oracle, via the C ABI.

* quadrature cells: bit-exact, the oracle evaluated on the GPU's own decoded FP32 sample positions
  (a floating-point decision taken in the same precision);
* reference positions X_q (Newton inversion of the decoder), mass and reference volume, v_trial,
  vhat_{n+1}: 1e-5 relative, or K times the oracle's measured sensitivity to one FP32 rounding of
  its inputs where the quantity amplifies it (tests/fp32_bounds.py);
* inside flags: identical except for points whose X_q lies within 1e-3 h of an occupancy box face
  (h the box side), where FP32 and FP64 inversions may legitimately decide differently; those points
  take the GPU's decision on both sides;
the oracle is given the FP32 values of the decoder, the reference positions and the latents
that the GPU uses (FP32 decoder on the CUDA cores).
"""
import numpy as np
import pytest

import fp32_bounds as FB
import oracle.decoder as OD
import oracle.mpm as OM
import oracle.rom as OR
import synth.scenes as S

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def _rom_scene(sc, k, seed):
    return OR.RomScene(X=sc.x.copy(), mass=sc.p_mass, vol=sc.p_vol, E=float(sc.E[0]), nu=float(sc.nu[0]),
                       dx=sc.dx, dt=sc.dt, n_grid=sc.n_grid, gravity=sc.gravity, bc=sc.bc, bc_width=sc.bc_width,
                       material=sc.material, transfer=sc.transfer, n_samples=k, seed=seed, quadrature="eulerian")


def _order_key(x, dx, ell, n, d):
    """(cell id, sub-point id) of Eulerian points at (c + (j + 1/2) / ell) dx, as one sortable key."""
    u = np.asarray(x, np.float64) / dx
    c = np.floor(u).astype(np.int64)
    j = np.floor((u - c) * ell).astype(np.int64)
    cl = np.zeros(len(u), np.int64)
    jl = np.zeros(len(u), np.int64)
    for a in range(d):
        cl = cl * n + c[:, a]
        jl = jl * ell + j[:, a]
    return cl * ell ** d + jl, cl


def _check_step(sc, p, k, seed, projection=1, transfer=None, m_kin=0):
    import torch
    from paper_2109_12390_gb300.decoder import Decoder, PRIMAL
    from paper_2109_12390_gb300.rom import ROM
    d, r = sc.dim, p.r
    if transfer is not None:
        sc.transfer = transfer
    dec = Decoder.from_params(p)
    dec.set_precision(True)
    rom = ROM.from_scene(dec, sc, n_samples=k, seed=seed, projection=projection, quadrature=1)
    if m_kin:
        rom.set_kinematic(sc.kin_group, sc.kin_vel, min_samples=m_kin)
    rng = np.random.default_rng(seed)
    xh = 0.3 * rng.normal(size=r)
    vh = rng.normal(size=r)
    rom.set_state(xh, vh, xh - sc.dt * vh, 0)
    rom.step(1)
    assert rom.status() == 0
    dbg = rom.debug()
    samples = dbg["samples"]
    if m_kin:
        want = OR.kinematic_sample_set(seed, 0, 0, len(sc.x), k, sc.kin_group, m_kin)
    else:
        want = OR.sample_set(seed, 0, 0, len(sc.x), k)
    np.testing.assert_array_equal(samples, want)
    # the GPU's own decoded sample positions (same kernel and rows as the step's sample decode)
    Xs = np.ascontiguousarray(sc.x[samples], np.float32)
    out = dec.eval(torch.from_numpy(Xs).cuda(), torch.from_numpy(xh.astype(np.float32)[None]).cuda(),
                   [PRIMAL] + [dec.dxhat(j) for j in range(r)]).cpu().numpy()
    xs = out[0].astype(np.float64)
    assert rel(xs, OD.decode(p, sc.x[samples], xh)) < 1e-6
    qg = rom.quadrature_points()
    rs = _rom_scene(sc, k, seed)
    if m_kin:
        rs.kin_group, rs.kin_vel, rs.kin_min_samples = sc.kin_group, sc.kin_vel, m_kin
        g = sc.kin_group[samples]
        assert np.array_equal(dbg["v_trial"][g >= 0], sc.kin_vel[g[g >= 0]].astype(np.float32))
    # the oracle on the FP32 values the GPU uses
    p32, xh32, vh32 = FB.f32_decoder(p), FB.f32(xh), FB.f32(vh)
    rs.X = FB.f32(rs.X)
    quad = OR.eulerian_quadrature(p32, rs, xh32, vh32, samples, xs)
    basis, cells, xq, Xq, FX, vq, mq, V0, inside = quad
    # point sets: same cells, same points
    key_g, cells_g = _order_key(qg["x"], sc.dx, rs.ell, sc.n_grid, d)
    np.testing.assert_array_equal(np.unique(cells_g), cells)
    key_o, _ = _order_key(xq, sc.dx, rs.ell, sc.n_grid, d)
    assert len(key_g) == len(key_o) and len(np.unique(key_g)) == len(key_g)
    og, oo = np.argsort(key_g), np.argsort(key_o)
    np.testing.assert_array_equal(key_g[og], key_o[oo])
    np.testing.assert_allclose(qg["x"][og], xq[oo], rtol=0, atol=1e-6 * sc.dx + 1e-7)
    # inside flags, up to points within 1e-3 h of a box face
    h = rs.vol ** (1.0 / d)
    origin = sc.x.min(0) - 0.5 * h
    fr = (Xq - origin) / h
    border = np.abs(fr - np.round(fr)).min(1) < 1e-3
    inside_g = np.zeros(len(Xq), bool)
    inside_g[oo] = qg["mass"][og] > 0
    np.testing.assert_array_equal(inside_g[~border], inside[~border])
    override = (np.nonzero(border)[0], inside_g[border])

    # the local step, and the same step with the decoder and latents perturbed by one FP32 ulp
    # (the cells and points stay those of the GPU's own sample positions)
    def run(pp, x_, v_):
        return OR.eulerian_local_dynamics(pp, rs, x_, v_, samples, xs, inside_override=override)

    v_trial, x_trial, quad = run(p32, xh32, vh32)
    rng = np.random.default_rng(77)
    v_p, _, quad_p = run(FB.perturb_decoder(p32, rng), FB.perturb(xh32, rng), FB.perturb(vh32, rng))
    Xq, mq, V0, inside = quad[3], quad[6], quad[7], quad[8]
    # inversion: converged points agree with the FP64 Newton iterate
    conv = np.linalg.norm(OD.decode(p32, Xq, xh32) - xq, axis=1) < rs.newton_tol * sc.dx
    Xg = np.empty_like(Xq)
    Xg[oo] = qg["X"][og]
    err_X = np.abs(Xg - Xq)[conv].max()
    sens_X = np.abs(quad_p[3] - Xq)[conv].max()
    lim_X = max(1e-5 * np.abs(Xq).max(), FB.K * sens_X)
    print(f"inversion: max error {err_X / sc.dx:.3e} dx, sensitivity {sens_X / sc.dx:.3e} dx, bound {lim_X / sc.dx:.3e} dx")
    assert err_X < lim_X
    mg = np.empty_like(mq)
    mg[oo] = qg["mass"][og]
    vg = np.empty_like(V0)
    vg[oo] = qg["V0"][og]
    assert inside.sum() > 0
    for name, got, ref, pert in (("mass", mg, mq, quad_p[6]), ("volume", vg, V0, quad_p[7]),
                                 ("v_trial", dbg["v_trial"], v_trial, v_p)):
        err, sens = rel(got, ref), FB.rel(pert, ref)
        print(f"{name}: error {err:.3e} sensitivity {sens:.3e} bound {FB.bound(sens):.3e}")
        assert err < FB.bound(sens), name
    assert rel(dbg["x_trial"], x_trial) < 1e-6
    _, vh1, _, step = rom.get_state()
    assert step == 1
    FB.check_velocity_projection(p, sc.x[samples], xh, dbg["v_trial"].astype(np.float64), vh1, "eulerian",
                                 vhat_n=vh)
    rom.close()
    dec.close()
    return int(border.sum()), len(xq), int(inside.sum())


@pytest.mark.parametrize("transfer", [OM.MLS, OM.PIC])
def test_eulerian_step_2d(transfer):
    sc = S.block_2d(side=32, dt=5e-5, origin=(0.4, 0.3), E=1e3)
    X = sc.x
    p = S.near_identity_decoder(7, 2, 4, 1, X_min=X.min(0), X_range=X.max(0) - X.min(0), eps=3e-3)
    nb, nq, ni = _check_step(sc, p, 64, 3, transfer=transfer)
    print(f"2D Eulerian: {nq} points, {ni} inside, {nb} within 1e-3 h of a box face")


def test_eulerian_step_2d_deep_decoder_position_projection():
    sc = S.block_2d(side=32, dt=5e-5, origin=(0.4, 0.3), E=1e3)
    X = sc.x
    p = S.near_identity_decoder(9, 2, 4, 5, X_min=X.min(0), X_range=X.max(0) - X.min(0), eps=3e-3)
    _check_step(sc, p, 64, 5, projection=0)


def test_eulerian_step_benchmark_size():
    """The Eulerian step at the benchmark's size and launch configuration (4096 particles, 256
    samples, r = 16, 5 hidden layers on the FP32 decoder path, 3 Gauss-Newton iterations, about
    5,000 quadrature points): one step against the oracle, then 20 steps run clean."""
    from paper_2109_12390_gb300.decoder import Decoder
    from paper_2109_12390_gb300.rom import ROM
    sc = S.block_2d(side=64, dt=5e-5, origin=(0.375, 0.3), E=1e3)
    X = sc.x
    p = S.near_identity_decoder(9, 2, 16, 5, X_min=X.min(0), X_range=X.max(0) - X.min(0), eps=3e-3)
    nb, nq, ni = _check_step(sc, p, 256, 5, projection=0)
    assert nq > 4000 and ni > 3000
    dec = Decoder.from_params(p)
    dec.set_precision(True)
    rom = ROM.from_scene(dec, sc, n_samples=256, seed=5, quadrature=1)
    rng = np.random.default_rng(5)
    xh = 0.3 * rng.normal(size=16)
    vh = rng.normal(size=16)
    rom.set_state(xh, vh, xh - sc.dt * vh, 0)
    rom.step(20)
    assert rom.status() == 0
    xh1, vh1, _, step = rom.get_state()
    assert step == 20 and np.isfinite(xh1).all() and np.isfinite(vh1).all()
    rom.close()
    dec.close()


def test_eulerian_step_kinematic_boundaries():
    """Kinematic (Dirichlet) groups with the Eulerian quadrature: the sample set adds each group's
    smallest-hash particles (bit-exact), kinematic samples take their prescribed trial velocity,
    and the quadrature cells, points and the other trial velocities match the oracle around the
    enlarged sample set."""
    sc = S.clamped_bar_2d(side=32)
    X = sc.x
    p = S.near_identity_decoder(21, 2, 4, 1, X_min=X.min(0), X_range=X.max(0) - X.min(0), eps=3e-3)
    _check_step(sc, p, 48, 6, projection=0, m_kin=5)


def test_eulerian_step_3d():
    sc = S.cube_3d(seed=2, side=12, n_grid=64, dt=5e-5, bottom=0.3)
    X = sc.x
    p = S.near_identity_decoder(11, 3, 4, 1, X_min=X.min(0), X_range=X.max(0) - X.min(0), eps=1e-3)
    _check_step(sc, p, 48, 13)


def test_eulerian_translation_free_fall():
    """Hand-set linear decoder g = X + xhat: with the Eulerian quadrature the reduced step still
    follows the full-order free fall (closed form) and the oracle's reduced step, same samples."""
    from paper_2109_12390_gb300.decoder import Decoder
    from paper_2109_12390_gb300.rom import ROM
    sc = S.block_2d(side=16, dt=5e-5, origin=(0.375, 0.375), v0=np.array([0.2, 0.3]))
    X = sc.x
    lo, rg = X.min(0), X.max(0) - X.min(0)
    p = S.xavier_decoder(0, 2, 2, 128, 0, OD.IDENTITY, X_min=lo, X_range=rg)
    p.W[0] = np.concatenate([np.diag(rg), np.eye(2)], axis=1)
    p.b[0] = np.array(lo, np.float64)
    dec = Decoder.from_params(p)
    rom = ROM.from_scene(dec, sc, n_samples=12, seed=4, quadrature=1)
    v0 = sc.v[0]
    rom.set_state(np.zeros(2), v0, -sc.dt * v0, 0)
    rs = _rom_scene(sc, 12, 4)
    st = OR.RomState(xhat=np.zeros(2), vhat=v0.copy(), xhat_prev=-sc.dt * v0)
    for n in range(10):
        rec = {}
        st = OR.rom_step(p, rs, st, rec)
        rom.step(1)
        np.testing.assert_array_equal(rom.debug()["samples"], rec["samples"])
    assert rom.status() == 0
    xh, vh, _, step = rom.get_state()
    assert step == 10
    np.testing.assert_allclose(vh, v0 + 10 * sc.dt * sc.gravity[:2], rtol=1e-5)
    np.testing.assert_allclose(xh, st.xhat, rtol=1e-5, atol=1e-9)
    q = rom.quadrature_points()
    assert (q["mass"] > 0).any()
    # translation: J = 1, every inside point carries rho0 (dx / 2)^2
    m = q["mass"][q["mass"] > 0]
    np.testing.assert_allclose(m, sc.p_mass / sc.p_vol * (sc.dx / 2) ** 2, rtol=1e-5)
