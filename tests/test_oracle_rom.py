"""Pins of the FP64 reduced-order oracle (Algorithms 2, 3, 5, 6, 7)."""
import os

import numpy as np
import pytest

import oracle.decoder as D
import oracle.mpm as M
import oracle.rom as R
import synth.scenes as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_known_answers():
    vals = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) if l.startswith("0x")]
    got = [int(R.splitmix64_out(np.uint64(0), np.uint64(k))) for k in range(3)]
    assert got == vals


def test_bottom_k_against_full_sort_and_uniformity():
    P, k = 500, 37
    h = R.sample_hash(5, 2, 9, np.arange(P, dtype=np.uint64))
    ref = sorted(range(P), key=lambda p: (int(h[p]), p))[:k]
    assert list(R.sample_set(5, 2, 9, P, k)) == sorted(ref)
    # every particle is drawn with probability k / P
    counts = np.zeros(P)
    steps = 400
    for s in range(steps):
        counts[R.sample_set(1, 0, s, P, k)] += 1
    expect = steps * k / P
    chi2 = np.sum((counts - expect) ** 2 / expect)
    assert chi2 < P + 5 * np.sqrt(2 * P)          # chi-square with P-1 dof, ~5 sigma bound
    assert len(np.unique(R.sample_set(1, 0, 0, P, k))) == k


def test_neighbourhood_brute_force():
    rng = np.random.default_rng(3)
    for d in (2, 3):
        n, dx = 16, 1.0 / 16
        x = 0.3 + 0.4 * rng.uniform(size=(64, d))
        samples = np.array(sorted(rng.choice(64, 6, replace=False)))
        basis, neigh = R.neighbourhood(x, samples, dx, n)
        # brute force: explicit node tuples
        def stencil(p):
            b = [int(np.floor(x[p, k] / dx - 0.5)) for k in range(d)]
            out = set()
            for off in np.ndindex(*(3,) * d):
                out.add(tuple(b[k] + off[k] for k in range(d)))
            return out
        I = set()
        for p in samples:
            I |= stencil(p)
        lin = sorted(sum(t[k] * n ** (d - 1 - k) for k in range(d)) for t in I)
        assert list(basis) == lin
        Nset = [q for q in range(64) if q not in set(samples) and stencil(q) & I]
        assert list(neigh) == Nset


def _translation_decoder(d, X_min, X_range):
    """g(X; xhat) = X + xhat as a one-layer linear network (r = d)."""
    dec = S.xavier_decoder(0, d, d, 8, 0, D.IDENTITY, X_min=X_min, X_range=X_range)
    dec.W[0] = np.concatenate([np.diag(X_range), np.eye(d)], axis=1)
    dec.b[0] = np.array(X_min, np.float64)
    return dec


def test_rom_reproduces_free_fall_exactly():
    sc = S.block_2d(side=16, dt=5e-5, v0=np.array([0.2, 0.3]))
    X = sc.x.copy()
    dec = _translation_decoder(2, X.min(0), X.max(0) - X.min(0))
    rs = R.RomScene(X=X, mass=sc.p_mass, vol=sc.p_vol, E=1e4, nu=0.3, dx=sc.dx, dt=sc.dt, n_grid=sc.n_grid,
                    gravity=sc.gravity, bc=sc.bc, bc_width=sc.bc_width, material=sc.material,
                    transfer=sc.transfer, n_samples=12, seed=4)
    st = R.rom_init(dec, X, sc.v[0], sc.dt)
    np.testing.assert_allclose(st.xhat, 0.0, atol=1e-14)
    np.testing.assert_allclose(st.vhat, sc.v[0], atol=1e-14)
    fom = sc.copy()
    for n in range(1, 11):
        st = R.rom_step(dec, rs, st)
        M.step(fom, 1)
        np.testing.assert_allclose(D.decode(dec, X, st.xhat), fom.x, atol=1e-13)
    assert not st.no_decrease
    g = sc.gravity[:2]
    np.testing.assert_allclose(st.vhat, sc.v[0] + 10 * sc.dt * g, atol=1e-12)


def test_gauss_newton_equals_qr_least_squares_for_linear_decoder():
    rng = np.random.default_rng(6)
    d, r = 3, 2          # a linear decoder's latent Jacobian is shared by all points: rank <= d
    dec = S.xavier_decoder(9, d, r, 8, 0, D.IDENTITY, bias_scale=0.5)
    Xs = rng.uniform(size=(11, d))
    target = rng.uniform(size=(11, d))
    xh, flag = R.gauss_newton(dec, Xs, target, rng.normal(size=r), iters=1)
    assert not flag
    # closed form via QR of the affine map xhat -> g
    _, _, J = D.jacobians(dec, Xs, np.zeros(r))
    A = J.reshape(-1, r)
    b = (target - D.decode(dec, Xs, np.zeros(r))).reshape(-1)
    Q, Rm = np.linalg.qr(A)
    sol = np.linalg.solve(Rm, Q.T @ b)
    np.testing.assert_allclose(xh, sol, rtol=1e-12, atol=1e-12)


def test_gauss_newton_reaches_the_nonlinear_least_squares_minimiser():
    """Alg. 6 on a nonlinear (ELU) decoder: with a consistent target it recovers the latent that
    produced it to round-off within 5 iterations (Gauss-Newton converges quadratically at zero
    residual); with a noisy target it reaches the minimiser that scipy's Levenberg-Marquardt finds
    from the same start; from a far start the backtracking keeps every iteration's objective at
    or below the previous one."""
    so = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(31)
    d, r = 2, 3
    X = rng.uniform(0.3, 0.6, size=(20, d))
    dec = S.xavier_decoder(7, d, r, 16, 2, D.ELU, X_min=X.min(0), X_range=X.max(0) - X.min(0),
                           out_scale=np.full(d, 0.2), bias_scale=0.2)
    xt = rng.normal(size=r)
    exact = D.decode(dec, X, xt)
    for pert in (0.3, 1.0):
        x0 = xt + pert * np.random.default_rng(1).normal(size=r)
        xh, flag = R.gauss_newton(dec, X, exact, x0, iters=5)
        np.testing.assert_allclose(xh, xt, rtol=0, atol=1e-13)
    noisy = exact + 0.002 * rng.normal(size=exact.shape)

    def f(z):
        return (D.decode(dec, X, z) - noisy).reshape(-1)

    x0 = xt + 1.0 * rng.normal(size=r)
    ref = so.least_squares(f, x0, xtol=1e-15, ftol=1e-15, gtol=1e-15, method="lm").x
    xh, _ = R.gauss_newton(dec, X, noisy, x0, iters=40)
    np.testing.assert_allclose(xh, ref, rtol=0, atol=1e-7)
    z = xt + 3.0 * rng.normal(size=r)
    obj = [f(z) @ f(z)]
    for _ in range(8):
        z, _ = R.gauss_newton(dec, X, noisy, z, iters=1)
        obj.append(f(z) @ f(z))
    assert np.all(np.diff(obj) <= 0) and obj[-1] < 1e-2 * obj[0]


def test_gauss_newton_record_and_replay_of_line_search_choices():
    """Algorithm 6's backtracking: the record of each iteration lists the objective at every trial
    2^-m; the search took the first trial with sufficient decrease; the next iteration's f0
    (formed from the decoder's value at the new iterate, not from the record) equals the chosen
    trial's objective; replaying the choices reproduces the searched run exactly; and a far start
    makes the search halve at least once."""
    rng = np.random.default_rng(31)
    d, r = 2, 3
    X = rng.uniform(0.3, 0.6, size=(20, d))
    dec = S.xavier_decoder(7, d, r, 16, 2, D.ELU, X_min=X.min(0), X_range=X.max(0) - X.min(0),
                           out_scale=np.full(d, 0.2), bias_scale=0.2)
    target = D.decode(dec, X, rng.normal(size=r)) + 0.002 * rng.normal(size=(20, d))
    x0 = 3.0 * rng.normal(size=r)
    rec = []
    xh, _ = R.gauss_newton(dec, X, target, x0, iters=6, record=rec)
    picks = []
    for it in rec:
        ok = it["f"] <= it["f0"] + 1e-4 * 0.5 ** np.arange(len(it["f"])) * it["slope"]
        picks.append(int(np.argmax(ok)) if ok.any() else -1)
    assert max(picks) > 0
    for i in range(len(rec) - 1):
        if picks[i] >= 0:
            assert rec[i + 1]["f0"] == pytest.approx(rec[i]["f"][picks[i]], rel=1e-12)
    xr, _ = R.gauss_newton(dec, X, target, x0, iters=6, steps=picks)
    np.testing.assert_array_equal(xr, xh)
    # a different choice gives a different (and here worse) result
    other = list(picks)
    other[0] = picks[0] + 1
    xo, _ = R.gauss_newton(dec, X, target, x0, iters=1, steps=other[:1])
    x1, _ = R.gauss_newton(dec, X, target, x0, iters=1)
    assert not np.array_equal(xo, x1)


def test_velocity_only_matches_position_velocity_to_second_order():
    rng = np.random.default_rng(1)
    d, r = 2, 3
    dec = S.xavier_decoder(2, d, r, 16, 3, D.ELU, bias_scale=0.3)
    Xs = rng.uniform(size=(20, d))
    xh = 0.3 * rng.normal(size=r)
    v_trial = rng.normal(size=(20, d))
    diffs = []
    for dt in (2e-3, 1e-3, 5e-4):
        x_trial = D.decode(dec, Xs, xh) + dt * v_trial
        vh = R.project_velocity(dec, Xs, xh, v_trial)
        x_vo = xh + dt * vh
        x_pv, _ = R.gauss_newton(dec, Xs, x_trial, xh, iters=6)
        diffs.append(np.linalg.norm(x_pv - x_vo))
    assert diffs[0] / diffs[1] == pytest.approx(4.0, rel=0.1)
    assert diffs[1] / diffs[2] == pytest.approx(4.0, rel=0.1)


def test_position_error_toy():
    err = R.PositionError()
    err.add(np.array([[1.0, 0.0], [0.0, 2.0], [1.0, 1.0]]), np.array([[1.0, 0.0], [0.0, 2.0], [1.0, 0.0]]))
    err.add(np.array([[0.0, 0.0], [3.0, 0.0], [0.0, 0.0]]), np.array([[0.0, 1.0], [3.0, 0.0], [0.0, 0.0]]))
    # numerator: 1 + 1 = 2; denominator: 1 + 4 + 1 + 1 + 9 = 16 -> 100 * sqrt(2) / 4
    assert err.percent() == pytest.approx(100 * np.sqrt(2) / 4, rel=1e-15)


def test_ridge_projection_equals_augmented_least_squares():
    """The ridge option: argmin |J a - b|^2 + rho tr(J^T J)/r |a|^2 equals the plain
    least-squares solution of the stacked system [J; sqrt(lam) I] a = [b; 0]."""
    rng = np.random.default_rng(12)
    J = rng.normal(size=(40, 6)) @ np.diag([1, 1, 1, 1e-2, 1e-3, 1e-3])
    b = rng.normal(size=40)
    rho = 1e-3
    lam = rho * np.trace(J.T @ J) / 6
    aug = np.linalg.lstsq(np.vstack([J, np.sqrt(lam) * np.eye(6)]), np.concatenate([b, np.zeros(6)]), rcond=None)[0]
    np.testing.assert_allclose(R.lstsq(J, b, rho), aug, rtol=1e-10, atol=1e-12)
    # rho -> 0 recovers the least-squares fit on the well-determined directions
    np.testing.assert_allclose(J @ R.lstsq(J, b, 1e-14), J @ R.lstsq(J, b), rtol=1e-6, atol=1e-8)


def test_ridge_velocity_projection_penalises_the_change_from_vhat_n():
    """With the ridge, the velocity projection equals the stacked least-squares problem
    [J; sqrt(lam) I] v = [v_trial; sqrt(lam) vhat_n]: near-null latent directions keep vhat_n
    (a constant latent velocity that J reproduces exactly is a fixed point for any ridge), and
    ridge = 0 is the plain fit."""
    rng = np.random.default_rng(13)
    d, r = 2, 4
    X = rng.uniform(0.3, 0.6, size=(30, d))
    dec = S.xavier_decoder(2, d, r, 16, 2, D.ELU, X_min=X.min(0), X_range=X.max(0) - X.min(0),
                           out_scale=np.full(d, 0.1), bias_scale=0.2)
    xh = 0.2 * rng.normal(size=r)
    vh_n = rng.normal(size=r)
    _, _, Jq = D.jacobians(dec, X, xh)
    J = Jq.reshape(-1, r)
    vt = (J @ vh_n).reshape(-1, d)
    for rho in (0.0, 1e-4, 1e-1):
        np.testing.assert_allclose(R.project_velocity(dec, X, xh, vt, rho, vh_n), vh_n, rtol=1e-9, atol=1e-11)
    vt2 = vt + 0.3 * rng.normal(size=vt.shape)
    rho = 1e-2
    lam = rho * np.trace(J.T @ J) / r
    aug = np.linalg.lstsq(np.vstack([J, np.sqrt(lam) * np.eye(r)]),
                          np.concatenate([vt2.reshape(-1), np.sqrt(lam) * vh_n]), rcond=None)[0]
    np.testing.assert_allclose(R.project_velocity(dec, X, xh, vt2, rho, vh_n), aug, rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(R.project_velocity(dec, X, xh, vt2, 0.0, vh_n),
                               np.linalg.lstsq(J, vt2.reshape(-1), rcond=None)[0], rtol=1e-9, atol=1e-11)


def test_reference_gradient_makes_the_decoded_initial_state_stress_free():
    """f_reference: with G_p the inverse decoded gradient at xhat_ref, the stress-carrying gradient
    at xhat_ref is the identity exactly, so a body at rest (vhat = 0, g = 0) in the decoded
    reference configuration gets zero trial velocity; without the correction the decoder's
    gradient error at rest produces stress and motion."""
    from oracle import mpm as OM
    sc = S.block_2d(side=8, dt=5e-5, origin=(0.4, 0.4), E=1e4)
    rng = np.random.default_rng(5)
    # a linear decoder g = A X + E xhat whose gradient A at rest is 1 % off the identity
    lo, rng_ = sc.x.min(0), sc.x.max(0) - sc.x.min(0)
    dec = S.xavier_decoder(0, 2, 3, 128, 0, D.IDENTITY, X_min=lo, X_range=rng_)
    A = np.eye(2) + 0.01 * rng.uniform(-1, 1, (2, 2))
    dec.W[0] = np.concatenate([A @ np.diag(rng_), 0.01 * rng.normal(size=(2, 3))], axis=1)
    dec.b[0] = A @ lo
    xh = 0.1 * rng.normal(size=3)
    rs = R.RomScene(X=sc.x.copy(), mass=sc.p_mass, vol=sc.p_vol, E=1e4, nu=0.3, dx=sc.dx, dt=sc.dt,
                    n_grid=sc.n_grid, gravity=np.zeros(3), bc=sc.bc, bc_width=sc.bc_width,
                    material=OM.NEO_HOOKEAN, transfer=OM.MLS, n_samples=16, seed=1)
    x_all = D.decode(dec, sc.x, xh)
    samples = R.sample_set(1, 0, 0, len(sc.x), 16)
    v0, _, _, _ = R.local_dynamics(dec, rs, xh, np.zeros(3), samples, x_all)
    assert np.abs(v0).max() > 1e-6           # stress from the decoder's gradient error
    rs.F_ref_inv = R.reference_inverse(dec, sc.x, xh)
    _, FX, _ = D.jacobians(dec, sc.x, xh)
    np.testing.assert_allclose(np.einsum("pik,pkj->pij", FX, rs.F_ref_inv), np.broadcast_to(np.eye(2), FX.shape),
                               atol=1e-12)
    v1, _, _, _ = R.local_dynamics(dec, rs, xh, np.zeros(3), samples, x_all)
    assert np.abs(v1).max() < 1e-9 * np.abs(v0).max()


# ---------------------------------------------------------------- Eulerian quadrature (Alg. 4)


def test_eulerian_cells_brute_force():
    """Cells whose ell = 2 quadrature points reach a basis node: enumerate every cell's points and
    their stencils directly."""
    n, d, dx = 16, 2, 1.0 / 16
    basis = np.array([5 * n + 7, 9 * n + 9])
    cells = R.eulerian_cells(basis, d, n)
    want = []
    for c in range(n * n):
        ci = np.array(np.unravel_index(c, (n, n)))
        if ci.min() < 1 or ci.max() > n - 3:
            continue
        pts, _ = R.eulerian_points(np.array([c]), d, n, dx, 2)
        nodes = R.stencil_nodes(pts, dx, n)
        if np.isin(nodes, basis).any():
            want.append(c)
    np.testing.assert_array_equal(cells, want)


def test_eulerian_points_tile_their_cells():
    """ell^d points per cell at the centres of the ell^d equal sub-cells (Section 3.2.2): each
    point lies inside its own cell, the sub-cell volumes add up to the cells' volume, and in 3D the
    points of one cell are the sub-cell centres written out by hand."""
    n, dx = 16, 1.0 / 16
    for d in (2, 3):
        cells = np.array([3, 5 * n + 7, 2 * n + 9] if d == 2 else [3, (5 * n + 7) * n + 2])
        for ell in (1, 2, 3):
            pts, vol = R.eulerian_points(cells, d, n, dx, ell)
            assert pts.shape == (len(cells) * ell ** d, d)
            owner = np.ravel_multi_index(tuple(np.floor(pts / dx).astype(np.int64).T), (n,) * d)
            np.testing.assert_array_equal(owner, np.repeat(cells, ell ** d))
            assert vol * len(pts) == pytest.approx(len(cells) * dx ** d, rel=1e-14)
            assert len(np.unique(pts, axis=0)) == len(pts)
    pts, _ = R.eulerian_points(np.array([(1 * n + 2) * n + 3]), 3, n, dx, 2)
    want = [[(1 + a / 2 + 0.25) * dx, (2 + b / 2 + 0.25) * dx, (3 + c / 2 + 0.25) * dx]
            for a in range(2) for b in range(2) for c in range(2)]
    np.testing.assert_allclose(pts, want, rtol=0, atol=1e-15)


def test_reference_domain_is_the_union_of_particle_boxes():
    """Inside test of the reference domain (Section 3.2.2: a point belongs to the body when it lies
    in the reference configuration): an L-shaped body with a hole on a lattice of spacing h,
    against the union of the particles' boxes [X_p - h/2, X_p + h/2)^d tested point by point.
    h is a power of two, so box faces are exact and points on them are tested too."""
    h = 0.25
    for d in (2, 3):
        ks = np.array(list(np.ndindex(*(6,) * d)))
        keep = ~((ks[:, 0] >= 3) & (ks[:, 1] >= 3))          # L shape
        keep &= ~np.all(ks[:, :2] == [1, 1], axis=1)           # a hole
        X = 1.0 + (ks[keep] + 0.5) * h
        origin, shape, occ = R.reference_occupancy(X, h)
        rng = np.random.default_rng(5 + d)
        Xq = np.concatenate([rng.uniform(0.5, 3.0, size=(4000, d)),
                             1.0 + rng.integers(-2, 9, size=(2000, d)) * (h / 2)])
        got = R.inside_reference(Xq, origin, h, shape, occ)
        lo, hi = X - h / 2, X + h / 2
        want = np.array([np.any(np.all((lo <= q) & (q < hi), axis=1)) for q in Xq])
        np.testing.assert_array_equal(got, want)
        assert want.any() and not want.all()


def test_decoder_inversion():
    """Newton inversion of g(X; xhat) = x: exact in one iteration for a decoder affine in X, and to
    round-off for an ELU decoder started from a perturbed reference position."""
    rng = np.random.default_rng(21)
    X = rng.uniform(0.3, 0.6, size=(40, 2))
    lin = _translation_decoder(2, X.min(0), X.max(0) - X.min(0))
    lin.W[0][:, :2] = lin.W[0][:, :2] @ np.array([[1.1, 0.2], [-0.1, 0.9]])
    xh = np.array([0.01, -0.02])
    x = D.decode(lin, X, xh)
    Xi, res = R.invert_decoder(lin, x, xh, X + 0.01, 1)
    np.testing.assert_allclose(Xi, X, atol=1e-13)
    dec = S.xavier_decoder(4, 2, 3, 32, 2, D.ELU, X_min=X.min(0), X_range=X.max(0) - X.min(0),
                           out_shift=X.mean(0), out_scale=np.full(2, 0.1), bias_scale=0.1)
    dec.W[0][:, :2] *= 0.3
    xh = 0.1 * rng.normal(size=3)
    x = D.decode(dec, X, xh)
    _, FX, _ = D.jacobians(dec, X, xh)
    assert np.abs(np.linalg.det(FX)).min() > 0
    Xi, res = R.invert_decoder(dec, x, xh, X + 1e-3 * rng.normal(size=X.shape), 6)
    assert res.max() < 1e-13
    np.testing.assert_allclose(Xi, X, atol=1e-11)


def test_eulerian_quadrature_mass_and_free_fall():
    """Translation decoder g = X + xhat with the body aligned to the quadrature grid: when the
    samples' cells cover the whole block, the inside quadrature points carry exactly the
    particles' total mass; and the Eulerian reduced step reproduces the full-order free fall."""
    sc = S.block_2d(side=16, dt=5e-5, origin=(0.375, 0.375), v0=np.array([0.2, 0.3]))
    X = sc.x.copy()
    dec = _translation_decoder(2, X.min(0), X.max(0) - X.min(0))
    rs = R.RomScene(X=X, mass=sc.p_mass, vol=sc.p_vol, E=1e4, nu=0.3, dx=sc.dx, dt=sc.dt, n_grid=sc.n_grid,
                    gravity=sc.gravity, bc=sc.bc, bc_width=sc.bc_width, material=sc.material,
                    transfer=sc.transfer, n_samples=len(X), seed=4, quadrature="eulerian")
    xh = np.array([2, -1]) * sc.dx / 2          # a shift by whole quadrature spacings keeps the alignment
    samples = np.arange(len(X))
    q = R.eulerian_quadrature(dec, rs, xh, np.zeros(2), samples, D.decode(dec, X, xh))
    mq, inside = q[6], q[8]
    assert inside.sum() == len(X)              # ell = 2 on a block at dx / 2 spacing: one point per particle
    np.testing.assert_allclose(mq.sum(), sc.p_mass * len(X), rtol=1e-14)
    rs.n_samples = 12
    st = R.rom_init(dec, X, sc.v[0], sc.dt)
    fom = sc.copy()
    for _ in range(5):
        st = R.rom_step(dec, rs, st)
        M.step(fom, 1)
        np.testing.assert_allclose(D.decode(dec, X, st.xhat), fom.x, atol=1e-13)


def test_kinematic_sample_set_brute_force():
    """Every kinematic group contributes its min(m, |g|) smallest-(hash, id) particles to the sample
    set; the bottom-k draw comes first, the group extras (not already drawn) after it."""
    rng = np.random.default_rng(0)
    P, k, m = 500, 40, 5
    groups = np.full(P, -1, np.int32)
    groups[rng.choice(P, 30, replace=False)] = 0
    groups[rng.choice(np.nonzero(groups < 0)[0], 3, replace=False)] = 1     # smaller than m
    for step in range(4):
        smp = R.kinematic_sample_set(9, 2, step, P, k, groups, m)
        h = R.sample_hash(9, 2, step, np.arange(P, dtype=np.uint64))
        order = sorted(range(P), key=lambda p: (int(h[p]), p))
        base = sorted(order[:k])
        assert list(smp[:k]) == base
        assert len(set(smp.tolist())) == len(smp)
        want = set(base)
        for g in (0, 1):
            members = [p for p in order if groups[p] == g]
            want |= set(members[:m])
            assert sum(groups[smp] == g) >= min(m, len(members))
        assert set(smp.tolist()) == want


@pytest.mark.parametrize("quadrature", ["lagrangian", "eulerian"])
def test_kinematic_trial_velocities_and_translation(quadrature):
    """Kinematic samples take their prescribed velocity; with a translation decoder and every group
    moving at the body's velocity the reduced step follows the translation exactly, with either
    quadrature."""
    sc = S.clamped_bar_2d(side=16, top_velocity=(0.0, 0.0))
    v0 = np.array([0.2, -0.1])
    sc.kin_vel = np.array([v0, v0])
    sc.v = np.broadcast_to(v0, sc.x.shape).copy()
    X = sc.x.copy()
    dec = _translation_decoder(2, X.min(0), X.max(0) - X.min(0))
    rs = R.RomScene(X=X, mass=sc.p_mass, vol=sc.p_vol, E=float(sc.E[0]), nu=float(sc.nu[0]), dx=sc.dx,
                    dt=sc.dt, n_grid=sc.n_grid, gravity=sc.gravity, bc=sc.bc, bc_width=sc.bc_width,
                    material=sc.material, transfer=sc.transfer, n_samples=12, seed=4,
                    kin_group=sc.kin_group, kin_vel=sc.kin_vel, quadrature=quadrature)
    st = R.RomState(xhat=np.zeros(2), vhat=v0.copy(), xhat_prev=-sc.dt * v0)
    for n in range(5):
        rec = {}
        st = R.rom_step(dec, rs, st, rec)
        g = sc.kin_group[rec["samples"]]
        assert (g == 0).sum() >= 5 and (g == 1).sum() >= 5
        np.testing.assert_allclose(rec["v_trial"][g >= 0], np.broadcast_to(v0, ((g >= 0).sum(), 2)), rtol=0,
                                   atol=0)
    np.testing.assert_allclose(st.xhat, 5 * sc.dt * v0, rtol=1e-12, atol=1e-15)
    # a moving group with another velocity: its samples report it, the rest keep the grid velocity
    vt = np.zeros((3, 2))
    rs.kin_vel = np.array([[0.0, 0.0], [1.0, 2.0]])
    smp = np.array([np.nonzero(sc.kin_group == 1)[0][0], np.nonzero(sc.kin_group == -1)[0][0],
                    np.nonzero(sc.kin_group == 0)[0][0]])
    v, xt = R.prescribe_kinematic(rs, smp, X[smp], vt + 0.5)
    np.testing.assert_array_equal(v, [[1.0, 2.0], [0.5, 0.5], [0.0, 0.0]])
    np.testing.assert_allclose(xt, X[smp] + sc.dt * v, rtol=0, atol=1e-16)
