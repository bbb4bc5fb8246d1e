"""Pins of the FP64 MPM oracle (Algorithm 1) against closed forms, invariants and brute force."""
import itertools
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg

import oracle.mpm as M
import synth.scenes as S


def _piecewise_N(t):
    t = abs(t)
    if t < 0.5:
        return 0.75 - t * t
    if t < 1.5:
        return 0.5 * (1.5 - t) ** 2
    return 0.0


def test_bspline_brute_force_and_moments():
    rng = np.random.default_rng(0)
    dx = 1.0 / 128
    x = rng.uniform(0.1, 0.9, size=500)
    base = M.stencil_base(x[:, None], dx)[:, 0]
    fx = x / dx - base
    w, dw = M.bspline(fx)
    for p in range(50):
        for k in range(3):
            assert w[p, k] == pytest.approx(_piecewise_N(x[p] / dx - (base[p] + k)), abs=1e-15)
            # derivative against central differences of the piecewise definition (in cells)
            h = 1e-6
            fd = (_piecewise_N(x[p] / dx + h - (base[p] + k)) - _piecewise_N(x[p] / dx - h - (base[p] + k))) / (2 * h)
            assert dw[p, k] == pytest.approx(fd, abs=1e-8)
    r = (base[:, None] + np.arange(3)) * dx - x[:, None]
    np.testing.assert_allclose(w.sum(1), 1.0, atol=1e-15)                      # partition of unity
    np.testing.assert_allclose((w * r).sum(1), 0.0, atol=1e-17)               # linear reproduction
    np.testing.assert_allclose((w * r * r).sum(1), dx * dx / 4, rtol=1e-12)   # MLS moment D = dx^2/4
    np.testing.assert_allclose(dw.sum(1), 0.0, atol=1e-14)                     # sum grad N = 0
    np.testing.assert_allclose((dw * r / dx).sum(1), 1.0, rtol=1e-12)          # sum x_i grad N_i = 1


def test_cell_keys_brute_force_exact():
    rng = np.random.default_rng(1)
    n, dx = 128, 1.0 / 128
    x = rng.uniform(0.05, 0.95, size=(200, 3)).astype(np.float32).astype(np.float64)
    keys = M.cell_keys(x, dx, n)
    for p in range(200):
        b = []
        for k in range(3):
            q = Fraction(float(x[p, k])) * 128 - Fraction(1, 2)
            b.append(q.numerator // q.denominator)
        assert keys[p] == (b[0] * n + b[1]) * n + b[2]
    perm, offs = M.bin_sort(keys, n ** 3)
    assert np.all(np.diff(keys[perm]) >= 0)
    # stability: equal keys keep index order
    same = np.diff(keys[perm]) == 0
    assert np.all(np.diff(perm)[same] > 0)
    assert offs[-1] == 200


def _random_state(rng, P, d, spread=0.1, center=0.5):
    x = center + rng.uniform(-spread, spread, size=(P, d))
    v = rng.uniform(-1, 1, size=(P, d))
    F = S.random_deformation(rng, P, d, 0.2)
    C = rng.uniform(-5, 5, size=(P, d, d))
    return x, v, F, C


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("transfer", [M.MLS, M.PIC])
@pytest.mark.parametrize("material", [M.NEO_HOOKEAN, M.FIXED_COROTATED])
def test_p2g_conserves_mass_momentum_angular(d, transfer, material):
    rng = np.random.default_rng(2 + d)
    n, dx, dt = 32, 1.0 / 32, 1e-4
    P = 300 if d == 2 else 150
    x, v, F, C = _random_state(rng, P, d, 0.2)
    mass, vol = 0.7, 1e-3
    mu, lam = M.lame(1e4, 0.3)
    m, p = M.p2g(x, v, F, C, mass, vol, mu, lam, dx=dx, dt=dt, n_grid=n, material=material, transfer=transfer)
    assert m.sum() == pytest.approx(P * mass, rel=1e-13)
    np.testing.assert_allclose(p.reshape(-1, d).sum(0), mass * v.sum(0), atol=1e-11)
    if transfer != M.MLS:
        return
    xi = np.stack(np.indices(m.shape), -1).reshape(-1, d) * dx
    pi = p.reshape(-1, d)
    if d == 2:
        Lg = np.sum(xi[:, 0] * pi[:, 1] - xi[:, 1] * pi[:, 0])
        Lp = mass * np.sum(x[:, 0] * v[:, 1] - x[:, 1] * v[:, 0] + dx * dx / 4 * (C[:, 1, 0] - C[:, 0, 1]))
        assert Lg == pytest.approx(Lp, rel=1e-11, abs=1e-13)
    else:
        Lg = np.cross(xi, pi).sum(0)
        eps = np.zeros((3, 3, 3))
        for a, b, c in itertools.permutations(range(3)):
            eps[a, b, c] = np.linalg.det(np.eye(3)[[a, b, c]])
        Lp = mass * (np.cross(x, v).sum(0) + dx * dx / 4 * np.einsum("abc,pcb->a", eps, C))
        np.testing.assert_allclose(Lg, Lp, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("transfer", [M.MLS, M.PIC])
def test_rigid_rotation_reproduced(d, transfer):
    rng = np.random.default_rng(7)
    n, dx, dt = 32, 1.0 / 32, 1e-3
    P = 200
    x = 0.5 + rng.uniform(-0.15, 0.15, size=(P, d))
    A = rng.normal(size=(d, d))
    W = A - A.T
    c = rng.normal(size=d)
    v = c + x @ W.T
    F = np.broadcast_to(np.eye(d), (P, d, d)).copy()
    C = np.broadcast_to(W, (P, d, d)).copy() if transfer == M.MLS else np.zeros((P, d, d))
    mu, lam = M.lame(1e4, 0.3)
    m, p = M.p2g(x, v, F, C, 1.0, 1e-3, mu, lam, dx=dx, dt=dt, n_grid=n, material=M.FIXED_COROTATED, transfer=transfer)
    vg = M.grid_update(m, p, dt=dt, gravity=np.zeros(3), bc=M.BC_STICKY, bc_width=0)
    if transfer == M.PIC:
        # PIC grid velocity is a smoothed field; check the gradient transfer on an exactly linear grid field
        xi = np.stack(np.indices(m.shape), -1) * dx
        vg = c + xi @ W.T
    xn, vn, Fn, Cn = M.g2p(x, F, vg, dx=dx, dt=dt, transfer=transfer)
    np.testing.assert_allclose(vn, v, atol=1e-12)
    if transfer == M.MLS:
        np.testing.assert_allclose(Cn, C, atol=1e-10)
    np.testing.assert_allclose(Fn, np.broadcast_to(np.eye(d) + dt * W, Fn.shape), atol=1e-12)
    np.testing.assert_allclose(xn, x + dt * v, atol=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
def test_free_fall_closed_form(dim):
    s = S.block_2d(side=8) if dim == 2 else S.cube_3d(side=6, jitter=0.0, bottom=0.4)
    s.v[:] = 0.3
    x0, v0 = s.x.copy(), s.v.copy()
    g = s.gravity[:dim]
    n = 25
    M.step(s, n)
    expect = x0 + n * s.dt * v0 + s.dt ** 2 * g * n * (n + 1) / 2
    np.testing.assert_allclose(s.x, expect, atol=1e-13)
    np.testing.assert_allclose(s.v, v0 + n * s.dt * g, atol=1e-12)
    np.testing.assert_allclose(s.F, np.broadcast_to(np.eye(dim), s.F.shape), atol=1e-12)


@pytest.mark.parametrize("material", [M.NEO_HOOKEAN, M.FIXED_COROTATED])
def test_rest_state_does_not_move(material):
    s = S.block_2d(side=8)
    s.material = material
    s.v[:] = 0.0
    s.gravity[:] = 0.0
    x0 = s.x.copy()
    M.step(s, 10)
    np.testing.assert_array_equal(s.x, x0)
    assert np.abs(s.v).max() == 0.0
    F = np.broadcast_to(np.eye(3), (4, 3, 3))
    assert np.abs(M.pk1(F, material, 10.0, 20.0)).max() < 1e-12


def _rot(rng, d):
    Q, _ = np.linalg.qr(rng.normal(size=(d, d)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    return Q


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("material", [M.NEO_HOOKEAN, M.FIXED_COROTATED])
def test_stress_closed_form_fd_invariance(d, material):
    rng = np.random.default_rng(11 + d)
    mu, lam = M.lame(1e4, 0.3)
    # closed form at F = R diag(s)
    R = _rot(rng, d)
    sig = rng.uniform(0.7, 1.4, size=d)
    F = R @ np.diag(sig)
    J = np.prod(sig)
    if material == M.NEO_HOOKEAN:
        diag = mu * (sig - 1 / sig) + lam * np.log(J) / sig
    else:
        diag = 2 * mu * (sig - 1) + lam * (J - 1) * J / sig
    np.testing.assert_allclose(M.pk1(F, material, mu, lam), R @ np.diag(diag), rtol=1e-12, atol=1e-9)
    # P = dPsi/dF by central differences
    for _ in range(3):
        F = S.random_deformation(rng, 1, d, 0.25)[0]
        P = M.pk1(F, material, mu, lam)
        fd = np.zeros_like(F)
        h = 1e-6
        for a in range(d):
            for b in range(d):
                E = np.zeros_like(F)
                E[a, b] = h
                fd[a, b] = (M.energy(F + E, material, mu, lam) - M.energy(F - E, material, mu, lam)) / (2 * h)
        np.testing.assert_allclose(P, fd, rtol=1e-6, atol=1e-4)
        Q = _rot(rng, d)
        np.testing.assert_allclose(M.pk1(Q @ F, material, mu, lam), Q @ P, rtol=1e-10, atol=1e-8)
        tau = M.kirchhoff(F, material, mu, lam)
        np.testing.assert_allclose(tau, tau.T, atol=1e-8)


@pytest.mark.parametrize("d", [2, 3])
def test_polar_against_textbook(d):
    rng = np.random.default_rng(5)
    F = S.random_deformation(rng, 50, d, 0.4)
    R = M.polar_rotation(F)
    for k in range(50):
        Rk, Sk = scipy.linalg.polar(F[k])
        np.testing.assert_allclose(R[k], Rk, atol=1e-12)
        np.testing.assert_allclose(R[k].T @ R[k], np.eye(d), atol=1e-13)
        assert np.linalg.det(R[k]) == pytest.approx(1.0, abs=1e-13)
        Sm = R[k].T @ F[k]
        np.testing.assert_allclose(Sm, Sm.T, atol=1e-13)
        assert np.all(np.linalg.eigvalsh(0.5 * (Sm + Sm.T)) > 0)


def test_walls():
    n = 16
    m = np.ones((n, n, n))
    p = np.ones((n, n, n, 3)) * np.array([0.5, -2.0, 0.25])
    v = M.grid_update(m, p, dt=0.0, gravity=np.zeros(3), bc=M.BC_SLIP_FLOOR, bc_width=3)
    # interior untouched
    np.testing.assert_array_equal(v[5, 5, 5], [0.5, -2.0, 0.25])
    # slip floor: only v_y clamped at >= 0
    np.testing.assert_array_equal(v[5, 1, 5], [0.5, 0.0, 0.25])
    # corner of floor and x wall is sticky
    np.testing.assert_array_equal(v[1, 1, 5], [0.0, 0.0, 0.0])
    # x walls, z walls and the top are sticky
    for idx in [(2, 6, 6), (13, 6, 6), (6, 6, 0), (6, 13, 6)]:
        np.testing.assert_array_equal(v[idx], 0.0)
    np.testing.assert_array_equal(v[12, 12, 12], [0.5, -2.0, 0.25])
    v2 = M.grid_update(m[:, :, 0], p[:, :, 0, :2], dt=0.0, gravity=np.zeros(3), bc=M.BC_STICKY, bc_width=3)
    assert np.abs(v2[:3]).max() == 0 and np.abs(v2[-3:]).max() == 0
    assert np.abs(v2[:, :3]).max() == 0 and np.abs(v2[:, -3:]).max() == 0
    np.testing.assert_array_equal(v2[3:-3, 3:-3], np.broadcast_to([0.5, -2.0], (n - 6, n - 6, 2)))


def _momenta(s, d):
    """Total linear momentum and APIC angular momentum sum_p m (x_p x v_p + (dx^2/4) eps:C_p)."""
    p = (s.p_mass * s.v).sum(0)
    x, v, C = s.x, s.v, s.C
    if d == 2:
        L = s.p_mass * ((x[:, 0] * v[:, 1] - x[:, 1] * v[:, 0]).sum() + s.dx ** 2 / 4 * (C[:, 1, 0] - C[:, 0, 1]).sum())
        return p, np.atleast_1d(L)
    L = s.p_mass * (np.cross(x, v).sum(0) + s.dx ** 2 / 4 * np.stack(
        [C[:, 2, 1] - C[:, 1, 2], C[:, 0, 2] - C[:, 2, 0], C[:, 1, 0] - C[:, 0, 1]], 1).sum(0))
    return p, L


@pytest.mark.parametrize("d", [2, 3])
def test_free_stressed_steps_conserve_momenta(d):
    """No gravity, no wall contact, random velocities and deformation: 20 full MLS steps keep the
    total linear momentum and the APIC angular momentum to round-off (symmetric Kirchhoff stress,
    mass-weighted affine transfer); PIC keeps the linear momentum but not the angular one."""
    for transfer in (M.MLS, M.PIC):
        if d == 2:
            sc = S.block_2d(side=16, dt=5e-5, origin=(0.45, 0.45), E=5e3)
        else:
            sc = S.cube_3d(side=8, n_grid=64, dt=5e-5, bottom=0.45)
        rng = np.random.default_rng(1)
        sc.transfer = transfer
        sc.gravity = np.zeros(3)
        sc.v = 0.3 * rng.normal(size=sc.v.shape)
        sc.F = S.random_deformation(rng, sc.n_particles, d, 0.02)
        sc.C[:] = 0.0
        M.step(sc, 1)   # C becomes the grid-consistent affine velocity
        p0, L0 = _momenta(sc, d)
        M.step(sc, 20)
        p1, L1 = _momenta(sc, d)
        assert np.abs(p1 - p0).max() <= 1e-12 * np.abs(p0).max()
        if transfer == M.MLS:
            assert np.abs(L1 - L0).max() <= 1e-12 * np.abs(L0).max()
        else:
            assert np.abs(L1 - L0).max() > 1e-4 * np.abs(L0).max()


def _rot2(a):
    return np.array([[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]])


def _rot3(rng):
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    return q * np.sign(np.linalg.det(q))


def test_plastic_return_closed_forms():
    """Material 2: singular values clamped to [1 - theta_c, 1 + theta_s], rotations kept."""
    lo, hi = 1 - 2.5e-2, 1 + 7.5e-3
    R1, R2 = _rot2(0.3), _rot2(-1.1)
    F = R1 @ np.diag([1.2, 0.9]) @ R2.T
    out = M.plastic_return(F[None], lo, hi)[0]
    np.testing.assert_allclose(out, R1 @ np.diag([hi, lo]) @ R2.T, rtol=0, atol=1e-14)
    rng = np.random.default_rng(0)
    Q1, Q2 = _rot3(rng), _rot3(rng)
    F3 = Q1 @ np.diag([1.02, 0.99, 0.95]) @ Q2.T
    out3 = M.plastic_return(F3[None], lo, hi)[0]
    np.testing.assert_allclose(out3, Q1 @ np.diag([hi, 0.99, lo]) @ Q2.T, rtol=0, atol=1e-14)
    # inside the bounds: unchanged, bit for bit
    Fe = Q1 @ np.diag([1.005, 0.99, 0.98]) @ Q2.T
    assert np.array_equal(M.plastic_return(Fe[None], lo, hi)[0], Fe)


def test_plastic_return_invariants():
    rng = np.random.default_rng(1)
    lo, hi = 0.9, 1.05
    F = np.eye(3)[None] + 0.2 * rng.normal(size=(200, 3, 3))
    F = F[np.linalg.det(F) > 0.2]
    out = M.plastic_return(F, lo, hi)
    s = np.linalg.svd(out, compute_uv=False)
    assert s.min() >= lo - 1e-12 and s.max() <= hi + 1e-12
    np.testing.assert_allclose(M.polar_rotation(out), M.polar_rotation(F), rtol=0, atol=1e-12)
    np.testing.assert_allclose(M.plastic_return(out, lo, hi), out, rtol=0, atol=1e-13)


def test_plastic_material_with_wide_bounds_is_the_elastic_material():
    sc = S.block_2d(side=8, dt=5e-5)
    rng = np.random.default_rng(2)
    sc.F = S.random_deformation(rng, sc.n_particles, 2, 0.05)
    sc.material = M.FIXED_COROTATED
    a = sc.copy()
    b = sc.copy()
    b.material = M.FIXED_COROTATED_PLASTIC
    b.theta_c, b.theta_s = 0.9, 10.0
    M.step(a, 5)
    M.step(b, 5)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.F, b.F)
    # with the snow bounds the same motion yields plastically: the singular values stay inside
    c = sc.copy()
    c.material = M.FIXED_COROTATED_PLASTIC
    M.step(c, 5)
    s = np.linalg.svd(c.F, compute_uv=False)
    assert s.max() <= 1 + c.theta_s + 1e-12 and s.min() >= 1 - c.theta_c - 1e-12
    assert not np.allclose(c.F, a.F)


def test_kinematic_particles_follow_their_prescribed_motion():
    """Dirichlet particles: the held group stays in place, the moving group translates at its
    velocity exactly, the free particles are pulled along; with every group id -1 the step is the
    plain one."""
    sc = S.clamped_bar_2d(side=16)
    a = sc.copy()
    n = 30
    M.step(a, n)
    g = sc.kin_group
    assert np.array_equal(a.x[g == 0], sc.x[g == 0])
    np.testing.assert_allclose(a.x[g == 1], sc.x[g == 1] + n * sc.dt * sc.kin_vel[1], rtol=0, atol=1e-14)
    assert np.all(a.C[g >= 0] == 0) and np.all(a.v[g == 1] == sc.kin_vel[1])
    assert np.abs(a.v[g == -1]).max() > 0.05          # the free particles are dragged
    b = sc.copy()
    b.kin_group = np.full(sc.n_particles, -1, np.int32)
    c = sc.copy()
    c.kin_group, c.kin_vel = None, None
    M.step(b, 5)
    M.step(c, 5)
    assert np.array_equal(b.x, c.x) and np.array_equal(b.F, c.F)


def test_p2g_conservation_over_random_clouds():
    """The mass, linear-momentum and (MLS) angular-momentum identities of the transfer, over
    randomly drawn clouds, dimensions, transfers and materials (property-based)."""
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")

    @hyp.settings(max_examples=30, deadline=None, derandomize=True)
    @hyp.given(seed=st.integers(0, 2 ** 31 - 1), d=st.sampled_from([2, 3]),
               transfer=st.sampled_from([M.MLS, M.PIC]), material=st.sampled_from([M.NEO_HOOKEAN, M.FIXED_COROTATED]),
               P=st.integers(1, 60), spread=st.floats(0.0, 0.3))
    def check(seed, d, transfer, material, P, spread):
        rng = np.random.default_rng(seed)
        n, dx, dt = 32, 1.0 / 32, 1e-4
        x, v, F, C = _random_state(rng, P, d, spread)
        mass, vol = float(rng.uniform(0.1, 2.0)), 1e-3
        mu, lam = M.lame(float(rng.uniform(1e3, 5e4)), 0.3)
        m, p = M.p2g(x, v, F, C, mass, vol, mu, lam, dx=dx, dt=dt, n_grid=n, material=material, transfer=transfer)
        assert m.sum() == pytest.approx(P * mass, rel=1e-12)
        np.testing.assert_allclose(p.reshape(-1, d).sum(0), mass * v.sum(0), rtol=1e-10, atol=1e-10)
        if transfer == M.MLS:
            xi = np.stack(np.indices(m.shape), -1).reshape(-1, d) * dx
            pi = p.reshape(-1, d)
            if d == 2:
                Lg = np.sum(xi[:, 0] * pi[:, 1] - xi[:, 1] * pi[:, 0])
                Lp = mass * np.sum(x[:, 0] * v[:, 1] - x[:, 1] * v[:, 0] + dx * dx / 4 * (C[:, 1, 0] - C[:, 0, 1]))
                assert Lg == pytest.approx(Lp, rel=1e-10, abs=1e-11)
            else:
                eps = np.zeros((3, 3, 3))
                for a, b, c in itertools.permutations(range(3)):
                    eps[a, b, c] = np.linalg.det(np.eye(3)[[a, b, c]])
                Lp = mass * (np.cross(x, v).sum(0) + dx * dx / 4 * np.einsum("abc,pcb->a", eps, C))
                np.testing.assert_allclose(np.cross(xi, pi).sum(0), Lp, rtol=1e-10, atol=1e-11)

    check()
