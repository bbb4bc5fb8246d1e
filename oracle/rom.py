"""FP64 oracle of the reduced-order step (Algorithms 2, 3, 5, 6, 7).  Test infrastructure only.

Algorithm 2: (1) full-space kinematics at quadrature points (Algorithm 3,
Lagrangian quadrature), (2) full-space dynamics of the sample material points
(Algorithm 5), (3) reduced-space dynamics by projection (Algorithm 6,
position-velocity, or Algorithm 7, velocity-only).

Algorithm 3: x_n^p = g(X^p; xhat_n) for the samples; the basis set I is every
node whose basis function is non-zero at a sample; the neighbour set N holds
every other material point with a non-zero basis function in I; at P u N the
deformation gradient is dg/dX and the velocity (dg/dxhat) vhat_n; quadrature
masses are the particle masses.

Algorithm 5: particle-to-grid from the quadrature points onto I (no affine
velocity term), the grid update of Algorithm 1 on I, grid-to-particle to the
samples only: v_trial, x_trial = x_n + dt v_trial.  F is not evolved (it comes
from the decoder, Remark in Section 3.2.3).

Algorithm 6: vhat_{n+1} = argmin sum_P |(dg/dxhat)(X^p; xhat_n) vhat - v_trial|^2;
xhat_{n+1} = argmin sum_P |g(X^p; xhat) - x_trial|^2 by Gauss-Newton with
backtracking, initial guess 2 xhat_n - xhat_{n-1} (Section 5).
Algorithm 7: vhat_{n+1} as above, xhat_{n+1} = xhat_n + dt vhat_{n+1}.

Readings where the paper is silent (listed in the design notes):
  * sampling: uniform without replacement, re-drawn every step (Section 3.2.1),
    as the k particles with the smallest 64-bit hash h(seed, instance, step, p),
    ties broken by p; h chains three SplitMix64 outputs (Steele, Lea and Flood
    2014): h = out(out(out(seed, instance), step), p) where out(s, k) is the
    (k+1)-th output of the SplitMix64 generator seeded with s;
  * stencil membership (integer) decides "N_i != 0" (equal except on the
    zero-weight support boundary);
  * Gauss-Newton: a fixed number of iterations (3); the step solves the
    linearised least-squares problem; Armijo backtracking with c = 1e-4 and
    step halving, at most 10 halvings; if no trial decreases the objective the
    iterate is kept and the ``no_decrease`` flag is raised;
  * at the first step xhat_{-1} = xhat_0 - dt vhat_0;
  * optional reference gradient (f_reference): the quadrature points' stress
    uses F = (dg/dX)(X; xhat_n) [(dg/dX)(X; xhat_ref)]^-1 with xhat_ref the
    fitted initial latent state (for initial states with F = I), so that the
    decoder's error in representing the undeformed body is not a strain;
  * quadrature-point affine velocity (MLS transfer only): Algorithm 5 gives the
    quadrature points C = 0, which matches the paper's PIC full-order model;
    with the MLS/APIC full-order model the option ``affine = "decoded"`` gives
    them the affine velocity of the decoded motion, C = (dv/dX) (dg/dX)^-1 with
    v = (dg/dxhat) vhat, the state an APIC particle of that motion carries;
  * optional ridge rho: the projections then solve min |J a - b|^2 +
    rho (tr(J^T J) / r) |a|^2 (Tikhonov regularisation of the least-squares
    problems for latent Jacobians with near-null directions; rho = 0 is the
    paper's plain least squares), where a is the increment of the unknown
    from its prior: the Gauss-Newton step from the current iterate
    (Levenberg-Marquardt damping) and, for the velocity, the change from
    vhat_n (a penalty on vhat itself would pull the latent velocity to zero
    and damp the motion);
  * initial latent state by the least-squares fit of Eq. essentialSpecInt over
    all particles (Gauss-Newton from zero, then a linear least-squares fit of
    the initial velocity).

Pins (tests/test_oracle_rom.py): SplitMix64 known answers, bottom-k against a
full sort, sampling uniformity, neighbour sets against brute-force
enumeration, exact reproduction of the full-order free fall with a hand-set
linear decoder g = X + xhat, Gauss-Newton against a QR least-squares solve for
a linear decoder, O(dt^2) agreement of the two projections (Appendix A), the
error metric on a hand-computed toy.
"""
from __future__ import annotations

import dataclasses
import itertools

import numpy as np

from . import decoder as D
from . import mpm as M

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_out(state, k):
    """(k+1)-th output of SplitMix64 seeded with ``state`` (uint64 arrays, wrapping)."""
    with np.errstate(over="ignore"):
        z = np.asarray(state, np.uint64) + GOLDEN * (np.asarray(k, np.uint64) + np.uint64(1))
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def sample_hash(seed, inst, step, p):
    s = splitmix64_out(np.uint64(seed), np.uint64(inst))
    s = splitmix64_out(s, np.uint64(step))
    return splitmix64_out(s, np.asarray(p, np.uint64))


def sample_set(seed, inst, step, n_particles, k):
    """Indices of the k particles with the smallest hash (ties by index), ascending."""
    h = sample_hash(seed, inst, step, np.arange(n_particles, dtype=np.uint64))
    order = np.lexsort((np.arange(n_particles), h))
    return np.sort(order[:k])


def stencil_nodes(x, dx, n_grid):
    """Linear node ids (n, 3^d) of the quadratic stencils at positions x."""
    d = x.shape[1]
    base = M.stencil_base(x, dx)
    out = []
    for off in M.stencil_offsets(d):
        node = base + np.array(off)
        lin = np.zeros(len(x), np.int64)
        for k in range(d):
            lin = lin * n_grid + node[:, k]
        out.append(lin)
    return np.stack(out, axis=1)


def kinematic_sample_set(seed, inst, step, n_particles, k, groups, m_kin):
    """Sample set with kinematic boundaries (Section 3.2.1: their material points are included;
    Section 5: at least 5 per boundary).  The k particles with the smallest hash (ascending), then,
    for each kinematic group g in order, those of its min(m_kin, |g|) particles of smallest (hash,
    id) that are not already drawn (ascending)."""
    base = sample_set(seed, inst, step, n_particles, k)
    h = sample_hash(seed, inst, step, np.arange(n_particles, dtype=np.uint64))
    taken = np.zeros(n_particles, bool)
    taken[base] = True
    parts = [base]
    groups = np.asarray(groups)
    for g in range(int(groups.max()) + 1 if groups.size else 0):
        ids = np.nonzero(groups == g)[0]
        first = ids[np.lexsort((ids, h[ids]))][:m_kin]
        extra = np.sort(first[~taken[first]])
        taken[extra] = True
        parts.append(extra)
    return np.concatenate(parts).astype(np.int64)


def prescribe_kinematic(rs, samples, x_samples, v_trial):
    """Trial state of kinematic samples: their prescribed velocity (the Dirichlet condition enforced
    in the full-space update, Section 3.2.1)."""
    if rs.kin_group is None:
        return v_trial, x_samples + rs.dt * v_trial
    g = np.asarray(rs.kin_group)[samples]
    m = g >= 0
    v = v_trial.copy()
    v[m] = np.asarray(rs.kin_vel, np.float64)[g[m]]
    return v, x_samples + rs.dt * v


def neighbourhood(x_all, samples, dx, n_grid):
    """Algorithm 3 sets: basis set I (sorted node ids) and neighbour set N (sorted particle ids)."""
    nodes = stencil_nodes(x_all, dx, n_grid)
    basis = np.unique(nodes[samples])
    hit = np.isin(nodes, basis).any(axis=1)
    hit[samples] = False
    return basis, np.nonzero(hit)[0]


# ----------------------------------------------------------- Eulerian quadrature (Algorithm 4)


def eulerian_cells(basis, d, n_grid):
    """Grid cells whose quadrature points can reach a node of the basis set I: a point in cell c
    has stencil base c - 1 or c, so its stencil covers nodes c - 1 .. c + 2; node i is reached from
    cells i - 2 .. i + 1 along every axis.  Sorted linear cell ids (cell c = lower corner node c),
    clipped to cells whose stencils stay in the grid."""
    nodes = np.array(basis, np.int64)
    coords = np.stack(np.unravel_index(nodes, (n_grid,) * d), axis=1)
    cells = set()
    for off in itertools.product(range(-2, 2), repeat=d):
        c = coords + np.array(off)
        ok = np.all((c >= 1) & (c <= n_grid - 3), axis=1)
        cells.update(np.ravel_multi_index(tuple(c[ok].T), (n_grid,) * d).tolist())
    return np.array(sorted(cells), np.int64)


def eulerian_points(cells, d, n_grid, dx, ell):
    """ell^d evenly spaced quadrature points per cell, (c + (q + 1/2) / ell) dx, each with volume
    (dx / ell)^d (Section 3.2.2); ordered by cell, then q lexicographically."""
    coords = np.stack(np.unravel_index(cells, (n_grid,) * d), axis=1).astype(np.float64)
    offs = (np.array(list(itertools.product(range(ell), repeat=d)), np.float64) + 0.5) / ell
    pts = (coords[:, None, :] + offs[None, :, :]) * dx
    return pts.reshape(-1, d), (dx / ell) ** d


def invert_decoder(dec, x, xhat, X0, iters):
    """Newton's method on g(X; xhat) = x (Section 3.2.2): X <- X - (dg/dX)^-1 (g(X) - x).
    Returns X and the final residual norms."""
    X = np.array(X0, np.float64)
    for _ in range(iters):
        g, FX, _ = D.jacobians(dec, X, xhat)
        X = X - np.linalg.solve(FX, (g - x)[..., None])[..., 0]
    g = D.decode(dec, X, xhat)
    return X, np.linalg.norm(g - x, axis=1)


def reference_occupancy(X, h):
    """The reference domain as the union of the particles' volume boxes (side h = V0^(1/d), centred
    on the reference positions): returns (origin, shape, occupied flags) of a box grid of spacing
    h whose cell k holds particle positions in [origin + k h, origin + (k + 1) h)."""
    origin = X.min(0) - 0.5 * h
    idx = np.floor((X - origin) / h).astype(np.int64)
    shape = tuple(idx.max(0) + 1)
    occ = np.zeros(shape, bool)
    occ[tuple(idx.T)] = True
    return origin, shape, occ


def inside_reference(Xq, origin, h, shape, occ):
    idx = np.floor((Xq - origin) / h).astype(np.int64)
    ok = np.all((idx >= 0) & (idx < np.array(shape)), axis=1)
    out = np.zeros(len(Xq), bool)
    out[ok] = occ[tuple(idx[ok].T)]
    return out


@dataclasses.dataclass
class RomScene:
    """Static data of one reduced-order instance."""
    X: np.ndarray            # (P, d) reference positions
    mass: float
    vol: float
    E: float
    nu: float
    dx: float
    dt: float
    n_grid: int
    gravity: np.ndarray
    bc: int
    bc_width: int
    material: int
    transfer: int
    n_samples: int
    seed: int
    inst: int = 0
    gn_iters: int = 3
    armijo_c: float = 1e-4
    max_halvings: int = 10
    projection: str = "position-velocity"   # or "velocity-only"
    ridge: float = 0.0                       # rho of the regularised projections
    affine: str = "zero"                     # quadrature-point C: "zero" or "decoded"
    F_ref_inv: np.ndarray | None = None      # (P, d, d) inverse reference gradients (f_reference option)
    quadrature: str = "lagrangian"           # or "eulerian" (Algorithm 4)
    ell: int = 2                             # Eulerian quadrature points per cell per dimension
    newton_iters: int = 4                    # decoder inversion iterations
    newton_tol: float = 1e-3                 # converged: final residual below newton_tol * dx
    kin_group: np.ndarray | None = None      # kinematic group per particle (-1: free)
    kin_vel: np.ndarray | None = None        # prescribed velocity per group (n_groups, d)
    kin_min_samples: int = 5                 # samples forced from each kinematic group


@dataclasses.dataclass
class RomState:
    xhat: np.ndarray
    vhat: np.ndarray
    xhat_prev: np.ndarray
    step: int = 0
    no_decrease: bool = False


def local_dynamics(dec, rs: RomScene, xhat, vhat, samples, x_all):
    """Algorithms 3 and 5: trial velocities and positions of the samples.

    Returns (v_trial, x_trial, basis, neighbours).
    """
    basis, neigh = neighbourhood(x_all, samples, rs.dx, rs.n_grid)
    quad = np.concatenate([samples, neigh])
    _, FX, _ = D.jacobians(dec, rs.X[quad], xhat)
    vq, dvdX = D.velocity_gradient(dec, rs.X[quad], xhat, vhat)
    xq = x_all[quad]
    d = xq.shape[1]
    if rs.affine == "decoded" and rs.transfer == M.MLS:
        # affine velocity of the decoded motion: C = (dv/dX) F^-1
        Cq = np.einsum("pik,pkj->pij", dvdX, np.linalg.inv(FX))
    else:
        Cq = np.zeros((len(quad), d, d))
    # stress from the gradient measured against the decoded reference configuration (option)
    Fs = FX if rs.F_ref_inv is None else np.einsum("pik,pkj->pij", FX, rs.F_ref_inv[quad])
    mu, lam = M.lame(rs.E, rs.nu)
    m, p = M.p2g(xq, vq, Fs, Cq, rs.mass, rs.vol, mu, lam, dx=rs.dx,
                 dt=rs.dt, n_grid=rs.n_grid, material=rs.material, transfer=rs.transfer)
    vg = M.grid_update(m, p, dt=rs.dt, gravity=rs.gravity, bc=rs.bc, bc_width=rs.bc_width)
    xs = x_all[samples]
    base = M.stencil_base(xs, rs.dx)
    w, _ = M.bspline(xs / rs.dx - base)
    v_trial = np.zeros((len(samples), d))
    for off in M.stencil_offsets(d):
        node = base + np.array(off)
        weight = np.ones(len(samples))
        for k in range(d):
            weight = weight * w[:, k, off[k]]
        v_trial += weight[:, None] * vg[tuple(node[:, k] for k in range(d))]
    v_trial, x_trial = prescribe_kinematic(rs, samples, xs, v_trial)
    return v_trial, x_trial, basis, neigh


def reference_inverse(dec, X, xhat_ref):
    """Inverse gradients [(dg/dX)(X_p; xhat_ref)]^-1 of the decoded reference configuration (the
    f_reference option: F = (dg/dX)(X; xhat_n) G_p, so the decoder's approximation error of the
    undeformed configuration produces no stress)."""
    _, FX, _ = D.jacobians(dec, X, xhat_ref)
    return np.linalg.inv(FX)


def eulerian_quadrature(dec, rs: RomScene, xhat, vhat, samples, x_samples, X_guess=None, inside_override=None):
    """Algorithm 4: quadrature points on the cells around the basis set of the samples, their
    reference positions by inverting the decoder, kinematics there by Eqs. defGrad and timederOne,
    mass rho0 V_q / J.  Points whose reference position is outside the reference domain (or whose
    inversion does not converge) carry no mass.  Returns (basis, cells, points x_q, reference X_q,
    F_q, v_q, mass_q, reference volume V_q / J_q, inside flags).  ``inside_override`` (index array,
    flag array) replaces the inside decision of the listed points (a decision taken elsewhere in
    another precision)."""
    d = rs.X.shape[1]
    nodes = stencil_nodes(x_samples, rs.dx, rs.n_grid)
    basis = np.unique(nodes)
    cells = eulerian_cells(basis, d, rs.n_grid)
    xq, Vq = eulerian_points(cells, d, rs.n_grid, rs.dx, rs.ell)
    if X_guess is None:
        X_guess = xq - (x_samples - rs.X[samples]).mean(0)
    Xq, resid = invert_decoder(dec, xq, xhat, X_guess, rs.newton_iters)
    h = rs.vol ** (1.0 / d)
    origin, shape, occ = reference_occupancy(rs.X, h)
    inside = inside_reference(Xq, origin, h, shape, occ) & (resid < rs.newton_tol * rs.dx)
    if inside_override is not None:
        inside[inside_override[0]] = inside_override[1]
    _, FX, _ = D.jacobians(dec, Xq, xhat)
    _, vq = D.jvp_latent(dec, Xq, xhat, vhat)
    J = np.linalg.det(FX)
    rho0 = rs.mass / rs.vol
    V0 = np.where(inside, Vq / np.where(J > 0, J, 1.0), 0.0)
    return basis, cells, xq, Xq, FX, vq, rho0 * V0, V0, inside


def eulerian_local_dynamics(dec, rs: RomScene, xhat, vhat, samples, x_samples, X_guess=None, inside_override=None):
    """Algorithm 5 with the Eulerian quadrature points of Algorithm 4: P2G from the points inside
    the body onto the basis set, grid update, G2P to the samples.  Returns (v_trial, x_trial, and
    the quadrature data of eulerian_quadrature)."""
    q = eulerian_quadrature(dec, rs, xhat, vhat, samples, x_samples, X_guess, inside_override)
    basis, cells, xq, Xq, FX, vq, mq, V0, inside = q
    d = xq.shape[1]
    mu, lam = M.lame(rs.E, rs.nu)
    sel = inside
    m, p = M.p2g(xq[sel], vq[sel], FX[sel], np.zeros((int(sel.sum()), d, d)), mq[sel], V0[sel], mu, lam,
                 dx=rs.dx, dt=rs.dt, n_grid=rs.n_grid, material=rs.material, transfer=rs.transfer)
    vg = M.grid_update(m, p, dt=rs.dt, gravity=rs.gravity, bc=rs.bc, bc_width=rs.bc_width)
    xs = x_samples
    base = M.stencil_base(xs, rs.dx)
    w, _ = M.bspline(xs / rs.dx - base)
    v_trial = np.zeros((len(samples), d))
    for off in M.stencil_offsets(d):
        node = base + np.array(off)
        weight = np.ones(len(samples))
        for k in range(d):
            weight = weight * w[:, k, off[k]]
        v_trial += weight[:, None] * vg[tuple(node[:, k] for k in range(d))]
    v_trial, x_trial = prescribe_kinematic(rs, samples, xs, v_trial)
    return v_trial, x_trial, q


def lstsq(A, b, ridge=0.0):
    """argmin |A x - b|^2 (+ ridge * tr(A^T A) / n * |x|^2 when ridge > 0)."""
    if ridge > 0:
        M = A.T @ A
        lam = ridge * np.trace(M) / M.shape[0]
        return np.linalg.solve(M + lam * np.eye(M.shape[0]), A.T @ b)
    return np.linalg.lstsq(A, b, rcond=None)[0]


def project_velocity(dec, Xs, xhat_n, v_trial, ridge=0.0, vhat_n=None):
    """Eq. nonlinear_projection:vel / linear_projection: LSQ fit of v_trial by dg/dxhat at xhat_n.
    With ridge > 0 the regularised fit penalises the change of the latent velocity from vhat_n
    (a reading for ill-conditioned latent Jacobians: unresolved directions keep their previous
    velocity instead of being pulled to zero): vhat = vhat_n + argmin |J a - (v_trial - J vhat_n)|^2
    + ridge tr(J^T J)/r |a|^2.  With ridge = 0 this is the plain fit."""
    _, _, Jq = D.jacobians(dec, Xs, xhat_n)
    J = Jq.reshape(-1, dec.r)
    if vhat_n is None:
        vhat_n = np.zeros(dec.r)
    return vhat_n + lstsq(J, v_trial.reshape(-1) - J @ vhat_n, ridge)


def gauss_newton(dec, Xs, x_trial, xhat0, iters, c=1e-4, max_halvings=10, ridge=0.0, steps=None, record=None):
    """Eq. nonlinear_projection:pos by Gauss-Newton with backtracking; returns (xhat, no_decrease).
    With ridge > 0 every step solves the ridge-regularised linearised problem.

    Backtracking tries alpha = 1, 1/2, ... and takes the first alpha with sufficient decrease,
    ||r(xhat + alpha delta)||^2 <= f0 + c alpha slope.  With `steps` (one entry per iteration: the
    m of the step 2^-m to take, or -1 for none) that choice is given instead of searched for, so
    that a run whose choices were made at a different precision can be replayed.  `record`, a list,
    receives per iteration a dict with f0, slope and f: the objective at every trial 2^-m, m = 0 ..
    max_halvings (evaluated only when record is given)."""
    xh = np.array(xhat0, np.float64)
    flag = False
    target = x_trial.reshape(-1)
    for it in range(iters):
        g, _, Jq = D.jacobians(dec, Xs, xh)
        res = g.reshape(-1) - target
        J = Jq.reshape(-1, dec.r)
        delta = lstsq(J, -res, ridge)
        f0 = res @ res
        slope = 2.0 * res @ (J @ delta)

        def objective(m):
            r1 = D.decode(dec, Xs, xh + 0.5 ** m * delta).reshape(-1) - target
            return r1 @ r1

        if record is not None:
            record.append(dict(f0=f0, slope=slope, f=np.array([objective(m) for m in range(max_halvings + 1)])))
        if steps is not None:
            pick = int(steps[it])
        else:
            pick = -1
            for m in range(max_halvings + 1):
                if objective(m) <= f0 + c * 0.5 ** m * slope:
                    pick = m
                    break
        if pick >= 0:
            xh = xh + 0.5 ** pick * delta
        elif np.linalg.norm(delta) > 1e-10 * (1.0 + np.linalg.norm(xh)):
            flag = True
    return xh, flag


def rom_step(dec, rs: RomScene, st: RomState, record=None):
    """Algorithm 2 with Lagrangian quadrature; returns the new RomState."""
    P = len(rs.X)
    if rs.kin_group is None:
        samples = sample_set(rs.seed, rs.inst, st.step, P, rs.n_samples)
    else:
        samples = kinematic_sample_set(rs.seed, rs.inst, st.step, P, min(rs.n_samples, P), rs.kin_group,
                                       rs.kin_min_samples)
    if rs.quadrature == "eulerian":
        x_all = None
        x_s = D.decode(dec, rs.X[samples], st.xhat)
        v_trial, x_trial, q = eulerian_local_dynamics(dec, rs, st.xhat, st.vhat, samples, x_s)
        basis, neigh = q[0], np.zeros(0, np.int64)
    else:
        x_all = D.decode(dec, rs.X, st.xhat)
        v_trial, x_trial, basis, neigh = local_dynamics(dec, rs, st.xhat, st.vhat, samples, x_all)
    Xs = rs.X[samples]
    vhat_new = project_velocity(dec, Xs, st.xhat, v_trial, rs.ridge, st.vhat)
    if rs.projection == "velocity-only":
        xhat_new, flag = st.xhat + rs.dt * vhat_new, False
    else:
        guess = 2.0 * st.xhat - st.xhat_prev
        xhat_new, flag = gauss_newton(dec, Xs, x_trial, guess, rs.gn_iters, rs.armijo_c, rs.max_halvings,
                                      rs.ridge)
    if record is not None:
        record.update(samples=samples, basis=basis, neigh=neigh, x_all=x_all, v_trial=v_trial,
                      x_trial=x_trial)
    return RomState(xhat=xhat_new, vhat=vhat_new, xhat_prev=st.xhat.copy(), step=st.step + 1,
                    no_decrease=st.no_decrease or flag)


def rom_init(dec, X, V0, dt, xhat_guess=None, iters=30):
    """Eq. essentialSpecInt: least-squares fit of xhat_0 (to X) and vhat_0 (to V0) over all particles."""
    xh = np.zeros(dec.r) if xhat_guess is None else np.array(xhat_guess, np.float64)
    for _ in range(iters):
        g, _, Jq = D.jacobians(dec, X, xh)
        res = (g - X).reshape(-1)
        J = Jq.reshape(-1, dec.r)
        delta = lstsq(J, -res)
        f0 = res @ res
        alpha = 1.0
        for _h in range(20):
            r1 = (D.decode(dec, X, xh + alpha * delta) - X).reshape(-1)
            if r1 @ r1 <= f0 + 1e-4 * alpha * 2.0 * res @ (J @ delta):
                break
            alpha *= 0.5
        xh = xh + alpha * delta
        if np.linalg.norm(alpha * delta) < 1e-13 * (1 + np.linalg.norm(xh)):
            break
    _, _, Jq = D.jacobians(dec, X, xh)
    vh = lstsq(Jq.reshape(-1, dec.r), np.broadcast_to(V0, X.shape).reshape(-1))
    return RomState(xhat=xh, vhat=vh, xhat_prev=xh - dt * vh, step=0)


class PositionError:
    """Accumulated position error of Section 5 (in percent)."""

    def __init__(self):
        self.num = 0.0
        self.den = 0.0

    def add(self, x_rom, x_fom):
        self.num += float(np.sum((np.asarray(x_rom) - np.asarray(x_fom)) ** 2))
        self.den += float(np.sum(np.asarray(x_fom) ** 2))

    def percent(self):
        return 100.0 * np.sqrt(self.num) / np.sqrt(self.den)
