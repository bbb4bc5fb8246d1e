"""FP64 oracle of the explicit MPM step (Algorithm 1, Section 2.2).  Test infrastructure only.

Algorithm 1 of the paper, one symplectic-Euler step:
  1. particle to grid: m_i = sum_p N_i(x_p) m_p, (m v)_i = sum_p N_i m_p v_p,
     f_i = -sum_p V0_p tau_p grad N_i(x_p) (tau = J sigma = P F^T, Section 2.1
     footnote: J rho = rho0 so (J / rho0) sigma m_p = V0 tau), f^e_i = m_i g;
  2. grid update: v_i <- v_i + dt (f_i + f^e_i) / m_i, lumped mass (Eq. spaceDiscTwo);
  3. grid to particle: v_p = sum_i N_i v_i, F_p <- (1 + dt sum_i v_i (x) grad N_i) F_p;
  4. advection: x_p <- x_p + dt v_p.

Readings where the paper is silent (each listed in the design notes):
  * basis: quadratic B-splines on a uniform grid of spacing dx, nodes x_i = i dx,
    stencil base = floor(x / dx - 0.5), nodes base + {0, 1, 2}^d;
  * transfer: MLS-MPM with APIC affine velocity C_p (default) or the literal
    PIC form of Algorithm 1 with exact basis gradients (``transfer = PIC``);
    in MLS mode the basis gradient is replaced by its moving-least-squares
    counterpart (4 / dx^2) N_i (x_i - x_p) and F is updated with C_p;
  * constitutive laws: neo-Hookean and fixed-corotated (Stomakhin et al. 2012,
    the paper's material), Lame parameters from (E, nu); a plastic variant of
    the fixed-corotated material (material 2: after the F update the singular
    values are clamped to [1 - theta_c, 1 + theta_s], Stomakhin et al. 2013
    without hardening) for plastic bodies, which the reduced model does not
    cover;
  * the internal force enters the grid momentum as dt f_i (same arithmetic as
    the grid update of Algorithm 1, summed before the division by m_i);
  * boundaries: nodes with any index < w or > n - 1 - w are wall nodes; sticky
    walls zero the velocity; the slip floor clamps v_y >= 0 on the low-y band
    and leaves the other walls sticky;
  * nodes with m_i == 0 get zero velocity;
  * kinematic (Dirichlet) particles of group g take the prescribed velocity v_g after the grid
    to particle transfer, move with it and carry C = 0 (their F follows the grid).

Pins (tests/test_oracle_mpm.py): partition of unity and linear reproduction of
the weights, brute-force piecewise basis, exact mass and linear-momentum
transfer, zero net internal force, angular-momentum transfer identity of APIC,
exact rigid translation / rotation reproduction, symplectic free fall in closed
form, zero stress at rest, stress against finite differences of the energy,
rotation invariance, polar factor against a textbook routine.
"""
from __future__ import annotations

import itertools
import numpy as np

MLS, PIC = 0, 1
NEO_HOOKEAN, FIXED_COROTATED, FIXED_COROTATED_PLASTIC = 0, 1, 2
BC_STICKY, BC_SLIP_FLOOR = 0, 1


# ----------------------------------------------------------------------------- basis


def stencil_base(x: np.ndarray, dx: float) -> np.ndarray:
    """Lowest stencil node per axis: floor(x / dx - 0.5), integer."""
    return np.floor(x / dx - 0.5).astype(np.int64)


def bspline(fx: np.ndarray):
    """Quadratic B-spline weights of the 3 stencil nodes and their derivatives.

    ``fx = x / dx - base`` lies in [0.5, 1.5).  Node k sits at distance
    t = fx - k (in cells) and N(t) = 3/4 - t^2 for |t| < 1/2,
    (3/2 - |t|)^2 / 2 for 1/2 <= |t| < 3/2, 0 beyond.  Returns ``w[..., k]``
    and ``dw[..., k] = dN/dx * dx`` (derivative with respect to x_p in cells).
    """
    w = np.stack([0.5 * (1.5 - fx) ** 2, 0.75 - (fx - 1.0) ** 2, 0.5 * (fx - 0.5) ** 2], axis=-1)
    dw = np.stack([fx - 1.5, -2.0 * (fx - 1.0), fx - 0.5], axis=-1)
    return w, dw


def stencil_offsets(d: int):
    return list(itertools.product(range(3), repeat=d))


def cell_keys(x: np.ndarray, dx: float, n_grid: int) -> np.ndarray:
    """Linear index of the stencil base node, first axis slowest (row-major)."""
    base = stencil_base(x, dx)
    key = np.zeros(len(x), np.int64)
    for k in range(x.shape[1]):
        key = key * n_grid + base[:, k]
    return key


def bin_sort(keys: np.ndarray, n_keys: int):
    """Stable counting sort of particle indices by key; returns (perm, offsets)."""
    perm = np.argsort(keys, kind="stable")
    counts = np.bincount(keys, minlength=n_keys)
    offsets = np.concatenate([[0], np.cumsum(counts)])
    return perm, offsets


# ----------------------------------------------------------------------- constitutive


def lame(E, nu):
    mu = E / (2.0 * (1.0 + nu))
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    return mu, lam


def polar_rotation(F: np.ndarray) -> np.ndarray:
    """Rotation R of F = R S with det R = +1, from the SVD F = U diag(s) V^T.

    When det U or det V is negative its last column is negated (the sign moves
    to the smallest singular value), so R = U V^T is a proper rotation; for
    det F > 0 this is the polar factor.
    """
    U, s, Vt = np.linalg.svd(F)
    detU = np.linalg.det(U)
    detV = np.linalg.det(Vt)
    U = U.copy()
    Vt = Vt.copy()
    U[..., :, -1] *= np.where(detU < 0, -1.0, 1.0)[..., None]
    Vt[..., -1, :] *= np.where(detV < 0, -1.0, 1.0)[..., None]
    return U @ Vt


def signed_svd(F):
    """F = U diag(s) V^T with U, V proper rotations (det +1): when det U or det V is negative the
    last column is negated and the sign moves to the smallest singular value."""
    U, s, Vt = np.linalg.svd(F)
    detU = np.linalg.det(U)
    detV = np.linalg.det(Vt)
    U, s, Vt = U.copy(), s.copy(), Vt.copy()
    flipU = detU < 0
    flipV = detV < 0
    U[..., :, -1] *= np.where(flipU, -1.0, 1.0)[..., None]
    Vt[..., -1, :] *= np.where(flipV, -1.0, 1.0)[..., None]
    s[..., -1] *= np.where(flipU ^ flipV, -1.0, 1.0)
    return U, s, Vt


def plastic_return(F, lo, hi):
    """Return mapping of the plastic material (material 2): the elastic deformation gradient keeps
    its rotations, its singular values are clamped to [lo, hi] (lo = 1 - theta_c, hi = 1 +
    theta_s), the excess is plastic flow (Stomakhin et al. 2013, without hardening).  Particles
    whose singular values are all inside the bounds keep F unchanged."""
    U, s, Vt = signed_svd(F)
    c = np.clip(s, lo, hi)
    out = np.array(F, np.float64, copy=True)
    moved = np.any(c != s, axis=-1)
    out[moved] = np.einsum("pij,pj,pjk->pik", U[moved], c[moved], Vt[moved])
    return out


def kinematic_override(x, xn, vn, Cn, group, kin_vel, dt):
    """Essential (Dirichlet) boundary of Section 2: particles of kinematic group g (group >= 0) take
    the prescribed velocity kin_vel[g] and move with it, x_{n+1} = x_n + dt v_g, carrying no affine
    velocity (C = 0); F follows the grid like every particle.  Other particles are unchanged."""
    m = np.asarray(group) >= 0
    if not np.any(m):
        return xn, vn, Cn
    xn, vn, Cn = xn.copy(), vn.copy(), Cn.copy()
    vg = np.asarray(kin_vel, np.float64)[np.asarray(group)[m]]
    vn[m] = vg
    xn[m] = x[m] + dt * vg
    Cn[m] = 0.0
    return xn, vn, Cn


def energy(F, material, mu, lam):
    """Strain energy density Psi(F) per unit reference volume."""
    d = F.shape[-1]
    J = np.linalg.det(F)
    if material == NEO_HOOKEAN:
        lnJ = np.log(J)
        return 0.5 * mu * (np.einsum("...ij,...ij->...", F, F) - d) - mu * lnJ + 0.5 * lam * lnJ ** 2
    sig = np.linalg.svd(F, compute_uv=False)
    sig = sig.copy()
    sig[..., -1] *= np.sign(J)
    return mu * np.sum((sig - 1.0) ** 2, axis=-1) + 0.5 * lam * (J - 1.0) ** 2


def pk1(F, material, mu, lam):
    """First Piola-Kirchhoff stress P = dPsi/dF.

    neo-Hookean:      P = mu (F - F^-T) + lam ln(J) F^-T
    fixed-corotated:  P = 2 mu (F - R) + lam (J - 1) J F^-T
    """
    J = np.linalg.det(F)
    FinvT = np.swapaxes(np.linalg.inv(F), -1, -2)
    if material == NEO_HOOKEAN:
        return mu * (F - FinvT) + (lam * np.log(J))[..., None, None] * FinvT
    R = polar_rotation(F)
    return 2.0 * mu * (F - R) + (lam * (J - 1.0) * J)[..., None, None] * FinvT


def kirchhoff(F, material, mu, lam):
    """Kirchhoff stress tau = J sigma = P F^T (Section 2.1: P = J sigma F^-T)."""
    return pk1(F, material, mu, lam) @ np.swapaxes(F, -1, -2)


# -------------------------------------------------------------------------- transfers


def p2g(x, v, F, C, mass, vol, mu, lam, *, dx, dt, n_grid, material, transfer):
    """Particle-to-grid transfer of Algorithm 1 (step 1) for one instance.

    Returns dense grids ``m`` (n^d) and ``p`` (n^d, d) where ``p`` is the grid
    momentum m_i v_i plus the impulse dt f_i of the internal force.  Particles
    whose stencil leaves the grid raise ValueError.
    """
    P, d = x.shape
    base = stencil_base(x, dx)
    if len(x) and (base.min() < 0 or base.max() + 2 >= n_grid):
        raise ValueError("particle stencil outside the grid")
    fx = x / dx - base
    w, dw = bspline(fx)
    tau = kirchhoff(F, material, mu, lam) if P else np.zeros((0, d, d))
    shape = (n_grid,) * d
    m = np.zeros(shape)
    p = np.zeros(shape + (d,))
    # mass and reference volume: one value for all particles, or one per particle
    mass = np.broadcast_to(np.asarray(mass, np.float64), (P,))
    vol = np.broadcast_to(np.asarray(vol, np.float64), (P,))
    if transfer == MLS:
        affine = mass[:, None, None] * C - (dt * 4.0 / dx ** 2) * vol[:, None, None] * tau
    for off in stencil_offsets(d):
        node = base + np.array(off)
        weight = np.ones(P)
        for k in range(d):
            weight = weight * w[:, k, off[k]]
        dpos = node * dx - x
        if transfer == MLS:
            mom = weight[:, None] * (mass[:, None] * v + np.einsum("pij,pj->pi", affine, dpos))
        else:
            grad = np.empty((P, d))
            for a in range(d):
                g = dw[:, a, off[a]] / dx
                for k in range(d):
                    if k != a:
                        g = g * w[:, k, off[k]]
                grad[:, a] = g
            mom = weight[:, None] * mass[:, None] * v - dt * vol[:, None] * np.einsum("pij,pj->pi", tau, grad)
        idx = tuple(node[:, k] for k in range(d))
        np.add.at(m, idx, weight * mass)
        np.add.at(p, idx, mom)
    return m, p


def wall_mask(n_grid: int, d: int, width: int):
    """Per-axis boolean arrays lo[k][i] (i < width) and hi[k][i] (i > n - 1 - width)."""
    i = np.arange(n_grid)
    return i < width, i > n_grid - 1 - width


def grid_update(m, p, *, dt, gravity, bc, bc_width):
    """Grid step of Algorithm 1: v_i = (m v)_i / m_i + dt g, then the walls."""
    d = m.ndim
    n = m.shape[0]
    v = np.zeros_like(p)
    occ = m > 0
    v[occ] = p[occ] / m[occ][:, None] + dt * np.asarray(gravity[:d])
    lo, hi = wall_mask(n, d, bc_width)
    idx = np.indices(m.shape)
    sticky = np.zeros(m.shape, bool)
    for k in range(d):
        if bc == BC_SLIP_FLOOR and k == 1:
            sticky |= hi[idx[k]]
        else:
            sticky |= lo[idx[k]] | hi[idx[k]]
    if bc == BC_SLIP_FLOOR:
        floor = lo[idx[1]]
        v[..., 1] = np.where(floor, np.maximum(v[..., 1], 0.0), v[..., 1])
    v[sticky] = 0.0
    return v


def g2p(x, F, vgrid, *, dx, dt, transfer):
    """Grid-to-particle transfer and advection of Algorithm 1 (steps 3 and 4).

    Returns the new (x, v, F, C).  MLS: C_p = 4 / dx^2 sum_i N_i v_i (x_i - x_p)^T
    and F <- (1 + dt C_p) F.  PIC: grad v = sum_i v_i (x) grad N_i, C_p = 0.
    """
    P, d = x.shape
    base = stencil_base(x, dx)
    fx = x / dx - base
    w, dw = bspline(fx)
    vp = np.zeros((P, d))
    B = np.zeros((P, d, d))
    for off in stencil_offsets(d):
        node = base + np.array(off)
        weight = np.ones(P)
        for k in range(d):
            weight = weight * w[:, k, off[k]]
        vi = vgrid[tuple(node[:, k] for k in range(d))]
        vp += weight[:, None] * vi
        if transfer == MLS:
            dpos = node * dx - x
            B += weight[:, None, None] * np.einsum("pi,pj->pij", vi, dpos)
        else:
            grad = np.empty((P, d))
            for a in range(d):
                g = dw[:, a, off[a]] / dx
                for k in range(d):
                    if k != a:
                        g = g * w[:, k, off[k]]
                grad[:, a] = g
            B += np.einsum("pi,pj->pij", vi, grad)
    if transfer == MLS:
        Cn = (4.0 / dx ** 2) * B
        gradv = Cn
    else:
        Cn = np.zeros((P, d, d))
        gradv = B
    Fn = (np.eye(d) + dt * gradv) @ F
    xn = x + dt * vp
    return xn, vp, Fn, Cn


# ------------------------------------------------------------------------------ step


def instance_params(scene, k):
    mu, lam = lame(scene.E[k], scene.nu[k])
    return mu, lam


def step(scene, n_steps: int = 1, return_grid: bool = False):
    """Advance every instance of ``scene`` (a synth.scenes.Scene) by n_steps in place."""
    d = scene.dim
    grids = []
    for _ in range(n_steps):
        grids = []
        for k in range(scene.n_inst):
            s = slice(int(scene.inst_offsets[k]), int(scene.inst_offsets[k + 1]))
            mu, lam = instance_params(scene, k)
            m, p = p2g(scene.x[s], scene.v[s], scene.F[s], scene.C[s], scene.p_mass, scene.p_vol,
                       mu, lam, dx=scene.dx, dt=scene.dt, n_grid=scene.n_grid,
                       material=scene.material, transfer=scene.transfer)
            vg = grid_update(m, p, dt=scene.dt, gravity=scene.gravity, bc=scene.bc,
                             bc_width=scene.bc_width)
            xn, vn, Fn, Cn = g2p(scene.x[s], scene.F[s], vg, dx=scene.dx, dt=scene.dt,
                                 transfer=scene.transfer)
            if scene.material == FIXED_COROTATED_PLASTIC:
                Fn = plastic_return(Fn, 1.0 - scene.theta_c, 1.0 + scene.theta_s)
            if scene.kin_group is not None:
                xn, vn, Cn = kinematic_override(scene.x[s], xn, vn, Cn, scene.kin_group[s], scene.kin_vel,
                                                scene.dt)
            scene.x[s], scene.v[s], scene.F[s], scene.C[s] = xn, vn, Fn, Cn
            if return_grid:
                grids.append((m, p, vg))
    return grids if return_grid else None


def health(scene):
    """Stability monitor: (min J, max J, max |v|, any NaN)."""
    J = np.linalg.det(scene.F)
    return (float(J.min()), float(J.max()), float(np.abs(scene.v).max()),
            bool(np.isnan(scene.x).any() or np.isnan(scene.F).any()))
