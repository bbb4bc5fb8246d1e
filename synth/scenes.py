"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only draws numbers: particle lattices, jitter, material and
initial-velocity parameters, network initial weights.  It holds none of the
method's arithmetic (no transfer, no stress, no network evaluation), so the
oracle and the CUDA path can both consume it without sharing any of the
computation they are compared on.

Scene recipes (the paper's own scenes and data are not available; these are
elastic bodies under gravity and impact shaped like them: lattice of particles
at 2 per cell per dimension, E of order 1e4 Pa, nu = 0.3):

* ``block_2d``   64 x 64 particles at dx/2 spacing, a 0.25 m square block in a
                 unit box on a 128^2 grid, one initial velocity per body drawn
                 from U[-0.5, 0.5]^2.
* ``cube_3d``    64^3 lattice at dx/2 spacing with U[-0.2 dx, 0.2 dx] jitter per
                 component, a 0.25 m cube on a 128^3 grid, E ~ U[5e3, 5e4],
                 dropped at 1 m/s onto the floor.
* ``batch_2d``   n instances of 2D blocks with particle counts drawn from
                 U[20k, 120k] (rounded to 4 w h), (E, v0) from
                 U[5e3, 1.5e4] x U[-0.5, 0.5]^2, on a 256^2 grid (box side 2),
                 dt = 5e-5 (the elastic-wave CFL number c dt / dx stays
                 below 0.95 over the whole E range; at E = 5e4 or dt = 1e-4
                 the explicit step diverges on impact).
"""
from __future__ import annotations

import dataclasses
import numpy as np


@dataclasses.dataclass
class Scene:
    """A batch of independent MPM instances laid out back to back.

    Arrays are float64 on the host; consumers cast to their own precision.
    ``inst_offsets[k]:inst_offsets[k+1]`` are the particles of instance k.
    """
    dim: int
    n_grid: int
    dx: float
    dt: float
    gravity: np.ndarray          # (3,)
    bc: int                      # 0 sticky walls, 1 slip floor (+ sticky elsewhere)
    bc_width: int
    material: int                # 0 neo-Hookean, 1 fixed-corotated
    transfer: int                # 0 MLS/APIC, 1 PIC with exact basis gradients
    rho: float
    p_vol: float                 # particle reference volume V0
    E: np.ndarray                # (n_inst,)
    nu: np.ndarray               # (n_inst,)
    inst_offsets: np.ndarray     # (n_inst + 1,) int64
    x: np.ndarray                # (P, d)
    v: np.ndarray                # (P, d)
    F: np.ndarray                # (P, d, d)
    C: np.ndarray                # (P, d, d)
    # plastic material (material 2): singular values of F kept in [1 - theta_c, 1 + theta_s]
    theta_c: float = 2.5e-2
    theta_s: float = 7.5e-3
    # kinematic boundaries: group id per particle (-1: free) and the prescribed velocity of each
    # group (n_groups, d); None: no kinematic particles
    kin_group: np.ndarray | None = None
    kin_vel: np.ndarray | None = None

    @property
    def n_inst(self) -> int:
        return len(self.E)

    @property
    def n_particles(self) -> int:
        return int(self.inst_offsets[-1])

    @property
    def p_mass(self) -> float:
        return self.rho * self.p_vol

    def copy(self) -> "Scene":
        return dataclasses.replace(
            self, gravity=self.gravity.copy(), E=self.E.copy(), nu=self.nu.copy(),
            inst_offsets=self.inst_offsets.copy(), x=self.x.copy(), v=self.v.copy(),
            F=self.F.copy(), C=self.C.copy(),
            kin_group=None if self.kin_group is None else self.kin_group.copy(),
            kin_vel=None if self.kin_vel is None else self.kin_vel.copy())

    def subset_instances(self, ids) -> "Scene":
        ids = list(ids)
        parts = [np.arange(self.inst_offsets[i], self.inst_offsets[i + 1]) for i in ids]
        sel = np.concatenate(parts)
        offs = np.concatenate([[0], np.cumsum([len(p) for p in parts])]).astype(np.int64)
        return dataclasses.replace(
            self, gravity=self.gravity.copy(), E=self.E[ids].copy(), nu=self.nu[ids].copy(),
            inst_offsets=offs, x=self.x[sel].copy(), v=self.v[sel].copy(),
            F=self.F[sel].copy(), C=self.C[sel].copy())


def _lattice(counts, spacing, origin):
    axes = [origin[k] + (np.arange(counts[k]) + 0.5) * spacing for k in range(len(counts))]
    grids = np.meshgrid(*axes, indexing="ij")
    # particle order: first axis slowest, last axis fastest
    return np.stack([g.reshape(-1) for g in grids], axis=-1)


def _identity_state(x):
    P, d = x.shape
    F = np.broadcast_to(np.eye(d), (P, d, d)).copy()
    C = np.zeros((P, d, d))
    return F, C


def block_2d(seed: int = 1, side: int = 64, E: float | None = None,
             v0: np.ndarray | None = None, dt: float = 1e-4,
             origin=(0.375, 0.2)) -> Scene:
    """Square neo-Hookean block: side x side particles at dx/2 spacing."""
    rng = np.random.default_rng(seed)
    n_grid, dx = 128, 1.0 / 128
    x = _lattice((side, side), dx / 2, origin)
    if v0 is None:
        v0 = rng.uniform(-0.5, 0.5, size=2)
    v = np.broadcast_to(np.asarray(v0, np.float64), x.shape).copy()
    F, C = _identity_state(x)
    return Scene(dim=2, n_grid=n_grid, dx=dx, dt=dt, gravity=np.array([0.0, -9.8, 0.0]),
                 bc=0, bc_width=3, material=0, transfer=0, rho=1.0, p_vol=(dx / 2) ** 2,
                 E=np.array([1e4 if E is None else E]), nu=np.array([0.3]),
                 inst_offsets=np.array([0, len(x)], np.int64), x=x, v=v, F=F, C=C)


def cube_3d(seed: int = 2, side: int = 64, n_grid: int = 128, dt: float = 5e-5,
            jitter: float = 0.2, bottom: float = 0.05, v0=(0.0, -1.0, 0.0)) -> Scene:
    """Fixed-corotated cube: side^3 jittered lattice at dx/2 spacing."""
    rng = np.random.default_rng(seed)
    dx = 1.0 / n_grid
    width = side * dx / 2
    origin = (0.5 - width / 2, bottom, 0.5 - width / 2)
    x = _lattice((side, side, side), dx / 2, origin)
    E = rng.uniform(5e3, 5e4)
    x = x + rng.uniform(-jitter * dx, jitter * dx, size=x.shape)
    v = np.broadcast_to(np.asarray(v0, np.float64), x.shape).copy()
    F, C = _identity_state(x)
    return Scene(dim=3, n_grid=n_grid, dx=dx, dt=dt, gravity=np.array([0.0, -9.8, 0.0]),
                 bc=1, bc_width=3, material=1, transfer=0, rho=1.0, p_vol=(dx / 2) ** 3,
                 E=np.array([E]), nu=np.array([0.3]),
                 inst_offsets=np.array([0, len(x)], np.int64), x=x, v=v, F=F, C=C)


def batch_2d(seed: int = 3, n_inst: int = 16, count_range=(20000, 120000),
             n_grid: int = 256, dt: float = 5e-5, fixed_side: int | None = None,
             E_range=(5e3, 1.5e4), origin_y: float = 0.1) -> Scene:
    """Uneven batch of 2D neo-Hookean blocks on a 256^2 grid (box side 2).

    Particle count per instance ~ U[count_range], rounded to 4 w h with a near
    square w x h block of cells (4 particles per cell).  ``fixed_side`` instead
    gives every instance the same side x side particle block (the training set
    for the reduced model of the 4096-particle scene).
    """
    rng = np.random.default_rng(seed)
    dx = 1.0 / 128
    xs, vs, Es, offs = [], [], [], [0]
    box = n_grid * dx
    for _ in range(n_inst):
        if fixed_side is None:
            c = rng.uniform(*count_range)
            w = max(1, int(round(np.sqrt(c / 4))))
            h = max(1, int(round(c / (4 * w))))
            nx, ny = 2 * w, 2 * h
        else:
            nx = ny = fixed_side
        E = rng.uniform(*E_range)
        v0 = rng.uniform(-0.5, 0.5, size=2)
        origin = (box / 2 - nx * dx / 4, origin_y * box)
        x = _lattice((nx, ny), dx / 2, origin)
        xs.append(x)
        vs.append(np.broadcast_to(v0, x.shape).copy())
        Es.append(E)
        offs.append(offs[-1] + len(x))
    x = np.concatenate(xs)
    v = np.concatenate(vs)
    F, C = _identity_state(x)
    return Scene(dim=2, n_grid=n_grid, dx=dx, dt=dt, gravity=np.array([0.0, -9.8, 0.0]),
                 bc=0, bc_width=3, material=0, transfer=0, rho=1.0, p_vol=(dx / 2) ** 2,
                 E=np.array(Es), nu=np.full(n_inst, 0.3),
                 inst_offsets=np.array(offs, np.int64), x=x, v=v, F=F, C=C)


def random_deformation(rng: np.random.Generator, P: int, d: int, scale: float = 0.2):
    """Random F = I + scale * U(-1,1) with det > 0 (resampled until positive)."""
    F = np.eye(d) + scale * rng.uniform(-1, 1, size=(P, d, d))
    bad = np.linalg.det(F) <= 0.05
    while bad.any():
        F[bad] = np.eye(d) + scale * rng.uniform(-1, 1, size=(int(bad.sum()), d, d))
        bad = np.linalg.det(F) <= 0.05
    return F


# ----------------------------------------------------------------------------------
# decoder parameters


@dataclasses.dataclass
class DecoderParams:
    """Multilayer perceptron g(X; xhat) = out_scale * MLP([Xn, xhat]) + out_shift.

    ``W[l]`` has shape (out, in).  Layer 0 maps d + r inputs to ``width``;
    ``n_hidden - 1`` square layers follow; the last layer maps to d.  With
    ``n_hidden == 0`` the network is a single linear map (in -> d) and
    ``activation`` is ignored.  ``X_min``/``X_range`` give the min-max input
    normalisation Xn = (X - X_min) / X_range.
    """
    d: int
    r: int
    width: int
    n_hidden: int
    activation: int              # 0 ELU, 1 identity
    W: list
    b: list
    X_min: np.ndarray
    X_range: np.ndarray
    out_shift: np.ndarray
    out_scale: np.ndarray

    def copy(self) -> "DecoderParams":
        return dataclasses.replace(self, W=[w.copy() for w in self.W], b=[v.copy() for v in self.b],
                                   X_min=self.X_min.copy(), X_range=self.X_range.copy(),
                                   out_shift=self.out_shift.copy(), out_scale=self.out_scale.copy())

    def flat(self) -> np.ndarray:
        return np.concatenate([a.reshape(-1) for pair in zip(self.W, self.b) for a in pair])


def xavier_decoder(seed: int, d: int, r: int, width: int = 128, n_hidden: int = 5,
                   activation: int = 0, X_min=None, X_range=None, out_shift=None,
                   out_scale=None, bias_scale: float = 0.0) -> DecoderParams:
    """Xavier-uniform initial weights (Glorot and Bengio 2010); biases zero unless asked."""
    rng = np.random.default_rng(seed)
    dims = [d + r] + [width] * n_hidden + [d]
    W, b = [], []
    for l in range(len(dims) - 1):
        fan_in, fan_out = dims[l], dims[l + 1]
        lim = np.sqrt(6.0 / (fan_in + fan_out))
        W.append(rng.uniform(-lim, lim, size=(fan_out, fan_in)))
        b.append(rng.uniform(-bias_scale, bias_scale, size=fan_out) if bias_scale else np.zeros(fan_out))
    return DecoderParams(
        d=d, r=r, width=width, n_hidden=n_hidden, activation=activation, W=W, b=b,
        X_min=np.zeros(d) if X_min is None else np.asarray(X_min, np.float64),
        X_range=np.ones(d) if X_range is None else np.asarray(X_range, np.float64),
        out_shift=np.zeros(d) if out_shift is None else np.asarray(out_shift, np.float64),
        out_scale=np.ones(d) if out_scale is None else np.asarray(out_scale, np.float64))


def near_identity_decoder(seed: int, d: int, r: int, n_hidden: int = 1, X_min=None, X_range=None,
                          eps: float = 1e-3, width: int = 128) -> DecoderParams:
    """ELU network whose output is X plus a small nonlinear function of (X, xhat).

    The first d hidden units of every layer carry the normalised inputs X_n + 1 (positive, so the
    ELU passes them through); the output layer maps them back to X.  The remaining units are
    Xavier-initialised and enter the output with weights of size eps, so dg/dX = I + O(eps / X_range)
    and the decoded motion stays invertible (a configuration the inversion of the decoder and the
    reference-domain test see in a deformed body)."""
    p = xavier_decoder(seed, d, r, width, n_hidden, 0, X_min=X_min, X_range=X_range, bias_scale=0.2)
    rng = np.random.default_rng(seed + 1)
    for l in range(n_hidden):
        W, b = p.W[l], p.b[l]
        W[:d, :] = 0.0
        W[:d, :d] = np.eye(d)
        b[:d] = 1.0 if l == 0 else 0.0
    Wo = p.W[-1]
    Wo[:, :] = eps * rng.uniform(-1, 1, size=Wo.shape)
    Wo[:, :d] = np.diag(p.X_range)
    p.b[-1][:] = p.X_min - p.X_range
    return p


def refine_block_2d(sc: Scene, factor: int = 2) -> Scene:
    """The same single 2D block (a dx/2 lattice) discretised `factor` times finer: particles at
    (dx / factor) / 2 spacing over the same extent, a grid of factor x n_grid nodes, the same
    material and initial velocity (super-resolution scenes of Section 5)."""
    assert sc.dim == 2 and sc.n_inst == 1
    h = sc.dx / 2
    lo = sc.x.min(0) - 0.5 * h
    counts = np.round((sc.x.max(0) + 0.5 * h - lo) / h).astype(int)
    dxf = sc.dx / factor
    x = _lattice(tuple(counts * factor), dxf / 2, lo)
    v = np.broadcast_to(sc.v[0], x.shape).copy()
    F, C = _identity_state(x)
    return dataclasses.replace(sc, n_grid=sc.n_grid * factor, dx=dxf, p_vol=(dxf / 2) ** 2,
                               inst_offsets=np.array([0, len(x)], np.int64), x=x, v=v, F=F, C=C,
                               gravity=sc.gravity.copy(), E=sc.E.copy(), nu=sc.nu.copy())


def clamped_bar_2d(seed: int = 5, side: int = 32, top_velocity=(0.4, -0.3), layers: int = 2,
                   dt: float = 5e-5) -> Scene:
    """Square block whose bottom `layers` particle rows are held still and whose top rows move at a
    fixed velocity (two kinematic boundaries, as in the tension / torsion scenes of Section 5);
    gravity off, neo-Hookean."""
    sc = block_2d(seed=seed, side=side, dt=dt, origin=(0.375, 0.375), E=5e3, v0=np.zeros(2))
    sc.gravity = np.zeros(3)
    y = sc.x[:, 1]
    ys = np.unique(np.round(y, 12))
    g = np.full(sc.n_particles, -1, np.int32)
    g[y <= ys[layers - 1] + 1e-12] = 0
    g[y >= ys[-layers] - 1e-12] = 1
    sc.kin_group = g
    sc.kin_vel = np.array([[0.0, 0.0], list(top_velocity)], np.float64)
    sc.v = np.where((g == 1)[:, None], sc.kin_vel[1], 0.0)
    return sc
