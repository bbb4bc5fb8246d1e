"""FP64 oracle of the implicit neural decoder g(X; xhat) and its training.  Test infrastructure only.

Section 3.1 (kinematic restriction, Eq. kinematicRestriction): phi(X; t) = g(X; xhat(t)).
Eq. defGrad: the deformation gradient is dg/dX; Eq. timederOne: the velocity is
(dg/dxhat) xhat_dot.  Section 4: g is a multilayer perceptron with ELU
activations (continuously differentiable, so both derivatives exist); its input
X is min-max normalised and its output standardised (Appendix B).  The loss of
Section 4.2 is, per (snapshot, particle),
    |g - phi|^2 + lambda_F |dg/dX - F|_F^2 + lambda_v |(dg/dxhat) (xhat_{n+1} - xhat_n) / dt - v|^2,
averaged over the minibatch here.  The latent table (one xhat per snapshot,
optimised with the weights) is the alternative to the encoder that the Remark
of Section 4.1 allows.  Adam (Appendix B) uses the PyTorch defaults
beta1 = 0.9, beta2 = 0.999, eps = 1e-8.

Derivatives are plain chain rule: forward-mode tangents for dg/dX and
dg/dxhat, hand-written reverse mode (including the ELU'' terms that the
tangent penalties need) for the training gradients.

Pins (tests/test_oracle_decoder.py): tangents against central differences;
a linear (identity-activation) network whose Jacobians are exactly its weight
blocks; loss gradients against central differences of the loss; Adam's
closed-form behaviour under a constant gradient; the Appendix B scaling maps the training X
onto [0, 1] with both ends attained and standardises the snapshot positions (zero mean, unit
population variance), checked by brute force on small sets.
"""
from __future__ import annotations

import numpy as np

ELU, IDENTITY = 0, 1


def act(z, kind):
    if kind == IDENTITY:
        return z
    return np.where(z > 0, z, np.expm1(np.minimum(z, 0.0)))


def act_d1(z, kind):
    if kind == IDENTITY:
        return np.ones_like(z)
    return np.where(z > 0, 1.0, np.exp(np.minimum(z, 0.0)))


def act_d2(z, kind):
    if kind == IDENTITY:
        return np.zeros_like(z)
    return np.where(z > 0, 0.0, np.exp(np.minimum(z, 0.0)))


def _inputs(dec, X, xhat):
    X = np.atleast_2d(np.asarray(X, np.float64))
    xhat = np.asarray(xhat, np.float64)
    if xhat.ndim == 1:
        xhat = np.broadcast_to(xhat, (len(X), dec.r))
    return np.concatenate([(X - dec.X_min) / dec.X_range, xhat], axis=1)


def forward(dec, X, xhat, tangents=(), keep=False):
    """Evaluate g and directional derivatives.

    ``tangents`` is a list of (dX, dxhat) input directions, each (n, d) and
    (n, r) (or broadcastable).  Returns g (n, d), the list of dg along each
    direction (n, d), and, with ``keep``, the per-layer records
    [(h_in, z, t_in list, zdot list)] that the reverse pass needs.
    """
    h = _inputs(dec, X, xhat)
    n = len(h)
    ts = []
    for dX, dxh in tangents:
        dX = np.broadcast_to(np.asarray(dX, np.float64), (n, dec.d))
        dxh = np.broadcast_to(np.asarray(dxh, np.float64), (n, dec.r))
        ts.append(np.concatenate([dX / dec.X_range, dxh], axis=1))
    records = []
    L = len(dec.W)
    for l in range(L):
        z = h @ dec.W[l].T + dec.b[l]
        zd = [t @ dec.W[l].T for t in ts]
        if keep:
            records.append((h, z, ts, zd))
        if l < L - 1:
            s1 = act_d1(z, dec.activation)
            h = act(z, dec.activation)
            ts = [s1 * q for q in zd]
        else:
            h, ts = z, zd
    g = h * dec.out_scale + dec.out_shift
    gd = [t * dec.out_scale for t in ts]
    return (g, gd, records) if keep else (g, gd)


def decode(dec, X, xhat):
    return forward(dec, X, xhat)[0]


def jacobians(dec, X, xhat):
    """g, dg/dX (n, d, d) with [p, i, k] = dg_i/dX_k, dg/dxhat (n, d, r)."""
    d, r = dec.d, dec.r
    dirs = [(np.eye(d)[k], np.zeros(r)) for k in range(d)] + [(np.zeros(d), np.eye(r)[j]) for j in range(r)]
    g, gd = forward(dec, X, xhat, dirs)
    dgdX = np.stack(gd[:d], axis=-1)
    dgdxh = np.stack(gd[d:], axis=-1) if r else np.zeros((len(g), d, 0))
    return g, dgdX, dgdxh


def jvp_latent(dec, X, xhat, u):
    """(dg/dxhat)(X; xhat) u for a latent direction u (r,) or (n, r)."""
    g, gd = forward(dec, X, xhat, [(np.zeros(dec.d), u)])
    return g, gd[0]


def velocity_gradient(dec, X, xhat, u):
    """Decoded velocity v = (dg/dxhat) u (Eq. timederOne with xhat_dot = u) and its
    material gradient dv/dX (n, d, d), [p, i, k] = dv_i/dX_k, by forward-over-forward
    chain rule: along the layers carry z, the latent tangent s (direction u), the
    X tangents t_k and the mixed tangents m_k = d s / d X_k, with
        s' = act'(z) (W s),  t_k' = act'(z) (W t_k),
        m_k' = act''(z) (W s)(W t_k) + act'(z) (W m_k).
    The spatial velocity gradient of the decoded motion is (dv/dX) (dg/dX)^-1."""
    d, r = dec.d, dec.r
    h = _inputs(dec, X, xhat)
    n = len(h)
    u = np.broadcast_to(np.asarray(u, np.float64), (n, r))
    s = np.concatenate([np.zeros((n, d)), u], axis=1)
    ts = [np.broadcast_to(np.concatenate([np.eye(d)[k] / dec.X_range, np.zeros(r)]), (n, d + r)) for k in range(d)]
    ms = [np.zeros((n, d + r)) for _ in range(d)]
    L = len(dec.W)
    for l in range(L):
        W = dec.W[l]
        z = h @ W.T + dec.b[l]
        zs = s @ W.T
        zt = [t @ W.T for t in ts]
        zm = [m @ W.T for m in ms]
        if l < L - 1:
            a1, a2 = act_d1(z, dec.activation), act_d2(z, dec.activation)
            h = act(z, dec.activation)
            s = a1 * zs
            ts = [a1 * q for q in zt]
            ms = [a2 * zs * q + a1 * mq for q, mq in zip(zt, zm)]
        else:
            s, ms = zs, zm
    v = s * dec.out_scale
    dvdX = np.stack([m * dec.out_scale for m in ms], axis=-1)
    return v, dvdX


# ------------------------------------------------------------------------------ training


def loss_and_grads(dec, X, xhat, x_t, F_t, v_t, u, mask_v, lam_F, lam_v):
    """Minibatch loss of Section 4.2 and its gradients.

    Per point p: latent xhat[p], target position x_t[p], deformation gradient
    F_t[p] (d, d), velocity v_t[p], latent finite-difference velocity u[p] =
    (xhat_{n+1} - xhat_n) / dt_snap, mask_v[p] in {0, 1} (0 where the snapshot
    has no successor).  Returns (loss, gW list, gb list, g_xhat (n, r), g_u (n, r)),
    the loss averaged over the n points.
    """
    d, r = dec.d, dec.r
    n = len(X)
    dirs = [(np.eye(d)[k], np.zeros(r)) for k in range(d)] + [(np.zeros(d), u)]
    g, gd, rec = forward(dec, X, xhat, dirs, keep=True)
    e1 = g - x_t
    e2 = [gd[k] - F_t[:, :, k] for k in range(d)]
    e3 = (gd[d] - v_t) * mask_v[:, None]
    loss = (np.sum(e1 ** 2) + lam_F * sum(np.sum(e ** 2) for e in e2) + lam_v * np.sum(e3 ** 2)) / n
    # adjoints of the network outputs (before the output scaling)
    hbar = 2.0 * e1 / n * dec.out_scale
    tbar = [2.0 * lam_F * e / n * dec.out_scale for e in e2] + [2.0 * lam_v * e3 / n * dec.out_scale]
    L = len(dec.W)
    gW = [None] * L
    gb = [None] * L
    for l in range(L - 1, -1, -1):
        h_in, z, t_in, zd = rec[l]
        if l < L - 1:
            s1 = act_d1(z, dec.activation)
            s2 = act_d2(z, dec.activation)
            zbar = s1 * hbar + sum(s2 * zd[j] * tbar[j] for j in range(len(tbar)))
            zdbar = [s1 * tb for tb in tbar]
        else:
            zbar, zdbar = hbar, tbar
        gW[l] = zbar.T @ h_in + sum(zdbar[j].T @ t_in[j] for j in range(len(zdbar)))
        gb[l] = zbar.sum(axis=0)
        hbar = zbar @ dec.W[l]
        tbar = [zb @ dec.W[l] for zb in zdbar]
    g_xhat = hbar[:, d:]
    g_u = tbar[d][:, d:]
    return loss, gW, gb, g_xhat, g_u


def batch_loss_grads(dec, latents, batch, dt_snap, lam_F, lam_v):
    """Loss and gradients for a minibatch drawn from a snapshot store.

    ``latents`` (S, r) is the latent table; ``batch`` holds per point: X, snap
    (index into latents), next (index of the successor snapshot or -1), x, F, v.
    Returns (loss, gW, gb, g_latents (S, r)).
    """
    snap = batch["snap"]
    nxt = batch["next"]
    has = nxt >= 0
    xh = latents[snap]
    u = np.where(has[:, None], (latents[np.where(has, nxt, snap)] - xh) / dt_snap, 0.0)
    loss, gW, gb, g_xh, g_u = loss_and_grads(dec, batch["X"], xh, batch["x"], batch["F"], batch["v"],
                                            u, has.astype(np.float64), lam_F, lam_v)
    gl = np.zeros_like(latents)
    np.add.at(gl, snap, g_xh - g_u / dt_snap * has[:, None])
    np.add.at(gl, nxt[has], g_u[has] / dt_snap)
    return loss, gW, gb, gl


class Adam:
    """Adam (Kingma and Ba 2015) over a list of arrays, updated in place."""

    def __init__(self, params, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.params = params
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps
        self.m = [np.zeros_like(p) for p in params]
        self.v = [np.zeros_like(p) for p in params]
        self.t = 0

    def step(self, grads, lr=None):
        lr = self.lr if lr is None else lr
        self.t += 1
        for p, g, m, v in zip(self.params, grads, self.m, self.v):
            m *= self.b1
            m += (1 - self.b1) * g
            v *= self.b2
            v += (1 - self.b2) * g * g
            mhat = m / (1 - self.b1 ** self.t)
            vhat = v / (1 - self.b2 ** self.t)
            p -= lr * mhat / (np.sqrt(vhat) + self.eps)


def lr_schedule(step, n_steps, lr0=1e-3, lr1=1e-6):
    """Geometric decay from lr0 to lr1 over the run (Appendix B: 1e-3 -> 1e-6)."""
    if n_steps <= 1:
        return lr0
    return lr0 * (lr1 / lr0) ** (step / (n_steps - 1))


def appendix_b_scaling(X, x):
    """Input and output scaling of Appendix B, by definition: per coordinate, the minimum and the
    range (max - min) of the reference positions X (n, d), and the mean and the population
    standard deviation (1/N) of the positions x (N, d) of every snapshot row.  Returns
    (X_min, X_range, out_shift, out_scale), the fields the decoder's input and output maps use."""
    X = np.asarray(X, np.float64)
    x = np.asarray(x, np.float64)
    lo = X.min(axis=0)
    hi = X.max(axis=0)
    mean = x.sum(axis=0) / x.shape[0]
    std = np.sqrt(((x - mean) ** 2).sum(axis=0) / x.shape[0])
    return lo, hi - lo, mean, std
