"""FP32 parity bounds derived from the measured sensitivity of each quantity (test infrastructure).

The GPU path computes in FP32, the oracle in FP64.  The stated bound is 1e-5, norm-wise relative.
Some quantities amplify FP32 rounding, and no FP32 computation can meet 1e-5 on them:
- a difference of nearly equal terms, such as F - R in the stress or the increment of a latent;
- a least-squares solve with an ill-conditioned Jacobian;
- a trajectory whose stress waves carry rounding from step to step.

For each such quantity the bound is K times its measured sensitivity, never below 1e-5.  The FP64
oracle is run again on perturbed inputs:
- for a single evaluation, every input (latents, positions, velocities, the decoder's biases and
  scaling) is multiplied by 1 +- u, with u = 2^-24 (one unit in the last place of FP32) and
  random signs, and the decoder's weights by 1 +- sqrt(n) u, n the layer's fan-in (the
  backward error of its FP32 dot products, below);
- for a trajectory, the state is rounded to FP32 after every step, which is the rounding FP32
  storage alone forces.
The perturbed run's deviation from the plain oracle is the sensitivity.

K = 10.  The GPU also rounds the result of every operation, not only its inputs.  The
probabilistic error bound of an n-term FP32 dot product grows like sqrt(n) u (Higham and Mary,
SIAM J. Sci. Comput. 2019).  With the decoder's hidden width n = 128 that is sqrt(128) ~ 11 units
of rounding; the 27-term sums of the 3D transfer give sqrt(27) ~ 5.
"""
from __future__ import annotations

import numpy as np

import oracle.mpm as OM

U32 = 2.0 ** -24
K = 10.0
FLOOR = 1e-5


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def bound(sens):
    """The parity bound for a quantity of measured sensitivity `sens` (1e-5 at least)."""
    return max(FLOOR, K * float(sens))


def f32(a):
    """The FP32 value of every element, held in FP64 (the inputs the GPU actually uses)."""
    return np.asarray(a, np.float64).astype(np.float32).astype(np.float64)


def perturb(a, rng):
    """a (1 +- u) elementwise, random signs: one FP32 unit in the last place."""
    a = np.asarray(a, np.float64)
    return a * (1.0 + U32 * rng.choice((-1.0, 1.0), size=a.shape))


def f32_decoder(p):
    """The decoder with every parameter and scaling field rounded to FP32 (the GPU's copy)."""
    q = p.copy()
    q.W = [f32(w) for w in q.W]
    q.b = [f32(v) for v in q.b]
    q.X_min, q.X_range, q.out_shift, q.out_scale = (f32(q.X_min), f32(q.X_range), f32(q.out_shift),
                                                    f32(q.out_scale))
    return q


def perturb_decoder(p, rng):
    """The decoder with the backward error of its FP32 evaluation: each layer's weights perturbed
    by sqrt(n) u with random signs (n its fan-in; the probabilistic backward error of an n-term
    FP32 dot product accumulated in order, Higham and Mary 2019), biases and scaling by u."""
    q = p.copy()
    q.W = [w * (1.0 + np.sqrt(w.shape[1]) * U32 * rng.choice((-1.0, 1.0), size=w.shape)) for w in q.W]
    q.b = [perturb(v, rng) for v in q.b]
    q.X_min, q.X_range, q.out_shift, q.out_scale = (perturb(q.X_min, rng), perturb(q.X_range, rng),
                                                    perturb(q.out_shift, rng), perturb(q.out_scale, rng))
    return q


# Split-BF16 square layers (decoder precision 2): each activation and weight is hi + lo with
# hi = bf16(v) (|v - hi| <= 2^-9 |v|) and lo the BF16 rounding of v - hi (error <= 2^-18 |v|), and
# the product keeps A_hi W_hi + A_hi W_lo + A_lo W_hi: the two operand residuals and the dropped
# A_lo W_lo term are each at most 2^-18 of the product.
SPLIT_PRODUCT = 3.0 * 2.0 ** -18


def perturb_decoder_split(p, rng):
    """The backward error of the split-BF16 evaluation: the FP32 model of perturb_decoder, with
    the weights of the square hidden layers (all but the first and the output layer) perturbed
    by SPLIT_PRODUCT with random signs instead (the error of each product, which does not
    accumulate over the sum beyond the FP32 rounding already in the model)."""
    q = perturb_decoder(p, rng)
    for l in range(1, len(p.W) - 1):
        q.W[l] = p.W[l] * (1.0 + SPLIT_PRODUCT * rng.choice((-1.0, 1.0), size=p.W[l].shape))
    return q


DECODER_MODELS = {"fp32": perturb_decoder, "split": perturb_decoder_split}


def sensitivity(fn, args, rng=None, decoder_args=(), model="fp32"):
    """Relative deviation of fn(*args) when every float array argument is perturbed by one FP32
    ulp (decoder arguments, given by position in decoder_args, have all their parameters
    perturbed by the backward error of the decoder arithmetic `model`).  Integer arrays (index
    sets) and scalars are passed unchanged."""
    rng = np.random.default_rng(12345) if rng is None else rng
    base = fn(*args)
    pert = []
    for i, a in enumerate(args):
        if i in decoder_args:
            pert.append(DECODER_MODELS[model](a, rng))
        elif isinstance(a, np.ndarray) and a.dtype.kind == "f":
            pert.append(perturb(a, rng))
        else:
            pert.append(a)
    return rel(fn(*pert), base), base


def fom_fp32_storage_run(sc, steps):
    """The FP64 oracle run of `steps` steps with the particle state rounded to FP32 before the
    first step and after every step."""
    run = sc.copy()
    for name in ("x", "v", "F", "C"):
        setattr(run, name, f32(getattr(run, name)))
    for _ in range(steps):
        OM.step(run, 1)
        for name in ("x", "v", "F", "C"):
            setattr(run, name, f32(getattr(run, name)))
    return run


def c_scale(ref):
    """C is a velocity gradient: it is measured against max(|C|, |v| / dx), so that rounding-level
    C (a rigid motion) is not divided by rounding."""
    return max(np.linalg.norm(ref.C), np.linalg.norm(ref.v) / ref.dx)


def fom_errors(x, v, F, Cm, ref):
    errs = dict(x=rel(x, ref.x), v=rel(v, ref.v), F=rel(F, ref.F))
    errs["C"] = float(np.linalg.norm(np.asarray(Cm, np.float64) - ref.C) / c_scale(ref))
    return errs


def fom_bounds(sc, ref, steps):
    """Per-quantity bounds for an N-step full-order trajectory from `sc` whose plain FP64 oracle
    result is `ref`: the sensitivity is the FP32-storage run's deviation from `ref`."""
    run = fom_fp32_storage_run(sc, steps)
    sens = fom_errors(run.x, run.v, run.F, run.C, ref)
    return {k: bound(s) for k, s in sens.items()}, sens


# ----------------------------------------------------------------------------- reduced step
# The GPU's reduced step consumes FP32 copies of the decoder's parameters, of the reference
# positions and of the latent state; the oracle is given exactly those values (f32_*), so that
# the comparison measures the GPU's arithmetic, and the bound its sensitivity.


def check_trial_velocity(p, rs, xh, vh, samples, x_all, got, label="", model="fp32"):
    """v_trial of Algorithm 5 (the oracle's local step on the GPU's own decoded positions x_all
    and sample set) within the derived bound; returns the oracle's v_trial."""
    import dataclasses

    import oracle.rom as OR
    rs32 = dataclasses.replace(rs, X=f32(rs.X))

    def fn(pp, X_, x_, v_, xa_):
        return OR.local_dynamics(pp, dataclasses.replace(rs32, X=X_), x_, v_, samples, xa_)[0]

    sens, ref = sensitivity(fn, (f32_decoder(p), rs32.X, f32(xh), f32(vh), np.asarray(x_all, np.float64)),
                            decoder_args=(0,), model=model)
    err = rel(got, ref)
    print(f"{label} v_trial error {err:.3e} sensitivity {sens:.3e} bound {bound(sens):.3e}")
    assert err < bound(sens), (label, err, sens)
    return ref


# Every normal-equations solve of the GPU carries a ridge of at least 1e-10 tr(J^T J) / r (the
# minimum-norm limit for rank-deficient J^T J), on the increment from the previous value; the
# oracle is given the same problem.
RIDGE_FLOOR = 1e-10


def check_velocity_projection(p, Xs, xh, v_trial, got, label="", ridge=0.0, vhat_n=None, model="fp32"):
    """vhat of the velocity least-squares fit (on the GPU's own trial velocities), as the
    increment from vhat_n (zero if None) with ridge max(ridge, 1e-10)."""
    ridge = max(ridge, RIDGE_FLOOR)
    import oracle.rom as OR

    def fn(pp, X_, x_, v_):
        return OR.project_velocity(pp, X_, x_, v_, ridge=ridge, vhat_n=vhat_n)

    sens, ref = sensitivity(fn, (f32_decoder(p), f32(Xs), f32(xh), np.asarray(v_trial, np.float64)),
                            decoder_args=(0,), model=model)
    err = rel(got, ref)
    print(f"{label} vhat error {err:.3e} sensitivity {sens:.3e} bound {bound(sens):.3e}")
    assert err < bound(sens), (label, err, sens)
    return ref


def line_search_band(p, rec, dt_v, model="fp32"):
    """Rounding band of the sufficient-decrease margins f(2^-m) - f0 - c 2^-m slope of one
    Gauss-Newton iteration (rec: the oracle's record of it).  The GPU forms every residual row
    from an FP32 secant s = g(xhat) - g(xhat_n) (r = s - dt v_trial), whose relative error is that
    of an n-term FP32 dot product, sqrt(n) u (n the widest fan-in).  An error e in the rows moves
    |r|^2 by 2 r.e to first order, at most 2 |r| |e| <= 2 sqrt(n) u |r| (|r| + |dt v_trial|); the
    band is K times that for the trial and for f0 together."""
    n = max(w.shape[1] for w in p.W)
    rel_row = np.sqrt(n) * U32 if model == "fp32" else SPLIT_PRODUCT
    rs = np.sqrt(np.maximum(rec["f"], 0.0))
    r0 = np.sqrt(max(rec["f0"], 0.0))
    return 2.0 * K * rel_row * (rs * (rs + dt_v) + r0 * (r0 + dt_v))


def check_line_search_picks(p, records, picks, dt_v, c=1e-4, label="", model="fp32"):
    """Every line-search choice of the GPU is a valid outcome of the backtracking rule in exact
    arithmetic up to the rounding band: each trial before the chosen one fails the condition or
    lies within the band, and the chosen one meets it or lies within the band (with -1, none is
    chosen, so every trial fails or lies within the band).  Returns the number of choices that
    differ from the FP64 one (possible only within the band)."""
    open_choices = 0
    for i, (m, rec) in enumerate(zip(picks, records)):
        f = rec["f"]
        margins = f - (rec["f0"] + c * 0.5 ** np.arange(len(f)) * rec["slope"])
        band = line_search_band(p, rec, dt_v, model)
        last = int(m) if m >= 0 else len(f)
        assert np.all(margins[:last] > -band[:last]), (label, i, m, margins[:last], band[:last])
        if m >= 0:
            assert margins[m] <= band[m], (label, i, m, margins[m], band[m])
        first = int(np.argmax(margins <= 0)) if np.any(margins <= 0) else -1
        open_choices += int(first != m)
    return open_choices


def check_gauss_newton_increment(p, Xs, xh, xh_prev, v_trial, dt, got_xh1, iters=3, label="", ridge=0.0,
                                 picks=None, model="fp32"):
    """xhat_{n+1} - xhat_n of Algorithm 6 (Gauss-Newton from 2 xhat_n - xhat_{n-1} towards the
    trial positions g(X; xhat_n) + dt v_trial, on the GPU's own trial velocities).  The GPU forms
    the residual as [g(xhat_k) - g(xhat_n)] - dt v_trial (secant rows), never rounding the trial
    positions themselves, so the perturbed inputs are the decoder, X, xhat_n, v_trial and the
    initial guess, and the trial positions follow from them in FP64.

    Backtracking is a discrete choice the GPU makes on its FP32 residual rows.  Once an iteration
    has reached the rounding level of those rows, the sufficient-decrease margin of a trial can be
    smaller than their rounding, and the GPU and the FP64 oracle may then take different step
    lengths, both correct; the increments differ by a fraction of that iteration's step.  With
    `picks` (the GPU's choices, ROM.line_search_picks) every choice is checked to be valid within
    the rounding band, and the oracle replays the GPU's choices."""
    import oracle.decoder as OD
    import oracle.rom as OR
    dt32 = float(np.float32(dt))
    init = 2 * np.asarray(xh, np.float64) - np.asarray(xh_prev, np.float64)
    pf = f32_decoder(p)
    Xs32 = f32(Xs)
    vt = np.asarray(v_trial, np.float64)
    xh = np.asarray(xh, np.float64)
    rid = max(ridge, RIDGE_FLOOR)
    if picks is not None:
        records = []
        x_trial = OD.decode(pf, Xs32, xh) + dt32 * vt
        OR.gauss_newton(pf, Xs32, x_trial, init, iters, ridge=rid, steps=picks, record=records)
        n_open = check_line_search_picks(pf, records, picks, dt32 * np.linalg.norm(vt), label=label, model=model)
        print(f"{label} line-search choices {[int(m) for m in picks]}, {n_open} of them other than the FP64 "
              f"choice, within the rounding band")

    def fn(pp, X_, xh_, vt_, i_):
        x_trial = OD.decode(pp, X_, xh_) + dt32 * vt_
        return OR.gauss_newton(pp, X_, x_trial, i_, iters, ridge=rid, steps=picks)[0] - xh_

    sens, ref = sensitivity(fn, (pf, Xs32, xh, vt, init), decoder_args=(0,), model=model)
    err = rel(np.asarray(got_xh1) - xh, ref)
    print(f"{label} GN increment error {err:.3e} sensitivity {sens:.3e} bound {bound(sens):.3e}")
    assert err < bound(sens), (label, err, sens)
    return ref + xh
