"""End-to-end use of the library: full-order snapshots -> decoder training -> reduced-order
simulation -> accumulated position error against the full-order model (Section 5).

Everything numeric runs in libmpmrom.so; this module only sequences the C-ABI calls
and keeps device tensors alive.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np
import torch

from .decoder import Decoder
from .mpm import MPM
from .rom import ROM, metric_accumulate
from .train import Trainer, generate_snapshots


def decoder_for_snapshots(snaps, r, seed=0, width=128, n_hidden=5, activation=0):
    """Xavier-initialised decoder (seeded initial weights) whose Appendix B scaling (min-max of
    the training X, standardisation of the snapshot positions) is computed by the library from
    the snapshots (decoder_fit_scaling).  Returns the decoder and its initial parameters with
    the fitted scaling read back."""
    import synth.scenes as S
    d = snaps["dim"]
    p = S.xavier_decoder(seed, d, r, width, n_hidden, activation)
    dec = Decoder.from_params(p)
    dec.fit_scaling(snaps)
    norm = torch.empty(4 * d, dtype=torch.float32, device="cuda")
    dec.get_params(None, norm)
    nm = norm.cpu().numpy().astype(np.float64)
    p.X_min, p.X_range, p.out_shift, p.out_scale = nm[:d], nm[d:2 * d], nm[2 * d:3 * d], nm[3 * d:]
    return dec, p


def train(snaps, decoder, *, steps, batch=65536, lambda_F=100.0, lambda_v=0.01, lr0=1e-3, lr1=1e-6, seed=0,
          report_every=0, encoder_subset=0):
    """Trains the decoder with a latent table (encoder_subset = 0) or with the encoder of Section 4.1 on
    encoder_subset particles per snapshot."""
    dt_snap = float(snaps["dt_snap"])
    tr = Trainer(decoder, snaps, lambda_F=lambda_F, lambda_v=lambda_v, dt_snap=dt_snap, lr0=lr0, lr1=lr1,
                 batch=batch, total_steps=steps, seed=seed, encoder_subset=encoder_subset)
    history = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    done = 0
    chunk = report_every if report_every > 0 else steps
    while done < steps:
        n = min(chunk, steps - done)
        tr.step(n)
        done += n
        history.append((done, tr.loss()[0]))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    return tr, history, wall


@dataclasses.dataclass
class RomRun:
    error_percent: float
    rom_steps_per_s: float
    fom_steps_per_s: float
    status: int
    steps: int
    error_percent_at: dict = dataclasses.field(default_factory=dict)   # step -> accumulated error so far


def fom_positions(scene, steps, device="cuda"):
    """Positions of the full-order run at steps 0..steps (device tensor (steps+1, P, d)) and its steps/s."""
    ctx = MPM.from_scene(scene)
    ctx.load_numpy(scene.x, scene.v, scene.F, scene.C)
    P, d = scene.n_particles, scene.dim
    xs = torch.empty((steps + 1, P, d), dtype=torch.float32, device=device)
    ctx.get_state(xs[0])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for n in range(1, steps + 1):
        ctx.step(1)
        ctx.get_state(xs[n])
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    # pure stepping rate (no per-step read-back)
    ctx.load_numpy(scene.x, scene.v, scene.F, scene.C)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.step(steps)
    torch.cuda.synchronize()
    rate = steps / (time.perf_counter() - t0)
    status = ctx.status()
    ctx.close()
    return xs, rate, status


def rom_error(decoder, scene, fom_xs, *, n_samples=256, seed=4, gn_iters=3, projection=0, fit_iters=20, ridge=0.0,
              affine=0, f_reference=0, quadrature=0, ell=0, newton_iters=0, checkpoints=()):
    """Runs the reduced model from the least-squares initial condition (Eq. essentialSpecInt) for as
    many steps as fom_xs has, accumulating the Section 5 error on the device."""
    steps = fom_xs.shape[0] - 1
    rom = ROM.from_scene(decoder, scene, n_samples=n_samples, seed=seed, gn_iters=gn_iters, projection=projection,
                         ridge=ridge, affine=affine, f_reference=f_reference, quadrature=quadrature, ell=ell,
                         newton_iters=newton_iters)
    rom.fit_initial(scene.x, scene.v, iters=fit_iters)
    acc = torch.zeros(2, dtype=torch.float64, device="cuda")
    xr = torch.empty_like(fom_xs[0])
    rom.decode_all(xr)
    metric_accumulate(xr, fom_xs[0], acc)
    rom.step(1)  # capture the graph outside the timed loop
    torch.cuda.synchronize()
    # restart from the initial state and time the steps with the metric accumulation
    rom.fit_initial(scene.x, scene.v, iters=fit_iters)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    marks = {}
    for n in range(1, steps + 1):
        rom.step(1)
        rom.decode_all(xr)
        metric_accumulate(xr, fom_xs[n], acc)
        if n in checkpoints:
            marks[n] = acc.clone()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    num, den = acc.cpu().numpy()
    at = {}
    for n, a in marks.items():
        nn, dd = a.cpu().numpy()
        at[n] = 100.0 * float(np.sqrt(nn / dd))
    # pure stepping rate
    rom.fit_initial(scene.x, scene.v, iters=fit_iters)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rom.step(steps)
    torch.cuda.synchronize()
    rate = steps / (time.perf_counter() - t0)
    status = rom.status()
    rom.close()
    return RomRun(error_percent=100.0 * float(np.sqrt(num / den)), rom_steps_per_s=rate, fom_steps_per_s=float("nan"),
                  status=status, steps=steps, error_percent_at=at)


def build_serving_batch(decoders, roms, concurrency, precision=None):
    """Sets the decoders' expected concurrency (the FP32 tiling of their calls) and, if given, their
    square-layer arithmetic (1 FP32 CUDA cores, 2 split BF16 tensor cores), then captures the batch
    of reduced-order contexts (one graph launch per step for all of them)."""
    from .rom import RomBatch
    for dec in decoders:
        dec.set_concurrency(int(concurrency))
        if precision is not None:
            dec.set_precision(int(precision))
    return RomBatch(roms)


def autotune_serving(decoders, roms, candidates=(1, 8, 32, 128, 512), precisions=(1, 2), trial_steps=4):
    """Decoder arithmetic and tiling for batched serving, chosen by measurement: for the FP32
    CUDA-core arithmetic each candidate concurrency k (how many decoder calls are expected to run
    at once, which sets how many SMs one call's tiles spread over), and the split-BF16 tensor-core
    arithmetic (128-row tiles, no tiling choice); each configuration's batch is captured and
    `trial_steps` batch steps are timed on the device.  Returns ((precision, k) of the fastest,
    {"precision/k": ms per batch step}).  The trial steps advance the contexts."""
    times = {}
    configs = []
    for prec in precisions:
        for k in (candidates if prec == 1 else candidates[:1]):
            if k > max(1, len(roms)) and k != candidates[0]:
                continue
            configs.append((int(prec), int(k)))
    for prec, k in configs:
        batch = build_serving_batch(decoders, roms, k, prec)
        batch.step(1)                       # first launch: graph upload
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        batch.step(trial_steps)
        b.record()
        torch.cuda.synchronize()
        times[(prec, k)] = a.elapsed_time(b) / trial_steps
        batch.close()
    best = min(times, key=times.get)
    return best, {f"{p}/{k}": t for (p, k), t in times.items()}
