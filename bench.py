"""Benchmark of the hot path: MPM particle-steps/s on the 3D fixed-corotated cube, and the
reduced-order model's steps/s against the full-order model at its measured position error.

Workload (N = 1): 262,144 particles (64^3 jittered lattice at dx/2), 128^3
grid, fixed-corotated material with the polar factor refined by a compensated-FP32 rotation
correction (the FP64 one is a reported variant), slip floor, dt = 5e-5, MLS-MPM; the timed
steps follow an untimed pre-roll to the slip-floor contact.  A step is one explicit MPM step of every instance
(binning, particle-to-grid, grid update, grid-to-particle).  Inputs are
resident in HBM when the timed region starts; L2 is flushed (a 256 MiB write)
before every timed step, outside its CUDA-event interval.

The reduced-order leg (key "rom"; skipped with --no-rom) generates snapshots with the GPU
full-order model, trains the decoder on the GPU, runs the reduced model on a held-out 2D impact
scene and reports its steps/s next to the full-order steps/s on the same scene, with the
accumulated relative position error of Section 5.

With torchrun (N > 1) every rank runs an independent replica of the workload
(the single-scene step does not shard; batched instances would shard by
instance with no exchange): weak scaling, max time over ranks.

``--impl reference`` times the FP64 CPU oracle (the deliberately slow,
obviously correct restatement of the paper's algorithm) on the host cores
instead, on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth.scenes as S  # noqa: E402

METRIC = "MPM particle-steps/s vs ROM steps/s at \u22641e-2 rel. position err, 1 GB300"
UNIT = "particle-steps/s"
WORKLOAD = ("3D fixed-corotated cube, 262144 particles, 128^3 grid, MLS-MPM, polar factor refined by a "
            "compensated-FP32 (double-FP32) rotation correction, dt=5e-5, slip floor")
# algorithmic bytes per particle-step (3D): particle state read + written once,
# x, v (3 each), F, C (9 each) in FP32 = 2 x 96 B; active grid nodes ~1/8 per
# particle x 56 B (clear + scatter 16, update 28, gather 12) = 7 B
ALGO_BYTES_3D = 2 * 96 + 7
L2_FLUSH_BYTES = 256 << 20
# the cube's lowest particles reach the slip band (nodes j < 3) after about 450 steps; the timed
# steps start after this untimed pre-roll, so that they include the floor contact
PRE_ROLL = 600
# the rotation correction of the polar factor: compensated FP32 (Dot2 sums, as accurate as twice
# the working precision); the FP64 correction is reported as a variant
HEADLINE_POLAR_EFT = 1
# DRAM bytes (read + write) of one launch of the fused step kernel on this workload, from one ncu
# capture of the current kernel (dram__bytes_read.sum + dram__bytes_write.sum; first timed step
# after the pre-roll).  Reads: x, F, particle id and binning permutation (56 B per particle) and
# the node tiles; v and C are not read (G2P recomputes them).  The written state is still in the
# write-back L2 when the kernel ends.
FUSED_DRAM_BYTES_NCU = 16_716_800 + 45_824


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi around the timed region.

    The sampler is running (first sample read) before the region starts and keeps running until
    a sample after its end has arrived; the summary uses the samples from the last one before
    the region to the first one after it (a region shorter than the sampling period is
    bracketed by its neighbours)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index, period_ms=50):
        self.index = index
        self.period_ms = period_ms
        self.proc = None
        self.samples = []   # (host time, line)

    def _reader(self):
        for line in self.proc.stdout:
            if line.strip():
                self.samples.append((time.perf_counter(), line))

    def __enter__(self):
        import threading
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(self.period_ms)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._reader, daemon=True).start()
            deadline = time.perf_counter() + 10.0
            while not self.samples and time.perf_counter() < deadline and self.proc.poll() is None:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        self.t0 = time.perf_counter()
        return self

    def __exit__(self, *a):
        self.t1 = time.perf_counter()
        if self.proc is not None:
            deadline = time.perf_counter() + 2.0
            while (not self.samples or self.samples[-1][0] <= self.t1) and time.perf_counter() < deadline:
                time.sleep(0.01)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        before = [i for i, (t, _) in enumerate(self.samples) if t <= self.t0]
        after = [i for i, (t, _) in enumerate(self.samples) if t > self.t1]
        lo = before[-1] if before else 0
        hi = after[0] if after else len(self.samples) - 1
        self.lines = [l for _, l in self.samples[lo:hi + 1]]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "window_ms": 1e3 * (self.t1 - self.t0)}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def _cpu_model():
    """CPU model string of this host (x86 'model name', or the Arm implementer / part ids)."""
    try:
        info = open("/proc/cpuinfo").read().splitlines()
    except OSError:
        return "unknown"
    fields = {}
    for line in info:
        if ":" in line:
            k, v = line.split(":", 1)
            fields.setdefault(k.strip(), v.strip())
    if "model name" in fields:
        return fields["model name"]
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return " ".join(f"{k} {fields[k]}" for k in ("CPU implementer", "CPU part") if k in fields) or "unknown"


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def _cube_sub_block(k, side=64):
    """Sub-block k (of the 8 octants of the cube, cycled) of the benchmark's cube as its own scene:
    32,768 particles of the 262,144."""
    sc = S.cube_3d(side=side)
    c = sc.x.mean(0)
    q = k % 8
    mask = np.ones(sc.n_particles, bool)
    for a in range(3):
        hi = (q >> a) & 1
        mask &= (sc.x[:, a] >= c[a]) if hi else (sc.x[:, a] < c[a])
    sub = sc.copy()
    sub.x, sub.v, sub.F, sub.C = sc.x[mask], sc.v[mask], sc.F[mask], sc.C[mask]
    sub.inst_offsets = np.array([0, int(mask.sum())])
    return sub


def _oracle_fom_task(args):
    """One worker of the CPU baseline: FP64 oracle steps of its own sub-block for ~seconds."""
    k, seconds, min_steps = args
    import oracle.mpm as OM
    sub = _cube_sub_block(k)
    t0 = time.perf_counter()
    steps = 0
    while steps < min_steps or time.perf_counter() - t0 < seconds:
        OM.step(sub, 1)
        steps += 1
    return sub.n_particles * steps, time.perf_counter() - t0


def _spawn_pool(n):
    """Process pool started with 'spawn' (safe after CUDA initialisation); one BLAS / OpenMP thread
    per worker, so that n workers use n cores."""
    import multiprocessing as mp
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    return mp.get_context("spawn").Pool(n)


def oracle_fom_throughput(n_procs, seconds):
    """Particle-steps/s of the FP64 oracle on n_procs host cores: each worker steps its own
    32,768-particle sub-block of the cube for ~seconds; the aggregate is the sum of the
    particle-steps over the longest worker's time."""
    with _spawn_pool(n_procs) as pool:
        res = pool.map(_oracle_fom_task, [(k, seconds, 1) for k in range(n_procs)], chunksize=1)
    work = sum(r[0] for r in res)
    wall = max(r[1] for r in res)
    return work / wall, work


def cpu_baseline_fom(sc, seconds=8.0):
    """The FP64 oracle as it stands, on bounded samples of the benchmark's cube: one core, then
    every host core (one process per core, each on its own 32,768-particle sub-block)."""
    one, _ = oracle_fom_throughput(1, seconds)
    cores = _host_cores()
    allc, _ = oracle_fom_throughput(cores, seconds)
    return {"value": allc, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": _cpu_model(),
            "single_core": {"value": one, "cores": 1},
            "sample": f"FP64 numpy oracle steps of 32,768-particle octants of the {sc.n_particles}-particle cube, "
                      f"~{seconds:.0f} s per worker; 'value' on all {cores} host cores (one process each), "
                      "'single_core' on one"}


# reduced-order leg (Sections 3-5): 2D neo-Hookean blocks of 4096 particles on 128^2 (dt = 5e-5,
# sticky walls, floor impact).  Training set: 32 trajectories with (E, v0) ~ U[5e3, 1.5e4] x
# U[-0.5, 0.5]^2, snapshots every 10 steps; test set: 4 held-out draws from the same box, each
# against its own full-order run.  The error is the accumulated relative position error of
# Section 5 after 2000 reduced steps (the step count of the reduced-order benchmark) and after
# 4000 (0.2 s, the same physical time as 2000 steps at dt = 1e-4).
ROM_STEPS = 4000
ROM_CHECKPOINT = 2000
ROM_TRAIN_STEPS = 12000
ROM_TRAIN_INSTANCES = 32
ROM_TESTS = 4
ENCODER_SUBSET = 1024
ROM_SETTINGS = dict(n_samples=256, gn_iters=3, projection=0, ridge=1e-1, affine=0, f_reference=1)
ROM_DECODER_FP32 = True     # reduced-step decoder calls in FP32 on the CUDA cores (training stays BF16)


def _rom_tests(steps, n_tests=ROM_TESTS):
    from paper_2109_12390_gb300 import pipeline as PL
    rng = np.random.default_rng(44)
    tests = []
    for _ in range(n_tests):
        E = float(rng.uniform(5e3, 1.5e4))
        v0 = rng.uniform(-0.5, 0.5, size=2)
        sc = S.block_2d(seed=4, side=64, dt=5e-5, origin=(0.375, 0.06), E=E, v0=v0)
        fx, rate, status = PL.fom_positions(sc, steps)
        tests.append(dict(scene=sc, fom=fx, fom_rate=rate, fom_status=status, E=E, v0=v0.tolist()))
    return tests


def cpu_baseline_rom(dec, sc, r, max_seconds=20.0):
    """The FP64 oracle's reduced step (Algorithms 2, 3, 5, 6), as it stands, with the trained
    decoder's parameters, on the first held-out scene: whole steps until ~max_seconds, one thread."""
    import torch
    import oracle.decoder as OD
    import oracle.rom as OR
    try:
        from threadpoolctl import threadpool_limits
        limiter = threadpool_limits(1)
    except Exception:  # pragma: no cover
        limiter = None
    p = S.xavier_decoder(0, sc.dim, r, 128, 5, OD.ELU)
    params = torch.empty(dec.n_params, dtype=torch.float32, device="cuda")
    norm = torch.empty(4 * sc.dim, dtype=torch.float32, device="cuda")
    dec.get_params(params, norm)
    torch.cuda.synchronize()
    flat = params.cpu().numpy().astype(np.float64)
    off = 0
    for l in range(len(p.W)):
        n = p.W[l].size
        p.W[l] = flat[off:off + n].reshape(p.W[l].shape)
        off += n
        n = p.b[l].size
        p.b[l] = flat[off:off + n]
        off += n
    nm = norm.cpu().numpy().astype(np.float64)
    d = sc.dim
    p.X_min, p.X_range, p.out_shift, p.out_scale = nm[:d], nm[d:2 * d], nm[2 * d:3 * d], nm[3 * d:]
    rs = OR.RomScene(X=sc.x.copy(), mass=sc.p_mass, vol=sc.p_vol, E=float(sc.E[0]), nu=float(sc.nu[0]), dx=sc.dx,
                     dt=sc.dt, n_grid=sc.n_grid, gravity=sc.gravity, bc=sc.bc, bc_width=sc.bc_width,
                     material=sc.material, transfer=sc.transfer, n_samples=ROM_SETTINGS["n_samples"], seed=4,
                     gn_iters=ROM_SETTINGS["gn_iters"], ridge=ROM_SETTINGS["ridge"])
    st = OR.RomState(xhat=np.zeros(r), vhat=np.zeros(r), xhat_prev=np.zeros(r))
    t0 = time.perf_counter()
    steps = 0
    while True:
        st = OR.rom_step(p, rs, st)
        steps += 1
        if time.perf_counter() - t0 > max_seconds or steps >= 5:
            break
    dt = time.perf_counter() - t0
    if limiter is not None and hasattr(limiter, "unregister"):
        limiter.unregister()
    return {"value": steps / dt, "unit": "ROM steps/s", "cores": 1, "kind": "oracle",
            "sample": f"{steps} FP64 oracle reduced step(s) of the first held-out scene, single thread"}


def rom_serving(dec, n_inst=8, steps=200):
    """Many independent reduced-order instances served concurrently, one CUDA stream and one
    captured step graph each (held-out (E, v0) draws of the same scene).  Returns the aggregate
    reduced steps/s over all instances and the per-step latency distribution."""
    import torch
    from paper_2109_12390_gb300.rom import ROM
    rng = np.random.default_rng(55)
    dec.set_concurrency(n_inst)   # fewer, fuller FP32 tiles per call: the instances share the SMs
    roms, streams = [], []
    for _ in range(n_inst):
        E = float(rng.uniform(5e3, 1.5e4))
        v0 = rng.uniform(-0.5, 0.5, size=2)
        sc = S.block_2d(seed=4, side=64, dt=5e-5, origin=(0.375, 0.06), E=E, v0=v0)
        rom = ROM.from_scene(dec, sc, seed=4, **{k: v for k, v in ROM_SETTINGS.items()})
        rom.fit_initial(sc.x, sc.v, iters=20)
        roms.append(rom)
        streams.append(torch.cuda.Stream())
    for rom, st in zip(roms, streams):
        rom.step(2, stream=st)            # graph capture outside the timed region
    torch.cuda.synchronize()
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
          for _ in range(n_inst)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_start.record()
    for st in streams:
        st.wait_event(t_start)
    for k in range(steps):
        for i, (rom, st) in enumerate(zip(roms, streams)):
            ev[i][k][0].record(st)
            rom.step(1, stream=st)
            ev[i][k][1].record(st)
    for st in streams:
        torch.cuda.current_stream().wait_stream(st)
    t_end.record()
    torch.cuda.synchronize()
    wall_ms = t_start.elapsed_time(t_end)
    lat = np.array([[a.elapsed_time(b) for a, b in ev[i]] for i in range(n_inst)]).ravel()
    status = [rom.status() for rom in roms]
    for rom in roms:
        rom.close()
    dec.set_concurrency(1)
    return {"instances": n_inst, "steps_each": steps, "aggregate_rom_steps_per_s": n_inst * steps / (wall_ms * 1e-3),
            "latency_ms_p50": float(np.percentile(lat, 50)), "latency_ms_p99": float(np.percentile(lat, 99)),
            "status_words": status, "how": "one CUDA stream and one captured step graph per instance"}


def rom_batch_serving(dec16, snaps, n_inst=384, steps=40, n_recon_inst=64):
    """Batched reduced-order serving: n_inst independent instances of the 2D block scene (held-out
    (E, v0) draws), sample sets uneven in 64..1024, latent size cycled over r = 8, 16, 32 (the
    trained r = 16 decoder; untrained Xavier decoders with the same scaling for r = 8 and 32, for
    timing), all stepped by one CUDA graph launch per step.  The decoders' FP32 tiling is chosen
    by the autotuner of the pipeline.  Reports the aggregate reduced steps/s, the per-step latency
    distribution (every instance advances one step per launch) and a BF16 reconstruction: one
    1,048,576-point decoder pass (4096 instance latents x 256 points) timed, and the full-particle
    BF16 reconstruction of the first r = 16 instances scored against their full-order runs."""
    import torch
    from paper_2109_12390_gb300 import pipeline as PL
    from paper_2109_12390_gb300.decoder import PRIMAL
    from paper_2109_12390_gb300.rom import ROM, metric_accumulate
    rng = np.random.default_rng(77)
    decs = {16: dec16}
    for r in (8, 32):
        decs[r], _ = PL.decoder_for_snapshots(snaps, r, seed=r)
        decs[r].set_precision(True)
    settings = {k: v for k, v in ROM_SETTINGS.items() if k != "n_samples"}
    roms, plan = [], []
    t0 = time.perf_counter()
    for i in range(n_inst):
        r = (8, 16, 32)[i % 3]
        k = int(rng.integers(64, 1025))
        E = float(rng.uniform(5e3, 1.5e4))
        v0 = rng.uniform(-0.5, 0.5, size=2)
        sc = S.block_2d(seed=4, side=64, dt=5e-5, origin=(0.375, 0.06), E=E, v0=v0)
        rom = ROM.from_scene(decs[r], sc, n_samples=k, seed=100 + i, **settings)
        rom.fit_initial(sc.x, sc.v, iters=20)
        roms.append(rom)
        plan.append((r, k, sc))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    (best_prec, best_k), tune = PL.autotune_serving(list(decs.values()), roms)
    batch = PL.build_serving_batch(list(decs.values()), roms, best_k, best_prec)
    batch.step(1)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in ev:
        a.record()
        batch.step(1)
        b.record()
    torch.cuda.synchronize()
    lat = np.array([a.elapsed_time(b) for a, b in ev])
    status = [rom.status() for rom in roms]
    n_steps_done = roms[0].get_state()[3]
    batch.close()
    # reconstruction: full-particle BF16 decode of the first r = 16 instances against their FOM runs
    for dec in decs.values():
        dec.set_precision(False)
    idx16 = [i for i, (r, _, _) in enumerate(plan) if r == 16][:n_recon_inst]
    acc = torch.zeros(2, dtype=torch.float64, device="cuda")
    for i in idx16:
        sc = plan[i][2]
        fx, _, _ = PL.fom_positions(sc, n_steps_done)
        xh = torch.from_numpy(roms[i].get_state()[0].astype(np.float32)[None]).cuda()
        Xg = torch.from_numpy(sc.x.astype(np.float32)).cuda()
        xr = dec16.eval(Xg, xh, [PRIMAL])[0]
        metric_accumulate(xr, fx[n_steps_done], acc)
    num, den = acc.cpu().numpy()
    # one 1,048,576-point BF16 decoder pass: 4096 latents (the r = 16 members' states, tiled) x 256
    lat16 = np.stack([roms[i].get_state()[0] for i in idx16]).astype(np.float32)
    lat_all = torch.from_numpy(np.resize(lat16, (4096, 16))).cuda()
    X0 = plan[idx16[0]][2].x.astype(np.float32)
    pts = torch.from_numpy(X0[rng.integers(0, len(X0), size=4096 * 256)]).cuda()
    lid = torch.arange(4096, dtype=torch.int32, device="cuda").repeat_interleave(256)
    out = dec16.eval(pts, lat_all, [PRIMAL], lat_idx=lid)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(5):
        dec16.eval(pts, lat_all, [PRIMAL], lat_idx=lid, out=out)
    b.record()
    torch.cuda.synchronize()
    recon_ms = a.elapsed_time(b) / 5
    flop_row = 2 * ((2 + 16) * 128 + 4 * 128 * 128 + 128 * 2)
    for dec in decs.values():
        dec.set_precision(True)
        dec.set_concurrency(1)
    for rom in roms:
        rom.close()
    for r in (8, 32):
        decs[r].close()
    return {"instances": n_inst, "latent_dims": [8, 16, 32], "samples_range": [64, 1024],
            "samples_mean": float(np.mean([k for _, k, _ in plan])), "steps": steps,
            "aggregate_rom_steps_per_s": n_inst * steps / (float(lat.sum()) * 1e-3),
            "batch_step_ms_p50": float(np.percentile(lat, 50)), "batch_step_ms_p99": float(np.percentile(lat, 99)),
            "status_words_nonzero_by_r": {r: int(sum(1 for w, (rr, _, _) in zip(status, plan) if w and rr == r))
                                          for r in (8, 16, 32)},
            "setup_seconds": setup_s,
            "reading": "the reduced step is throughput-bound on its FP32 decoder work (the batch step takes about "
                       "the sum of the instances' steps): one launch serves them all, it does not add concurrency",
            "autotune": {"chosen_precision": {1: "FP32 CUDA cores", 2: "split BF16 tensor cores"}[best_prec],
                         "chosen_concurrency": best_k, "ms_per_batch_step": tune,
                         "what": "precision/concurrency: square-layer arithmetic (1 FP32 CUDA cores, 2 split "
                                 "BF16 tensor cores) and decoder_set_concurrency (FP32 tiles per call), timed"},
            "how": "one CUDA graph launch per step: every instance's step graph a parallel branch",
            "decoders": "r = 16 trained; r = 8 and 32 untrained (Xavier, same scaling), timing only",
            "reconstruction": {"points": 4096 * 256, "bf16_ms": recon_ms,
                               "tflops": 4096 * 256 * flop_row / (recon_ms * 1e-3) / 1e12,
                               "rel_position_error_vs_fom": float(np.sqrt(num / den)),
                               "error_instances": len(idx16), "error_after_steps": int(n_steps_done),
                               "error_how": "full-particle BF16 decode of the r = 16 members vs their FOM runs"}}


def rom_large_p_3d(steps=5):
    """The reduced step where hyper-reduction is meant to pay: the 3D benchmark cube (262,144
    particles, 128^3) with the Eulerian quadrature (Algorithm 4, whose decoder work does not grow
    with the particle count) at 256 and 32 samples, the Lagrangian quadrature at 256, against the
    full-order step on the same scene.  The decoder is an untrained near-identity 3 + 16 -> 128 x 5
    -> 3 ELU network on the FP32 path: the reduced steps/s are timings, the error is not scored."""
    import torch
    import oracle.decoder as OD
    from paper_2109_12390_gb300.decoder import Decoder
    from paper_2109_12390_gb300.mpm import MPM
    from paper_2109_12390_gb300.rom import ROM
    sc = S.cube_3d()
    X = sc.x
    p = S.near_identity_decoder(3, 3, 16, 5, X_min=X.min(0) - 0.05, X_range=X.max(0) - X.min(0) + 0.1, eps=1e-3)
    dec = Decoder.from_params(p)
    dec.set_precision(True)
    ev = lambda: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    fom = MPM.from_scene(sc, polar_eft=HEADLINE_POLAR_EFT)
    fom.load_numpy(sc.x, sc.v, sc.F, sc.C)
    fom.step(5)
    a, b = ev()
    a.record()
    fom.step(50)
    b.record()
    torch.cuda.synchronize()
    fom_ms = a.elapsed_time(b) / 50
    fom.close()
    out = {"particles": sc.n_particles, "fom_steps_per_s": 1e3 / fom_ms, "decoder": "untrained near-identity, FP32",
           "runs": []}
    for quad, k in ((1, 256), (1, 32), (0, 256)):
        rom = ROM.from_scene(dec, sc, n_samples=k, seed=5, projection=0, quadrature=quad)
        rom.fit_initial(sc.x, sc.v, iters=5)
        rom.step(1)
        torch.cuda.synchronize()
        a, b = ev()
        a.record()
        rom.step(steps)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        run = {"quadrature": "eulerian" if quad else "lagrangian", "n_samples": k, "rom_steps_per_s": 1e3 / ms,
               "rom_ms_per_step": ms, "fom_over_rom": ms / fom_ms, "status_word": rom.status()}
        if quad:
            run["quadrature_points"] = int(rom.quadrature_points()["x"].shape[0])
        out["runs"].append(run)
        rom.close()
    dec.close()
    return out


def rom_leg(r=16, train_steps=None, steps=None):
    """Snapshots from the GPU full-order model, decoder training on the GPU, reduced-order runs on
    held-out scenes and their accumulated position error (Section 5) against the full-order runs;
    plus the gain of the trained network over an untrained one and over a trained linear manifold
    (the same network with identity activations)."""
    train_steps = ROM_TRAIN_STEPS if train_steps is None else train_steps
    steps = ROM_STEPS if steps is None else steps
    ck = min(ROM_CHECKPOINT, steps)
    import torch
    from paper_2109_12390_gb300 import pipeline as PL
    from paper_2109_12390_gb300.train import generate_snapshots
    train_sc = S.batch_2d(seed=3, n_inst=ROM_TRAIN_INSTANCES, fixed_side=64, n_grid=128, origin_y=0.06)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    snaps = generate_snapshots(train_sc, ROM_STEPS, 10)
    torch.cuda.synchronize()
    t_snap = time.perf_counter() - t0
    dec, _ = PL.decoder_for_snapshots(snaps, r, seed=0)
    tr, hist, t_train = PL.train(snaps, dec, steps=train_steps)
    loss = hist[-1][1]
    tr.close()
    dec.set_precision(ROM_DECODER_FP32)
    tests = _rom_tests(steps)
    per_test = []
    for t in tests:
        run = PL.rom_error(dec, t["scene"], t["fom"], seed=4, checkpoints=(ck,), **ROM_SETTINGS)
        per_test.append(dict(E=t["E"], v0=t["v0"], rel_error_at_checkpoint=run.error_percent_at[ck] / 100.0,
                             rel_error_full=run.error_percent / 100.0, rom_steps_per_s=run.rom_steps_per_s,
                             fom_steps_per_s=t["fom_rate"], rom_status_word=run.status,
                             fom_status_word=t["fom_status"]))
    err_ck = float(np.mean([q["rel_error_at_checkpoint"] for q in per_test]))
    err_full = float(np.mean([q["rel_error_full"] for q in per_test]))
    rom_rate = float(np.mean([q["rom_steps_per_s"] for q in per_test]))
    fom_rate = float(np.mean([q["fom_steps_per_s"] for q in per_test]))
    # gain of the network: untrained decoder and trained linear manifold, first test, same settings
    t0s = tests[0]
    fx_ck = t0s["fom"][:ck + 1]
    untrained, _ = PL.decoder_for_snapshots(snaps, r, seed=0)
    untrained.set_precision(ROM_DECODER_FP32)
    e_untrained = PL.rom_error(untrained, t0s["scene"], fx_ck, seed=4, **ROM_SETTINGS).error_percent / 100.0
    lin, _ = PL.decoder_for_snapshots(snaps, r, seed=0, activation=1)
    trl, histl, t_lin = PL.train(snaps, lin, steps=max(1, train_steps // 4))
    trl.close()
    lin.set_precision(ROM_DECODER_FP32)
    e_linear = PL.rom_error(lin, t0s["scene"], fx_ck, seed=4, **ROM_SETTINGS).error_percent / 100.0
    # Eulerian quadrature (Algorithm 4) on the first test: it has no particle ids at its points, so
    # no reference-gradient correction; the Lagrangian quadrature without it is the like-for-like
    eul_settings = dict(ROM_SETTINGS, f_reference=0)
    e_eul = PL.rom_error(dec, t0s["scene"], t0s["fom"], seed=4, checkpoints=(ck,), quadrature=1, **eul_settings)
    e_lag = PL.rom_error(dec, t0s["scene"], t0s["fom"], seed=4, checkpoints=(ck,), **eul_settings)
    eulerian = {"rel_error_at_checkpoint": e_eul.error_percent_at[ck] / 100.0,
                "rel_error_full": e_eul.error_percent / 100.0, "rom_steps_per_s": e_eul.rom_steps_per_s,
                "status_word": e_eul.status, "ell": 2, "newton_iters": 4,
                "lagrangian_same_settings": {"rel_error_at_checkpoint": e_lag.error_percent_at[ck] / 100.0,
                                             "rel_error_full": e_lag.error_percent / 100.0,
                                             "rom_steps_per_s": e_lag.rom_steps_per_s},
                "settings": eul_settings, "steps": ck}
    # decoder trained with the encoder of Section 4.1 (1024 of the 4096 particles per snapshot) in
    # place of the latent table, same steps and settings; first test
    enc_dec, _ = PL.decoder_for_snapshots(snaps, r, seed=0)
    tre, histe, t_enc = PL.train(snaps, enc_dec, steps=train_steps, encoder_subset=ENCODER_SUBSET)
    tre.close()
    enc_dec.set_precision(ROM_DECODER_FP32)
    e_enc = PL.rom_error(enc_dec, t0s["scene"], t0s["fom"], seed=4, checkpoints=(ck,), **ROM_SETTINGS)
    encoder = {"subset": ENCODER_SUBSET, "training_steps": train_steps, "training_seconds": t_enc,
               "ms_per_step": 1e3 * t_enc / train_steps, "final_loss": histe[-1][1],
               "rel_error_at_checkpoint": e_enc.error_percent_at[ck] / 100.0,
               "rel_error_full": e_enc.error_percent / 100.0, "status_word": e_enc.status, "steps": ck,
               "latent_table_same_test": per_test[0]["rel_error_at_checkpoint"]}
    # the paper's plain settings (least squares without the ridge, no reference gradient) beside
    # the tuned ones, same decoder, first test
    plain_settings = dict(ROM_SETTINGS, ridge=0.0, f_reference=0)
    e_plain = PL.rom_error(dec, t0s["scene"], t0s["fom"], seed=4, checkpoints=(ck,), **plain_settings)
    fin = lambda v: float(v) if np.isfinite(v) else None
    plain = {"settings": plain_settings, "rel_error_at_checkpoint": fin(e_plain.error_percent_at.get(ck, np.nan) / 100.0),
             "rel_error_full": fin(e_plain.error_percent / 100.0), "status_word": e_plain.status,
             "tuned_same_test": {"rel_error_at_checkpoint": per_test[0]["rel_error_at_checkpoint"],
                                 "rel_error_full": per_test[0]["rel_error_full"]}}
    cpu = cpu_baseline_rom(dec, tests[0]["scene"], r)
    serving = rom_serving(dec, n_inst=8, steps=min(200, steps))
    batched_serving = rom_batch_serving(dec, snaps)
    large_p = rom_large_p_3d()
    return {
        "cpu_baseline": cpu,
        "serving": serving,
        "batched_serving": batched_serving,
        "large_p_3d": large_p,
        "scene": "2D neo-Hookean block 64x64 (4096 particles), 128^2 grid, nu=0.3, dt=5e-5, sticky walls, floor "
                 f"impact; decoder 2+{r}->128x5->2 ELU trained on {ROM_TRAIN_INSTANCES} trajectories, "
                 f"(E, v0) ~ U[5e3,1.5e4] x U[-0.5,0.5]^2; {len(tests)} held-out test draws",
        "rom_steps_per_s": rom_rate, "fom_steps_per_s": fom_rate, "speedup": rom_rate / fom_rate,
        "rel_position_error": err_ck, "error_steps": ck, "rel_position_error_full": err_full, "full_steps": steps,
        "meets_1e-2": {f"at_{ck}_steps_{ck * 5e-5:.2f}s": bool(err_ck <= 1e-2),
                       f"at_{steps}_steps_{steps * 5e-5:.2f}s": bool(err_full <= 1e-2)},
        "paper_plain_settings": plain,
        "per_test": per_test,
        "settings": dict(ROM_SETTINGS, latent_dim=r, decoder="FP32 CUDA cores" if ROM_DECODER_FP32 else "BF16 tcgen05"),
        "gain": {"trained": per_test[0]["rel_error_at_checkpoint"], "untrained_xavier": e_untrained,
                 "trained_linear_manifold": e_linear, "linear_training_steps": max(1, train_steps // 4),
                 "steps": ck},
        "eulerian_quadrature": eulerian,
        "encoder": encoder,
        "training": {"steps": train_steps, "batch_points": 65536, "seconds": t_train,
                     "points_per_s": train_steps * 65536 / t_train, "ms_per_step": 1e3 * t_train / train_steps,
                     "final_loss": loss, "snapshot_seconds": t_snap, "snapshots": int(snaps["n_snap"])},
    }


_SUB_CACHE = {}


def _oracle_fom_step_task(k):
    """One oracle step of sub-block k, whose state this worker keeps between calls."""
    import oracle.mpm as OM
    if k not in _SUB_CACHE:
        _SUB_CACHE[k] = _cube_sub_block(k)
    sub = _SUB_CACHE[k]
    t0 = time.perf_counter()
    OM.step(sub, 1)
    return sub.n_particles, time.perf_counter() - t0


def run_reference(args, ws, rank):
    """The FP64 oracle on every host core: one timed step is one oracle step of each worker's own
    32,768-particle octant of the cube, all workers at once (a bounded sample of the workload)."""
    if rank != 0:
        return
    cores = _host_cores()
    times, work = [], 0
    with _spawn_pool(cores) as pool:
        for i in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            res = pool.map(_oracle_fom_step_task, range(cores), chunksize=1)
            dt = time.perf_counter() - t0
            if i >= args.warmup:
                times.append(dt)
                work += sum(r[0] for r in res)
    per = float(np.mean(times))
    value = work / float(np.sum(times))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": f"one FP64 oracle step of a 32,768-particle octant per "
                                                      f"host core ({cores} cores) per timed step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": _cpu_model(),
                             "sample": f"{cores} processes, each stepping its own 32,768-particle octant of the "
                                       "cube with the FP64 numpy oracle"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batched_snapshot_leg(dev, steps=400, every=10):
    """16 instances of the 2D block with particle counts uneven in 20k-120k and (E, v0) drawn from a
    seeded box, on a 256^2 grid, stepped together in one context (one launch per kernel per step
    for all instances), positions of every 10th step copied into a device snapshot store.
    Returns particle-steps/s over `steps` steps with the snapshot copies inside the timing."""
    import torch
    from paper_2109_12390_gb300.mpm import MPM
    sc = S.batch_2d(seed=3)
    P = sc.n_particles
    ctx = MPM.from_scene(sc)
    ctx.load_numpy(sc.x, sc.v, sc.F, sc.C)
    J = steps // every
    xs = torch.empty((J, P, 2), dtype=torch.float32, device=dev)
    ctx.step(every)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for j in range(J):
        ctx.step(every)
        ctx.get_state(xs[j])
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    out = {"instances": sc.n_inst, "particles": P,
           "counts": [int(c) for c in np.diff(sc.inst_offsets)], "grid": "256^2", "steps": steps,
           "snapshot_every": every, "ms_per_step": ms / steps, "particle_steps_per_s": P * steps / (ms * 1e-3),
           "status_word": ctx.status(), "how": "CUDA events around all steps and snapshot copies"}
    ctx.close()
    return out


def run_ours(args, ws, rank, local):
    import torch
    from paper_2109_12390_gb300.mpm import MPM

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    sc = S.cube_3d()
    P = sc.n_particles
    ctx = MPM.from_scene(sc, polar_eft=HEADLINE_POLAR_EFT)
    stream = torch.cuda.current_stream()
    ctx.load_numpy(sc.x, sc.v, sc.F, sc.C)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    # untimed pre-roll: the cube falls onto the slip floor, so that the timed steps are in contact
    ctx.step(PRE_ROLL)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    ctx.step_profiled(args.warmup, flush=flush)
    assert ctx.status() == 0, "unstable state during warm-up"
    barrier()
    with Clocks(local) as clk:
        # all K steps enqueued at once, events at the step boundaries on the launching stream (none
        # between a step's kernels); the L2 flush runs between steps, outside the timed intervals
        step_ms = ctx.step_timed(args.steps, flush=flush)
    barrier()
    # the K steps that follow, with events around every kernel: the kernel durations of the roofline
    kern = ctx.step_profiled(args.steps, flush=flush)
    torch.cuda.synchronize()
    status = ctx.status()
    total_ms = float(np.sum(step_ms))
    from paper_2109_12390_gb300.dist import max_over_ranks
    total_ms = max_over_ranks(total_ms, device=dev)
    fused_ms = float(kern[:, 0].mean())
    peak, peak_kind = _peaks()
    achieved = ALGO_BYTES_3D * P / (fused_ms * 1e-3) / 1e9

    # the same workload with the compensated-FP32 rotation correction of the polar factor, and a
    # scaled-up cube (2,097,152 particles on 256^3, working set far above L2)
    variants = {}
    plastic = sc.copy()
    plastic.material = 2   # plastic fixed-corotated (singular values clamped), second workload
    other = 1 - HEADLINE_POLAR_EFT
    extra = () if args.profile else ((("polar_eft" if other else "polar_fp64"), sc, other, PRE_ROLL),
                                     ("cube_2M_256", S.cube_3d(side=128, n_grid=256, dt=2.5e-5), HEADLINE_POLAR_EFT, 0),
                                     ("plastic_cube", plastic, HEADLINE_POLAR_EFT, PRE_ROLL))
    for name, vsc, eft, pre in extra:
        vctx = MPM.from_scene(vsc, polar_eft=eft)
        vctx.load_numpy(vsc.x, vsc.v, vsc.F, vsc.C)
        vctx.step(pre)
        vctx.step_profiled(args.warmup, flush=flush)
        vs = vctx.step_timed(min(args.steps, 20), flush=flush)
        vk = vctx.step_profiled(min(args.steps, 20), flush=flush)
        vf = float(vk[:, 0].mean())
        variants[name] = {"particles": vsc.n_particles, "polar": "compensated FP32" if eft else "FP64",
                          "ms_per_step": float(vs.mean()), "fused_ms": vf, "pre_roll_steps": pre,
                          "particle_steps_per_s": vsc.n_particles / (float(vs.mean()) * 1e-3),
                          "fused_gbs": ALGO_BYTES_3D * vsc.n_particles / (vf * 1e-3) / 1e9,
                          "status_word": vctx.status(), "material": int(vsc.material)}
        variants[name]["fused_frac"] = variants[name]["fused_gbs"] / _peaks()[0]
        vctx.close()

    # batched snapshot generation (16 uneven 2D instances of 20k-120k particles on 256^2 in one
    # context, every 10th step's positions stored on the device)
    if not args.profile:
        variants["batched_16_uneven_2d"] = batched_snapshot_leg(dev)

    # end to end through the public API: pinned host state in, one step, state out
    d = sc.dim
    hx = torch.from_numpy(sc.x.astype(np.float32)).pin_memory()
    hv = torch.from_numpy(sc.v.astype(np.float32)).pin_memory()
    hF = torch.from_numpy(sc.F.astype(np.float32).reshape(P, d * d)).pin_memory()
    hC = torch.from_numpy(sc.C.astype(np.float32).reshape(P, d * d)).pin_memory()
    ox, ov, oF, oC = [torch.empty_like(t).pin_memory() for t in (hx, hv, hF, hC)]
    e2e_ms = []
    for i in range(0 if args.profile else args.warmup + args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.set_state(hx, hv, hF, hC)
        ctx.step(1)
        ctx.get_state(ox, ov, oF, oC)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_total = float(np.sum(e2e_ms)) if e2e_ms else float("nan")
    e2e_total = max_over_ranks(e2e_total, device=dev)
    bytes_io = 4 * P * (2 * d + 2 * d * d)

    if rank == 0:
        line = {
            "metric": METRIC, "value": ws * P * args.steps / (total_ms * 1e-3), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "particles": P, "grid": "128^3", "l2": "flushed before every timed step",
                       "timed_steps": f"{PRE_ROLL + args.warmup + 1}..{PRE_ROLL + args.warmup + args.steps} "
                                      "(after an untimed pre-roll to the slip-floor contact)",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": FUSED_DRAM_BYTES_NCU, "kernel": "mpm_g2p2g",
                         "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                         "algorithmic_bytes_per_launch": ALGO_BYTES_3D * P, "kernel_ms": fused_ms},
            "kernels_ms": {"mpm_g2p2g": fused_ms, "mpm_scan": float(kern[:, 1].mean()),
                           "mpm_permute": float(kern[:, 2].mean()),
                           "how": "CUDA events around each kernel over the K steps after the timed region"},
            "e2e": None if args.profile else {"value": ws * P * args.steps / (e2e_total * 1e-3), "unit": UNIT,
                                              "h2d_bytes_per_step": bytes_io, "d2h_bytes_per_step": bytes_io},
            "variants": variants,
            "gpu_launches": 3 * args.steps,
            "clocks": clk.summary(),
            "status_word": status,
        }
        if not (args.no_cpu_baseline or args.profile):
            line["cpu_baseline"] = cpu_baseline_fom(sc)
        if not (args.no_rom or args.profile):
            line["rom"] = rom_leg(train_steps=args.rom_train_steps, steps=args.rom_steps)
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-rom", action="store_true", help="skip the reduced-order leg (training + ROM run)")
    ap.add_argument("--rom-train-steps", type=int, default=ROM_TRAIN_STEPS, help="decoder training steps")
    ap.add_argument("--rom-steps", type=int, default=ROM_STEPS, help="reduced-order (and full-order) steps")
    ap.add_argument("--profile", action="store_true",
                    help="only the warm-up and the timed steps (for profiler launch lists)")
    args = ap.parse_args()
    ws, rank, local = _dist()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
