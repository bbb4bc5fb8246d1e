"""GPU decoder training (Section 4.2 loss, Appendix B Adam) against the FP64 oracle via the C ABI.

Gradients of one minibatch (the GPU's own draw, handed to the oracle) are compared per
parameter block at 2e-2 relative norm-wise (BF16 tensor-core GEMMs, FP32 accumulation).
"""
import numpy as np
import pytest

import oracle.decoder as OD
import synth.scenes as S

pytestmark = pytest.mark.gpu
TOL = 2e-2


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def _store(d=2, n_inst=2, J=5, side=8, seed=0):
    """Synthetic snapshot store (random smooth-ish targets) in the snapshot_desc layout."""
    import torch
    rng = np.random.default_rng(seed)
    sc = S.batch_2d(seed=seed, n_inst=n_inst, fixed_side=side) if d == 2 else None
    X = sc.x
    P = len(X)
    xs = X[None] + 0.01 * rng.normal(size=(J, P, d))
    vs = rng.normal(size=(J, P, d))
    Fs = np.eye(d)[None, None] + 0.05 * rng.normal(size=(J, P, d, d))
    S_ = J * n_inst
    snaps = dict(dim=d, n_inst=n_inst, inst_offsets=np.ascontiguousarray(sc.inst_offsets, np.int64),
                 X=torch.from_numpy(X.astype(np.float32)).cuda(), n_snap=S_,
                 snap_inst=np.array([s % n_inst for s in range(S_)], np.int32),
                 snap_next=np.array([s + n_inst if s + n_inst < S_ else -1 for s in range(S_)], np.int32),
                 x=torch.from_numpy(xs.reshape(-1, d).astype(np.float32)).cuda(),
                 v=torch.from_numpy(vs.reshape(-1, d).astype(np.float32)).cuda(),
                 F=torch.from_numpy(Fs.reshape(-1, d * d).astype(np.float32)).cuda())
    host = dict(X=X, x=xs, v=vs, F=Fs, P=P, J=J)
    return snaps, host


def _oracle_batch(host, snaps, bs, bp):
    n_inst = snaps["n_inst"]
    offs = snaps["inst_offsets"]
    j = bs // n_inst
    inst = bs % n_inst
    pidx = offs[inst] + bp
    f32 = lambda a: a.astype(np.float32).astype(np.float64)
    return {"X": f32(host["X"][pidx]), "snap": bs.astype(np.int64),
            "next": snaps["snap_next"][bs].astype(np.int64),
            "x": f32(host["x"][j, pidx]), "F": f32(host["F"][j, pidx]), "v": f32(host["v"][j, pidx])}


def test_gradients_match_oracle():
    from paper_2109_12390_gb300.decoder import Decoder
    from paper_2109_12390_gb300.train import Trainer
    d, r = 2, 8
    snaps, host = _store(d)
    X = host["X"]
    p = S.xavier_decoder(1, d, r, 128, 5, OD.ELU, X_min=X.min(0), X_range=X.max(0) - X.min(0),
                         out_shift=X.mean(0), out_scale=np.full(d, 0.1), bias_scale=0.2)
    dec = Decoder.from_params(p)
    lat0 = 0.5 * np.random.default_rng(3).normal(size=(snaps["n_snap"], r)).astype(np.float32)
    lamF, lamv, dts = 3.0, 0.05, 0.01
    tr = Trainer(dec, snaps, lambda_F=lamF, lambda_v=lamv, dt_snap=dts, batch=1000, total_steps=10, latents0=lat0)
    gp, gl, bs, bp, loss = tr.gradients()
    batch = _oracle_batch(host, snaps, bs, bp)
    pf = p.copy()
    for l in range(len(pf.W)):
        pf.W[l] = pf.W[l].astype(np.float32).astype(np.float64)
        pf.b[l] = pf.b[l].astype(np.float32).astype(np.float64)
    L, gW, gb, glat = OD.batch_loss_grads(pf, lat0.astype(np.float64), batch, np.float32(dts), lamF, lamv)
    assert loss == pytest.approx(L, rel=TOL)
    off = 0
    for l in range(len(pf.W)):
        nW = pf.W[l].size
        assert rel(gp[off:off + nW].reshape(pf.W[l].shape), gW[l]) < TOL, ("W", l)
        off += nW
        nb = pf.b[l].size
        assert rel(gp[off:off + nb], gb[l]) < TOL, ("b", l)
        off += nb
    assert rel(gl, glat) < TOL


def test_adam_first_step_and_loss_decrease():
    from paper_2109_12390_gb300.decoder import Decoder
    from paper_2109_12390_gb300.train import Trainer
    d, r = 2, 8
    snaps, host = _store(d, seed=4)
    X = host["X"]
    p = S.xavier_decoder(2, d, r, 128, 5, OD.ELU, X_min=X.min(0), X_range=X.max(0) - X.min(0),
                         out_shift=X.mean(0), out_scale=np.full(d, 0.05))
    dec = Decoder.from_params(p)
    tr = Trainer(dec, snaps, lambda_F=1.0, lambda_v=0.01, dt_snap=0.01, batch=2048, total_steps=300,
                 lr0=1e-3, lr1=1e-4, latents0=np.zeros((snaps["n_snap"], r), np.float32))
    gp, _, _, _, loss0 = tr.gradients()
    before = np.empty(dec.n_params, np.float32)
    dec.get_params(before, None)
    tr.step(1)
    after = np.empty(dec.n_params, np.float32)
    dec.get_params(after, None)
    import torch
    torch.cuda.synchronize()
    # Adam's first step is -lr g / (|g| + eps): -lr sign(g) where |g| >> eps
    big = np.abs(gp) > 1e-5
    np.testing.assert_allclose((after - before)[big], -1e-3 * np.sign(gp[big]), rtol=1e-3, atol=2e-7)
    tr.step(299)
    loss1, step = tr.loss()
    assert step == 300
    assert tr.status() == 0
    assert loss1 < 0.5 * loss0


def test_fit_scaling_matches_appendix_b_definition():
    """decoder_fit_scaling (Appendix B min-max of X, mean / population std of the snapshot
    positions) against the oracle's definition on the same FP32 values, over a store with
    uneven instances; then the decoder's outputs use exactly that scaling."""
    import torch
    from paper_2109_12390_gb300.decoder import Decoder, PRIMAL
    sc = S.batch_2d(seed=5, n_inst=3)
    d, P = 2, sc.n_particles
    rng = np.random.default_rng(5)
    J = 3
    xs = sc.x[None] + 0.02 * rng.normal(size=(J, P, d)) + np.array([0.1, -0.05])
    snaps = dict(dim=d, n_inst=3, inst_offsets=np.ascontiguousarray(sc.inst_offsets, np.int64),
                 X=torch.from_numpy(sc.x.astype(np.float32)).cuda(), n_snap=J * 3,
                 snap_inst=np.array([s % 3 for s in range(J * 3)], np.int32),
                 snap_next=np.array([s + 3 if s + 3 < J * 3 else -1 for s in range(J * 3)], np.int32),
                 x=torch.from_numpy(xs.reshape(-1, d).astype(np.float32)).cuda(), v=None, F=None)
    p = S.xavier_decoder(1, d, 4, 128, 2, OD.ELU)
    dec = Decoder.from_params(p)
    dec.fit_scaling(snaps)
    norm = torch.empty(4 * d, dtype=torch.float32, device="cuda")
    dec.get_params(None, norm)
    got = norm.cpu().numpy().astype(np.float64)
    want = np.concatenate(OD.appendix_b_scaling(sc.x.astype(np.float32), xs.reshape(-1, d).astype(np.float32)))
    # min of FP32 values is exact; the range max - min is one FP32 rounding of its exact value
    np.testing.assert_array_equal(got[:2 * d], want[:2 * d].astype(np.float32))
    assert rel(got[2 * d:], want[2 * d:]) < 1e-6          # FP64 sums, one FP32 rounding
    p.X_min, p.X_range, p.out_shift, p.out_scale = want[:d], want[d:2 * d], want[2 * d:3 * d], want[3 * d:]
    X = sc.x[:64].astype(np.float32)
    xh = rng.normal(size=4).astype(np.float32)
    out = dec.eval(torch.from_numpy(X).cuda(), torch.from_numpy(xh[None]).cuda(), [PRIMAL]).cpu().numpy()[0]
    ref = OD.decode(p, X.astype(np.float64), xh.astype(np.float64))
    assert rel(out, ref) < TOL
    dec.close()


def test_data_parallel_shards_sum_to_the_whole_minibatch():
    """Data-parallel training on one GPU, the all-reduce done by hand: two shard trainers (shard_index
    0 and 1 of 2, 1024 points each) draw the two halves of the 2048-point minibatch of an unsharded
    trainer; the sum of their gradients is the unsharded gradient (FP32 summation order only), and
    after both apply the summed gradients the two replicas are bit-identical and moved as the
    unsharded trainer's one step."""
    import torch
    from paper_2109_12390_gb300.decoder import Decoder
    from paper_2109_12390_gb300.train import Trainer
    d, r = 2, 8
    snaps, host = _store(d, seed=6)
    X = host["X"]
    p = S.xavier_decoder(3, d, r, 128, 5, OD.ELU, X_min=X.min(0), X_range=X.max(0) - X.min(0),
                         out_shift=X.mean(0), out_scale=np.full(d, 0.1), bias_scale=0.2)
    lat0 = 0.5 * np.random.default_rng(7).normal(size=(snaps["n_snap"], r)).astype(np.float32)
    kw = dict(lambda_F=3.0, lambda_v=0.05, dt_snap=0.01, total_steps=10, latents0=lat0, seed=11)
    dec_full = Decoder.from_params(p)
    full = Trainer(dec_full, snaps, batch=2048, **kw)
    gp, gl, _, _, loss_full = full.gradients()
    decs = [Decoder.from_params(p) for _ in range(2)]
    shards = [Trainer(dk, snaps, batch=1024, shard_index=k, shard_count=2, **kw) for k, dk in enumerate(decs)]
    bufs = [t.gradient_buffers() for t in shards]
    for t, (g0, g1) in zip(shards, bufs):
        t.compute_gradients(g0, g1)
    s0 = bufs[0][0] + bufs[1][0]
    s1 = bufs[0][1] + bufs[1][1]
    torch.cuda.synchronize()
    assert rel(s0.cpu().numpy(), gp) < 1e-5
    assert rel(s1.cpu().numpy(), gl.ravel()) < 1e-5
    assert sum(t.loss()[0] for t in shards) == pytest.approx(loss_full, rel=1e-6)
    before = np.empty(dec_full.n_params, np.float32)
    dec_full.get_params(before, None)
    for t in shards:
        t.apply_gradients(s0, s1)
    full.step(1)
    after = [np.empty(dec_full.n_params, np.float32) for _ in range(3)]
    for dk, a in zip(decs + [dec_full], after):
        dk.get_params(a, None)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(after[0], after[1])
    assert rel(after[0] - before, after[2] - before) < 1e-3      # Adam's first step is -lr sign(g)
    for t in shards:
        assert t.loss()[1] == 1 and t.status() == 0
    np.testing.assert_array_equal(shards[0].latents(), shards[1].latents())


def test_instance_sharded_snapshots_match_the_whole_batch():
    """Batched snapshot generation sharded by whole instances (dist.scene_shard), the shards run one
    after the other on this GPU as two ranks would run them: concatenated in rank order, the
    snapshots equal those of the whole batch in one context up to the order of float atomics (the
    bound is ten times the difference between two runs of the whole batch, at least 1e-6 of the
    state's scale)."""
    import torch
    from paper_2109_12390_gb300.dist import scene_shard
    from paper_2109_12390_gb300.train import generate_snapshots
    sc = S.batch_2d(seed=9, n_inst=5, count_range=(3000, 9000), n_grid=128, origin_y=0.06)
    steps, every = 200, 50
    J = steps // every + 1
    full = generate_snapshots(sc, steps, every)
    twin = generate_snapshots(sc, steps, every)
    assert full["status"] == 0
    parts = [generate_snapshots(scene_shard(sc, r, 2)[0], steps, every) for r in range(2)]
    for key, c in (("x", 2), ("v", 2), ("F", 4)):
        cat = torch.cat([p[key].reshape(J, -1, c) for p in parts], dim=1).reshape(-1, c).cpu().numpy()
        ref = full[key].cpu().numpy()
        noise = np.abs(twin[key].cpu().numpy() - ref).max()
        scale = np.abs(ref).max()
        assert np.abs(cat - ref).max() <= max(10 * noise, 1e-6 * scale), key
