"""GPU encoder (Section 4.1, Table 1) trained with the decoder, against the FP64 oracle via the C ABI.

* latents of every snapshot: 1e-5 relative (FP32 convolutions and fully connected layers);
* encoder parameter gradients, given the GPU's own per-snapshot latent gradients: 1e-4 relative
  per parameter block (FP32 sums over snapshots and positions);
* the decoder gradients with encoder latents: 2e-2 (BF16 tensor-core GEMMs, as in the table case).
"""
import numpy as np
import pytest

import oracle.decoder as OD
import oracle.encoder as OE
import synth.scenes as S
from test_gpu_train import _oracle_batch, _store

pytestmark = pytest.mark.gpu
N_SUB = 200


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def _setup(seed=0, r=8):
    from paper_2109_12390_gb300.decoder import Decoder
    from paper_2109_12390_gb300.train import Trainer
    d = 2
    snaps, host = _store(d, n_inst=2, J=5, side=16, seed=seed)
    X = host["X"]
    p = S.xavier_decoder(1, d, r, 128, 5, OD.ELU, X_min=X.min(0), X_range=X.max(0) - X.min(0),
                         out_shift=X.mean(0), out_scale=np.full(d, 0.1), bias_scale=0.2)
    dec = Decoder.from_params(p)
    tr = Trainer(dec, snaps, lambda_F=3.0, lambda_v=0.05, dt_snap=0.01, batch=1000, total_steps=50,
                 encoder_subset=N_SUB, seed=7)
    return snaps, host, p, dec, tr


def _snapshot_positions(snaps, host):
    """(n_snap, P_inst, d) positions of every snapshot (all instances here have the same size)."""
    n_inst, offs = snaps["n_inst"], snaps["inst_offsets"]
    out = []
    for s in range(snaps["n_snap"]):
        j, inst = s // n_inst, s % n_inst
        out.append(host["x"][j, offs[inst]:offs[inst + 1]])
    return np.stack(out)


def _oracle_encoder(tr, d, r):
    vec, ss = tr.encoder_params()
    tmpl = OE.xavier_encoder(0, d, r, N_SUB)
    enc = OE.unflatten(tmpl, vec.astype(np.float64))
    enc.shift, enc.scale = ss[:d].astype(np.float64), ss[d:].astype(np.float64)
    return enc, vec


def test_encoder_latents_match_oracle():
    snaps, host, p, dec, tr = _setup()
    d, r = 2, dec.r
    enc, _ = _oracle_encoder(tr, d, r)
    xs = _snapshot_positions(snaps, host)
    # standardisation: mean and standard deviation of the subset positions over all snapshots
    ids = OE.subset_ids(xs.shape[1], N_SUB)
    sub = xs[:, ids].astype(np.float32).astype(np.float64)
    np.testing.assert_allclose(enc.shift, sub.reshape(-1, d).mean(0), rtol=1e-5)
    np.testing.assert_allclose(enc.scale, sub.reshape(-1, d).std(0), rtol=1e-4)
    ref = OE.encode(enc, sub)
    got = tr.encode(xs.astype(np.float32))
    assert rel(got, ref) < 1e-5
    tr.gradients()   # one forward of the training step fills the per-snapshot latents
    assert rel(tr.latents(), ref) < 1e-5
    assert enc.lengths == [2 * N_SUB, 198, 97, 46]


def test_encoder_gradients_match_oracle():
    snaps, host, p, dec, tr = _setup(seed=1)
    d, r = 2, dec.r
    # non-zero biases so that every gradient block is exercised
    vec, ss = tr.encoder_params()
    rng = np.random.default_rng(5)
    enc0 = OE.unflatten(OE.xavier_encoder(0, d, r, N_SUB), vec.astype(np.float64))
    enc0.conv_b = 0.2 * rng.normal(size=len(enc0.conv_w))
    enc0.b1 = 0.2 * rng.normal(size=32)
    tr.set_encoder_params(OE.flatten(enc0).astype(np.float32))
    enc, _ = _oracle_encoder(tr, d, r)
    xs = _snapshot_positions(snaps, host)
    ids = OE.subset_ids(xs.shape[1], N_SUB)
    u = OE.encoder_input(enc, xs[:, ids].astype(np.float32).astype(np.float64))
    gp, gl, bs, bp, loss = tr.gradients()
    ge = tr.last_encoder_gradients
    ref = OE.vjp(enc, u, gl.astype(np.float64))
    o = 0
    for l in range(len(enc.conv_w)):
        assert rel(ge[o:o + 6], ref["conv_w"][l]) < 1e-4, ("conv w", l)
        assert rel(ge[o + 6:o + 7], [ref["conv_b"][l]]) < 1e-4, ("conv b", l)
        o += 7
    for key in ("W1", "b1", "W2", "b2"):
        n = ref[key].size
        assert rel(ge[o:o + n], ref[key].ravel()) < 1e-4, key
        o += n
    assert o == len(ge)
    # the decoder's gradients with the encoder's latents (the integration of the two)
    lat = OE.forward(enc, u)
    batch = _oracle_batch(host, snaps, bs, bp)
    pf = p.copy()
    for l in range(len(pf.W)):
        pf.W[l] = pf.W[l].astype(np.float32).astype(np.float64)
        pf.b[l] = pf.b[l].astype(np.float32).astype(np.float64)
    L, gW, gb, glat = OD.batch_loss_grads(pf, lat, batch, np.float32(0.01), 3.0, 0.05)
    assert loss == pytest.approx(L, rel=2e-2)
    assert rel(gl, glat) < 2e-2


def test_training_with_encoder_reduces_loss():
    snaps, host, p, dec, tr = _setup(seed=2)
    tr.step(1)
    l0, _ = tr.loss()
    vec0, _ = tr.encoder_params()
    tr.step(49)
    l1, step = tr.loss()
    vec1, _ = tr.encoder_params()
    assert step == 50 and tr.status() == 0
    assert np.isfinite(l1) and l1 < l0
    assert np.abs(vec1 - vec0).max() > 0      # Adam moves the encoder, not a table


def test_encoder_arguments():
    from paper_2109_12390_gb300 import _abi
    from paper_2109_12390_gb300.decoder import Decoder
    from paper_2109_12390_gb300.train import Trainer
    snaps, host, p, dec, tr = _setup(seed=3)
    assert tr.encode(np.zeros((0, 256, 2), np.float32)).shape == (0, dec.r)
    with pytest.raises(_abi.MpmError):
        Trainer(dec, snaps, dt_snap=0.01, batch=100, total_steps=1, encoder_subset=257)   # larger than an instance
    with pytest.raises(_abi.MpmError):
        Trainer(dec, snaps, dt_snap=0.01, batch=100, total_steps=1, encoder_subset=8)     # 2 x 8 < 32 inputs
    table = Trainer(dec, snaps, dt_snap=0.01, batch=100, total_steps=1)
    with pytest.raises(_abi.MpmError):
        table.encoder_params()                                                            # no encoder
