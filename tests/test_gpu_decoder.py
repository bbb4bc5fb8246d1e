"""GPU parity of the decoder g(X; xhat) and its Jacobians (BF16 tensor cores) against the FP64 oracle.

Tolerance: 2e-2 relative, norm-wise per quantity, for the BF16 square layers
(FP32 accumulation); the network output is compared without the output shift
(out_shift would otherwise hide errors of the learned part).  FP32-only paths
(linear decoder, one hidden layer, the CUDA-core path) are held to 1e-5.  Second-derivative
(mixed) rows: in FP32 at 1e-5 away from the ELU'' jump at z = 0; in BF16 against a bound derived
from the oracle evaluated with the GPU's BF16 operand rounding.
"""
import numpy as np
import pytest

import oracle.decoder as OD
import synth.scenes as S

pytestmark = pytest.mark.gpu
TOL_BF16 = 2e-2


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def _dec_params(d, r, n_hidden=5, act=OD.ELU, seed=0):
    lo = np.full(d, 0.3)
    return S.xavier_decoder(seed, d, r, 128, n_hidden, act, X_min=lo, X_range=np.full(d, 0.3),
                            out_shift=np.full(d, 0.5), out_scale=np.full(d, 0.1), bias_scale=0.2)


def _points(n, d, r, n_lat=1, seed=1):
    rng = np.random.default_rng(seed)
    X = 0.3 + 0.3 * rng.uniform(size=(n, d))
    lat = rng.normal(scale=0.7, size=(n_lat, r))
    idx = rng.integers(0, n_lat, size=n).astype(np.int32)
    return X, lat, idx


def _gpu(*arrays):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrays]


@pytest.mark.parametrize("d,r,n", [(2, 16, 1000), (3, 16, 777), (2, 8, 1), (3, 32, 300), (3, 13, 200), (2, 38, 50)])
def test_forward_and_jacobians(d, r, n):
    """Includes r = 13 (latents loaded one by one rather than as float4) and r = 38 (beyond the
    tensor-core kernel's 36-latent input layout: the FP32 kernel)."""
    import torch
    from paper_2109_12390_gb300.decoder import Decoder, PRIMAL
    p = _dec_params(d, r)
    dec = Decoder.from_params(p)
    X, lat, idx = _points(n, d, r, n_lat=3)
    Xg, latg, idxg = _gpu(X.astype(np.float32), lat.astype(np.float32), idx)
    kinds = [PRIMAL] + [1 + k for k in range(d)] + [dec.dxhat(j) for j in range(r)]
    out = dec.eval(Xg, latg, kinds, lat_idx=idxg).cpu().numpy()
    torch.cuda.synchronize()
    assert dec.status() == 0
    Xr = X.astype(np.float32).astype(np.float64)
    xh = lat.astype(np.float32).astype(np.float64)[idx]
    g, JX, Jq = OD.jacobians(p, Xr, xh)
    assert rel(out[0] - 0.5, g - 0.5) < TOL_BF16
    assert rel(np.stack(out[1:1 + d], -1), JX) < TOL_BF16
    assert rel(np.stack(out[1 + d:], -1), Jq) < TOL_BF16


def test_jvp_and_secant_rows():
    from paper_2109_12390_gb300.decoder import Decoder, PRIMAL, JVP, SECANT
    d, r, n = 2, 16, 2000
    p = _dec_params(d, r, seed=3)
    dec = Decoder.from_params(p)
    X, lat, idx = _points(n, d, r, n_lat=4, seed=4)
    rng = np.random.default_rng(5)
    u = rng.normal(size=lat.shape)
    Xg, latg, idxg, ug = _gpu(X.astype(np.float32), lat.astype(np.float32), idx, u.astype(np.float32))
    out = dec.eval(Xg, latg, [PRIMAL, JVP], lat_idx=idxg, dirs=ug).cpu().numpy()
    Xr = X.astype(np.float32).astype(np.float64)
    xh = lat.astype(np.float32).astype(np.float64)[idx]
    uu = u.astype(np.float32).astype(np.float64)[idx]
    _, jv = OD.jvp_latent(p, Xr, xh, uu)
    assert rel(out[1], jv) < TOL_BF16
    # secant rows resolve latent increments far below BF16 resolution
    for scale in (1e-2, 1e-4, 1e-6):
        delta = (scale * u).astype(np.float32)
        (dg,) = _gpu(delta)
        sec = dec.eval(Xg, latg, [PRIMAL, SECANT], lat_idx=idxg, dirs=dg).cpu().numpy()[1]
        ref = OD.decode(p, Xr, xh + delta.astype(np.float64)[idx]) - OD.decode(p, Xr, xh)
        assert rel(sec, ref) < TOL_BF16, scale


def _bf16(a):
    """Round to the nearest BF16 value (ties to even), held in FP64."""
    u = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _velocity_gradient_bf16_operands(p, X, xh, u):
    """The oracle's forward-over-forward dv/dX with the operands the tensor-core path rounds to
    BF16 rounded the same way: the weights of the square hidden layers and every row that enters
    them (activations, latent and X tangents, mixed tangents).  The first and last layers stay in
    FP64, as they are FP32 on the GPU."""
    d, r = p.d, p.r
    h = np.concatenate([(X - p.X_min) / p.X_range, xh], axis=1)
    n = len(h)
    s = np.concatenate([np.zeros((n, d)), np.broadcast_to(u, (n, r))], axis=1)
    ts = [np.broadcast_to(np.concatenate([np.eye(d)[k] / p.X_range, np.zeros(r)]), (n, d + r)) for k in range(d)]
    ms = [np.zeros((n, d + r)) for _ in range(d)]
    L = len(p.W)
    for l in range(L):
        W = p.W[l]
        if 0 < l < L - 1:
            W = _bf16(W)
            h, s = _bf16(h), _bf16(s)
            ts = [_bf16(t) for t in ts]
            ms = [_bf16(m) for m in ms]
        z = h @ W.T + p.b[l]
        zs, zt, zm = s @ W.T, [t @ W.T for t in ts], [m @ W.T for m in ms]
        if l < L - 1:
            a1, a2 = OD.act_d1(z, p.activation), OD.act_d2(z, p.activation)
            h = OD.act(z, p.activation)
            s = a1 * zs
            ts = [a1 * q for q in zt]
            ms = [a2 * zs * q + a1 * mq for q, mq in zip(zt, zm)]
        else:
            s, ms = zs, zm
    return np.stack([m * p.out_scale for m in ms], axis=-1)


def _mixed_bf16_bound(p, Xr, xh, uu, G):
    """Bound of the BF16 mixed rows: a second derivative through four BF16 layers, whose terms
    act''(z)(W u)(W t) and act'(z)(W m) partly cancel and whose act'' jumps at z = 0, so the BF16
    rounding of the operands costs far more than for first derivatives.  The sensitivity is the
    deviation of the oracle evaluated with exactly the GPU's BF16 operand rounding; the GPU's
    remaining difference is its FP32 accumulation order, so twice that (at least 2e-2) bounds it."""
    sens = rel(_velocity_gradient_bf16_operands(p, Xr, xh, uu), G)
    return max(TOL_BF16, 2.0 * sens), sens


def _away_from_kink(p, Xr, xh, band):
    """Points whose every hidden pre-activation z lies outside |z| < band * RMS(z of its layer):
    ELU'' jumps at z = 0 (1 below, 0 above), so at a point with a pre-activation within rounding
    of 0 the FP32 and FP64 evaluations may take opposite sides, and both values are correct
    second derivatives of the one-sided branches.  Mixed rows are compared at the other points."""
    _, _, rec = OD.forward(p, Xr, xh, keep=True)
    ok = np.ones(len(Xr), bool)
    for l in range(len(p.W) - 1):
        z = rec[l][1]
        ok &= (np.abs(z) >= band * np.sqrt(np.mean(z * z))).all(axis=1)
    return ok


@pytest.mark.parametrize("d,n_hidden,tol", [(2, 5, None), (3, 5, None), (2, 1, 1e-5), (3, 1, 1e-5)])
def test_mixed_rows_velocity_gradient(d, n_hidden, tol):
    """Mixed rows d/dX_k of the JVP row against the oracle's forward-over-forward dv/dX:
    5 hidden layers on the tensor cores (BF16), one hidden layer in FP32.  The JVP and
    tangent rows of the same call keep the first-derivative tolerance."""
    from paper_2109_12390_gb300.decoder import Decoder, PRIMAL, JVP, mixed, dX
    r, n = 16, 1500
    p = _dec_params(d, r, n_hidden=n_hidden, seed=21)
    dec = Decoder.from_params(p)
    X, lat, idx = _points(n, d, r, n_lat=3, seed=22)
    u = np.random.default_rng(23).normal(size=lat.shape)
    Xg, latg, idxg, ug = _gpu(X.astype(np.float32), lat.astype(np.float32), idx, u.astype(np.float32))
    kinds = [PRIMAL] + [dX(k) for k in range(d)] + [JVP] + [mixed(dX(k)) for k in range(d)]
    out = dec.eval(Xg, latg, kinds, lat_idx=idxg, dirs=ug).cpu().numpy()
    assert dec.status() == 0
    Xr = X.astype(np.float32).astype(np.float64)
    xh = lat.astype(np.float32).astype(np.float64)[idx]
    uu = u.astype(np.float32).astype(np.float64)[idx]
    v, G = OD.velocity_gradient(p, Xr, xh, uu)
    _, JX, _ = OD.jacobians(p, Xr, xh)
    tol1 = TOL_BF16 if tol is None else tol
    assert rel(np.stack(out[1:1 + d], -1), JX) < tol1
    assert rel(out[1 + d], v) < tol1
    if tol is None:
        tol, sens = _mixed_bf16_bound(p, Xr, xh, uu, G)
        print(f"BF16 mixed rows: error {rel(np.stack(out[2 + d:], -1), G):.3e}, operand-rounding sensitivity "
              f"{sens:.3e}, bound {tol:.3e}")
        assert rel(np.stack(out[2 + d:], -1), G) < tol
    else:
        ok = _away_from_kink(p, Xr, xh, 1e-5)
        assert ok.mean() > 0.95, ok.mean()
        assert rel(np.stack(out[2 + d:], -1)[ok], G[ok]) < tol


def test_mixed_rows_of_affine_network_vanish_and_need_partners():
    import torch
    from paper_2109_12390_gb300 import _abi
    from paper_2109_12390_gb300.decoder import Decoder, PRIMAL, JVP, mixed, dX
    d, r, n = 2, 4, 200
    for n_hidden in (0, 3):
        p = _dec_params(d, r, n_hidden=n_hidden, act=OD.IDENTITY, seed=24)
        dec = Decoder.from_params(p)
        X, lat, idx = _points(n, d, r, seed=25)
        Xg, latg, ug = _gpu(X.astype(np.float32), lat.astype(np.float32), np.ones_like(lat, np.float32))
        out = dec.eval(Xg, latg, [PRIMAL, dX(0), dX(1), JVP, mixed(dX(0)), mixed(dX(1))], dirs=ug).cpu().numpy()
        assert np.abs(out[4:]).max() == 0.0
    with pytest.raises(_abi.MpmError):
        dec.eval(Xg, latg, [PRIMAL, JVP, mixed(dX(0))], dirs=ug)   # no dX_0 tangent row
    with pytest.raises(_abi.MpmError):
        dec.eval(Xg, latg, [PRIMAL, dX(0), mixed(dX(0))], dirs=ug)  # no JVP row


@pytest.mark.parametrize("d,r,n", [(2, 16, 1000), (3, 8, 333), (2, 16, 37), (3, 8, 5)])
def test_fp32_cuda_core_path_deep_decoder(d, r, n):
    """decoder_set_precision(fp32): the 5-hidden-layer decoder evaluated in FP32 on the CUDA cores
    matches the FP64 oracle to FP32 accuracy for every row kind (primal, tangents, JVP, secant,
    mixed), and the BF16 tensor-core path stays available on the same object.  The small sizes
    pack a few rows per tile, so tiles start in the middle of a point's rows."""
    from paper_2109_12390_gb300.decoder import Decoder, PRIMAL, JVP, SECANT, dX, mixed
    p = _dec_params(d, r, seed=31)
    dec = Decoder.from_params(p)
    X, lat, idx = _points(n, d, r, n_lat=3, seed=32)
    u = 0.3 * np.random.default_rng(33).normal(size=lat.shape)
    Xg, latg, idxg, ug = _gpu(X.astype(np.float32), lat.astype(np.float32), idx, u.astype(np.float32))
    Xr = X.astype(np.float32).astype(np.float64)
    xh = lat.astype(np.float32).astype(np.float64)[idx]
    uu = u.astype(np.float32).astype(np.float64)[idx]
    g, JX, Jq = OD.jacobians(p, Xr, xh)
    v, G = OD.velocity_gradient(p, Xr, xh, uu)
    dec.set_precision(True)
    kinds = [PRIMAL] + [dX(k) for k in range(d)] + [JVP] + [mixed(dX(k)) for k in range(d)]
    out = dec.eval(Xg, latg, kinds, lat_idx=idxg, dirs=ug).cpu().numpy()
    assert dec.status() == 0
    assert rel(out[0] - 0.5, g - 0.5) < 1e-5
    assert rel(np.stack(out[1:1 + d], -1), JX) < 1e-5
    assert rel(out[1 + d], v) < 1e-5
    # ELU'' jumps at z = 0: mixed rows are compared at 1e-5 at the points whose pre-activations
    # are all clear of the kink by far more than FP32 rounding
    ok = _away_from_kink(p, Xr, xh, 1e-5)
    assert ok.mean() > 0.95, ok.mean()
    assert rel(np.stack(out[2 + d:], -1)[ok], G[ok]) < 1e-5
    out2 = dec.eval(Xg, latg, [PRIMAL] + [dec.dxhat(j) for j in range(r)], lat_idx=idxg).cpu().numpy()
    assert rel(np.stack(out2[1:], -1), Jq) < 1e-5
    sec = dec.eval(Xg, latg, [PRIMAL, SECANT], lat_idx=idxg, dirs=ug).cpu().numpy()[1]
    ref = OD.decode(p, Xr, xh + uu) - OD.decode(p, Xr, xh)
    assert rel(sec, ref) < 1e-5
    dec.set_precision(False)
    out3 = dec.eval(Xg, latg, [PRIMAL], lat_idx=idxg).cpu().numpy()
    assert 1e-6 < rel(out3[0] - 0.5, g - 0.5) < TOL_BF16


@pytest.mark.parametrize("d,r,n", [(2, 16, 1000), (3, 8, 333), (2, 16, 37)])
def test_split_bf16_tensor_path_deep_decoder(d, r, n):
    """decoder_set_precision(2): split-BF16 square layers on the tensor cores.  Every row kind
    (primal, tangents, JVP, latent Jacobian, secant, mixed) against the FP64 oracle within the bound
    derived from the split arithmetic's backward error (square-layer products perturbed by
    3 * 2^-18, the rest by the FP32 model; 10 times the oracle's response, at least 1e-5); mixed
    rows away from the ELU'' jump by more than that error.  The split path must also be well
    inside the BF16 path's error on the same call."""
    import fp32_bounds as FB
    from paper_2109_12390_gb300.decoder import Decoder, PRIMAL, JVP, SECANT, dX, mixed
    p = _dec_params(d, r, seed=51)
    dec = Decoder.from_params(p)
    X, lat, idx = _points(n, d, r, n_lat=3, seed=52)
    u = 0.3 * np.random.default_rng(53).normal(size=lat.shape)
    Xg, latg, idxg, ug = _gpu(X.astype(np.float32), lat.astype(np.float32), idx, u.astype(np.float32))
    Xr = X.astype(np.float32).astype(np.float64)
    xh = lat.astype(np.float32).astype(np.float64)[idx]
    uu = u.astype(np.float32).astype(np.float64)[idx]
    pf = FB.f32_decoder(p)
    kinds = [PRIMAL] + [dX(k) for k in range(d)] + [JVP] + [mixed(dX(k)) for k in range(d)]
    dec.set_precision(2)
    out = dec.eval(Xg, latg, kinds, lat_idx=idxg, dirs=ug).cpu().numpy()
    out2 = dec.eval(Xg, latg, [PRIMAL] + [dec.dxhat(j) for j in range(r)], lat_idx=idxg).cpu().numpy()
    sec = dec.eval(Xg, latg, [PRIMAL, SECANT], lat_idx=idxg, dirs=ug).cpu().numpy()[1]
    assert dec.status() == 0

    def quantities(pp, X_, xh_, uu_):
        g, JX, Jq = OD.jacobians(pp, X_, xh_)
        v, G = OD.velocity_gradient(pp, X_, xh_, uu_)
        return dict(g=g - pp.out_shift, JX=JX, v=v, Jq=Jq, sec=OD.decode(pp, X_, xh_ + uu_) - OD.decode(pp, X_, xh_), G=G)

    ref = quantities(pf, Xr, xh, uu)
    rng = np.random.default_rng(54)
    pert = quantities(FB.perturb_decoder_split(pf, rng), FB.perturb(Xr, rng), FB.perturb(xh, rng), FB.perturb(uu, rng))
    # the split arithmetic moves a pre-activation by up to about 1e-4 of its layer's RMS: points
    # with one inside 3e-4 RMS of the kink are left out of the mixed rows (about a fifth here,
    # with 640 pre-activations per point)
    ok = _away_from_kink(p, Xr, xh, 3e-4)
    assert ok.sum() >= min(n, 10) and ok.mean() > 0.4, ok.mean()
    got = dict(g=out[0] - p.out_shift, JX=np.stack(out[1:1 + d], -1), v=out[1 + d], Jq=np.stack(out2[1:], -1),
               sec=sec, G=np.stack(out[2 + d:], -1))
    for k in got:
        sel = ok if k == "G" else slice(None)
        sens = rel(pert[k][sel], ref[k][sel])
        err = rel(got[k][sel], ref[k][sel])
        print(f"split {k}: error {err:.3e} sensitivity {sens:.3e} bound {FB.bound(sens):.3e}")
        assert err < FB.bound(sens), (k, err, sens)
    dec.set_precision(0)
    bf = dec.eval(Xg, latg, [PRIMAL], lat_idx=idxg).cpu().numpy()[0]
    assert rel(got["g"], ref["g"]) < 0.05 * rel(bf - p.out_shift, ref["g"])


def test_linear_and_single_hidden_layer_fp32():
    from paper_2109_12390_gb300.decoder import Decoder, PRIMAL
    for n_hidden, act in [(0, OD.IDENTITY), (1, OD.ELU)]:
        d, r, n = 3, 6, 513
        p = _dec_params(d, r, n_hidden=n_hidden, act=act, seed=7)
        dec = Decoder.from_params(p)
        X, lat, idx = _points(n, d, r, n_lat=2, seed=8)
        Xg, latg, idxg = _gpu(X.astype(np.float32), lat.astype(np.float32), idx)
        kinds = [PRIMAL] + [1 + k for k in range(d)] + [dec.dxhat(j) for j in range(r)]
        out = dec.eval(Xg, latg, kinds, lat_idx=idxg).cpu().numpy()
        g, JX, Jq = OD.jacobians(p, X.astype(np.float32).astype(np.float64),
                                 lat.astype(np.float32).astype(np.float64)[idx])
        assert rel(out[0] - 0.5, g - 0.5) < 1e-5
        assert rel(np.stack(out[1:1 + d], -1), JX) < 1e-5
        assert rel(np.stack(out[1 + d:], -1), Jq) < 1e-5


def test_identity_activation_tensor_path_is_weight_product():
    from paper_2109_12390_gb300.decoder import Decoder, PRIMAL
    d, r, n = 2, 4, 130
    p = _dec_params(d, r, n_hidden=3, act=OD.IDENTITY, seed=9)
    dec = Decoder.from_params(p)
    X, lat, idx = _points(n, d, r, seed=10)
    Xg, latg = _gpu(X.astype(np.float32), lat.astype(np.float32))
    out = dec.eval(Xg, latg, [PRIMAL] + [dec.dxhat(j) for j in range(r)]).cpu().numpy()
    prod = p.W[3] @ p.W[2] @ p.W[1] @ p.W[0]
    Jq = np.stack(out[1:], -1)
    assert rel(Jq, np.broadcast_to(0.1 * prod[:, d:], Jq.shape)) < TOL_BF16


def test_reconstruction_size_sampled():
    """1,048,576 points (4096 latents x 256 points) forward; sampled points against the oracle."""
    import torch
    from paper_2109_12390_gb300.decoder import Decoder, PRIMAL
    d, r, n = 2, 16, 1 << 20
    p = _dec_params(d, r, seed=11)
    dec = Decoder.from_params(p)
    X, lat, idx = _points(n, d, r, n_lat=4096, seed=12)
    Xg, latg, idxg = _gpu(X.astype(np.float32), lat.astype(np.float32), idx)
    out = dec.eval(Xg, latg, [PRIMAL], lat_idx=idxg)
    torch.cuda.synchronize()
    assert dec.status() == 0
    rng = np.random.default_rng(13)
    sel = np.concatenate([rng.choice(n, 2000, replace=False), [0, n - 1]])
    g = OD.decode(p, X[sel].astype(np.float32).astype(np.float64),
                  lat.astype(np.float32).astype(np.float64)[idx[sel]])
    assert rel(out[0].cpu().numpy()[sel] - 0.5, g - 0.5) < TOL_BF16


def test_empty_and_bad_arguments():
    import torch
    from paper_2109_12390_gb300 import _abi
    from paper_2109_12390_gb300.decoder import Decoder, PRIMAL
    p = _dec_params(2, 4)
    dec = Decoder.from_params(p)
    X = torch.zeros((0, 2), device="cuda")
    lat = torch.zeros((1, 4), device="cuda")
    out = dec.eval(X, lat, [PRIMAL])
    assert out.shape == (1, 0, 2)
    with pytest.raises(_abi.MpmError):
        dec.eval(torch.zeros((3, 2), device="cuda"), lat, [5, PRIMAL])   # primal must come first
    with pytest.raises(_abi.MpmError):
        dec.eval(torch.zeros((3, 2), device="cuda"), lat, [PRIMAL, 999])


@pytest.mark.parametrize("fp32,tol", [(True, 1e-5), (False, TOL_BF16)])
def test_secant_rows_along_direction_blocks(fp32, tol):
    """DECODER_SECANT_DIR + m: several secants of one point, each along its own direction block of
    the point's latent row (dirs laid out (n_lat, n_dirs, r)), sharing the point's primal row; the
    reduced step's line search evaluates its 11 trial steps this way."""
    from paper_2109_12390_gb300.decoder import Decoder, PRIMAL, secant_dir
    d, r, n, nd = 2, 8, 300, 3
    p = _dec_params(d, r, seed=41)
    dec = Decoder.from_params(p)
    dec.set_precision(fp32)
    X, lat, idx = _points(n, d, r, n_lat=2, seed=42)
    u = (1e-3 * np.random.default_rng(43).normal(size=(len(lat), nd, r))).astype(np.float32)
    Xg, latg, idxg, ug = _gpu(X.astype(np.float32), lat.astype(np.float32), idx, u)
    out = dec.eval(Xg, latg, [PRIMAL] + [secant_dir(m) for m in range(nd)], lat_idx=idxg, dirs=ug).cpu().numpy()
    assert dec.status() == 0
    Xr = X.astype(np.float32).astype(np.float64)
    xh = lat.astype(np.float32).astype(np.float64)[idx]
    g0 = OD.decode(p, Xr, xh)
    for m in range(nd):
        ref = OD.decode(p, Xr, xh + u.astype(np.float64)[idx, m]) - g0
        assert rel(out[1 + m], ref) < tol, (m, rel(out[1 + m], ref))
