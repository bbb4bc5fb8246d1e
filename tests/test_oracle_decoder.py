"""Pins of the FP64 decoder oracle: finite differences, linear special case, Adam closed form."""
import numpy as np
import pytest

import oracle.decoder as D
import synth.scenes as S


def _small_dec(seed=0, d=2, r=3, width=16, n_hidden=3, activation=D.ELU):
    return S.xavier_decoder(seed, d, r, width, n_hidden, activation, X_min=np.full(d, 0.3),
                            X_range=np.full(d, 0.4), out_shift=np.linspace(0.2, 0.6, d),
                            out_scale=np.linspace(0.05, 0.2, d), bias_scale=0.3)


def test_activation_derivatives():
    z = np.linspace(-3, 3, 61)
    z = z[np.abs(z) > 1e-3]
    h = 1e-6
    fd1 = (D.act(z + h, D.ELU) - D.act(z - h, D.ELU)) / (2 * h)
    fd2 = (D.act_d1(z + h, D.ELU) - D.act_d1(z - h, D.ELU)) / (2 * h)
    np.testing.assert_allclose(D.act_d1(z, D.ELU), fd1, atol=1e-8)
    np.testing.assert_allclose(D.act_d2(z, D.ELU), fd2, atol=1e-7)
    assert D.act(np.array([-1.0]), D.ELU)[0] == pytest.approx(np.exp(-1) - 1, abs=1e-16)


@pytest.mark.parametrize("d", [2, 3])
def test_jacobians_against_central_differences(d):
    r = 4
    dec = _small_dec(1, d, r)
    rng = np.random.default_rng(2)
    X = 0.3 + 0.4 * rng.uniform(size=(7, d))
    xh = rng.normal(size=r)
    g, JX, Jq = D.jacobians(dec, X, xh)
    h = 1e-6
    for k in range(d):
        e = np.zeros(d)
        e[k] = h
        fd = (D.decode(dec, X + e, xh) - D.decode(dec, X - e, xh)) / (2 * h)
        np.testing.assert_allclose(JX[:, :, k], fd, rtol=1e-7, atol=1e-9)
    for j in range(r):
        e = np.zeros(r)
        e[j] = h
        fd = (D.decode(dec, X, xh + e) - D.decode(dec, X, xh - e)) / (2 * h)
        np.testing.assert_allclose(Jq[:, :, j], fd, rtol=1e-7, atol=1e-9)
    u = rng.normal(size=r)
    _, jv = D.jvp_latent(dec, X, xh, u)
    np.testing.assert_allclose(jv, np.einsum("pij,j->pi", Jq, u), atol=1e-13)


def test_linear_network_jacobians_are_weight_blocks():
    d, r = 3, 5
    dec = S.xavier_decoder(3, d, r, 8, 0, D.IDENTITY, X_min=np.full(d, 0.1), X_range=np.array([0.5, 0.25, 2.0]),
                           out_shift=np.ones(d), out_scale=np.array([2.0, 0.5, 1.0]), bias_scale=0.2)
    rng = np.random.default_rng(4)
    X = rng.uniform(size=(5, d))
    xh = rng.normal(size=r)
    g, JX, Jq = D.jacobians(dec, X, xh)
    W = dec.W[0]
    np.testing.assert_array_equal(Jq[0], dec.out_scale[:, None] * W[:, d:])
    np.testing.assert_allclose(JX[0], dec.out_scale[:, None] * W[:, :d] / dec.X_range[None, :], rtol=1e-15)
    # identity activation with hidden layers: Jacobian is the product of the weights
    dec2 = S.xavier_decoder(5, d, r, 6, 2, D.IDENTITY, bias_scale=0.1)
    _, JX2, Jq2 = D.jacobians(dec2, X, xh)
    prod = dec2.W[2] @ dec2.W[1] @ dec2.W[0]
    np.testing.assert_allclose(Jq2[0], prod[:, d:], atol=1e-14)
    np.testing.assert_allclose(JX2[3], prod[:, :d], atol=1e-14)


def test_loss_gradients_against_central_differences():
    d, r = 2, 3
    dec = _small_dec(7, d, r, width=8, n_hidden=3)
    rng = np.random.default_rng(8)
    S_snap, n = 4, 9
    latents = rng.normal(size=(S_snap, r))
    batch = {
        "X": 0.3 + 0.4 * rng.uniform(size=(n, d)),
        "snap": rng.integers(0, S_snap, size=n),
        "x": rng.uniform(size=(n, d)),
        "F": np.eye(d) + 0.1 * rng.normal(size=(n, d, d)),
        "v": rng.normal(size=(n, d)),
    }
    batch["next"] = np.where(batch["snap"] < S_snap - 1, batch["snap"] + 1, -1)
    dt, lF, lv = 0.05, 3.0, 0.2

    def L():
        return D.batch_loss_grads(dec, latents, batch, dt, lF, lv)[0]

    loss, gW, gb, gl = D.batch_loss_grads(dec, latents, batch, dt, lF, lv)
    h = 1e-6
    for l in range(len(dec.W)):
        for (a, b) in [(0, 0), (dec.W[l].shape[0] - 1, dec.W[l].shape[1] - 1), (1, 1)]:
            old = dec.W[l][a, b]
            dec.W[l][a, b] = old + h
            lp = L()
            dec.W[l][a, b] = old - h
            lm = L()
            dec.W[l][a, b] = old
            assert gW[l][a, b] == pytest.approx((lp - lm) / (2 * h), rel=1e-6, abs=1e-9)
        old = dec.b[l][0]
        dec.b[l][0] = old + h
        lp = L()
        dec.b[l][0] = old - h
        lm = L()
        dec.b[l][0] = old
        assert gb[l][0] == pytest.approx((lp - lm) / (2 * h), rel=1e-6, abs=1e-9)
    for s in range(S_snap):
        for j in range(r):
            old = latents[s, j]
            latents[s, j] = old + h
            lp = L()
            latents[s, j] = old - h
            lm = L()
            latents[s, j] = old
            assert gl[s, j] == pytest.approx((lp - lm) / (2 * h), rel=1e-6, abs=1e-9)


def test_adam_constant_gradient_closed_form():
    p = np.array([1.0, -2.0])
    g = np.array([0.3, -4.0])
    opt = D.Adam([p], lr=0.01)
    for k in range(1, 6):
        opt.step([g])
        # bias correction makes m_hat = g and v_hat = g^2 exactly for a constant gradient
        np.testing.assert_allclose(p, np.array([1.0, -2.0]) - k * 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    # invariance to a positive rescaling of the gradient (up to eps)
    q1, q2 = np.array([0.5]), np.array([0.5])
    o1, o2 = D.Adam([q1], lr=0.1), D.Adam([q2], lr=0.1)
    rng = np.random.default_rng(0)
    for _ in range(10):
        gg = rng.normal(size=1)
        o1.step([gg])
        o2.step([1000.0 * gg])
    assert q1[0] == pytest.approx(q2[0], rel=1e-6)
    assert D.lr_schedule(0, 100) == pytest.approx(1e-3)
    assert D.lr_schedule(99, 100) == pytest.approx(1e-6)


@pytest.mark.parametrize("d", [2, 3])
def test_velocity_gradient_against_central_differences(d):
    """dv/dX of the decoded velocity v = (dg/dxhat) u against central differences in X of
    the latent JVP (an independent forward-mode evaluation), and v against the JVP itself."""
    rng = np.random.default_rng(20 + d)
    r = 5
    X = rng.uniform(0.2, 0.8, size=(7, d))
    dec = S.xavier_decoder(3, d, r, 24, 3, D.ELU, X_min=X.min(0), X_range=X.max(0) - X.min(0) + 0.1,
                           out_shift=np.full(d, 0.5), out_scale=np.full(d, 0.3), bias_scale=0.3)
    xh = 0.4 * rng.normal(size=r)
    u = rng.normal(size=r)
    v, G = D.velocity_gradient(dec, X, xh, u)
    _, v_ref = D.jvp_latent(dec, X, xh, u)
    np.testing.assert_allclose(v, v_ref, rtol=1e-13, atol=1e-15)
    h = 1e-5
    for k in range(d):
        e = np.zeros(d)
        e[k] = h
        _, vp = D.jvp_latent(dec, X + e, xh, u)
        _, vm = D.jvp_latent(dec, X - e, xh, u)
        fd = (vp - vm) / (2 * h)
        assert np.linalg.norm(G[:, :, k] - fd) <= 1e-7 * np.linalg.norm(fd)


def test_velocity_gradient_of_affine_networks_is_zero():
    """Identity activation: g is affine in (X, xhat) jointly, so dv/dX vanishes exactly."""
    rng = np.random.default_rng(4)
    X = rng.uniform(size=(5, 2))
    dec = S.xavier_decoder(1, 2, 3, 16, 2, D.IDENTITY, X_min=X.min(0), X_range=X.max(0) - X.min(0))
    _, G = D.velocity_gradient(dec, X, rng.normal(size=3), rng.normal(size=3))
    assert np.abs(G).max() == 0.0


def test_jacobians_over_random_architectures():
    """Forward-mode Jacobians dg/dX and dg/dxhat and the latent JVP against central differences,
    over randomly drawn dimensions, latent sizes, depths, activations and inputs (property-based)."""
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")

    @hyp.settings(max_examples=25, deadline=None, derandomize=True)
    @hyp.given(seed=st.integers(0, 2 ** 31 - 1), d=st.sampled_from([2, 3]), r=st.integers(1, 6),
               n_hidden=st.integers(0, 4), act=st.sampled_from([D.ELU, D.IDENTITY]))
    def check(seed, d, r, n_hidden, act):
        rng = np.random.default_rng(seed)
        dec = S.xavier_decoder(seed % 1000, d, r, 16, n_hidden, act, bias_scale=0.3)
        X = rng.uniform(size=(5, d))
        xh = rng.normal(size=r)
        g, JX, Jq = D.jacobians(dec, X, xh)
        np.testing.assert_allclose(g, D.decode(dec, X, xh), rtol=0, atol=1e-14)
        h = 1e-6
        for k in range(d):
            e = np.zeros(d)
            e[k] = h
            fd = (D.decode(dec, X + e, xh) - D.decode(dec, X - e, xh)) / (2 * h)
            np.testing.assert_allclose(JX[:, :, k], fd, rtol=1e-6, atol=1e-8)
        for j in range(r):
            e = np.zeros(r)
            e[j] = h
            fd = (D.decode(dec, X, xh + e) - D.decode(dec, X, xh - e)) / (2 * h)
            np.testing.assert_allclose(Jq[:, :, j], fd, rtol=1e-6, atol=1e-8)
        u = rng.normal(size=r)
        _, jv = D.jvp_latent(dec, X, xh, u)
        np.testing.assert_allclose(jv, np.einsum("pij,j->pi", Jq, u), rtol=1e-12, atol=1e-13)

    check()


def test_appendix_b_scaling_maps_inputs_to_unit_box_and_standardises_outputs():
    """Pins of the Appendix B scaling: the min-max map sends the training X into [0, 1] with 0 and
    1 attained per coordinate; the output map standardises the snapshot positions (mean 0,
    population variance 1); both against brute-force loops on a small set."""
    rng = np.random.default_rng(7)
    X = rng.uniform(-0.3, 2.0, size=(37, 3)) * np.array([1.0, 0.2, 5.0])
    x = rng.normal(size=(211, 3)) * np.array([0.1, 3.0, 1e-3]) + np.array([0.5, -2.0, 7.0])
    lo, rg, mean, std = D.appendix_b_scaling(X, x)
    Xn = (X - lo) / rg
    assert Xn.min() >= 0.0 and Xn.max() <= 1.0
    np.testing.assert_allclose(Xn.min(0), 0.0, atol=1e-15)
    np.testing.assert_allclose(Xn.max(0), 1.0, rtol=1e-15)
    z = (x - mean) / std
    np.testing.assert_allclose(z.mean(0), 0.0, atol=1e-10)   # x - mean rounds at 7e-16 / 1e-3
    np.testing.assert_allclose((z ** 2).mean(0), 1.0, rtol=1e-12)
    for a in range(3):
        m = 0.0
        for i in range(len(x)):
            m += x[i, a]
        m /= len(x)
        v = 0.0
        for i in range(len(x)):
            v += (x[i, a] - m) ** 2
        assert abs(std[a] - np.sqrt(v / len(x))) <= 1e-12 * std[a]
        assert lo[a] == min(X[:, a]) and abs(lo[a] + rg[a] - max(X[:, a])) <= 4e-16 * abs(max(X[:, a]))
