"""Pins of the FP64 encoder oracle (Section 4.1, Table 1) against definitions outside it."""
import numpy as np

import oracle.encoder as E


def test_layer_lengths_follow_the_stopping_rule():
    # brute force: apply (L - 6) // 2 + 1 while the result is at least 32
    for L0 in (32, 37, 38, 69, 70, 71, 200, 2048, 8192):
        lens = [L0]
        while True:
            nxt = (lens[-1] - 6) // 2 + 1
            if nxt < 32:
                break
            lens.append(nxt)
        assert E.conv_lengths(L0) == lens
        assert lens[-1] >= 32 and (lens[-1] - 6) // 2 + 1 < 32
    assert E.conv_lengths(2048) == [2048, 1022, 509, 252, 124, 60]


def test_convolution_is_strided_correlation():
    rng = np.random.default_rng(0)
    h = rng.normal(size=(3, 101))
    w = rng.normal(size=6)
    z = E.conv_layer(h, w, 0.25)
    for s in range(3):
        ref = np.correlate(h[s], w, mode="valid")[::2] + 0.25
        np.testing.assert_allclose(z[s], ref, rtol=0, atol=1e-13)


def test_identity_encoder_is_product_of_layer_matrices():
    rng = np.random.default_rng(1)
    enc = E.xavier_encoder(2, 2, 4, 40, activation=E.IDENTITY)
    enc.conv_b = rng.normal(size=len(enc.conv_w))
    enc.b1 = rng.normal(size=32)
    enc.b2 = rng.normal(size=4)
    lens = enc.lengths
    M = np.eye(lens[0])
    c = np.zeros(lens[0])
    for l, (w, b) in enumerate(zip(enc.conv_w, enc.conv_b)):
        T = np.zeros((lens[l + 1], lens[l]))
        for i in range(lens[l + 1]):
            T[i, 2 * i:2 * i + 6] = w
        M = T @ M
        c = T @ c + b
    M = enc.W2 @ enc.W1 @ M
    c = enc.W2 @ (enc.W1 @ c + enc.b1) + enc.b2
    u = rng.normal(size=(5, lens[0]))
    np.testing.assert_allclose(E.forward(enc, u), u @ M.T + c, rtol=1e-12, atol=1e-12)


def test_standardised_particle_major_input():
    enc = E.xavier_encoder(0, 2, 3, 4, shift=[1.0, 2.0], scale=[2.0, 4.0])
    x = np.arange(16, dtype=np.float64).reshape(2, 4, 2)
    u = E.encoder_input(enc, x)
    assert u.shape == (2, 8)
    np.testing.assert_allclose(u[0, :4], [(0 - 1) / 2, (1 - 2) / 4, (2 - 1) / 2, (3 - 2) / 4])
    np.testing.assert_array_equal(E.subset_ids(4096, 1024)[:4], [0, 4, 8, 12])
    np.testing.assert_array_equal(E.subset_ids(10, 4), [0, 2, 5, 7])


def test_reverse_mode_gradients_match_central_differences():
    rng = np.random.default_rng(2)
    enc = E.xavier_encoder(3, 2, 3, 36)
    enc.conv_b = 0.3 * rng.normal(size=len(enc.conv_w))
    enc.b1 = 0.3 * rng.normal(size=32)
    u = rng.normal(size=(4, 72))
    g = rng.normal(size=(4, 3))
    grads = E.flatten_grads(E.vjp(enc, u, g))
    theta = E.flatten(enc)
    assert grads.shape == theta.shape
    loss = lambda th: float(np.sum(g * E.forward(E.unflatten(enc, th), u)))
    idx = rng.choice(len(theta), size=40, replace=False)
    idx = np.unique(np.concatenate([idx, np.arange(14), [len(theta) - 1]]))   # every conv parameter
    h = 1e-6
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        fd = (loss(theta + e) - loss(theta - e)) / (2 * h)
        assert abs(fd - grads[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, grads[i])
    np.testing.assert_allclose(E.flatten(E.unflatten(enc, theta)), theta, rtol=0, atol=0)
