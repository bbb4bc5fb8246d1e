"""FP64 oracle of the encoder network (Section 4.1, Table 1).  Test infrastructure only.

The encoder maps the deformed positions of a fixed subset of material points of one snapshot to
that snapshot's generalized coordinates, xhat = enc(x), and is trained together with the decoder
(the latent table of the Remark of Section 4.1 is the alternative).  Table 1 fixes the structure:
1D convolutions of kernel size 6 and stride 2 shrink the concatenated position vector to a length
d_conv, the smallest one reachable that is not below 32; a fully connected layer maps it to 32
values and a second one to the r generalized coordinates.

Readings (the paper is silent on these):
* the concatenation is particle-major, (x_1, y_1, x_2, y_2, ...), of positions standardised per
  coordinate, (x - shift) / scale;
* every convolution has one input and one output channel and a bias; ELU follows every layer but
  the last, which is linear (as in the decoder);
* the subset is fixed per instance: particle ids floor(j P / P_sub), j < P_sub.

Layer l (length L_l -> L_{l+1} = (L_l - 6) // 2 + 1):
    z_l[i] = b_l + sum_{k < 6} w_l[k] h_l[2 i + k],   h_{l+1} = ELU(z_l).

Pins (tests/test_oracle_encoder.py): each convolution against numpy.correlate of its input with
the kernel, every other output kept; the layer count and lengths against the stopping rule; an
identity-activation encoder against the product of its explicit (Toeplitz) layer matrices;
reverse-mode gradients against central differences of a scalar loss.
"""
from __future__ import annotations

import dataclasses

import numpy as np

KERNEL, STRIDE, FC_WIDTH, MIN_LEN = 6, 2, 32, 32
ELU, IDENTITY = 0, 1


def conv_lengths(L0):
    """Lengths L_0, L_1, ..., L_{n_conv}: convolve while the next length stays >= 32."""
    lens = [int(L0)]
    while (lens[-1] - KERNEL) // STRIDE + 1 >= MIN_LEN:
        lens.append((lens[-1] - KERNEL) // STRIDE + 1)
    return lens


def subset_ids(n_particles, n_sub):
    return (np.arange(n_sub) * n_particles) // n_sub


@dataclasses.dataclass
class EncoderParams:
    d: int
    r: int
    n_sub: int
    conv_w: list            # n_conv arrays (6,)
    conv_b: np.ndarray      # (n_conv,)
    W1: np.ndarray          # (32, d_conv)
    b1: np.ndarray          # (32,)
    W2: np.ndarray          # (r, 32)
    b2: np.ndarray          # (r,)
    shift: np.ndarray       # (d,)
    scale: np.ndarray       # (d,)
    activation: int = ELU

    @property
    def lengths(self):
        return conv_lengths(self.d * self.n_sub)


def xavier_encoder(seed, d, r, n_sub, shift=None, scale=None, activation=ELU):
    """Xavier-uniform weights (Glorot and Bengio 2010) with fan-in / fan-out of each layer's own
    linear map (a convolution: 6 in, 1 out), zero biases."""
    rng = np.random.default_rng(seed)
    lens = conv_lengths(d * n_sub)
    n_conv = len(lens) - 1
    lim = np.sqrt(6.0 / (KERNEL + 1))
    conv_w = [rng.uniform(-lim, lim, size=KERNEL) for _ in range(n_conv)]
    dc = lens[-1]
    l1 = np.sqrt(6.0 / (dc + FC_WIDTH))
    l2 = np.sqrt(6.0 / (FC_WIDTH + r))
    return EncoderParams(d=d, r=r, n_sub=n_sub, conv_w=conv_w, conv_b=np.zeros(n_conv),
                         W1=rng.uniform(-l1, l1, size=(FC_WIDTH, dc)), b1=np.zeros(FC_WIDTH),
                         W2=rng.uniform(-l2, l2, size=(r, FC_WIDTH)), b2=np.zeros(r),
                         shift=np.zeros(d) if shift is None else np.asarray(shift, np.float64),
                         scale=np.ones(d) if scale is None else np.asarray(scale, np.float64),
                         activation=activation)


def _act(z, kind):
    return z if kind == IDENTITY else np.where(z > 0, z, np.expm1(np.minimum(z, 0.0)))


def _act_d1(z, kind):
    return np.ones_like(z) if kind == IDENTITY else np.where(z > 0, 1.0, np.exp(np.minimum(z, 0.0)))


def encoder_input(enc, x_sub):
    """(n, n_sub, d) subset positions -> (n, d n_sub) standardised, particle-major."""
    x = np.asarray(x_sub, np.float64)
    return ((x - enc.shift) / enc.scale).reshape(len(x), -1)


def conv_layer(h, w, b):
    """z[:, i] = b + sum_k w[k] h[:, 2 i + k] for i < (L - 6) // 2 + 1."""
    L = h.shape[1]
    n_out = (L - KERNEL) // STRIDE + 1
    z = np.full((h.shape[0], n_out), float(b))
    for i in range(n_out):
        for k in range(KERNEL):
            z[:, i] += w[k] * h[:, STRIDE * i + k]
    return z


def forward(enc, u, keep=False):
    """u (n, L0) -> xhat (n, r); with keep, the per-layer (input, pre-activation) records."""
    h = np.asarray(u, np.float64)
    rec = []
    for w, b in zip(enc.conv_w, enc.conv_b):
        z = conv_layer(h, w, b)
        rec.append((h, z))
        h = _act(z, enc.activation)
    z1 = h @ enc.W1.T + enc.b1
    rec.append((h, z1))
    a = _act(z1, enc.activation)
    rec.append((a, None))
    xh = a @ enc.W2.T + enc.b2
    return (xh, rec) if keep else xh


def encode(enc, x_sub):
    return forward(enc, encoder_input(enc, x_sub))


def vjp(enc, u, g):
    """Reverse mode: for the loss sum_s g_s . xhat_s, the gradients of every parameter, summed
    over the rows of u.  Returns dict conv_w (list), conv_b, W1, b1, W2, b2."""
    _, rec = forward(enc, u, keep=True)
    g = np.asarray(g, np.float64)
    a = rec[-1][0]
    out = {"W2": g.T @ a, "b2": g.sum(0)}
    da = g @ enc.W2
    h_last, z1 = rec[-2]
    dz1 = da * _act_d1(z1, enc.activation)
    out["W1"] = dz1.T @ h_last
    out["b1"] = dz1.sum(0)
    dh = dz1 @ enc.W1
    n_conv = len(enc.conv_w)
    gw = [None] * n_conv
    gb = np.zeros(n_conv)
    for l in range(n_conv - 1, -1, -1):
        h_in, z = rec[l]
        dz = dh * _act_d1(z, enc.activation)
        gw[l] = np.array([sum(float(np.sum(dz[:, i] * h_in[:, STRIDE * i + k])) for i in range(z.shape[1]))
                          for k in range(KERNEL)])
        gb[l] = dz.sum()
        dprev = np.zeros_like(h_in)
        for i in range(z.shape[1]):
            for k in range(KERNEL):
                dprev[:, STRIDE * i + k] += enc.conv_w[l][k] * dz[:, i]
        dh = dprev
    out["conv_w"] = gw
    out["conv_b"] = gb
    return out


def flatten(enc):
    """Parameter vector in the order the library stores it: per convolution (w[0..5], b), then W1
    (row-major), b1, W2 (row-major), b2."""
    parts = []
    for w, b in zip(enc.conv_w, enc.conv_b):
        parts += [np.asarray(w, np.float64), np.array([b], np.float64)]
    parts += [enc.W1.ravel(), enc.b1, enc.W2.ravel(), enc.b2]
    return np.concatenate(parts)


def flatten_grads(gr):
    parts = []
    for w, b in zip(gr["conv_w"], gr["conv_b"]):
        parts += [np.asarray(w, np.float64), np.array([b], np.float64)]
    parts += [gr["W1"].ravel(), gr["b1"], gr["W2"].ravel(), gr["b2"]]
    return np.concatenate(parts)


def unflatten(enc, vec):
    """Parameters of the same shapes as enc's from a vector in the order of flatten()."""
    e = dataclasses.replace(enc)
    o = 0
    n_conv = len(enc.conv_w)
    e.conv_w, cb = [], []
    for _ in range(n_conv):
        e.conv_w.append(np.array(vec[o:o + KERNEL], np.float64))
        cb.append(float(vec[o + KERNEL]))
        o += KERNEL + 1
    e.conv_b = np.array(cb)
    n1 = enc.W1.size
    e.W1 = np.array(vec[o:o + n1], np.float64).reshape(enc.W1.shape)
    o += n1
    e.b1 = np.array(vec[o:o + FC_WIDTH], np.float64)
    o += FC_WIDTH
    n2 = enc.W2.size
    e.W2 = np.array(vec[o:o + n2], np.float64).reshape(enc.W2.shape)
    o += n2
    e.b2 = np.array(vec[o:o + enc.r], np.float64)
    return e
