"""Python surface of the implicit neural decoder (argument marshalling only).

All computation runs in libmpmrom.so (csrc/decoder.cu): the square hidden
layers as BF16 tcgen05 GEMMs with FP32 accumulation in tensor memory.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _abi
from .mpm import _ptr, _stream

PRIMAL, JVP, SECANT = _abi.DECODER_PRIMAL, _abi.DECODER_JVP, _abi.DECODER_SECANT


def dX(k):
    """Row kind of dg/dX_k."""
    return 1 + k


def secant_dir(m):
    """Kind of the secant row along the m-th direction of the point's latent row."""
    return 3000 + int(m)


def mixed(kind):
    """Row kind of d/d(input of tangent `kind`) of the JVP row; with kind = dX(k) this is
    the material gradient d/dX_k of the decoded velocity (dg/dxhat) u."""
    return _abi.DECODER_MIXED + int(kind)


class Decoder:
    def __init__(self, d, r, width=128, n_hidden=5, activation=0):
        L = _abi.lib()
        self.desc = _abi.DecoderDesc(d, r, width, n_hidden, activation)
        h = C.c_void_p()
        _abi.check(L.decoder_create(C.byref(self.desc), C.byref(h)))
        self._h = h
        self.d, self.r = d, r
        self.n_params = int(L.decoder_num_params(h))

    def dxhat(self, j):
        """Row kind of dg/dxhat_j."""
        return 1 + self.d + j

    @classmethod
    def from_params(cls, p):
        """From a synth.scenes.DecoderParams (FP64 host) -> FP32 device copy."""
        dec = cls(p.d, p.r, p.width, p.n_hidden, p.activation)
        dec.set_params(p.flat(), np.concatenate([p.X_min, p.X_range, p.out_shift, p.out_scale]))
        torch.cuda.synchronize()
        return dec

    def close(self):
        if getattr(self, "_h", None):
            _abi.lib().decoder_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params, norm, stream=None):
        f = lambda a: np.ascontiguousarray(a, np.float32) if isinstance(a, np.ndarray) else a
        self._keep = (f(params), f(norm))
        _abi.check(_abi.lib().decoder_set_params(self._h, _ptr(self._keep[0]), _ptr(self._keep[1]), _stream(stream)))

    def fit_scaling(self, snaps, stream=None):
        """Appendix B scaling from a snapshot dict (device X and x): decoder_fit_scaling."""
        from .train import snapshot_desc
        sd = snapshot_desc(snaps)
        _abi.check(_abi.lib().decoder_fit_scaling(self._h, C.byref(sd), _stream(stream)))

    def get_params(self, params=None, norm=None, stream=None):
        _abi.check(_abi.lib().decoder_get_params(self._h, _ptr(params), _ptr(norm), _stream(stream)))

    def eval(self, X, latents, kinds, lat_idx=None, dirs=None, out=None, stream=None):
        """X (n, d), latents (n_lat, r), lat_idx (n,) int32 | None, dirs (n_lat, r) | None: CUDA tensors.
        Returns out (R, n, d)."""
        kinds = [int(k) for k in kinds]
        n = X.shape[0]
        if out is None:
            out = torch.empty((len(kinds), n, self.d), dtype=torch.float32, device=X.device)
        karr = (C.c_int32 * len(kinds))(*kinds)
        _abi.check(_abi.lib().decoder_eval(self._h, _ptr(X), _ptr(lat_idx), _ptr(latents), _ptr(dirs), karr,
                                           len(kinds), n, _ptr(out), _stream(stream)))
        return out

    def set_precision(self, fp32):
        """Square-layer arithmetic of decoder_eval and of reduced-order contexts created afterwards:
        False / 0 BF16 tensor cores, True / 1 FP32 CUDA cores, 2 split BF16 (hi + lo operands,
        three products) on the tensor cores."""
        _abi.check(_abi.lib().decoder_set_precision(self._h, int(fp32)))

    def set_concurrency(self, k):
        """Expected number of concurrent calls on different streams (FP32 tiling; see
        decoder_set_concurrency)."""
        _abi.check(_abi.lib().decoder_set_concurrency(self._h, int(k)))

    def status(self, clear=True, stream=None):
        w = C.c_uint32()
        _abi.check(_abi.lib().decoder_status_word(self._h, C.byref(w), int(clear), _stream(stream)))
        return w.value
