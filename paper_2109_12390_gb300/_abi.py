"""ctypes declarations of the C ABI in include/mpmrom.h (argument marshalling only).

The shared library is built in-tree by ``paper_2109_12390_gb300.build`` into
``_lib/libmpmrom.so``.  If it is missing, :func:`lib` raises: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libmpmrom.so")

MPM_OK, MPM_EINVAL, MPM_ENOMEM, MPM_ECUDA, MPM_EUNSTABLE, MPM_ENOCONV, MPM_ETIMEOUT, MPM_ENOTIMPL = range(8)
STATUS_BITS = {
    1 << 0: "NONFINITE", 1 << 1: "INVERTED", 1 << 2: "OUT_OF_GRID", 1 << 3: "GN_NO_DECREASE",
    1 << 4: "CHOLESKY", 1 << 5: "TIMEOUT", 1 << 6: "CAPACITY",
}


class MpmConfig(C.Structure):
    _fields_ = [
        ("dim", C.c_int32), ("n_grid", C.c_int32), ("dx", C.c_float), ("dt", C.c_float),
        ("gravity", C.c_float * 3), ("bc", C.c_int32), ("bc_width", C.c_int32),
        ("material", C.c_int32), ("transfer", C.c_int32), ("rho", C.c_float), ("p_vol", C.c_float),
        ("n_inst", C.c_int32), ("E", C.POINTER(C.c_float)), ("nu", C.POINTER(C.c_float)),
        ("inst_offsets", C.POINTER(C.c_int64)), ("polar_eft", C.c_int32),
        ("plastic_compression", C.c_float), ("plastic_stretch", C.c_float),
    ]


class DecoderDesc(C.Structure):
    _fields_ = [("d", C.c_int32), ("r", C.c_int32), ("width", C.c_int32), ("n_hidden", C.c_int32),
                ("activation", C.c_int32)]


DECODER_PRIMAL, DECODER_JVP, DECODER_SECANT, DECODER_MIXED = 0, 1000, 1001, 2000


class RomConfig(C.Structure):
    _fields_ = [
        ("dim", C.c_int32), ("n_grid", C.c_int32), ("dx", C.c_float), ("dt", C.c_float),
        ("gravity", C.c_float * 3), ("bc", C.c_int32), ("bc_width", C.c_int32),
        ("material", C.c_int32), ("transfer", C.c_int32), ("rho", C.c_float), ("p_vol", C.c_float),
        ("E", C.c_float), ("nu", C.c_float), ("latent_dim", C.c_int32), ("n_samples", C.c_int32),
        ("seed", C.c_uint64), ("instance", C.c_int32), ("gn_iters", C.c_int32), ("projection", C.c_int32),
        ("ridge", C.c_float), ("affine", C.c_int32), ("f_reference", C.c_int32),
        ("quadrature", C.c_int32), ("ell", C.c_int32), ("newton_iters", C.c_int32), ("newton_tol", C.c_float),
    ]


class SnapshotDesc(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n_inst", C.c_int32), ("inst_offsets", C.c_void_p), ("X", C.c_void_p),
                ("n_snap", C.c_int32), ("snap_inst", C.c_void_p), ("snap_next", C.c_void_p),
                ("x", C.c_void_p), ("v", C.c_void_p), ("F", C.c_void_p)]


class TrainConfig(C.Structure):
    _fields_ = [("lambda_F", C.c_float), ("lambda_v", C.c_float), ("dt_snap", C.c_float), ("lr0", C.c_float),
                ("lr1", C.c_float), ("batch", C.c_int32), ("total_steps", C.c_int64), ("seed", C.c_uint64),
                ("encoder_subset", C.c_int32), ("shard_index", C.c_int32), ("shard_count", C.c_int32)]


class MpmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"mpmrom status {status}: {msg}")
        self.status = status


_lib = None

# (name, restype, argtypes); every symbol the header declares
SIGNATURES = [
    ("mpm_last_error", C.c_char_p, []),
    ("mpm_init", C.c_int, [C.POINTER(MpmConfig), C.POINTER(C.c_void_p)]),
    ("mpm_destroy", None, [C.c_void_p]),
    ("mpm_set_state", C.c_int, [C.c_void_p] + [C.c_void_p] * 4 + [C.c_void_p]),
    ("mpm_get_state", C.c_int, [C.c_void_p] + [C.c_void_p] * 4 + [C.c_void_p]),
    ("mpm_step", C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    ("mpm_set_kinematic", C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    ("mpm_step_profiled", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_size_t, C.POINTER(C.c_float), C.c_void_p]),
    ("mpm_step_timed", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_size_t, C.POINTER(C.c_float), C.c_void_p]),
    ("mpm_status_word", C.c_int, [C.c_void_p, C.POINTER(C.c_uint32), C.c_int, C.c_void_p]),
    ("mpm_debug_bins", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("mpm_num_block_keys", C.c_int64, [C.c_void_p]),
    ("mpm_step_noalloc", C.c_int, [C.POINTER(MpmConfig)] + [C.c_void_p] * 4 + [C.c_int, C.POINTER(C.c_uint32),
                                                                                C.c_void_p]),
    ("mpm_debug_grid", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("decoder_create", C.c_int, [C.POINTER(DecoderDesc), C.POINTER(C.c_void_p)]),
    ("decoder_destroy", None, [C.c_void_p]),
    ("decoder_num_params", C.c_int64, [C.c_void_p]),
    ("decoder_set_params", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("decoder_get_params", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("decoder_eval", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                               C.POINTER(C.c_int32), C.c_int, C.c_int64, C.c_void_p, C.c_void_p]),
    ("decoder_status_word", C.c_int, [C.c_void_p, C.POINTER(C.c_uint32), C.c_int, C.c_void_p]),
    ("decoder_set_precision", C.c_int, [C.c_void_p, C.c_int]),
    ("decoder_set_concurrency", C.c_int, [C.c_void_p, C.c_int]),
    ("rom_create", C.c_int, [C.POINTER(RomConfig), C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_void_p)]),
    ("rom_destroy", None, [C.c_void_p]),
    ("rom_set_state", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    ("rom_get_state", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("rom_fit_initial", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    ("rom_set_reference", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("rom_step", C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    ("rom_status_word", C.c_int, [C.c_void_p, C.POINTER(C.c_uint32), C.c_int, C.c_void_p]),
    ("rom_debug", C.c_int, [C.c_void_p] + [C.c_void_p] * 5 + [C.c_void_p]),
    ("rom_debug_line_search", C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_int32), C.c_void_p]),
    ("rom_debug_quadrature", C.c_int, [C.c_void_p, C.POINTER(C.c_int32)] + [C.c_void_p] * 4 + [C.c_void_p]),
    ("rom_decode_all", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("rom_set_kinematic", C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p]),
    ("rom_batch_create", C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(C.c_void_p)]),
    ("rom_batch_step", C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    ("rom_batch_destroy", None, [C.c_void_p]),
    ("rom_decode_points", C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    ("metric_accumulate", C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    ("decoder_fit_scaling", C.c_int, [C.c_void_p, C.POINTER(SnapshotDesc), C.c_void_p]),
    ("trainer_create", C.c_int, [C.c_void_p, C.POINTER(TrainConfig), C.POINTER(SnapshotDesc), C.c_void_p,
                                 C.POINTER(C.c_void_p)]),
    ("trainer_destroy", None, [C.c_void_p]),
    ("decoder_train", C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    ("trainer_gradient_sizes", C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    ("trainer_compute_gradients", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("trainer_apply_gradients", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("trainer_loss", C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_void_p]),
    ("trainer_get_latents", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("trainer_status_word", C.c_int, [C.c_void_p, C.POINTER(C.c_uint32), C.c_int, C.c_void_p]),
    ("trainer_gradients", C.c_int, [C.c_void_p] + [C.c_void_p] * 5 + [C.POINTER(C.c_double), C.c_void_p]),
    ("trainer_encoder_params", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int64), C.c_void_p]),
    ("trainer_set_encoder_params", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("trainer_encode", C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p]),
]


def lib():
    """The loaded libmpmrom.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2109_12390_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status):
    if status != MPM_OK:
        raise MpmError(status, lib().mpm_last_error().decode())
    return status


def status_names(word):
    return [name for bit, name in STATUS_BITS.items() if word & bit]
