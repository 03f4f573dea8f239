"""ctypes binding of the C ABI in include/bwt.h (argument marshalling only).

Every step of the transform runs in the CUDA library ``csrc/libbwt_gb300.so``;
this module passes pointers and sizes. PyTorch is used by callers for device
memory and streams only. There is no CPU fallback: if the library is missing
or no CUDA device is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
from pathlib import Path

from . import _build

(BWT_OK, BWT_EINVAL, BWT_ENOMEM, BWT_ECAPACITY, BWT_ECUDA, BWT_ETIMEOUT, BWT_EMISMATCH, BWT_ENOMODEL,
 BWT_ETOOBIG, BWT_EINTERNAL) = range(10)
STATUS_NAMES = ["BWT_OK", "BWT_EINVAL", "BWT_ENOMEM", "BWT_ECAPACITY", "BWT_ECUDA", "BWT_ETIMEOUT",
                "BWT_EMISMATCH", "BWT_ENOMODEL", "BWT_ETOOBIG", "BWT_EINTERNAL"]
NOALLOC_MAX_BYTES = 65536

F_GRAPH = 0x1
F_LEARNED = 0x2
F_PER_BLOCK_LAUNCH = 0x4
F_TIMING = 0x8


class PlanDesc(ctypes.Structure):
    _fields_ = [
        ("max_blocks", ctypes.c_uint32),
        ("max_total_bytes", ctypes.c_uint64),
        ("max_block_bytes", ctypes.c_uint32),
        ("radix_bits", ctypes.c_int),
        ("tile_keys", ctypes.c_int),
        ("flags", ctypes.c_uint32),
        ("model_path", ctypes.c_char_p),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("rounds", ctypes.c_uint32),
        ("radix_bits", ctypes.c_uint32),
        ("tile_keys", ctypes.c_uint32),
        ("kernel_launches", ctypes.c_uint64),
        ("radix_launches", ctypes.c_uint64),
        ("radix_keys", ctypes.c_uint64),
        ("radix_ms", ctypes.c_double),
        ("radix_bytes", ctypes.c_double),
        ("active_elements", ctypes.c_uint64),
        ("buckets_overflowed", ctypes.c_uint64),
        ("keys_overflowed", ctypes.c_uint64),
        ("max_bucket", ctypes.c_uint32),
        ("graph_replayed", ctypes.c_uint32),
        ("blocks_routed_plain", ctypes.c_uint32),
        ("blocks_routed_flat", ctypes.c_uint32),
        ("bucket_sq_sum", ctypes.c_uint64),
        ("buckets_nonempty", ctypes.c_uint64),
        ("round_radix_bits", ctypes.c_uint32),
        ("pad2_", ctypes.c_uint32),
        ("first_launches", ctypes.c_uint64),
        ("first_ms", ctypes.c_double),
        ("first_bytes", ctypes.c_double),
        ("chunk_launches", ctypes.c_uint64),
        ("chunk_ms", ctypes.c_double),
        ("chunk_keys", ctypes.c_uint64),
        ("chunk_bytes", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


# Every symbol the header declares (checked by the CPU test suite).
EXPORTS = [
    "bwt_plan_create", "bwt_forward_batch", "bwt_inverse_check", "bwt_inverse_batch", "bwt_plan_destroy",
    "bwt_rle_encode", "bwt_rle_decode", "bwt_vle_encode", "bwt_mtf_encode",
    "bwt_plan_last_status", "bwt_plan_stats", "bwt_plan_set_radix", "bwt_plan_debug_waits",
    "bwt_status_string", "bwt_last_cuda_error",
    "bwt_mlp_forward", "bwt_mlp_loss_grad", "bwt_mlp_adam_step", "bwt_model_train", "bwt_model_samples",
    "bwt_model_compile", "bwt_plan_set_splitters", "bwt_model_save", "bwt_model_load", "bwt_model_byte_norm",
    "bwt_forward_block_noalloc", "bwt_plan_autotune", "bwt_plan_set_round_radix",
]

MLP_NPARAMS = 1377
SPLITTERS = 4095
BUCKETS = 4096

_lib = None


def debug_build() -> bool:
    """True when the environment asks for the bounds-checked library (BWT_DEBUG=1)."""
    return os.environ.get("BWT_DEBUG", "") == "1"


def library_path() -> Path:
    return _build.BWT_DEBUG_SO if debug_build() else _build.BWT_SO


def load(build_if_missing: bool = True):
    """Load libbwt_gb300.so, or libbwt_gb300_debug.so with BWT_DEBUG=1
    (building it in-tree with nvcc if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    debug = debug_build()
    so = library_path()
    if not so.exists():
        if not build_if_missing and not debug:
            raise RuntimeError(f"{so} is missing: run __graft_entry__.build() first")
        _build.build_bwt(debug=debug)
    lib = ctypes.CDLL(str(so))
    vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32
    lib.bwt_plan_create.argtypes = [ctypes.POINTER(PlanDesc), ctypes.c_int, ctypes.POINTER(vp)]
    lib.bwt_plan_create.restype = ctypes.c_int
    lib.bwt_forward_batch.argtypes = [vp, vp, vp, u32, vp, vp, vp]
    lib.bwt_forward_batch.restype = ctypes.c_int
    lib.bwt_inverse_check.argtypes = [vp, u64, i32, vp]
    lib.bwt_inverse_check.restype = ctypes.c_int
    lib.bwt_inverse_batch.argtypes = [vp, vp, vp, u32, vp, vp, vp]
    lib.bwt_inverse_batch.restype = ctypes.c_int
    lib.bwt_rle_encode.argtypes = [vp, vp, vp, u32, vp, vp, vp, vp]
    lib.bwt_rle_encode.restype = ctypes.c_int
    lib.bwt_rle_decode.argtypes = [vp, vp, vp, vp, vp, u32, vp, vp]
    lib.bwt_rle_decode.restype = ctypes.c_int
    lib.bwt_vle_encode.argtypes = [vp, vp, vp, u32, vp, vp, vp, u64, vp, vp, vp]
    lib.bwt_vle_encode.restype = ctypes.c_int
    lib.bwt_mtf_encode.argtypes = [vp, vp, vp, u32, vp, vp]
    lib.bwt_mtf_encode.restype = ctypes.c_int
    lib.bwt_plan_destroy.argtypes = [vp]
    lib.bwt_plan_destroy.restype = ctypes.c_int
    lib.bwt_plan_last_status.argtypes = [vp]
    lib.bwt_plan_last_status.restype = ctypes.c_int
    lib.bwt_plan_stats.argtypes = [vp, ctypes.POINTER(Stats)]
    lib.bwt_plan_stats.restype = ctypes.c_int
    lib.bwt_plan_set_radix.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    lib.bwt_plan_set_radix.restype = ctypes.c_int
    lib.bwt_plan_set_round_radix.argtypes = [vp, ctypes.c_int]
    lib.bwt_plan_set_round_radix.restype = ctypes.c_int
    lib.bwt_plan_debug_waits.argtypes = [vp, u32, ctypes.c_int]
    lib.bwt_plan_debug_waits.restype = ctypes.c_int
    lib.bwt_status_string.argtypes = [ctypes.c_int]
    lib.bwt_status_string.restype = ctypes.c_char_p
    lib.bwt_last_cuda_error.argtypes = []
    lib.bwt_last_cuda_error.restype = ctypes.c_char_p
    f32 = ctypes.c_float
    lib.bwt_mlp_forward.argtypes = [vp, vp, u32, vp, vp]
    lib.bwt_mlp_loss_grad.argtypes = [vp, vp, vp, u32, vp, vp, vp]
    lib.bwt_mlp_adam_step.argtypes = [vp, vp, vp, vp, u32, f32, vp]
    lib.bwt_model_train.argtypes = [vp, vp, vp, u32, vp, u32, u32, f32, vp, vp]
    lib.bwt_model_samples.argtypes = [vp, vp, vp, u32, vp, u32, vp, vp, vp, vp]
    lib.bwt_model_compile.argtypes = [vp, vp, vp, vp]
    lib.bwt_model_byte_norm.argtypes = [vp, u64, vp, vp]
    lib.bwt_plan_set_splitters.argtypes = [vp, vp]
    lib.bwt_model_save.argtypes = [ctypes.c_char_p, vp, vp, vp]
    lib.bwt_model_load.argtypes = [ctypes.c_char_p, vp, vp, vp]
    lib.bwt_plan_autotune.argtypes = [vp, vp, vp, u32, vp, vp, vp, ctypes.c_char_p, ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_float)]
    lib.bwt_plan_autotune.restype = ctypes.c_int
    lib.bwt_forward_block_noalloc.argtypes = [vp, u32, vp, vp, vp]
    lib.bwt_forward_block_noalloc.restype = ctypes.c_int
    for name in ("bwt_mlp_forward", "bwt_mlp_loss_grad", "bwt_mlp_adam_step", "bwt_model_train",
                 "bwt_model_samples", "bwt_model_compile", "bwt_plan_set_splitters", "bwt_model_save",
                 "bwt_model_load", "bwt_model_byte_norm"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


class BWTError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        msg = f"{what}: {name}" if what else name
        if status == BWT_ECUDA and _lib is not None:
            msg += " (" + _lib.bwt_last_cuda_error().decode() + ")"
        super().__init__(msg)


def check(status: int, what: str = "") -> None:
    if status != BWT_OK:
        raise BWTError(status, what)
