"""CPU oracle for the forward BWT block sort -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference arms may import this package. It shares no code with the CUDA
path (``paper_1109_2348_gb300``) and never imports it. See ``bwt_oracle.c``
for the definition it implements (Section 3.1 of the paper: sort the rotations
of the block) and for how each routine is pinned.

Parity pin status: every routine here is pinned (brute force, hand-checked
words, inverse round trip, closed forms, finite differences); none is
"parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "bwt_oracle.c"
SO = HERE / "liboracle.so"

_lib = None


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (plain C99, pthreads, libm)."""
    if force or not SO.exists() or SRC.stat().st_mtime > SO.stat().st_mtime:
        tmp = SO.with_suffix(f".so.tmp{os.getpid()}")
        cmd = ["gcc", "-O2", "-std=c99", "-D_GNU_SOURCE", "-Wall", "-shared", "-fPIC", str(SRC),
               "-o", str(tmp), "-lpthread", "-lm"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + res.stdout + res.stderr)
        os.replace(tmp, SO)
    return SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(str(build()))
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        for name in ("oracle_bwt_bruteforce", "oracle_bwt_block"):
            f = getattr(lib, name)
            f.argtypes = [vp, i64, vp, ctypes.POINTER(i32), vp]
            f.restype = ctypes.c_int
        lib.oracle_bwt_batch.argtypes = [vp, vp, ctypes.c_int, vp, vp, ctypes.c_int]
        lib.oracle_bwt_batch.restype = ctypes.c_int
        lib.oracle_inverse_bwt.argtypes = [vp, i64, i32, vp]
        lib.oracle_inverse_bwt.restype = ctypes.c_int
        lib.oracle_mlp_nparams.argtypes = []
        lib.oracle_mlp_nparams.restype = ctypes.c_int
        lib.oracle_mlp_forward.argtypes = [vp, vp, i64, vp]
        lib.oracle_mlp_forward.restype = None
        lib.oracle_mlp_loss_grad.argtypes = [vp, vp, vp, i64, vp]
        lib.oracle_mlp_loss_grad.restype = ctypes.c_double
        lib.oracle_adam_step.argtypes = [vp, vp, vp, vp, i64, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_double]
        lib.oracle_adam_step.restype = None
        _lib = lib
    return _lib


def _u8(a) -> np.ndarray:
    if isinstance(a, (bytes, bytearray, str)):
        a = np.frombuffer(a.encode() if isinstance(a, str) else bytes(a), dtype=np.uint8)
    return np.ascontiguousarray(a, dtype=np.uint8)


def bwt_bruteforce(s, with_sa: bool = False):
    """(L, primary[, SA]) from the definition: a full cyclic comparison sort."""
    S = _u8(s)
    n = S.size
    L = np.empty(n, dtype=np.uint8)
    SA = np.empty(n, dtype=np.int32)
    p = ctypes.c_int32(-1)
    if _load().oracle_bwt_bruteforce(S.ctypes.data, n, L.ctypes.data, ctypes.byref(p), SA.ctypes.data):
        raise ValueError("empty block")
    return (L, p.value, SA) if with_sa else (L, p.value)


def bwt_block(s, with_sa: bool = False):
    """(L, primary[, SA]) by prefix doubling with qsort."""
    S = _u8(s)
    n = S.size
    L = np.empty(n, dtype=np.uint8)
    SA = np.empty(n, dtype=np.int32)
    p = ctypes.c_int32(-1)
    if _load().oracle_bwt_block(S.ctypes.data, n, L.ctypes.data, ctypes.byref(p), SA.ctypes.data):
        raise ValueError("empty block")
    return (L, p.value, SA) if with_sa else (L, p.value)


def bwt_batch(buf: np.ndarray, offsets: np.ndarray, threads: int | None = None):
    """(L uint8[N], primary int32[B]) for every block of a batch."""
    buf = _u8(buf)
    off = np.ascontiguousarray(offsets, dtype=np.uint64)
    nb = off.size - 1
    L = np.empty(buf.size, dtype=np.uint8)
    prim = np.empty(nb, dtype=np.int32)
    th = threads or os.cpu_count() or 1
    if _load().oracle_bwt_batch(buf.ctypes.data, off.ctypes.data, nb, L.ctypes.data, prim.ctypes.data, th):
        raise ValueError("empty block in batch")
    return L, prim


def inverse_bwt(L, primary: int) -> np.ndarray:
    L = _u8(L)
    out = np.empty(L.size, dtype=np.uint8)
    if _load().oracle_inverse_bwt(L.ctypes.data, L.size, int(primary), out.ctypes.data):
        raise ValueError("bad inverse arguments")
    return out


MLP_NPARAMS = 1377


def mlp_forward(params: np.ndarray, x: np.ndarray) -> np.ndarray:
    p = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 8)
    y = np.empty(x.shape[0], dtype=np.float64)
    _load().oracle_mlp_forward(p.ctypes.data, x.ctypes.data, x.shape[0], y.ctypes.data)
    return y


def mlp_loss_grad(params: np.ndarray, x: np.ndarray, t: np.ndarray):
    p = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 8)
    t = np.ascontiguousarray(t, dtype=np.float64)
    g = np.empty(MLP_NPARAMS, dtype=np.float64)
    loss = _load().oracle_mlp_loss_grad(p.ctypes.data, x.ctypes.data, t.ctypes.data, x.shape[0], g.ctypes.data)
    return loss, g


def adam_step(p, g, m, v, t: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place Adam update of float64 arrays p, m, v."""
    for a in (p, g, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    _load().oracle_adam_step(p.ctypes.data, g.ctypes.data, m.ctypes.data, v.ctypes.data, p.size, int(t),
                             lr, beta1, beta2, eps)
