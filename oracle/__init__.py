"""CPU oracle for the forward BWT block sort and the stages after it (run-length,
move-to-front and variable-length encoding) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference arms may import this package. It shares no code with the CUDA
path (``paper_1109_2348_gb300``) and never imports it. See ``bwt_oracle.c``
for the definition it implements (Section 3.1 of the paper: sort the rotations
of the block), ``stages_oracle.c`` for the later stages (Sections 3.2-3.4),
and both for how each routine is pinned.

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
SRCS = [SRC, HERE / "stages_oracle.c"]
SO = HERE / "liboracle.so"

_lib = None


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (plain C99, pthreads, libm)."""
    if force or not SO.exists() or any(s.stat().st_mtime > SO.stat().st_mtime for s in SRCS):
        tmp = SO.with_suffix(f".so.tmp{os.getpid()}")
        cmd = ["gcc", "-O2", "-std=c99", "-D_GNU_SOURCE", "-Wall", "-shared", "-fPIC", *map(str, SRCS),
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
        lib.oracle_rle_encode.argtypes = [vp, i64, vp, vp]
        lib.oracle_rle_encode.restype = i64
        lib.oracle_rle_decode.argtypes = [vp, vp, i64, vp]
        lib.oracle_rle_decode.restype = i64
        for name in ("oracle_mtf_encode", "oracle_mtf_decode"):
            getattr(lib, name).argtypes = [vp, i64, vp]
            getattr(lib, name).restype = None
        lib.oracle_vle_encode.argtypes = [vp, i64, vp, vp, vp, vp]
        lib.oracle_vle_encode.restype = i64
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


def rle_encode(s):
    """(chars uint8[runs], lens uint32[runs]): the maximal runs of s, in order."""
    S = _u8(s)
    chars = np.empty(S.size, dtype=np.uint8)
    lens = np.empty(S.size, dtype=np.uint32)
    k = _load().oracle_rle_encode(S.ctypes.data, S.size, chars.ctypes.data, lens.ctypes.data)
    return chars[:k].copy(), lens[:k].copy()


def rle_decode(chars, lens) -> np.ndarray:
    c = _u8(chars)
    ln = np.ascontiguousarray(lens, dtype=np.uint32)
    out = np.empty(int(ln.sum(dtype=np.uint64)), dtype=np.uint8)
    _load().oracle_rle_decode(c.ctypes.data, ln.ctypes.data, c.size, out.ctypes.data)
    return out


def rle_batch(buf, offsets):
    """Per-block runs of a batch: (chars, lens, run_offsets uint64[nb + 1])."""
    buf = _u8(buf)
    off = np.asarray(offsets, dtype=np.uint64)
    cs, ls, ro = [], [], [0]
    for b in range(off.size - 1):
        c, ln = rle_encode(buf[int(off[b]):int(off[b + 1])])
        cs.append(c)
        ls.append(ln)
        ro.append(ro[-1] + c.size)
    return (np.concatenate(cs) if cs else np.empty(0, np.uint8),
            np.concatenate(ls) if ls else np.empty(0, np.uint32), np.array(ro, dtype=np.uint64))


def mtf_encode(s) -> np.ndarray:
    S = _u8(s)
    out = np.empty(S.size, dtype=np.uint8)
    _load().oracle_mtf_encode(S.ctypes.data, S.size, out.ctypes.data)
    return out


def mtf_decode(s) -> np.ndarray:
    S = _u8(s)
    out = np.empty(S.size, dtype=np.uint8)
    _load().oracle_mtf_decode(S.ctypes.data, S.size, out.ctypes.data)
    return out


def vle_encode(s, code, length, with_pos: bool = False):
    """(bit stream uint8[ceil(bits / 8)], bits[, first bit of every codeword])."""
    S = _u8(s)
    code = np.ascontiguousarray(code, dtype=np.uint32)
    length = np.ascontiguousarray(length, dtype=np.uint8)
    total = int(length[S].astype(np.uint64).sum())
    out = np.zeros((total + 7) // 8, dtype=np.uint8)
    pos = np.empty(S.size, dtype=np.uint64) if with_pos else None
    bits = _load().oracle_vle_encode(S.ctypes.data, S.size, code.ctypes.data, length.ctypes.data, out.ctypes.data,
                                     pos.ctypes.data if with_pos else None)
    return (out, bits, pos) if with_pos else (out, bits)


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
