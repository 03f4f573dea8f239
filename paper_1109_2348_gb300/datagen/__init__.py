"""Seeded synthetic workloads for the BWT block sort.

This module only draws random bytes (see ``gen.c``); it holds none of the
transform's arithmetic, and both the CUDA path and the CPU oracle take their
inputs from it. The paper (Section 3.1) runs no experiments and names no
dataset, so the five workloads below are synthetic stand-ins shaped like bzip2
input blocks. Each block is (source, seed, size); a batch is the blocks
concatenated, with ``offsets[b] .. offsets[b+1]`` delimiting block b.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

from .. import _build

UNIFORM, MARKOV2_Z64, MARKOV3_Z96, RUNS16 = 0, 1, 2, 3
CONST, PERIOD7, PERIOD1000, FIBONACCI, MUTATED_UNIT = 4, 5, 6, 7, 8
SOURCE_NAMES = {
    UNIFORM: "uniform", MARKOV2_Z64: "markov2-zipf1.1-64", MARKOV3_Z96: "markov3-zipf1.2-96",
    RUNS16: "runs-geom50-16", CONST: "constant-0x61", PERIOD7: "period-7",
    PERIOD1000: "period-1000", FIBONACCI: "fibonacci", MUTATED_UNIT: "unit4096-mut5%",
}

BLOCK_900K = 900_000

_lib = None


def _load():
    global _lib
    if _lib is None:
        so = _build.build_datagen()
        lib = ctypes.CDLL(str(so))
        u64p = ctypes.POINTER(ctypes.c_uint64)
        lib.gen_block.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_uint64]
        lib.gen_block.restype = ctypes.c_int
        lib.gen_batch.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_int]
        lib.gen_batch.restype = ctypes.c_int
        lib.gen_uniform_ints.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, u64p]
        lib.gen_uniform_ints.restype = None
        lib.gen_uniform_unit.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p]
        lib.gen_uniform_unit.restype = None
        lib.gen_rng_probe.argtypes = [ctypes.c_uint64, u64p]
        lib.gen_rng_probe.restype = None
        lib.gen_splitmix_probe.argtypes = [ctypes.c_uint64, ctypes.c_int, u64p]
        lib.gen_splitmix_probe.restype = None
        lib.gen_permutation.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p]
        lib.gen_permutation.restype = None
        _lib = lib
    return _lib


def block(source: int, seed: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.uint8)
    if _load().gen_block(source, seed, out.ctypes.data, n) != 0:
        raise ValueError(f"unknown source {source}")
    return out


def uniform_ints(seed: int, count: int, lo: int, hi: int) -> np.ndarray:
    out = np.empty(count, dtype=np.uint64)
    _load().gen_uniform_ints(seed, count, lo, hi, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
    return out


def uniform_unit(seed: int, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.float64)
    _load().gen_uniform_unit(seed, count, out.ctypes.data)
    return out


def permutation(seed: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.uint32)
    _load().gen_permutation(seed, n, out.ctypes.data)
    return out


def rng_probe(seed: int) -> list[int]:
    out = (ctypes.c_uint64 * 8)()
    _load().gen_rng_probe(seed, out)
    return list(out)


def splitmix_probe(state: int, count: int) -> list[int]:
    out = (ctypes.c_uint64 * count)()
    _load().gen_splitmix_probe(state, count, out)
    return list(out)


@dataclass
class Workload:
    """A batch of independent blocks: block b is gen(sources[b], seeds[b], sizes[b])."""
    name: str
    sources: list[int]
    seeds: list[int]
    sizes: list[int]
    notes: dict = field(default_factory=dict)

    @property
    def num_blocks(self) -> int:
        return len(self.sizes)

    @property
    def total_bytes(self) -> int:
        return int(sum(self.sizes))

    def offsets(self) -> np.ndarray:
        off = np.zeros(len(self.sizes) + 1, dtype=np.uint64)
        np.cumsum(np.asarray(self.sizes, dtype=np.uint64), out=off[1:])
        return off

    def generate(self, threads: int | None = None, out: np.ndarray | None = None) -> tuple[np.ndarray, np.ndarray]:
        """Returns (bytes uint8[N], offsets uint64[B+1]); `out` may be a preallocated
        (e.g. pinned) uint8 buffer of at least N bytes."""
        off = self.offsets()
        n = int(off[-1])
        buf = np.empty(n, dtype=np.uint8) if out is None else out[:n]
        src = np.asarray(self.sources, dtype=np.int32)
        seed = np.asarray(self.seeds, dtype=np.uint64)
        th = threads or os.cpu_count() or 1
        if _load().gen_batch(len(self.sizes), src.ctypes.data, seed.ctypes.data, off.ctypes.data,
                             buf.ctypes.data, th) != 0:
            raise ValueError("bad source id in workload")
        return buf, off

    def reseeded(self, offset: int) -> "Workload":
        """The same shapes and sources with every seed shifted by `offset`:
        distinct units of work for another rank."""
        if offset == 0:
            return self
        return Workload(self.name + f"+seed{offset}", list(self.sources), [s + offset for s in self.seeds],
                        list(self.sizes), dict(self.notes))

    def subset(self, idx) -> "Workload":
        idx = list(idx)
        return Workload(self.name + f"[{len(idx)} blocks]", [self.sources[i] for i in idx],
                        [self.seeds[i] for i in idx], [self.sizes[i] for i in idx], dict(self.notes))


def markov2_block_100k() -> Workload:
    """One 100,000-byte block, order-2 Markov, 64 symbols, Zipf(1.1), seed 1."""
    return Workload("markov2-1x100000", [MARKOV2_Z64], [1], [100_000])


def mixed_64x900k(num_blocks: int = 64, n: int = BLOCK_900K) -> Workload:
    """Blocks of n bytes; block b draws from source b mod 3 (uniform, order-3
    Markov text-like, geometric runs) with seed 1000 + b."""
    srcs = [(UNIFORM, MARKOV3_Z96, RUNS16)[b % 3] for b in range(num_blocks)]
    return Workload(f"mixed3-{num_blocks}x{n}", srcs, [1000 + b for b in range(num_blocks)],
                    [n] * num_blocks)


DEGENERATE_SOURCES = [CONST, PERIOD7, PERIOD1000, FIBONACCI, MUTATED_UNIT]


def degenerate_5x900k(n: int = BLOCK_900K) -> Workload:
    """Constant, period-7, period-1000, Fibonacci word and mutated 4 KB unit."""
    return Workload(f"degenerate-5x{n}", list(DEGENERATE_SOURCES), [3000 + b for b in range(5)], [n] * 5)


def uneven_markov3(num_blocks: int = 256, lo: int = 10_000, hi: int = BLOCK_900K,
                   size_seed: int = 4000) -> Workload:
    """num_blocks order-3 Markov blocks with sizes uniform in [lo, hi]."""
    sizes = [int(x) for x in uniform_ints(size_seed, num_blocks, lo, hi)]
    return Workload(f"uneven-markov3-{num_blocks}x[{lo},{hi}]", [MARKOV3_Z96] * num_blocks,
                    [4001 + b for b in range(num_blocks)], sizes)


def learned_eval(num_blocks: int = 1200, n: int = BLOCK_900K) -> Workload:
    """Held-out evaluation set for the learned bucketing: order-3 Markov blocks
    (seeds 6000+) with every tenth block replaced by uniform random bytes (seeds
    7000+), i.e. 1,080 Markov + 120 uniform blocks at the default size."""
    srcs, seeds = [], []
    for b in range(num_blocks):
        if b % 10 == 9:
            srcs.append(UNIFORM); seeds.append(7000 + b // 10)
        else:
            srcs.append(MARKOV3_Z96); seeds.append(6000 + b)
    return Workload(f"learned-eval-{num_blocks}x{n}", srcs, seeds, [n] * num_blocks)


def learned_train(num_blocks: int = 100, n: int = BLOCK_900K) -> Workload:
    """Training blocks for the learned CDF: order-3 Markov, seeds 5000..5099."""
    return Workload(f"learned-train-{num_blocks}x{n}", [MARKOV3_Z96] * num_blocks,
                    [5000 + b for b in range(num_blocks)], [n] * num_blocks)


def config(k: int) -> Workload:
    """The five benchmark workloads at full size (1-based numbering)."""
    return {1: markov2_block_100k, 2: mixed_64x900k, 3: degenerate_5x900k,
            4: uneven_markov3, 5: learned_eval}[k]()
