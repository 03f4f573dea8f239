"""GPU inverse BWT (bwt_inverse_batch) against the oracle.

* Hand-worked words (tests/golden/bwt_words.txt): the GPU recovers each word
  from its L column and primary index.
* Every source, degenerate blocks (constant, periodic, Fibonacci, mutated
  unit) and sizes around the tile and sample strides: the GPU inverse of the
  oracle's (L, primary) equals the oracle's inverse of the same input, byte
  for byte.
* Round trips through the GPU forward transform, batched, in every sampling
  situation (the primary on a sampled row, n = 1, periodic blocks whose FL
  permutation has several cycles).
* A primary outside [0, n) is reported as BWT_EINVAL.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1109_2348_gb300 import Plan, _lib, datagen

from gpu_util import batch_from_blocks, gpu_bwt

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "bwt_words.txt")


def _gpu_inverse(L, off, prim, plan=None):
    import torch
    sizes = np.diff(off.astype(np.int64))
    own = plan is None
    if own:
        plan = Plan(max_blocks=off.size - 1, max_total_bytes=int(off[-1]), max_block_bytes=int(sizes.max()))
    try:
        d_L = torch.from_numpy(np.ascontiguousarray(L)).cuda()
        d_p = torch.from_numpy(np.ascontiguousarray(prim, dtype=np.int32)).cuda()
        out = plan.inverse(d_L, off, d_p)
        torch.cuda.synchronize()
        return out.cpu().numpy()
    finally:
        if own:
            plan.close()


def _words():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            w, L, p = line.split()
            rows.append((w, L, int(p)))
    return rows


def test_golden_words():
    rows = _words()
    L, off = batch_from_blocks([np.frombuffer(r[1].encode(), dtype=np.uint8) for r in rows])
    S, _ = batch_from_blocks([np.frombuffer(r[0].encode(), dtype=np.uint8) for r in rows])
    got = _gpu_inverse(L, off, np.array([r[2] for r in rows]))
    assert np.array_equal(got, S)


def _oracle_case(blocks):
    buf, off = batch_from_blocks(blocks)
    L, prim = oracle.bwt_batch(buf, off)
    want = np.concatenate([oracle.inverse_bwt(L[int(off[b]):int(off[b + 1])], int(prim[b]))
                           for b in range(off.size - 1)])
    assert np.array_equal(want, buf)  # the oracle's inverse recovers the input
    got = _gpu_inverse(L, off, prim)
    if not np.array_equal(got, want):
        bad = np.flatnonzero(got != want)
        raise AssertionError(f"{bad.size} bytes differ; first at {bad[0]}")


@pytest.mark.parametrize("src", [datagen.UNIFORM, datagen.MARKOV2_Z64, datagen.MARKOV3_Z96, datagen.RUNS16,
                                 datagen.CONST, datagen.PERIOD7, datagen.PERIOD1000, datagen.FIBONACCI,
                                 datagen.MUTATED_UNIT])
def test_every_source_matches_oracle(src):
    blocks = [datagen.block(src, 900 + i, n) for i, n in enumerate([1, 2, 3, 63, 64, 65, 4095, 4096, 4097,
                                                                     70_001])]
    _oracle_case(blocks)


def test_sizes_around_strides_matches_oracle():
    rng = np.random.default_rng(5)
    blocks = []
    for n in [1, 5, 8, 9, 127, 128, 129, 1023, 1024, 1025, 8191, 65_535, 65_536, 65_537, 262_145]:
        blocks.append(rng.integers(0, 4, n).astype(np.uint8))
    _oracle_case(blocks)


def test_periodic_blocks_matches_oracle():
    rng = np.random.default_rng(6)
    blocks = []
    for p, k in [(1, 5000), (2, 3000), (3, 777), (7, 129), (64, 64), (65, 100), (1000, 30), (4096, 3)]:
        u = rng.integers(0, 3, p).astype(np.uint8)
        blocks.append(np.tile(u, k))
    _oracle_case(blocks)


def test_round_trip_through_gpu_forward_mixed_workload():
    import torch
    w = datagen.config(2).subset(range(12))
    buf, off = w.generate()
    sizes = np.diff(off.astype(np.int64))
    with Plan(max_blocks=w.num_blocks, max_total_bytes=buf.size, max_block_bytes=int(sizes.max())) as plan:
        d_in = torch.from_numpy(buf).cuda()
        L, prim = plan.forward(d_in, off)
        back = plan.inverse(L, off, prim)
        torch.cuda.synchronize()
        assert torch.equal(back, d_in)


@pytest.mark.parametrize("cfg", [1, 3, 4])
def test_round_trip_full_workload(cfg):
    """GPU forward, then GPU inverse, of a whole benchmark workload: the one
    100,000-byte block, the degenerate blocks (constant and periodic: the
    primary's cycle covers one period and is repeated) and the 256 uneven
    blocks."""
    import torch
    from paper_1109_2348_gb300 import F_GRAPH
    w = datagen.config(cfg)
    buf, off = w.generate()
    sizes = np.diff(off.astype(np.int64))
    with Plan(max_blocks=w.num_blocks, max_total_bytes=buf.size, max_block_bytes=int(sizes.max()),
              flags=F_GRAPH) as plan:
        d_in = torch.from_numpy(buf).cuda()
        L, prim = plan.forward(d_in, off)
        back = plan.inverse(L, off, prim)
        torch.cuda.synchronize()
        assert torch.equal(back, d_in)


def test_bad_primary_is_einval():
    import torch
    buf = np.frombuffer(b"banana", dtype=np.uint8).copy()
    off = np.array([0, 6], dtype=np.uint64)
    with Plan(max_blocks=1, max_total_bytes=6, max_block_bytes=6) as plan:
        d_L = torch.from_numpy(buf).cuda()
        out = torch.empty_like(d_L)
        for bad in (6, -1):
            d_p = torch.tensor([bad], dtype=torch.int32, device="cuda")
            assert plan.inverse_into(d_L, off, d_p, out, raise_on_error=False) == _lib.BWT_EINVAL
        # the plan stays usable
        d_p = torch.tensor([3], dtype=torch.int32, device="cuda")
        L, _ = oracle.bwt_block(b"banana")
        d_L = torch.from_numpy(np.asarray(L)).cuda()
        plan.inverse_into(d_L, off, d_p, out)
        assert bytes(out.cpu().numpy()) == b"banana"
