"""GPU run-length, move-to-front and variable-length encoding against the
stage oracle (Sections 3.2-3.4): the paper's worked examples, every source
and degenerate block, sizes around the tile, batches of blocks (runs never
cross a block), round trips, and input errors reported as BWT_EINVAL."""
import os

import numpy as np
import pytest

import oracle
from paper_1109_2348_gb300 import Plan, _lib, datagen

from gpu_util import batch_from_blocks

pytestmark = pytest.mark.gpu


def _plan(buf, off):
    sizes = np.diff(off.astype(np.int64))
    return Plan(max_blocks=off.size - 1, max_total_bytes=max(1, int(off[-1])), max_block_bytes=int(sizes.max()))


def _rle_check(blocks):
    import torch
    buf, off = batch_from_blocks(blocks)
    ref_c, ref_l, ref_ro = oracle.rle_batch(buf, off)
    with _plan(buf, off) as plan:
        d_in = torch.from_numpy(buf).cuda()
        c, ln, ro = plan.rle_encode(d_in, off)
        assert np.array_equal(ro.cpu().numpy().astype(np.uint64), ref_ro)
        assert np.array_equal(c.cpu().numpy(), ref_c)
        assert np.array_equal(ln.cpu().numpy().astype(np.uint32), ref_l)
        back = plan.rle_decode(c, ln, ro, off)
        assert torch.equal(back, d_in)


def test_rle_fig1_fig2():
    _rle_check([np.frombuffer(b"AAABBCCC", dtype=np.uint8)])


@pytest.mark.parametrize("src", [datagen.UNIFORM, datagen.MARKOV2_Z64, datagen.MARKOV3_Z96, datagen.RUNS16,
                                 datagen.CONST, datagen.PERIOD7, datagen.PERIOD1000, datagen.FIBONACCI,
                                 datagen.MUTATED_UNIT])
def test_rle_every_source(src):
    _rle_check([datagen.block(src, 50 + i, n) for i, n in enumerate([1, 2, 4095, 4096, 4097, 100_003])])


def test_rle_runs_stop_at_block_edges():
    # the same byte across block boundaries and in many tiny blocks
    blocks = [np.full(n, 7, dtype=np.uint8) for n in [1, 1, 3, 4096, 5000, 1, 2]]
    blocks += [np.full(1, i % 2, dtype=np.uint8) for i in range(300)]
    _rle_check(blocks)


def test_rle_decode_rejects_bad_runs():
    import torch
    buf = np.frombuffer(b"AAABBCCC", dtype=np.uint8).copy()
    off = np.array([0, 8], dtype=np.uint64)
    with _plan(buf, off) as plan:
        chars = torch.tensor([65, 66, 67], dtype=torch.uint8, device="cuda")
        out = torch.empty(8, dtype=torch.uint8, device="cuda")
        ro = torch.tensor([0, 3], dtype=torch.int64, device="cuda")
        for bad in ([3, 2, 2], [3, 0, 5], [3, 2, 4]):  # short, zero length, long
            lens = torch.tensor(bad, dtype=torch.int32, device="cuda")
            assert plan.rle_decode_into(chars, lens, ro, off, out, raise_on_error=False) == _lib.BWT_EINVAL
        lens = torch.tensor([3, 2, 3], dtype=torch.int32, device="cuda")
        plan.rle_decode_into(chars, lens, ro, off, out)
        assert bytes(out.cpu().numpy()) == b"AAABBCCC"


def test_rle_full_mixed_workload():
    w = datagen.config(2)
    buf, off = w.generate()
    _rle_check([buf[int(off[b]):int(off[b + 1])] for b in range(w.num_blocks)])
