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


# ---- variable-length encoding ----------------------------------------------

def huffman_table(counts):
    """A Huffman code (lengths by the textbook merge of the two rarest
    weights, canonical code values) for the bytes with counts > 0; absent
    bytes get the 1-bit code 0 (never used)."""
    import heapq
    used = [c for c in range(256) if counts[c] > 0]
    length = np.ones(256, dtype=np.uint8)
    if len(used) == 1:
        length[used[0]] = 1
    else:
        heap = [(int(counts[c]), i, [c]) for i, c in enumerate(used)]
        heapq.heapify(heap)
        uid = len(heap)
        depth = {c: 0 for c in used}
        while len(heap) > 1:
            w1, _, a = heapq.heappop(heap)
            w2, _, b = heapq.heappop(heap)
            for c in a + b:
                depth[c] += 1
            heapq.heappush(heap, (w1 + w2, uid, a + b))
            uid += 1
        for c in used:
            length[c] = depth[c]
    code = np.zeros(256, dtype=np.uint32)
    nxt, prev = 0, 0
    for c in sorted(used, key=lambda c: (length[c], c)):
        nxt <<= int(length[c]) - prev
        code[c] = nxt
        nxt += 1
        prev = int(length[c])
    return code, length


def _vle_check(blocks, code=None, length=None):
    import torch
    buf, off = batch_from_blocks(blocks)
    if code is None:
        code, length = huffman_table(np.bincount(buf, minlength=256))
    with _plan(buf, off) as plan:
        out, byte_off, bits = plan.vle_encode(torch.from_numpy(buf).cuda(), off, code, length)
        out, byte_off, bits = out.cpu().numpy(), byte_off.cpu().numpy(), bits.cpu().numpy()
    for b in range(off.size - 1):
        ref, ref_bits = oracle.vle_encode(buf[int(off[b]):int(off[b + 1])], code, length)
        assert bits[b] == ref_bits
        assert byte_off[b + 1] - byte_off[b] == ref.size
        assert np.array_equal(out[byte_off[b]:byte_off[b + 1]], ref), b


def test_vle_fig3_lengths():
    lens = [1, 8, 16, 7, 14, 9, 4, 4]
    code = np.zeros(256, dtype=np.uint32)
    length = np.ones(256, dtype=np.uint8)
    for i, L in enumerate(lens):
        code[i] = (1 << L) - 1
        length[i] = L
    _vle_check([np.arange(8, dtype=np.uint8)], code, length)


@pytest.mark.parametrize("src", [datagen.UNIFORM, datagen.MARKOV3_Z96, datagen.RUNS16, datagen.CONST,
                                 datagen.FIBONACCI])
def test_vle_every_source(src):
    _vle_check([datagen.block(src, 70 + i, n) for i, n in enumerate([1, 3, 4095, 4096, 4097, 70_001])])


def test_vle_long_codes_and_many_blocks():
    rng = np.random.default_rng(8)
    code = rng.integers(0, 2**32, 256, dtype=np.uint64).astype(np.uint32)
    length = rng.integers(1, 33, 256).astype(np.uint8)
    length[:4] = 32
    blocks = [rng.integers(0, 256, int(n)).astype(np.uint8) for n in rng.integers(1, 9000, 40)]
    _vle_check(blocks, code, length)


def test_vle_rejects_bad_lengths_and_small_buffers():
    import torch
    buf = np.arange(10, dtype=np.uint8)
    off = np.array([0, 10], dtype=np.uint64)
    code = torch.zeros(256, dtype=torch.int32, device="cuda")
    with _plan(buf, off) as plan:
        d_in = torch.from_numpy(buf).cuda()
        bo = torch.empty(2, dtype=torch.int64, device="cuda")
        bits = torch.empty(1, dtype=torch.int64, device="cuda")
        length = torch.full((256,), 8, dtype=torch.uint8, device="cuda")
        length[3] = 0
        out = torch.empty(64, dtype=torch.uint8, device="cuda")
        assert plan.vle_encode_into(d_in, off, code, length, out, bo, bits, raise_on_error=False) == _lib.BWT_EINVAL
        length[3] = 8
        small = torch.empty(8, dtype=torch.uint8, device="cuda")  # 10 bytes of stream do not fit
        assert plan.vle_encode_into(d_in, off, code, length, small, bo, bits,
                                    raise_on_error=False) == _lib.BWT_ECAPACITY
        plan.vle_encode_into(d_in, off, code, length, out, bo, bits)
        assert int(bo[1]) == 10 and int(bits[0]) == 80


def test_vle_full_workload_with_its_huffman_table():
    w = datagen.config(2)
    buf, off = w.generate()
    _vle_check([buf[int(off[b]):int(off[b + 1])] for b in range(w.num_blocks)])


# ---- move-to-front encoding -------------------------------------------------

def _mtf_check(blocks, tile=0):
    import torch
    buf, off = batch_from_blocks(blocks)
    sizes = np.diff(off.astype(np.int64))
    with Plan(max_blocks=off.size - 1, max_total_bytes=int(off[-1]), max_block_bytes=int(sizes.max()),
              tile_keys=tile) as plan:
        got = plan.mtf_encode(torch.from_numpy(buf).cuda(), off).cpu().numpy()
    want = np.concatenate([oracle.mtf_encode(buf[int(off[b]):int(off[b + 1])]) for b in range(off.size - 1)])
    if not np.array_equal(got, want):
        bad = np.flatnonzero(got != want)
        raise AssertionError(f"{bad.size} positions differ, first {bad[0]}")


def test_mtf_hand_worked_words():
    _mtf_check([np.frombuffer(w, dtype=np.uint8) for w in (b"banana", b"aaab")])


@pytest.mark.parametrize("src", [datagen.UNIFORM, datagen.MARKOV2_Z64, datagen.MARKOV3_Z96, datagen.RUNS16,
                                 datagen.CONST, datagen.PERIOD7, datagen.PERIOD1000, datagen.FIBONACCI,
                                 datagen.MUTATED_UNIT])
def test_mtf_every_source(src):
    _mtf_check([datagen.block(src, 90 + i, n) for i, n in enumerate([1, 2, 4095, 4096, 4097, 50_001])])


@pytest.mark.parametrize("tile", [1024, 4096])
def test_mtf_chunks_chain_across_tiles(tile):
    rng = np.random.default_rng(9)
    blocks = [rng.integers(0, int(a), int(n)).astype(np.uint8)
              for a, n in zip(rng.choice([2, 5, 40, 256], 30), rng.integers(1, 30_000, 30))]
    _mtf_check(blocks, tile)


def test_mtf_of_the_bwt_output():
    import torch
    w = datagen.config(2).subset(range(9))
    buf, off = w.generate()
    L, _ = oracle.bwt_batch(buf, off)
    _mtf_check([L[int(off[b]):int(off[b + 1])] for b in range(w.num_blocks)])


def test_mtf_of_the_bwt_output_full_mixed_workload():
    """Move-to-front of the whole mixed workload's L column (57.6 MB, 64
    blocks of the three sources) against the oracle."""
    w = datagen.config(2)
    buf, off = w.generate()
    L, _ = oracle.bwt_batch(buf, off)
    _mtf_check([L[int(off[b]):int(off[b + 1])] for b in range(w.num_blocks)])


# ---- bounded waits of the single-pass scans -----------------------------------

@pytest.mark.parametrize("stage", ["rle_encode", "rle_decode", "vle_encode"])
def test_stage_scan_wait_times_out_and_the_plan_recovers(stage):
    """The first tile of each scan withholds its publish (the test knob), so
    the look-back wait behind it runs out after 2,000 polls: the call returns
    BWT_ETIMEOUT, and the next call on the same plan, with the knob off, is
    exact against the oracle. Uniform bytes give about one run a byte, so the
    decoding scan over the runs also spans several tiles."""
    import torch
    blocks = [datagen.block(datagen.UNIFORM, 90 + i, n) for i, n in enumerate([20_000, 13_001])]
    buf, off = batch_from_blocks(blocks)
    ref_c, ref_l, ref_ro = oracle.rle_batch(buf, off)
    code = np.arange(256, dtype=np.uint32)
    length = np.full(256, 8, dtype=np.uint8)  # every byte codes as itself
    with _plan(buf, off) as plan:
        d_in = torch.from_numpy(buf).cuda()
        n = buf.size
        chars = torch.empty_like(d_in)
        lens = torch.empty(n, dtype=torch.int32, device="cuda")
        ro = torch.empty(off.size, dtype=torch.int64, device="cuda")
        out = torch.empty(n, dtype=torch.uint8, device="cuda")
        vout = torch.empty(4 * n + 8, dtype=torch.uint8, device="cuda")
        bo = torch.empty(off.size, dtype=torch.int64, device="cuda")
        bits = torch.empty(off.size - 1, dtype=torch.int64, device="cuda")
        d_code = torch.from_numpy(code.view(np.int32)).cuda()
        d_len = torch.from_numpy(length).cuda()
        R = int(ref_ro[-1])
        if stage == "rle_decode":
            chars[:R].copy_(torch.from_numpy(ref_c))
            lens[:R].copy_(torch.from_numpy(ref_l.view(np.int32)))
            ro.copy_(torch.from_numpy(ref_ro.view(np.int64)))

        def call():
            if stage == "rle_encode":
                return plan.rle_encode_into(d_in, off, chars, lens, ro, raise_on_error=False)
            if stage == "rle_decode":
                return plan.rle_decode_into(chars, lens, ro, off, out, raise_on_error=False)
            return plan.vle_encode_into(d_in, off, d_code, d_len, vout, bo, bits, raise_on_error=False)

        plan.debug_waits(2000, True)
        assert call() == _lib.BWT_ETIMEOUT
        plan.debug_waits(0, False)
        assert call() == _lib.BWT_OK
        if stage == "rle_encode":
            assert np.array_equal(ro.cpu().numpy().view(np.uint64), ref_ro)
            assert np.array_equal(chars[:R].cpu().numpy(), ref_c)
            assert np.array_equal(lens[:R].cpu().numpy().view(np.uint32), ref_l)
        elif stage == "rle_decode":
            assert np.array_equal(out.cpu().numpy(), buf)
        else:
            assert int(bo[-1]) == n and np.array_equal(vout[:n].cpu().numpy(), buf)
