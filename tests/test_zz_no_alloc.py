"""The no-allocation entry point against the plan-based one and the oracle.

bwt_forward_block_noalloc serves callers that cannot allocate device memory
(and so cannot create a plan): it sorts one block of up to
BWT_NOALLOC_MAX_BYTES bytes using a fixed scratch array inside the library.
Here it is called through the C ABI, twice in a row on different blocks, and
each result must equal bwt_forward_batch's and the CPU oracle's byte for byte
(the tolerance of every other parity test). This file is collected last on
purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1109_2348_gb300 import Plan, _lib, datagen

pytestmark = pytest.mark.gpu


def _noalloc(lib, d_in, n, d_L, d_p, stream):
    return lib.bwt_forward_block_noalloc(ctypes.c_void_p(d_in.data_ptr()), n, ctypes.c_void_p(d_L.data_ptr()),
                                         ctypes.c_void_p(d_p.data_ptr()), ctypes.c_void_p(stream.cuda_stream))


def _plan_result(block: np.ndarray):
    import torch
    d_in = torch.from_numpy(block).cuda()
    off = np.array([0, block.size], dtype=np.uint64)
    with Plan(max_blocks=1, max_total_bytes=block.size, max_block_bytes=block.size) as plan:
        L, p = plan.forward(d_in, off)
        torch.cuda.synchronize()
        return L.cpu().numpy(), int(p.cpu().numpy()[0])


def test_noalloc_matches_plan_path_on_consecutive_calls():
    import torch
    lib = _lib.load()
    stream = torch.cuda.current_stream()
    cases = [datagen.block(datagen.MARKOV3_Z96, 71, _lib.NOALLOC_MAX_BYTES),
             datagen.block(datagen.PERIOD7, 72, 40_001),
             datagen.block(datagen.RUNS16, 73, 12_345),
             datagen.block(datagen.CONST, 74, 999),
             np.frombuffer(b"mississippi", dtype=np.uint8).copy(),
             # period 2, even length: identical rotations stay tied until 2h >= n ends the rounds
             np.frombuffer(b"ab" * 3000, dtype=np.uint8).copy(),
             # period 2 broken by an odd length: every rotation differs, found late
             np.frombuffer(b"ab" * 3000 + b"a", dtype=np.uint8).copy(),
             datagen.block(datagen.FIBONACCI, 76, 4181),
             datagen.block(datagen.UNIFORM, 75, 1)]
    for first, second in zip(cases[:-1], cases[1:]):
        outs = []
        for block in (first, second):  # two calls in a row share the scratch array
            d_in = torch.from_numpy(block).cuda()
            d_L = torch.empty_like(d_in)
            d_p = torch.full((1,), -1, dtype=torch.int32, device="cuda")
            assert _noalloc(lib, d_in, block.size, d_L, d_p, stream) == _lib.BWT_OK
            outs.append((d_L, d_p))
        torch.cuda.synchronize()
        for block, (d_L, d_p) in zip((first, second), outs):
            ref_L, ref_p = _plan_result(block)
            or_L, or_p = oracle.bwt_block(block)
            assert np.array_equal(ref_L, or_L) and ref_p == or_p
            assert np.array_equal(d_L.cpu().numpy(), or_L)
            assert int(d_p.cpu().numpy()[0]) == or_p


def test_noalloc_rejects_blocks_over_the_limit():
    import torch
    lib = _lib.load()
    stream = torch.cuda.current_stream()
    n = _lib.NOALLOC_MAX_BYTES + 1
    d_in = torch.zeros(n, dtype=torch.uint8, device="cuda")
    d_L = torch.empty_like(d_in)
    d_p = torch.empty(1, dtype=torch.int32, device="cuda")
    assert _noalloc(lib, d_in, n, d_L, d_p, stream) == _lib.BWT_ETOOBIG
    assert _noalloc(lib, d_in, 0, d_L, d_p, stream) == _lib.BWT_EINVAL


def test_noalloc_rejects_overlapping_buffers():
    """No two of input, L and primary may share a byte: partial overlaps and
    a primary slot inside either block are rejected before any launch."""
    import torch
    lib = _lib.load()
    stream = torch.cuda.current_stream()
    n = 1000
    buf = torch.zeros(3 * n, dtype=torch.uint8, device="cuda")
    p_ok = torch.empty(1, dtype=torch.int32, device="cuda")

    def call(i0, l0, p_tensor):
        return lib.bwt_forward_block_noalloc(ctypes.c_void_p(buf.data_ptr() + i0), n,
                                             ctypes.c_void_p(buf.data_ptr() + l0),
                                             ctypes.c_void_p(p_tensor), ctypes.c_void_p(stream.cuda_stream))

    assert call(0, n // 2, p_ok.data_ptr()) == _lib.BWT_EINVAL        # L starts inside the input
    assert call(n // 2, 0, p_ok.data_ptr()) == _lib.BWT_EINVAL        # input starts inside L
    assert call(0, n, buf.data_ptr() + n + 100) == _lib.BWT_EINVAL    # primary inside L
    assert call(n, 2 * n, buf.data_ptr() + n + 100) == _lib.BWT_EINVAL  # primary inside the input
    assert call(0, n, p_ok.data_ptr()) == _lib.BWT_OK                 # adjacent buffers are fine
    torch.cuda.synchronize()
