"""The no-allocation entry point against the plan-based one.

bwt_forward_block_noalloc serves callers that cannot allocate device memory
(and so cannot create a plan): it sorts one block of up to
BWT_NOALLOC_MAX_BYTES bytes using a fixed scratch array inside the library.
Here it is called through the C ABI, twice in a row on different blocks, and
each result must equal bwt_forward_batch's byte for byte (the tolerance of
every other parity test). This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

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
            assert np.array_equal(d_L.cpu().numpy(), ref_L)
            assert int(d_p.cpu().numpy()[0]) == ref_p


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
