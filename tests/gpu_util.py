"""Helpers shared by the GPU parity tests: run the CUDA path through the
C ABI and compare with the oracle byte for byte."""
from __future__ import annotations

import numpy as np

import oracle
from paper_1109_2348_gb300 import Plan, datagen


def gpu_bwt(buf: np.ndarray, off: np.ndarray, plan: Plan | None = None, **plan_kw):
    import torch
    d_in = torch.from_numpy(np.ascontiguousarray(buf)).cuda()
    own = plan is None
    if own:
        sizes = np.diff(off.astype(np.int64))
        plan = Plan(max_blocks=max(1, off.size - 1), max_total_bytes=max(1, int(off[-1])),
                    max_block_bytes=int(sizes.max()), **plan_kw)
    try:
        L, prim = plan.forward(d_in, off)
        torch.cuda.synchronize()
        assert plan.last_status() == 0, f"device-side status {plan.last_status()}"
        stats = plan.stats()
        return L.cpu().numpy(), prim.cpu().numpy(), stats
    finally:
        if own:
            plan.close()


def assert_matches_oracle(buf, off, L, prim, label=""):
    ref_L, ref_p = oracle.bwt_batch(buf, off)
    if not np.array_equal(prim, ref_p):
        bad = np.flatnonzero(prim != ref_p)
        raise AssertionError(f"{label}: primary differs in {bad.size} blocks, first {bad[:5]} "
                             f"got {prim[bad[:5]]} want {ref_p[bad[:5]]}")
    if not np.array_equal(L, ref_L):
        bad = np.flatnonzero(L != ref_L)
        blk = np.searchsorted(off, bad[0], side="right") - 1
        raise AssertionError(f"{label}: L differs at {bad.size} positions; first {bad[0]} (block {blk})")


def batch_from_blocks(blocks: list[np.ndarray]):
    off = np.zeros(len(blocks) + 1, dtype=np.uint64)
    off[1:] = np.cumsum([b.size for b in blocks])
    return np.concatenate(blocks).astype(np.uint8), off
