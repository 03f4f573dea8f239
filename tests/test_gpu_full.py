"""Full-size parity: every benchmark workload at its full size, in the launch
configurations bench.py times, compared with the oracle byte for byte in full
(the oracle runs on all host cores; the 1.08 GB learned-eval workload takes it
about half a minute). Workloads 5 and 2 also run as bench.py times them
(learned bucketing inside the batched graph: capture, then replay), workload 4
also with one launch chain per block."""
import numpy as np
import pytest

import oracle
from paper_1109_2348_gb300 import (F_GRAPH, F_LEARNED, F_PER_BLOCK_LAUNCH, F_TIMING, Plan, datagen,
                                   model)

from gpu_util import assert_matches_oracle

pytestmark = pytest.mark.gpu


def _run(w, flags=0, model_path=None, **kw):
    import torch
    buf, off = w.generate()
    sizes = np.diff(off.astype(np.int64))
    with Plan(max_blocks=w.num_blocks, max_total_bytes=buf.size, max_block_bytes=int(sizes.max()), flags=flags,
              model_path=model_path, **kw) as plan:
        d_in = torch.from_numpy(buf).cuda()
        L, prim = plan.forward(d_in, off)
        torch.cuda.synchronize()
        assert plan.last_status() == 0
        st = plan.stats()
        return buf, off, L.cpu().numpy(), prim.cpu().numpy(), st


def test_workload1_markov2_100k():
    buf, off, L, prim, _ = _run(datagen.config(1), flags=F_GRAPH)
    assert_matches_oracle(buf, off, L, prim, "workload 1")


def test_workload2_mixed_64x900k_graph():
    buf, off, L, prim, st = _run(datagen.config(2), flags=F_GRAPH)
    assert_matches_oracle(buf, off, L, prim, "workload 2")
    assert st["rounds"] >= 5


@pytest.mark.parametrize("cfg", [2, 4])
def test_workloads_2_and_4_with_16_bit_digits(cfg):
    buf, off, L, prim, st = _run(datagen.config(cfg), flags=F_GRAPH, radix_bits=16)
    assert st["radix_bits"] == 16
    assert_matches_oracle(buf, off, L, prim, f"workload {cfg}, 16-bit digits")


def test_workload3_degenerate_5x900k():
    buf, off, L, prim, st = _run(datagen.config(3), flags=F_GRAPH)
    assert_matches_oracle(buf, off, L, prim, "workload 3")
    assert prim[0] == 0 and st["rounds"] >= 15  # constant block: identity order after ~17 rounds


def test_workload4_uneven_256_graph():
    buf, off, L, prim, _ = _run(datagen.config(4), flags=F_GRAPH)
    assert_matches_oracle(buf, off, L, prim, "workload 4")


def test_workload4_uneven_256_one_launch_chain_per_block():
    buf, off, L, prim, _ = _run(datagen.config(4), flags=F_PER_BLOCK_LAUNCH)
    assert_matches_oracle(buf, off, L, prim, "workload 4, one launch chain per block")


@pytest.fixture(scope="module")
def trained_model_path(tmp_path_factory):
    m = model.train(num_samples=1_000_000, epochs=8)
    path = str(tmp_path_factory.mktemp("model") / "markov3.bwtmodel")
    m.save(path)
    return path


def test_workload5_learned_graph_as_benched(trained_model_path):
    """The configuration bench.py times by default: learned bucketing inside
    the batched CUDA graph on the 1,200-block learned-eval workload (1.08 GB),
    with a model trained as the bench trains it. The first call captures the
    graph, the second replays it; all 1,200 blocks of both outputs must equal
    the oracle's byte for byte, and the GPU inverse of the output must give the
    input back."""
    import torch
    w = datagen.config(5)
    buf, off = w.generate()
    ref_L, ref_p = oracle.bwt_batch(buf, off)
    with Plan(max_blocks=w.num_blocks, max_total_bytes=buf.size, max_block_bytes=900_000,
              flags=F_LEARNED | F_GRAPH, model_path=trained_model_path) as plan:
        d_in = torch.from_numpy(buf).cuda()
        d_L = torch.empty_like(d_in)
        d_p = torch.empty(w.num_blocks, dtype=torch.int32, device="cuda")
        for call in range(2):
            d_L.fill_(0)
            plan.forward_into(d_in, off, d_L, d_p)
            torch.cuda.synchronize()
            assert plan.last_status() == 0
            st = plan.stats()
            assert st["graph_replayed"] == call
            assert st["blocks_routed_plain"] == 0
            L, prim = d_L.cpu().numpy(), d_p.cpu().numpy()
            assert np.array_equal(prim, ref_p), f"call {call}: primary differs in {np.sum(prim != ref_p)} blocks"
            assert np.array_equal(L, ref_L), f"call {call}: L differs at {np.sum(L != ref_L)} positions"
        del d_in
    with Plan(max_blocks=w.num_blocks, max_total_bytes=buf.size, max_block_bytes=900_000) as inv:
        back = inv.inverse(torch.from_numpy(ref_L).cuda(), off, torch.from_numpy(ref_p).cuda())
        torch.cuda.synchronize()
        assert np.array_equal(back.cpu().numpy(), buf)


def test_workload4_learned_graph(trained_model_path):
    """The uneven workload (256 order-3 Markov blocks of 10,000 to 900,000
    bytes) through the learned bucketing in the batched graph, as bench.py
    times it beside the plain and per-block modes: every block equals the
    oracle, and every block is bucketed."""
    import torch
    w = datagen.config(4)
    buf, off = w.generate()
    sizes = np.diff(off.astype(np.int64))
    with Plan(max_blocks=w.num_blocks, max_total_bytes=buf.size, max_block_bytes=int(sizes.max()),
              flags=F_LEARNED | F_GRAPH, model_path=trained_model_path) as plan:
        d_in = torch.from_numpy(buf).cuda()
        L, prim = plan.forward(d_in, off)
        torch.cuda.synchronize()
        assert plan.last_status() == 0
        st = plan.stats()
        L, prim = L.cpu().numpy(), prim.cpu().numpy()
    assert_matches_oracle(buf, off, L, prim, "workload 4 learned+graph")
    assert st["blocks_routed_plain"] == 0, st


def test_workload2_learned_graph_as_benched(trained_model_path):
    """The configuration bench.py times by default: learned bucketing inside the
    batched CUDA graph on the mixed workload, with a model trained as the bench
    trains it. The first call captures the graph, the second replays it; both
    outputs must equal the oracle's."""
    import torch
    w = datagen.config(2)
    buf, off = w.generate()
    with Plan(max_blocks=w.num_blocks, max_total_bytes=buf.size, max_block_bytes=900_000,
              flags=F_LEARNED | F_GRAPH, model_path=trained_model_path) as plan:
        d_in = torch.from_numpy(buf).cuda()
        d_L = torch.empty_like(d_in)
        d_p = torch.empty(w.num_blocks, dtype=torch.int32, device="cuda")
        outs = []
        for _ in range(2):
            d_L.fill_(0)
            plan.forward_into(d_in, off, d_L, d_p)
            torch.cuda.synchronize()
            outs.append((d_L.cpu().numpy(), d_p.cpu().numpy(), plan.stats()))
    for i, (L, prim, st) in enumerate(outs):
        assert_matches_oracle(buf, off, L, prim, f"workload 2 learned+graph call {i}")
    st0, st1 = outs[0][2], outs[1][2]
    assert st1["graph_replayed"] == 1
    # the three sources take the three routes: Markov -> learned, uniform ->
    # equal-width, geometric runs -> plain radix
    assert st0["blocks_routed_flat"] >= 1 and st0["blocks_routed_plain"] >= 1
    assert st0["blocks_routed_flat"] + st0["blocks_routed_plain"] < w.num_blocks


def test_workload2_host_driven_modes(trained_model_path):
    """The mixed workload in the two host-driven launch modes: plain with
    events around every radix launch (the mode bench.py times its roofline
    in) and learned with host-driven rounds."""
    buf, off, L, prim, st = _run(datagen.config(2), flags=F_TIMING)
    assert_matches_oracle(buf, off, L, prim, "workload 2, host-driven with timing")
    assert st["first_launches"] == 8 and st["first_ms"] > 0
    buf, off, L, prim, st = _run(datagen.config(2), flags=F_LEARNED, model_path=trained_model_path)
    assert_matches_oracle(buf, off, L, prim, "workload 2, learned with host-driven rounds")


MAX_BLOCK = (1 << 30) - 1  # the largest block the interface takes


def test_max_block_constant_closed_form():
    """One block of the largest size, all bytes equal: every rotation is the
    same, so the order is by index, L = S and the primary index is 0."""
    import torch
    S = torch.full((MAX_BLOCK,), 0x61, dtype=torch.uint8, device="cuda")
    off = np.array([0, MAX_BLOCK], dtype=np.uint64)
    with Plan(max_blocks=1, max_total_bytes=MAX_BLOCK, max_block_bytes=MAX_BLOCK, flags=F_GRAPH) as plan:
        L, prim = plan.forward(S, off)
        torch.cuda.synchronize()
        st = plan.stats()
        assert bool(torch.equal(L, S)) and int(prim[0]) == 0
        assert st["rounds"] >= 26  # the doubling runs until the prefix length passes n
    del S, L


def test_max_block_uniform_round_trip():
    """One block of the largest size, uniform bytes: L is a permutation of S
    and the GPU inverse of (L, primary) gives S back."""
    import torch
    S = datagen.block(datagen.UNIFORM, 77, MAX_BLOCK)
    off = np.array([0, MAX_BLOCK], dtype=np.uint64)
    d_S = torch.from_numpy(S).cuda()
    with Plan(max_blocks=1, max_total_bytes=MAX_BLOCK, max_block_bytes=MAX_BLOCK, flags=F_GRAPH) as plan:
        L, prim = plan.forward(d_S, off)
        torch.cuda.synchronize()
        assert torch.equal(torch.bincount(L.to(torch.int64), minlength=256),
                           torch.bincount(d_S.to(torch.int64), minlength=256))
        back = plan.inverse(L, off, prim)
        torch.cuda.synchronize()
        assert bool(torch.equal(back, d_S))
