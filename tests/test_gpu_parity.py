"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle,
byte for byte on L and the primary index, for every source, edge cases,
every radix width and tile size, the batched graph mode and the per-block
launch mode. Full-size workloads are in test_gpu_full.py."""
import numpy as np
import pytest

from paper_1109_2348_gb300 import F_GRAPH, F_PER_BLOCK_LAUNCH, Plan, datagen

from gpu_util import assert_matches_oracle, batch_from_blocks, gpu_bwt

pytestmark = pytest.mark.gpu


def test_hand_words_and_tiny_blocks():
    words = [b"banana", b"abracadabra", b"mississippi", b"abab", b"aaaa", b"b", b"ba", b"abc", b"cba",
             b"aaaaaaab", b"abababababababab", b"zzzzzzzzz", b"\x00\xff\x00\xff\x00"]
    blocks = [np.frombuffer(w, dtype=np.uint8) for w in words]
    buf, off = batch_from_blocks(blocks)
    L, prim, _ = gpu_bwt(buf, off)
    assert_matches_oracle(buf, off, L, prim, "words")


@pytest.mark.parametrize("n", [1, 2, 3, 7, 8, 9, 15, 16, 17, 31, 32, 33, 63, 64, 65, 255, 1023, 1024, 1025,
                               2047, 2049, 4095, 4096, 4097, 8193])
def test_sizes_around_tiles(n):
    rng = np.random.default_rng(n)
    blocks = [rng.integers(0, 256, n, dtype=np.uint8), rng.integers(0, 2, n, dtype=np.uint8) + 97,
              np.full(n, 7, dtype=np.uint8), np.resize(rng.integers(0, 256, 3, dtype=np.uint8), n)]
    buf, off = batch_from_blocks(blocks)
    L, prim, _ = gpu_bwt(buf, off)
    assert_matches_oracle(buf, off, L, prim, f"n={n}")


@pytest.mark.parametrize("src", range(9))
def test_every_source_small(src):
    w = datagen.Workload("t", [src] * 3, [100 + src, 200 + src, 300 + src], [50_000, 12_345, 70_001])
    buf, off = w.generate()
    L, prim, st = gpu_bwt(buf, off)
    assert_matches_oracle(buf, off, L, prim, datagen.SOURCE_NAMES[src])


@pytest.mark.parametrize("rb", [8, 11, 16])
@pytest.mark.parametrize("tile", [1024, 2048, 4096])
def test_radix_and_tile_variants(rb, tile):
    w = datagen.Workload("t", [datagen.MARKOV3_Z96, datagen.RUNS16, datagen.UNIFORM, datagen.PERIOD1000,
                               datagen.FIBONACCI],
                         [1, 2, 3, 4, 5], [40_000, 30_001, 20_000, 25_000, 33_333])
    buf, off = w.generate()
    L, prim, _ = gpu_bwt(buf, off, radix_bits=rb, tile_keys=tile)
    assert_matches_oracle(buf, off, L, prim, f"rb={rb} tile={tile}")


def test_mixed_batch_scaled_down():
    w = datagen.mixed_64x900k(num_blocks=12, n=60_000)
    buf, off = w.generate()
    L, prim, st = gpu_bwt(buf, off)
    assert_matches_oracle(buf, off, L, prim, "mixed")
    assert st["rounds"] >= 1 and st["radix_launches"] >= 8


def test_degenerate_scaled_down():
    w = datagen.degenerate_5x900k(n=50_000)
    buf, off = w.generate()
    L, prim, st = gpu_bwt(buf, off)
    assert_matches_oracle(buf, off, L, prim, "degenerate")
    assert prim[0] == 0


def test_graph_mode_equals_oracle_and_replays():
    w = datagen.uneven_markov3(num_blocks=24, lo=1_000, hi=40_000)
    buf, off = w.generate()
    import torch
    d_in = torch.from_numpy(buf).cuda()
    with Plan(max_blocks=24, max_total_bytes=buf.size, max_block_bytes=40_000, flags=F_GRAPH) as plan:
        L = torch.empty_like(d_in)
        prim = torch.empty(24, dtype=torch.int32, device="cuda")
        plan.forward_into(d_in, off, L, prim)
        s1 = plan.stats()
        assert_matches_oracle(buf, off, L.cpu().numpy(), prim.cpu().numpy(), "graph first")
        L.zero_()
        prim.zero_()
        plan.forward_into(d_in, off, L, prim)
        s2 = plan.stats()
        assert s2["graph_replayed"] == 1 and s1["graph_replayed"] == 0
        assert s2["rounds"] == s1["rounds"] and s2["kernel_launches"] == s1["kernel_launches"]
        assert_matches_oracle(buf, off, L.cpu().numpy(), prim.cpu().numpy(), "graph replay")


def test_graph_mode_degenerate():
    w = datagen.degenerate_5x900k(n=30_000)
    buf, off = w.generate()
    L, prim, st = gpu_bwt(buf, off, flags=F_GRAPH)
    assert_matches_oracle(buf, off, L, prim, "graph degenerate")
    assert st["rounds"] >= 10


def test_per_block_launch_mode():
    w = datagen.uneven_markov3(num_blocks=10, lo=100, hi=30_000)
    buf, off = w.generate()
    L, prim, st = gpu_bwt(buf, off, flags=F_PER_BLOCK_LAUNCH)
    assert_matches_oracle(buf, off, L, prim, "per-block")


def test_device_offsets_and_reuse_of_plan():
    import torch
    w1 = datagen.mixed_64x900k(num_blocks=3, n=10_000)
    w2 = datagen.Workload("t", [datagen.RUNS16, datagen.CONST], [9, 9], [4_000, 25_000])
    with Plan(max_blocks=4, max_total_bytes=40_000, max_block_bytes=25_000) as plan:
        for w in (w1, w2, w1):
            buf, off = w.generate()
            d_in = torch.from_numpy(buf).cuda()
            d_off = torch.from_numpy(off.view(np.int64)).cuda()
            L, prim = plan.forward(d_in, d_off)
            assert_matches_oracle(buf, off, L.cpu().numpy(), prim.cpu().numpy(), w.name)


def test_argument_errors():
    import torch
    from paper_1109_2348_gb300 import _lib
    with Plan(max_blocks=2, max_total_bytes=100, max_block_bytes=60) as plan:
        d = torch.zeros(100, dtype=torch.uint8, device="cuda")
        L = torch.zeros(100, dtype=torch.uint8, device="cuda")
        p = torch.zeros(3, dtype=torch.int32, device="cuda")
        bad = [np.array([0, 10, 10], dtype=np.uint64),      # empty block
               np.array([1, 10], dtype=np.uint64),          # does not start at 0
               np.array([0, 61], dtype=np.uint64),          # block over max_block_bytes
               np.array([0, 50, 101], dtype=np.uint64),     # over max_total_bytes
               np.array([0, 10, 20, 30], dtype=np.uint64)]  # over max_blocks
        for off in bad:
            assert plan.forward_into(d, off, L, p, raise_on_error=False) == _lib.BWT_EINVAL
        assert plan.forward_into(d, np.array([0, 40], dtype=np.uint64), d, p, raise_on_error=False) == _lib.BWT_EINVAL
        assert plan.forward_into(d, np.array([0, 40, 100], dtype=np.uint64), L, p, raise_on_error=False) == _lib.BWT_OK


def test_bounded_wait_times_out_and_context_survives():
    """A look-back wait that nothing will satisfy runs out after the spin limit
    and the call reports BWT_ETIMEOUT; the next call on the same plan is exact."""
    import torch
    from paper_1109_2348_gb300 import _lib
    w = datagen.Workload("t", [datagen.UNIFORM], [1], [20_000])
    buf, off = w.generate()
    d_in = torch.from_numpy(buf).cuda()
    with Plan(max_blocks=1, max_total_bytes=buf.size, max_block_bytes=buf.size, tile_keys=1024) as plan:
        L = torch.empty_like(d_in)
        p = torch.empty(1, dtype=torch.int32, device="cuda")
        plan.debug_waits(2000, True)
        assert plan.forward_into(d_in, off, L, p, raise_on_error=False) == _lib.BWT_ETIMEOUT
        plan.debug_waits(0, False)
        plan.forward_into(d_in, off, L, p)
        assert_matches_oracle(buf, off, L.cpu().numpy(), p.cpu().numpy(), "after timeout")


def test_autotuner_picks_a_valid_config_and_caches_it(tmp_path):
    import json
    import torch
    w = datagen.uneven_markov3(num_blocks=16, lo=5_000, hi=60_000)
    buf, off = w.generate()
    d_in = torch.from_numpy(buf).cuda()
    cache = str(tmp_path / "tune.jsonl")
    with Plan(max_blocks=16, max_total_bytes=buf.size, max_block_bytes=60_000, flags=F_GRAPH) as plan:
        L = torch.empty_like(d_in)
        p = torch.empty(16, dtype=torch.int32, device="cuda")
        rb, tile, ms = plan.autotune(d_in, off, L, p, cache_path=cache, repeats=2)
        assert rb in (8, 11, 16) and tile in (1024, 2048, 4096) and ms > 0
        st = plan.stats()
        assert st["radix_bits"] == rb and st["tile_keys"] == tile
        assert_matches_oracle(buf, off, L.cpu().numpy(), p.cpu().numpy(), "autotuned")
        lines = [json.loads(x) for x in open(cache)]
        assert lines[-1]["radix_bits"] == rb and lines[-1]["tile_keys"] == tile
        cands = lines[-1]["candidates"]  # [radix_bits, tile_keys, round_radix_bits, ms], all timed
        assert len(cands) == 3 * 3 + 3 and all(c[3] > 0 for c in cands)
        assert {c[0] for c in cands} == {8, 11, 16}
        assert min(c[3] for c in cands) == pytest.approx(ms, rel=1e-3)
    with Plan(max_blocks=16, max_total_bytes=buf.size, max_block_bytes=60_000, flags=F_GRAPH) as plan2:
        L = torch.empty_like(d_in)
        p = torch.empty(16, dtype=torch.int32, device="cuda")
        rb2, tile2, _ = plan2.autotune(d_in, off, L, p, cache_path=cache, repeats=2)
        assert (rb2, tile2) == (rb, tile)
        assert len(open(cache).readlines()) == 1  # read back, no new sweep


@pytest.mark.parametrize("round_bits", [8, 10, 11])
def test_round_radix_widths(round_bits):
    import torch
    w = datagen.Workload("t", [datagen.RUNS16, datagen.PERIOD7, datagen.FIBONACCI, datagen.MUTATED_UNIT],
                         [21, 22, 23, 24], [70_000, 66_000, 50_001, 40_000])
    buf, off = w.generate()
    with Plan(max_blocks=4, max_total_bytes=buf.size, max_block_bytes=70_000) as plan:
        plan.set_round_radix(round_bits)
        L, prim = plan.forward(torch.from_numpy(buf).cuda(), off)
        assert plan.stats()["round_radix_bits"] == round_bits
        assert_matches_oracle(buf, off, L.cpu().numpy(), prim.cpu().numpy(), f"round bits {round_bits}")


@pytest.mark.parametrize("n, want", [(60_000, 8), (65_536, 8), (65_537, 10), (300_000, 10)])
def test_default_round_radix_follows_the_rank_width(n, want):
    """By default the rounds' digit width is 10 when that takes fewer passes
    than 8 over the batch's ranks (17 to 20 bits: two passes instead of
    three), else 8; the result is exact either way."""
    import torch
    w = datagen.Workload("t", [datagen.RUNS16], [31], [n])
    buf, off = w.generate()
    with Plan(max_blocks=1, max_total_bytes=n, max_block_bytes=n) as plan:
        L, prim = plan.forward(torch.from_numpy(buf).cuda(), off)
        st = plan.stats()
        assert st["round_radix_bits"] == want and st["rounds"] >= 1
        assert_matches_oracle(buf, off, L.cpu().numpy(), prim.cpu().numpy(), f"n={n}")


PART16 = 61440  # keys per part of a 16-bit pass


@pytest.mark.parametrize("flags", [0, F_GRAPH])
def test_radix16_parts_and_sub_tiles(flags):
    """16-bit digits: blocks that end just before, at and after a part and a
    4,096-key sub-tile, several parts a block, and tiny blocks whose 8-byte
    key wraps more than once."""
    rng = np.random.default_rng(16)
    sizes = [PART16 - 1, PART16, PART16 + 1, 2 * PART16 + 4097, 4095, 4096, 4097, 1, 2, 3, 7, 8, 9]
    srcs = [datagen.UNIFORM, datagen.MARKOV3_Z96, datagen.RUNS16, datagen.PERIOD7, datagen.FIBONACCI,
            datagen.MUTATED_UNIT, datagen.UNIFORM, datagen.UNIFORM, datagen.UNIFORM, datagen.CONST,
            datagen.UNIFORM, datagen.UNIFORM, datagen.UNIFORM]
    blocks = [datagen.block(src, 500 + i, n) for i, (src, n) in enumerate(zip(srcs, sizes))]
    blocks.append(rng.integers(0, 2, 70_000, dtype=np.uint8) + 97)  # few digits: long runs inside sub-tiles
    buf, off = batch_from_blocks(blocks)
    L, prim, st = gpu_bwt(buf, off, radix_bits=16, flags=flags)
    assert st["radix_bits"] == 16
    assert_matches_oracle(buf, off, L, prim, f"16-bit digits, flags={flags}")


def test_radix16_constant_block_is_one_run():
    """Every key of a constant block has the same digit in every pass: one run
    of 900,000 keys spans every part and sub-tile; the order stays the index
    order (L = S, primary 0)."""
    w = datagen.Workload("t", [datagen.CONST, datagen.MARKOV3_Z96], [1, 2], [900_000, 50_000])
    buf, off = w.generate()
    L, prim, _ = gpu_bwt(buf, off, radix_bits=16, flags=F_GRAPH)
    assert_matches_oracle(buf, off, L, prim, "16-bit, constant block")
    assert prim[0] == 0


def test_radix16_with_learned_bucketing():
    """With BWT_F_LEARNED and 16-bit digits, blocks the routing sends to the
    plain sort take 8-bit passes; the result is exact either way."""
    from paper_1109_2348_gb300 import F_LEARNED, model
    tiny = model.train(datagen.learned_train(num_blocks=2, n=50_000), num_samples=20_000, epochs=2)
    w = datagen.mixed_64x900k(num_blocks=6, n=70_000)
    buf, off = w.generate()
    import torch
    with Plan(max_blocks=6, max_total_bytes=buf.size, max_block_bytes=70_000, radix_bits=16,
              flags=F_LEARNED | F_GRAPH) as plan:
        model.install(plan, tiny.splitters)
        L, prim = plan.forward(torch.from_numpy(buf).cuda(), off)
        assert plan.last_status() == 0
        st = plan.stats()
        assert st["blocks_routed_plain"] >= 1
        assert_matches_oracle(buf, off, L.cpu().numpy(), prim.cpu().numpy(), "learned + 16-bit")


@pytest.mark.parametrize("src, n", [(datagen.MARKOV2_Z64, 100_000), (datagen.CONST, 50_000),
                                     (datagen.PERIOD7, 30_001), (datagen.RUNS16, 80_000),
                                     (datagen.UNIFORM, 20_000), (datagen.FIBONACCI, 40_000)])
def test_graph_skips_empty_rounds_and_sections_like_the_host_loop(src, n):
    """In graph mode the body's second round and each round's large-group
    sections are conditional nodes. On inputs from one round without large
    groups (uniform) to many rounds with them (constant, periodic,
    Fibonacci), the graph must run exactly the rounds the host-driven loop
    runs and give the oracle's output, on capture and on replay."""
    import torch
    w = datagen.Workload("t", [src], [77], [n])
    buf, off = w.generate()
    _, _, st_host = gpu_bwt(buf, off)
    d_in = torch.from_numpy(buf).cuda()
    L = torch.empty_like(d_in)
    prim = torch.empty(1, dtype=torch.int32, device="cuda")
    with Plan(max_blocks=1, max_total_bytes=n, max_block_bytes=n, flags=F_GRAPH) as plan:
        for call in range(2):
            L.zero_()
            plan.forward_into(d_in, off, L, prim)
            torch.cuda.synchronize()
            assert plan.last_status() == 0
            st = plan.stats()
            assert st["rounds"] == st_host["rounds"], (st["rounds"], st_host["rounds"])
            assert st["graph_replayed"] == call
            assert_matches_oracle(buf, off, L.cpu().numpy(), prim.cpu().numpy(), f"graph call {call}")
