"""GPU tests of the learned CDF model and the learned bucketing.

* The FP32 forward / loss gradient / Adam kernels against the float64 oracle
  on fixed weights and batches (relative 1e-4, absolute 1e-6).
* Training on samples the plain sorter produces lowers the loss; the compiled
  splitter table is sorted.
* The learned path equals the oracle byte for byte (held-out Markov blocks,
  uniform blocks that overflow, degenerate blocks, tiny blocks), whatever the
  splitter table.
* What the model gains: on held-out Markov blocks its buckets are far more
  even than the equal-width splitters of the method without it.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1109_2348_gb300 import F_GRAPH, F_LEARNED, Plan, _lib, datagen, model

from gpu_util import assert_matches_oracle, gpu_bwt

pytestmark = pytest.mark.gpu


def _vp(t):
    return ctypes.c_void_p(int(t.data_ptr()))


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _batch(seed, B):
    rng = np.random.default_rng(seed)
    p = model.init_params(seed).astype(np.float64)
    p += rng.normal(0, 0.05, p.size)  # biases away from zero so ReLUs are mixed
    x = rng.integers(0, 256, (B, 8)) / 255.0
    t = rng.random(B)
    return p, x, t


def test_mlp_forward_matches_oracle():
    import torch
    lib = _lib.load()
    p, x, _ = _batch(1, 1000)
    d_p = torch.from_numpy(p.astype(np.float32)).cuda()
    d_x = torch.from_numpy(x.astype(np.float32)).cuda()
    d_y = torch.empty(1000, dtype=torch.float32, device="cuda")
    assert lib.bwt_mlp_forward(_vp(d_p), _vp(d_x), 1000, _vp(d_y), _stream()) == 0
    ref = oracle.mlp_forward(p.astype(np.float32).astype(np.float64), x.astype(np.float32).astype(np.float64))
    got = d_y.cpu().numpy().astype(np.float64)
    assert np.allclose(got, ref, rtol=1e-4, atol=1e-6)


@pytest.mark.parametrize("B", [1, 63, 64, 4096, 5000])
def test_mlp_gradient_matches_oracle(B):
    import torch
    lib = _lib.load()
    p, x, t = _batch(B, B)
    p32, x32, t32 = p.astype(np.float32), x.astype(np.float32), t.astype(np.float32)
    d = [torch.from_numpy(a).cuda() for a in (p32, x32, t32)]
    d_g = torch.empty(_lib.MLP_NPARAMS, dtype=torch.float32, device="cuda")
    d_l = torch.empty(1, dtype=torch.float32, device="cuda")
    assert lib.bwt_mlp_loss_grad(_vp(d[0]), _vp(d[1]), _vp(d[2]), B, _vp(d_g), _vp(d_l), _stream()) == 0
    loss, g = oracle.mlp_loss_grad(p32.astype(np.float64), x32.astype(np.float64), t32.astype(np.float64))
    got = d_g.cpu().numpy().astype(np.float64)
    assert np.allclose(got, g, rtol=1e-4, atol=1e-6), np.max(np.abs(got - g))
    assert abs(float(d_l.cpu()[0]) - loss) <= 1e-4 * abs(loss) + 1e-6


def test_adam_step_matches_oracle():
    import torch
    lib = _lib.load()
    rng = np.random.default_rng(3)
    p = rng.normal(0, 1, _lib.MLP_NPARAMS)
    g = rng.normal(0, 1, _lib.MLP_NPARAMS)
    m = rng.normal(0, 0.1, _lib.MLP_NPARAMS)
    v = rng.random(_lib.MLP_NPARAMS) * 0.1
    d = [torch.from_numpy(a.astype(np.float32)).cuda() for a in (p, g, m, v)]
    for step in (1, 2, 7):
        assert lib.bwt_mlp_adam_step(_vp(d[0]), _vp(d[1]), _vp(d[2]), _vp(d[3]), step, ctypes.c_float(1e-3),
                                     _stream()) == 0
        oracle.adam_step(p, g, m, v, step, lr=1e-3)
    for dt, ref in zip(d, (p, g, m, v)):
        assert np.allclose(dt.cpu().numpy().astype(np.float64), ref, rtol=1e-4, atol=1e-6)


@pytest.fixture(scope="module")
def small_model():
    w = datagen.learned_train(num_blocks=12, n=200_000)
    return model.train(w, num_samples=200_000, epochs=6, batch=4096, lr=2e-3, seed=5000)


def test_training_lowers_loss_and_compiles_sorted_splitters(small_model):
    loss = small_model.epoch_loss
    assert loss[-1] < 0.5 * loss[0], loss
    assert loss[-1] < 0.01, loss
    s = small_model.splitters
    assert s.size == _lib.SPLITTERS and np.all(s[1:] >= s[:-1])


def test_training_samples_come_from_the_plain_sort():
    """A sample's target is its rotation's row / n in the plain sort and its
    inputs are the rotation's 8 bytes through the byte-value CDF; check both
    against the oracle's rotation order and a direct count on one block."""
    w = datagen.learned_train(num_blocks=1, n=30_000)
    d_x, d_t, d_norm = model.make_samples(w, 500, seed=9)
    buf, off = w.generate()
    _, _, SA = oracle.bwt_block(buf, with_sa=True)
    pos = datagen.uniform_ints(9, 500, 0, int(off[-1]) - 1)
    x = d_x.cpu().numpy()
    t = d_t.cpu().numpy()
    n = buf.size
    cnt = np.bincount(buf, minlength=256).astype(np.float64)
    norm_ref = (np.cumsum(cnt) - cnt + 0.5 * cnt) / n
    assert np.allclose(d_norm.cpu().numpy(), norm_ref, atol=1e-7)
    for s in range(500):
        k = int(pos[s])
        i = SA[k]
        want = norm_ref[buf[(i + np.arange(8)) % n]]
        assert np.allclose(x[s], want, atol=1e-6)
        assert abs(t[s] - k / n) < 1e-6


def _learned_run(buf, off, splitters, graph=False, **kw):
    import torch
    sizes = np.diff(off.astype(np.int64))
    flags = F_LEARNED | (F_GRAPH if graph else 0)
    with Plan(max_blocks=off.size - 1, max_total_bytes=buf.size, max_block_bytes=int(sizes.max()), flags=flags,
              **kw) as plan:
        model.install(plan, splitters)
        d_in = torch.from_numpy(buf).cuda()
        L, prim = plan.forward(d_in, off)
        torch.cuda.synchronize()
        return L.cpu().numpy(), prim.cpu().numpy(), plan.stats()


def test_learned_equals_oracle_on_held_out_blocks(small_model):
    w = datagen.learned_eval(num_blocks=20, n=150_000)
    buf, off = w.generate()
    L, prim, st = _learned_run(buf, off, small_model.splitters)
    assert_matches_oracle(buf, off, L, prim, "learned held-out")
    # the uniform blocks overflow the Markov-trained buckets and take the
    # equal-width fallback (their bytes are even over the key space)
    assert st["blocks_routed_flat"] >= 1 and st["blocks_routed_plain"] == 0, st


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("which", ["model", "equal_width"])
def test_learned_path_exact_for_any_splitters(small_model, which, graph):
    spl = small_model.splitters if which == "model" else model.equal_width_splitters()
    w = datagen.Workload("t", [datagen.CONST, datagen.PERIOD7, datagen.FIBONACCI, datagen.RUNS16, datagen.UNIFORM,
                               datagen.MARKOV3_Z96, datagen.MARKOV2_Z64],
                         [1, 2, 3, 4, 5, 6, 7], [30_000, 20_001, 25_000, 40_000, 3, 60_000, 7_777])
    buf, off = w.generate()
    L, prim, st = _learned_run(buf, off, spl, graph=graph)
    assert_matches_oracle(buf, off, L, prim, f"{which} graph={graph}")
    assert st["blocks_routed_plain"] >= 1, st  # the constant block overflows every bucketing


def _prefix_keys(block):
    """Every rotation's 8-byte big-endian prefix (cyclic), as the bucketing sees it."""
    n = block.size
    idx = (np.arange(n)[:, None] + np.arange(8)[None, :]) % n
    k = np.zeros(n, dtype=np.uint64)
    for j in range(8):
        k = (k << np.uint64(8)) | block[idx[:, j]].astype(np.uint64)
    return k


@pytest.mark.parametrize("graph", [False, True])
def test_overfull_buckets_big_chunk_sort_and_radix(small_model, graph):
    """A bucket above the 3,328-rotation chunk capacity is sorted whole by one
    CTA (512 threads up to 6,656 rotations, 1,024 up to 13,312) and by the
    overflow radix beyond; here one bucket of each of the last two kinds.
    Splitters merged on purpose give a learned-routed Markov block one bucket of
    each kind (sizes checked on the host first)."""
    w = datagen.Workload("t", [datagen.MARKOV3_Z96, datagen.MARKOV3_Z96], [11, 12], [300_000, 250_000])
    buf, off = w.generate()
    keys = _prefix_keys(buf[:300_000])
    spl = np.array(small_model.splitters, dtype=np.uint64).copy()

    def sizes(sp):
        return np.bincount(np.searchsorted(sp, keys, side="right"), minlength=sp.size + 1)

    base = sizes(spl)

    def merge_to(sp, j, lo, hi):
        """Splitters j+1 .. j+m set to splitter j: buckets j+1 .. j+m+1 become one,
        with m the first count that puts it in (lo, hi]."""
        for m in range(1, sp.size - j - 1):
            tot = int(base[j + 1:j + m + 2].sum())
            if lo < tot <= hi:
                t = sp.copy()
                t[j + 1:j + 1 + m] = t[j]
                return t, j + m + 1
            if tot > hi:
                break
        raise AssertionError("could not build the bucket")

    spl, end1 = merge_to(spl, 1000, 6_700, 13_312)  # above the 512-thread sort's 6,656
    assert end1 < 2600
    spl, _ = merge_to(spl, 2600, 20_000, 1 << 30)
    sz = sizes(spl)
    assert ((sz > 3_328) & (sz <= 13_312)).any() and (sz > 13_312).any(), sz.max()
    assert sz[sz > 3_328].sum() * 4 <= keys.size  # still routed to the learned buckets
    L, prim, st = _learned_run(buf, off, spl, graph=graph)
    assert_matches_oracle(buf, off, L, prim, f"over-full buckets graph={graph}")
    assert st["blocks_routed_plain"] == 0 and st["blocks_routed_flat"] == 0, st
    assert st["buckets_overflowed"] >= 2, st


def _with_repeats(block, frac, seg, seed):
    """A copy of `block` with segments of `seg` bytes copied elsewhere until
    about `frac` of its rotations share their first 8 bytes with another."""
    rng = np.random.default_rng(seed)
    b = block.copy()
    n = b.size
    for _ in range(max(1, int(frac * n / (2 * seg)))):
        src, dst = rng.integers(0, n - seg, 2)
        b[dst:dst + seg] = b[src:src + seg]
    return b


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("which", ["model", "equal_width"])
def test_lazy_and_stored_ranks(small_model, which, graph):
    """After the chunk sorts a bucketed block's doubling rounds read ranks
    either stored in full (more than 1/32 of its rotations in groups: filled
    after the chunk sorts) or found on demand (the bucket of the rotation's
    key, then a search of the bucket's sorted rows). Markov blocks with
    repeated segments put about 11% (stored), 0.9% and 0.9% (on demand) of
    their rotations in groups of two or more, a plain one none; every output
    is exact."""
    spl = small_model.splitters if which == "model" else model.equal_width_splitters()
    blocks = []
    for i, frac in enumerate([0.12, 0.015, 0.002, 0.0]):
        w = datagen.Workload("t", [datagen.MARKOV3_Z96], [40 + i], [120_000 + 7_001 * i])
        b, _ = w.generate()
        blocks.append(_with_repeats(b, frac, 600, 70 + i) if frac else b)
    from gpu_util import batch_from_blocks
    buf, off = batch_from_blocks(blocks)
    for blk in blocks[:3]:  # the intended share of group members, on the host
        keys = _prefix_keys(blk)
        _, inv, cnt = np.unique(keys, return_inverse=True, return_counts=True)
        share = (cnt[inv] > 1).mean()
        assert share > 0.0005, share
    L, prim, st = _learned_run(buf, off, spl, graph=graph)
    assert_matches_oracle(buf, off, L, prim, f"lazy ranks {which} graph={graph}")
    assert st["blocks_routed_plain"] == 0, st


@pytest.mark.parametrize("graph", [False, True])
def test_lazy_ranks_with_overfull_buckets(small_model, graph):
    """On-demand ranks whose rotations lie in over-full buckets: a Markov block
    with repeated segments (about 2% of its rotations in groups, so its
    groups of one keep their ranks unstored) whose splitters are merged so
    that one bucket goes to the 512-thread sort and one to the overflow
    radix (ranks stored in full there). The group members' successors are
    spread over the key range, so some lookups land in each kind of bucket."""
    w = datagen.Workload("t", [datagen.MARKOV3_Z96], [21], [300_000])
    base_block, _ = w.generate()
    blk = _with_repeats(base_block, 0.02, 400, 22)
    keys = _prefix_keys(blk)
    spl = np.array(small_model.splitters, dtype=np.uint64).copy()
    sizes = lambda sp: np.bincount(np.searchsorted(sp, keys, side="right"), minlength=sp.size + 1)  # noqa: E731
    base = sizes(spl)
    # merge buckets after 1000 until one holds 3,400..6,656 (the 512-thread sort), and after 2600
    # until one holds > 20,000 (the overflow radix)
    for j, lo, hi in ((1000, 3_400, 6_656), (2600, 20_000, 1 << 30)):
        for m in range(1, spl.size - j - 1):
            tot = int(base[j + 1:j + m + 2].sum())
            if lo < tot <= hi:
                spl[j + 1:j + 1 + m] = spl[j]
                break
        else:
            raise AssertionError("could not build the bucket")
        base = sizes(spl)
    sz = sizes(spl)
    assert ((sz > 3_328) & (sz <= 6_656)).any() and (sz > 13_312).any(), sz.max()
    _, inv, cnt = np.unique(keys, return_inverse=True, return_counts=True)
    share = (cnt[inv] > 1).mean()
    assert 0.005 < share < 1 / 32, share  # groups exist, and the block's ranks stay on demand
    buf, off = blk, np.array([0, blk.size], dtype=np.uint64)
    L, prim, st = _learned_run(buf, off, spl, graph=graph)
    assert_matches_oracle(buf, off, L, prim, f"lazy ranks with over-full buckets graph={graph}")
    assert st["blocks_routed_plain"] == 0 and st["buckets_overflowed"] >= 2, st


def test_large_blocks_near_and_over_the_chunk_limit(small_model):
    """Chunked blocks hold at most 1,024 chunks: a 1,400,000-byte Markov block
    still takes the learned buckets (about 450 chunks), a 1,700,000-byte one
    is routed to the plain radix; both are exact."""
    w = datagen.Workload("t", [datagen.MARKOV3_Z96, datagen.MARKOV3_Z96], [31, 32], [1_400_000, 1_700_000])
    buf, off = w.generate()
    L, prim, st = _learned_run(buf, off, small_model.splitters)
    assert_matches_oracle(buf, off, L, prim, "1.4 MB and 1.7 MB blocks")
    assert st["blocks_routed_plain"] == 1 and st["blocks_routed_flat"] == 0, st


def test_learned_graph_equals_oracle_and_replays(small_model):
    """Learned + batched: the learned stage (device-side routing included) and
    the doubling loop captured as one CUDA graph. The first call captures, the
    second replays; both are exact and route every block as the host-driven
    learned mode does."""
    import torch
    w = datagen.learned_eval(num_blocks=20, n=150_000)
    buf, off = w.generate()
    with Plan(max_blocks=20, max_total_bytes=buf.size, max_block_bytes=150_000, flags=F_LEARNED | F_GRAPH) as plan:
        model.install(plan, small_model.splitters)
        d_in = torch.from_numpy(buf).cuda()
        L = torch.empty_like(d_in)
        prim = torch.empty(20, dtype=torch.int32, device="cuda")
        for it in range(2):  # the same buffers: the second call replays the graph
            L.zero_()
            plan.forward_into(d_in, off, L, prim)
            torch.cuda.synchronize()
            st = plan.stats()
            assert_matches_oracle(buf, off, L.cpu().numpy(), prim.cpu().numpy(), f"learned graph call {it}")
            assert st["graph_replayed"] == it, st
    _, _, st_host = _learned_run(buf, off, small_model.splitters)
    for k in ("blocks_routed_flat", "blocks_routed_plain", "buckets_overflowed", "keys_overflowed", "bucket_sq_sum",
              "buckets_nonempty", "radix_keys"):
        assert st[k] == st_host[k], (k, st, st_host)


def test_learned_with_radix_variants(small_model):
    w = datagen.learned_eval(num_blocks=6, n=50_000)
    buf, off = w.generate()
    for rb, tile in ((8, 1024), (11, 2048)):
        L, prim, _ = _learned_run(buf, off, small_model.splitters, radix_bits=rb, tile_keys=tile)
        assert_matches_oracle(buf, off, L, prim, f"learned rb={rb} tile={tile}")


def test_what_the_model_gains(small_model):
    """The gain of the trained network. Against the plain sort: the learned
    buckets replace the 8 radix passes, so far fewer keys go through the
    radix. Against the same bucketing without a model (equal-width buckets on
    the top 12 key bits): the learned buckets are more even -- more of the
    4096 buckets are used and the in-bucket sort work (sum of squared bucket
    sizes) is smaller. All three give the identical transform."""
    w = datagen.learned_eval(num_blocks=9, n=300_000)  # 9 held-out Markov blocks
    buf, off = w.generate()
    L1, p1, s_model = _learned_run(buf, off, small_model.splitters)
    L2, p2, s_flat = _learned_run(buf, off, model.equal_width_splitters())
    L3, p3, s_plain = gpu_bwt(buf, off)
    assert np.array_equal(L1, L2) and np.array_equal(p1, p2)
    assert np.array_equal(L1, L3) and np.array_equal(p1, p3)
    assert s_model["blocks_routed_plain"] == 0, s_model
    assert s_model["radix_keys"] * 4 < s_plain["radix_keys"], (s_model, s_plain)
    assert s_model["buckets_nonempty"] > 2 * s_flat["buckets_nonempty"], (s_model, s_flat)
    assert s_model["bucket_sq_sum"] < s_flat["bucket_sq_sum"], (s_model, s_flat)


def test_model_file_round_trip(tmp_path, small_model):
    path = str(tmp_path / "m.bwtmodel")
    small_model.save(path)
    m2 = model.TrainedModel.load(path)
    assert np.array_equal(m2.params, small_model.params) and np.array_equal(m2.splitters, small_model.splitters)
    assert np.array_equal(m2.norm, small_model.norm)
    w = datagen.learned_eval(num_blocks=3, n=40_000)
    buf, off = w.generate()
    import torch
    with Plan(max_blocks=3, max_total_bytes=buf.size, max_block_bytes=40_000, flags=F_LEARNED,
              model_path=path) as plan:
        L, prim = plan.forward(torch.from_numpy(buf).cuda(), off)
        assert_matches_oracle(buf, off, L.cpu().numpy(), prim.cpu().numpy(), "model file")


def test_learned_without_model_reports_enomodel():
    import torch
    with Plan(max_blocks=1, max_total_bytes=100, max_block_bytes=100, flags=F_LEARNED) as plan:
        d = torch.zeros(100, dtype=torch.uint8, device="cuda")
        L = torch.empty_like(d)
        p = torch.empty(1, dtype=torch.int32, device="cuda")
        assert plan.forward_into(d, np.array([0, 100], dtype=np.uint64), L, p,
                                 raise_on_error=False) == _lib.BWT_ENOMODEL
    with pytest.raises(_lib.BWTError):
        Plan(max_blocks=1, max_total_bytes=100, max_block_bytes=100, flags=F_LEARNED, model_path="/nonexistent/m")
