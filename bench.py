"""Benchmark of the GB300 forward BWT block sort.

Default workload (learned-eval-1200x900000): 1,200 blocks of 900,000 bytes
(the bzip2 -9 block size), 1.08 GB -- 1,080 held-out order-3 Markov blocks and
120 uniform-random ones -- sorted by the learned-CDF bucketing in one batched,
graph-captured call with inputs resident in HBM (the model is trained on the
GPU first, outside the timed region); the plain batched path on the same batch
is timed beside it ("plain"). The other four workloads are timed after it in
their own launch modes ("workloads"). Prints one JSON line (rank 0). Metric:
input MB/s (10^6 bytes of blocks per second).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config 1..5]
                  [--mode learned|graph|host|perblock|learned-host]
                  [--impl ours|reference] [--no-workloads]

--impl reference times the CPU oracle (the only other place this script runs
it) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "BWT block-sort input MB/s on 1 GB300 (learned+batched vs plain), bit-exact"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", type=int, default=5)
    ap.add_argument("--blocks", type=int, default=0, help="use only the first N blocks of the workload")
    ap.add_argument("--mode", choices=["host", "graph", "perblock", "learned", "learned-host", "inverse", "stages"],
                    default="learned",
                    help="learned = learned bucketing + the batched graph launch; learned-host drives its rounds "
                         "from the host; inverse times the GPU inverse transform of the workload's BWT; stages "
                         "times the stages after it (run-length, move-to-front, variable-length encoding)")
    ap.add_argument("--radix-bits", type=int, default=0)
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--model", default=None, help="model file for --mode learned (trained in-process if absent)")
    ap.add_argument("--train-samples", type=int, default=1_000_000)
    ap.add_argument("--train-epochs", type=int, default=8)
    ap.add_argument("--compare-plain", action="store_true", help="also time the plain path on the same batch")
    ap.add_argument("--autotune", action="store_true", help="pick radix bits and tile size on this batch first")
    ap.add_argument("--autotune-cache", default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--verify", action="store_true", help="check every block with the host inverse")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the timing of the other workloads after the main one")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 20 ms from before the
    warm-up; only the samples taken inside the timed window (begin() .. end(),
    host clock at each line's arrival) are reported."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 20

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[tuple[float, str]] = []
        self.t0 = self.t1 = None
        self.interval_ms = self.INTERVAL_MS

    def start(self, wait_s: float = 3.0):
        for interval in (self.INTERVAL_MS, 200):  # 200 ms if this nvidia-smi refuses the short interval
            try:
                self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                              "--format=csv,noheader,nounits", "-lms", str(interval)],
                                             stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            except (OSError, FileNotFoundError):
                self.proc = None
                return
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
            t = time.perf_counter()
            while not self.lines and time.perf_counter() - t < wait_s and self.proc.poll() is None:
                time.sleep(0.01)  # sampling has started before the timed window opens
            if self.lines or self.proc.poll() is None:
                self.interval_ms = interval
                return

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def begin(self):
        self.t0 = time.perf_counter()

    def end(self):
        self.t1 = time.perf_counter()

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        lines = self.lines
        if self.t0 is not None and self.t1 is not None:
            inside = [ln for t, ln in lines if self.t0 <= t <= self.t1 + self.interval_ms / 1000]
            if not inside:  # a window shorter than one interval: the first sample after it opened
                inside = [ln for t, ln in lines if t >= self.t0][:1]
            lines = inside
        else:
            lines = [ln for _, ln in lines]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "interval_ms": self.interval_ms}


def workload(cfg: int, blocks: int = 0):
    from paper_1109_2348_gb300 import datagen
    w = datagen.config(cfg)
    if blocks and blocks < w.num_blocks:
        w = w.subset(range(blocks))
    return w


def rank_workload(cfg: int, blocks: int, rank: int, world: int):
    """Weak scaling: every rank sorts its own full batch of the workload, with
    seeds shifted by rank so the ranks' blocks are distinct units. Blocks are
    independent, so there is no data-path exchange between ranks."""
    w = workload(cfg, blocks)
    return w.reseeded(100_000 * rank) if world > 1 else w


def reduce_max(value: float, world: int, device=None) -> float:
    """Max over ranks (the slowest rank's time defines the job's time)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(bytes_per_rank: int, world: int, steps: int, t_ms: float) -> float:
    """Whole-job input MB/s: bytes all ranks sorted / the slowest rank's time."""
    return bytes_per_rank * world * steps / (t_ms / 1e3) / 1e6


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def cpu_sample(w, max_blocks: int):
    """A bounded sample of the workload for the oracle that keeps its mix of
    sources: each source contributes blocks in proportion to its share of the
    workload (at least one), spread evenly over that source's blocks."""
    k = min(max_blocks, w.num_blocks)
    by_src: dict[int, list[int]] = {}
    for i, s in enumerate(w.sources):
        by_src.setdefault(s, []).append(i)
    want = {s: max(1, int(round(k * len(ix) / w.num_blocks))) for s, ix in by_src.items()}
    while sum(want.values()) > k and any(v > 1 for v in want.values()):
        s = max(want, key=lambda q: want[q])
        want[s] -= 1
    order = []
    for s, ix in by_src.items():
        m = min(want[s], len(ix))
        order += [ix[int(j * len(ix) / m)] for j in range(m)]
    return w.subset(sorted(order))


def run_cpu_oracle(w, threads: int, repeats: int = 1):
    import oracle
    buf, off = w.generate()
    t0 = time.perf_counter()
    for _ in range(repeats):
        oracle.bwt_batch(buf, off, threads=threads)
    dt = (time.perf_counter() - t0) / repeats
    return buf.size / dt / 1e6, dt


def timed_cpu_baseline(w, cores: int, target_s: float = 12.0):
    """The oracle as it stands on the host cores, on a bounded sample of the
    workload sized to about target_s seconds: blocks taken round-robin over
    the workload's sources (the whole workload, repeated, if it is smaller)."""
    probe = cpu_sample(w, cores)
    _, dt = run_cpu_oracle(probe, cores)
    per_byte = dt / probe.total_bytes
    want = int(target_s / per_byte)
    if want >= w.total_bytes:
        sample, repeats = w, max(1, int(round(want / w.total_bytes)))
    else:
        k = max(cores, min(w.num_blocks, int(w.num_blocks * want / w.total_bytes)))
        sample, repeats = cpu_sample(w, k), 1
    mbs, dt = run_cpu_oracle(sample, cores, repeats)
    return {"value": round(mbs, 3), "unit": "MB/s", "cores": cores, "kind": "oracle",
            "sample": f"{sample.num_blocks} blocks ({sample.total_bytes} bytes) of {w.name}, {repeats} pass(es), "
                      f"{dt * repeats:.1f} s"}


# DRAM bytes (read + write) per key of one u64 onesweep pass as ncu counted
# them (1-pass metrics) for the current kernel on one full-size pass of the
# mixed3-64x900000 workload; None when the kernel has changed since.
ONESWEEP_DRAM_BYTES_PER_KEY = 23.37
# DRAM bytes (read + write) per rotation of the learned chunk sort
# (k_chunk_sort_name<256, 4, 0>) as ncu counted them for the current kernel on
# 24 blocks of the learned-eval workload; None when the kernel has changed since.
CHUNK_SORT_DRAM_BYTES_PER_KEY = 15.63


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = workload(args.config, args.blocks)
    cores = os.cpu_count() or 1
    sample = cpu_sample(w, cores)
    for _ in range(max(0, args.warmup)):
        pass  # the oracle has no warm state; warm-up steps are skipped
    times = []
    for _ in range(args.steps):
        mbs, dt = run_cpu_oracle(sample, cores)
        times.append(dt)
    dt = float(np.mean(times))
    v = sample.total_bytes / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "MB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic (seeded generators)",
            "config": {"workload": w.name, "sample": sample.name, "l2": "inputs of a step exceed L2 in working set"},
            "cpu_baseline": {"value": round(v, 3), "unit": "MB/s", "cores": cores, "kind": "oracle",
                             "sample": f"{sample.num_blocks} blocks ({sample.total_bytes} bytes) of {w.name}"},
            "e2e": {"value": round(v, 3), "unit": "MB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def make_model(args, local):
    """Trains the learned-CDF model on the GPU (outside every timed region)
    unless --model names a file; returns (path, description)."""
    if args.model:
        return args.model, None
    import tempfile
    from paper_1109_2348_gb300 import model as mdl
    t0 = time.perf_counter()
    trained = mdl.train(num_samples=args.train_samples, epochs=args.train_epochs, device=local)
    path = os.path.join(tempfile.mkdtemp(), "bwt.model")
    trained.save(path)
    return path, {"trained_s": round(time.perf_counter() - t0, 2), "samples": args.train_samples,
                  "epochs": args.train_epochs, "final_loss": float(trained.epoch_loss[-1]),
                  "train_blocks": "100 x 900000 order-3 Markov, seeds 5000..5099"}


class Runner:
    """One workload resident in HBM and the plans that time it."""

    def __init__(self, w, dev, local, flush):
        import torch
        self.w, self.dev, self.local, self.flush = w, dev, local, flush
        self.buf, self.off = w.generate()
        self.n = self.buf.size
        self.sizes = np.diff(self.off.astype(np.int64))
        self.pinned = torch.from_numpy(self.buf).pin_memory()
        self.d_in = self.pinned.to(dev)
        self.d_L = torch.empty_like(self.d_in)
        self.d_p = torch.empty(w.num_blocks, dtype=torch.int32, device=dev)
        self.stream = torch.cuda.current_stream()

    def plan(self, flags, rb=0, tk=0, model_path=None):
        from paper_1109_2348_gb300 import F_LEARNED, Plan
        return Plan(max_blocks=self.w.num_blocks, max_total_bytes=self.n, max_block_bytes=int(self.sizes.max()),
                    radix_bits=rb, tile_keys=tk, flags=flags, model_path=model_path if flags & F_LEARNED else None,
                    device=self.local)

    def warm(self, pl, count):
        import torch
        for _ in range(max(3, count)):
            pl.forward_into(self.d_in, self.off, self.d_L, self.d_p, self.stream)
        torch.cuda.synchronize()
        assert pl.last_status() == 0

    def timed(self, pl, steps):
        """`steps` calls, L2 flushed before each, CUDA events on the launch
        stream; no host synchronisation between the calls. Returns the step
        times and the statistics of the last call (every step is the same call
        on the same batch)."""
        import torch
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            self.flush.zero_()
            ev[i][0].record(self.stream)
            pl.forward_into(self.d_in, self.off, self.d_L, self.d_p, self.stream)
            ev[i][1].record(self.stream)
        torch.cuda.synchronize()
        assert pl.last_status() == 0
        return [a.elapsed_time(b) for a, b in ev], pl.stats()


def e2e_pipeline(R, plan, steps, world, dev, nsets: int = 3):
    """End to end through the public call: every step copies its input from
    pinned host memory to the device, sorts it with bwt_forward_batch and
    copies L and the primary indices back to pinned host memory, all inside
    the timed region. The copies run on their own streams (one per
    direction) and the sorts on one compute stream, ordered by events, with
    `nsets` buffer sets in flight, so step k+1's upload and step k-1's
    download overlap step k's sort; no call waits on the host. Returns the
    e2e record (input MB/s)."""
    import torch
    n = R.n
    st_h2d, st_cmp, st_d2h = (torch.cuda.Stream(device=dev) for _ in range(3))
    sets = [{"in": torch.empty_like(R.d_in), "L": torch.empty_like(R.d_in), "p": torch.empty_like(R.d_p),
             "hL": torch.empty(n, dtype=torch.uint8).pin_memory(),
             "hp": torch.empty(R.w.num_blocks, dtype=torch.int32).pin_memory()} for _ in range(nsets)]
    # warm-up: one full round trip through every buffer set (capture its
    # graph, touch its pinned host buffers), ordered on one stream
    with torch.cuda.stream(st_cmp):
        for s_ in sets:
            s_["in"].copy_(R.pinned, non_blocking=True)
            plan.forward_into(s_["in"], R.off, s_["L"], s_["p"], st_cmp)
            s_["hL"].copy_(s_["L"], non_blocking=True)
            s_["hp"].copy_(s_["p"], non_blocking=True)
    torch.cuda.synchronize()
    assert plan.last_status() == 0
    ev = lambda: torch.cuda.Event()  # noqa: E731
    up, done, down = [None] * steps, [None] * steps, [None] * steps
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(R.stream)
    for s_ in (st_h2d, st_cmp, st_d2h):
        s_.wait_event(e0)
    for i in range(steps):
        cur = sets[i % nsets]
        with torch.cuda.stream(st_h2d):
            if i >= nsets:
                st_h2d.wait_event(done[i - nsets])  # the sort that read this input buffer has finished
            cur["in"].copy_(R.pinned, non_blocking=True)
            up[i] = ev()
            up[i].record(st_h2d)
        st_cmp.wait_event(up[i])
        if i >= nsets:
            st_cmp.wait_event(down[i - nsets])  # this L buffer has been copied out
        plan.forward_into(cur["in"], R.off, cur["L"], cur["p"], st_cmp)
        done[i] = ev()
        done[i].record(st_cmp)
        with torch.cuda.stream(st_d2h):
            st_d2h.wait_event(done[i])
            cur["hL"].copy_(cur["L"], non_blocking=True)
            cur["hp"].copy_(cur["p"], non_blocking=True)
            down[i] = ev()
            down[i].record(st_d2h)
    for s_ in (st_h2d, st_cmp, st_d2h):
        R.stream.wait_stream(s_)
    e1.record(R.stream)
    torch.cuda.synchronize()
    assert plan.last_status() == 0
    e_ms = reduce_max(e0.elapsed_time(e1), world, dev)
    assert np.array_equal(sets[(steps - 1) % nsets]["hL"].numpy(), R.d_L.cpu().numpy())
    return {"value": round(n * world * steps / (e_ms / 1e3) / 1e6, 3), "unit": "MB/s",
            "h2d_bytes_per_step": int(n + R.off.nbytes), "d2h_bytes_per_step": int(n + 4 * R.w.num_blocks),
            "ms_per_step": round(e_ms / steps, 4),
            "pipelined": f"{nsets} buffer sets; uploads, sorts and downloads on three streams ordered by events"}


def ours(args):
    import torch
    from paper_1109_2348_gb300 import F_GRAPH, F_LEARNED, F_PER_BLOCK_LAUNCH, F_TIMING

    rank, world, local = dist_env()
    torch.cuda.set_device(local)  # before the process group, so its communicator is on this rank's GPU
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    learned = args.mode.startswith("learned")
    flags = {"host": F_TIMING, "graph": F_GRAPH, "perblock": F_PER_BLOCK_LAUNCH, "learned": F_LEARNED | F_GRAPH,
             "learned-host": F_LEARNED}[args.mode]
    model_path, model_info = make_model(args, local) if learned or (rank == 0 and not args.no_workloads) \
        else (None, None)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > L2 (129 MB)
    R = Runner(rank_workload(args.config, args.blocks, rank, world), dev, local, flush)
    w, n = R.w, R.n

    plan = R.plan(flags, args.radix_bits, args.tile, model_path)
    tuned = None
    if args.autotune:
        import tempfile
        cache = args.autotune_cache or os.path.join(tempfile.mkdtemp(), "autotune.jsonl")
        rb, tk, ms = plan.autotune(R.d_in, R.off, R.d_L, R.d_p, cache_path=cache, repeats=3, stream=R.stream)
        tuned = {"radix_bits": rb, "tile_keys": tk, "ms": round(ms, 4)}
    rb_used = tuned["radix_bits"] if tuned else args.radix_bits
    tk_used = tuned["tile_keys"] if tuned else args.tile

    sampler = ClockSampler(local)
    sampler.start()
    R.warm(plan, args.warmup)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.begin()
    step_ms, stats = R.timed(plan, args.steps)
    sampler.end()
    clocks = sampler.stop()
    launches = stats["kernel_launches"] * args.steps
    learned_stats = {k: stats[k] for k in ("blocks_routed_plain", "blocks_routed_flat", "buckets_overflowed",
                                           "keys_overflowed", "max_bucket", "bucket_sq_sum", "buckets_nonempty",
                                           "chunk_keys")} if learned else None
    t_ms = reduce_max(float(np.sum(step_ms)), world, dev)
    value = job_value(n, world, args.steps, t_ms)

    if args.verify and rank == 0:
        from paper_1109_2348_gb300 import bwt_inverse_check
        Lh = R.d_L.cpu().numpy()
        ph = R.d_p.cpu().numpy()
        for b in range(w.num_blocks):
            s, e = int(R.off[b]), int(R.off[b + 1])
            assert bwt_inverse_check(Lh[s:e], int(ph[b]), R.buf[s:e]) == 0, f"block {b} fails the inverse check"

    e2e = None
    if not args.no_e2e:
        e2e = e2e_pipeline(R, plan, args.steps, world, dev)

    plan.close()
    plain_cmp = None
    if learned or args.compare_plain:
        # the plain path on the same batch, batched the same way (graph)
        pg = R.plan(F_GRAPH, rb_used, tk_used)
        R.warm(pg, args.warmup)
        pms, pst = R.timed(pg, args.steps)
        pg.close()
        p_ms = reduce_max(float(np.sum(pms)), world, dev)
        plain_cmp = {"value": round(job_value(n, world, args.steps, p_ms), 3), "unit": "MB/s",
                     "mode": "plain radix, batched (graph)", "ms_per_step": round(p_ms / args.steps, 4),
                     "rounds": pst["rounds"]}
    peak, peak_kind = measured_peaks()

    def first_sort_roofline():
        # the plain first sort's u64 onesweep passes in host-driven mode with
        # CUDA events around every radix launch on the launch stream (events
        # cannot sit between the kernels of a graph replay): algorithmic bytes
        # (13 per key for the pass that packs the keys from the bytes, 24 for
        # the others) over their event time; traffic = the DRAM bytes per key
        # ncu measured for the current kernel, times the keys of one launch
        th = R.plan(F_TIMING, rb_used, tk_used)
        R.warm(th, 3)
        acc = {"ms": 0.0, "bytes": 0.0, "launches": 0, "keys": 0.0}
        for _ in range(max(1, args.steps // 2)):
            R.flush.zero_()
            th.forward_into(R.d_in, R.off, R.d_L, R.d_p, R.stream)
            st = th.stats()
            acc["ms"] += st["first_ms"]
            acc["bytes"] += st["first_bytes"]
            acc["launches"] += st["first_launches"]
            acc["keys"] += n * st["first_launches"]
        th.close()
        if acc["ms"] <= 0 or acc["launches"] == 0:
            return None  # small blocks: the one-cluster first sort has no separately timed passes
        achieved = acc["bytes"] / (acc["ms"] / 1e3) / 1e9
        per_launch_keys = acc["keys"] / max(1, acc["launches"])
        kname = ("k_hist16 + k_scan16_cols + k_scan16_digits + k_scatter16 (plain first-sort 16-bit pass)"
                 if stats["radix_bits"] == 16 else
                 f"k_onesweep<u64, {stats['radix_bits']}, {stats['tile_keys']}> (plain first-sort radix pass)")
        return {"bound": "hbm", "kernel": kname,
                "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "peak_source": peak_kind + " hbm_gbs",
                "traffic": None if ONESWEEP_DRAM_BYTES_PER_KEY is None or stats["radix_bits"] != 8 else
                round(ONESWEEP_DRAM_BYTES_PER_KEY * per_launch_keys),
                "algorithmic_bytes_per_launch": round(acc["bytes"] / max(1, acc["launches"])),
                "launches_timed": acc["launches"], "avg_launch_ms": round(acc["ms"] / max(1, acc["launches"]), 4)}

    def chunk_sort_roofline():
        # the learned step's dominant kernel, the 256-thread chunk sort, timed
        # in host-driven learned mode with CUDA events around its launch:
        # 16 algorithmic bytes per rotation it sorts (8-byte key and 4-byte
        # index read, SA entry written; ranks are stored only for the rare
        # group members) over its event time
        th = R.plan(F_TIMING | F_LEARNED, rb_used, tk_used, model_path)
        R.warm(th, 3)
        ms = by = 0.0
        la = keys = 0
        for _ in range(max(1, args.steps // 2)):
            R.flush.zero_()
            th.forward_into(R.d_in, R.off, R.d_L, R.d_p, R.stream)
            st = th.stats()
            ms += st["chunk_ms"]
            by += st["chunk_bytes"]
            la += st["chunk_launches"]
            keys += st["chunk_keys"]
        th.close()
        if ms <= 0 or la == 0:
            return None
        achieved = by / (ms / 1e3) / 1e9
        per_launch_keys = keys / la
        return {"bound": "hbm", "kernel": "k_chunk_sort_name<256, 4, 0> (learned chunk sort: sort, SA, naming)",
                "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "peak_source": peak_kind + " hbm_gbs",
                "traffic": None if CHUNK_SORT_DRAM_BYTES_PER_KEY is None else
                round(CHUNK_SORT_DRAM_BYTES_PER_KEY * per_launch_keys),
                "algorithmic_bytes_per_launch": round(by / la), "bytes_per_rotation": 16,
                "rotations_per_launch": round(per_launch_keys), "launches_timed": la,
                "avg_launch_ms": round(ms / la, 4)}

    roof, roof_plain = None, None
    if args.mode not in ("perblock",):
        roof_plain = first_sort_roofline()
        roof = chunk_sort_roofline() if learned else roof_plain
    if roof is None:
        roof = roof_plain
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = timed_cpu_baseline(w, os.cpu_count() or 1)
    del R
    others = None
    if rank == 0 and world == 1 and not args.no_workloads:
        others = other_workloads(args, dev, local, flush, model_path)
    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 3), "unit": "MB/s", "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": round(t_ms / args.steps, 4),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
                "data": "synthetic (seeded generators, no dataset)",
                "config": {"workload": w.name, "blocks": w.num_blocks, "bytes": n, "mode": args.mode,
                           "radix_bits": stats["radix_bits"], "tile_keys": stats["tile_keys"],
                           "rounds": stats["rounds"], "l2": "256 MB flush before every timed step",
                           "parallelism": f"block-sharded x{world} (each rank its own batch, no collective)"},
                "clocks": clocks, "gpu_launches": int(launches), "e2e": e2e, "roofline": roof,
                "cpu_baseline": cpu, "step_ms": [round(x, 3) for x in step_ms]}
        if plain_cmp:
            line["plain"] = plain_cmp
        if learned and roof_plain is not None:
            line["roofline_plain_first_sort"] = roof_plain
        if tuned:
            line["config"]["autotuned"] = tuned
        if learned_stats:
            line["config"]["learned"] = learned_stats
        if model_info:
            line["config"]["model"] = model_info
        if others:
            line["workloads"] = others
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def other_workloads(args, dev, local, flush, model_path):
    """The other workloads, each timed in its own launch modes on the same
    GPU (inputs resident in HBM, L2 flushed before every step, CUDA events on
    the launch stream): input MB/s and ms per step."""
    from paper_1109_2348_gb300 import F_GRAPH, F_LEARNED, F_PER_BLOCK_LAUNCH
    runs = {1: [("graph", F_GRAPH), ("graph_autotuned", F_GRAPH)],
            2: [("learned", F_LEARNED | F_GRAPH), ("graph", F_GRAPH)],
            3: [("graph", F_GRAPH)],
            4: [("graph", F_GRAPH), ("perblock", F_PER_BLOCK_LAUNCH), ("learned", F_LEARNED | F_GRAPH)],
            5: [("learned", F_LEARNED | F_GRAPH), ("graph", F_GRAPH)]}
    out = {}
    steps = max(3, min(args.steps, 10))
    for cfg in (1, 2, 3, 4, 5):
        if cfg == args.config:
            continue
        R = Runner(workload(cfg), dev, local, flush)
        res = {"workload": R.w.name, "blocks": R.w.num_blocks, "bytes": R.n}
        for label, fl in runs[cfg]:
            pl = R.plan(fl, model_path=model_path)
            tuned = None
            if label.endswith("autotuned"):  # the plan's autotuner picks digit width and tile size first
                rb, tk, _ = pl.autotune(R.d_in, R.off, R.d_L, R.d_p, repeats=3, stream=R.stream)
                tuned = {"radix_bits": rb, "tile_keys": tk}
            R.warm(pl, 3)
            k = 2 if label == "perblock" else steps
            ms, st = R.timed(pl, k)
            pl.close()
            t = float(np.sum(ms))
            res[label] = {"value": round(R.n * k / (t / 1e3) / 1e6, 3), "unit": "MB/s",
                          "ms_per_step": round(t / k, 4), "rounds": st["rounds"], "steps": k}
            if tuned:
                res[label]["autotuned"] = tuned
        out[f"config{cfg}"] = res
        del R
    return out


def inverse_bench(args):
    """The GPU inverse (bwt_inverse_batch) of the workload's BWT: output MB/s,
    every step's result compared with the input."""
    import torch
    from paper_1109_2348_gb300 import Plan

    rank, world, local = dist_env()
    torch.cuda.set_device(local)  # before the process group, so its communicator is on this rank's GPU
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    w = rank_workload(args.config, args.blocks, rank, world)
    buf, off = w.generate()
    n = buf.size
    sizes = np.diff(off.astype(np.int64))
    plan = Plan(max_blocks=w.num_blocks, max_total_bytes=n, max_block_bytes=int(sizes.max()), device=local)
    d_in = torch.from_numpy(buf).to(dev)
    d_L, d_p = plan.forward(d_in, off)
    d_out = torch.empty_like(d_in)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    sampler = ClockSampler(local)
    sampler.start()
    for _ in range(max(3, args.warmup)):
        plan.inverse_into(d_L, off, d_p, d_out, stream)
    torch.cuda.synchronize()
    assert torch.equal(d_out, d_in), "the GPU inverse does not give the input back"
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.begin()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches = 0
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        plan.inverse_into(d_L, off, d_p, d_out, stream)
        ev[i][1].record(stream)
        launches += plan.stats()["kernel_launches"]
    torch.cuda.synchronize()
    sampler.end()
    clocks = sampler.stop()
    assert torch.equal(d_out, d_in)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_ms = reduce_max(float(np.sum(step_ms)), world, dev)
    e2e = None
    if not args.no_e2e:
        hL = d_L.cpu().pin_memory()
        hp = d_p.cpu().pin_memory()
        ho = torch.empty(n, dtype=torch.uint8).pin_memory()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            d_L.copy_(hL, non_blocking=True)
            d_p.copy_(hp, non_blocking=True)
            plan.inverse_into(d_L, off, d_p, d_out, stream)
            ho.copy_(d_out, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e_ms = reduce_max(e0.elapsed_time(e1), world, dev)
        e2e = {"value": round(n * world * args.steps / (e_ms / 1e3) / 1e6, 3), "unit": "MB/s",
               "h2d_bytes_per_step": int(n + 4 * w.num_blocks + off.nbytes), "d2h_bytes_per_step": int(n)}
    plan.close()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        L_h, p_h = d_L.cpu().numpy(), d_p.cpu().numpy()
        t0 = time.perf_counter()
        done = 0
        b = 0
        while time.perf_counter() - t0 < 10.0 and b < w.num_blocks:
            s0, e0_ = int(off[b]), int(off[b + 1])
            oracle.inverse_bwt(L_h[s0:e0_], int(p_h[b]))
            done += e0_ - s0
            b += 1
        dt = time.perf_counter() - t0
        cpu = {"value": round(done / dt / 1e6, 3), "unit": "MB/s", "cores": 1, "kind": "oracle",
               "sample": f"{b} blocks ({done} bytes) of {w.name}, inverse LF walk, one thread, {dt:.1f} s"}
    if rank == 0:
        line = {"metric": "BWT inverse output MB/s on 1 GB300, bit-exact", "value": round(
                    job_value(n, world, args.steps, t_ms), 3), "unit": "MB/s", "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": round(t_ms / args.steps, 4), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic (seeded generators, no dataset)",
                "config": {"workload": w.name, "blocks": w.num_blocks, "bytes": n, "mode": "inverse",
                           "l2": "256 MB flush before every timed step"},
                "clocks": clocks, "gpu_launches": int(launches), "e2e": e2e, "roofline": None, "cpu_baseline": cpu,
                "step_ms": [round(x, 3) for x in step_ms]}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def huffman_lengths(counts):
    """Code lengths of a Huffman code for the bytes with counts > 0 (the host
    builds the table once: a precomputed table, as the paper proposes)."""
    import heapq
    used = [c for c in range(256) if counts[c] > 0]
    length = np.ones(256, dtype=np.uint8)
    if len(used) > 1:
        heap = [(int(counts[c]), i, [c]) for i, c in enumerate(used)]
        heapq.heapify(heap)
        depth = {c: 0 for c in used}
        uid = len(heap)
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


def stages_bench(args):
    """The stages of the paper's pipeline on the GPU, each timed with CUDA
    events (L2 flushed before every step): forward BWT of the workload ->
    run-length encoding of L -> move-to-front of the runs' bytes ->
    variable-length encoding of the result with a Huffman table built once
    from its histogram. Checked once on the GPU: run-length decoding gives L
    back and the inverse of (L, primary) gives the input back (parity of every
    stage with the oracle is the tests' job)."""
    import torch
    from paper_1109_2348_gb300 import F_GRAPH, Plan

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = rank_workload(args.config, args.blocks, rank, world)
    buf, off = w.generate()
    n = buf.size
    sizes = np.diff(off.astype(np.int64))
    plan = Plan(max_blocks=w.num_blocks, max_total_bytes=n, max_block_bytes=int(sizes.max()), flags=F_GRAPH,
                device=local)
    d_in = torch.from_numpy(buf).to(dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    d_L = torch.empty_like(d_in)
    d_p = torch.empty(w.num_blocks, dtype=torch.int32, device=dev)
    chars = torch.empty_like(d_in)
    lens = torch.empty(n, dtype=torch.int32, device=dev)
    run_off = torch.empty(w.num_blocks + 1, dtype=torch.int64, device=dev)
    mtf = torch.empty_like(d_in)
    vle = torch.empty(4 * n + 8, dtype=torch.uint8, device=dev)
    byte_off = torch.empty(w.num_blocks + 1, dtype=torch.int64, device=dev)
    bits = torch.empty(w.num_blocks, dtype=torch.int64, device=dev)

    def run_once(table=None):
        plan.forward_into(d_in, off, d_L, d_p, stream)
        plan.rle_encode_into(d_L, off, chars, lens, run_off, stream)
        ro = run_off.cpu().numpy().astype(np.uint64)  # the runs' block layout for the next stages
        R = int(ro[-1])
        plan.mtf_encode_into(chars[:R], ro, mtf, stream)
        if table is not None:
            plan.vle_encode_into(mtf[:R], ro, table[0], table[1], vle, byte_off, bits, stream)
        return ro, R

    ro, R = run_once()
    hist = np.bincount(mtf[:R].cpu().numpy(), minlength=256)
    code, length = huffman_lengths(hist)
    table = (torch.from_numpy(code.view(np.int32)).to(dev), torch.from_numpy(length).to(dev))
    for _ in range(max(3, args.warmup)):
        ro, R = run_once(table)
    torch.cuda.synchronize()
    # self-checks of the pipeline's output, on the GPU
    assert torch.equal(plan.rle_decode(chars[:R], lens[:R], run_off, off), d_L), "run-length round trip"
    assert torch.equal(plan.inverse(d_L, off, d_p), d_in), "inverse round trip"
    torch.cuda.synchronize()

    names = ["bwt", "rle", "mtf", "vle"]
    ms = {k: 0.0 for k in names}
    sampler = ClockSampler(local)
    sampler.start()
    torch.cuda.synchronize()
    sampler.begin()
    for _ in range(args.steps):
        flush.zero_()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        ev[0].record(stream)
        plan.forward_into(d_in, off, d_L, d_p, stream)
        ev[1].record(stream)
        plan.rle_encode_into(d_L, off, chars, lens, run_off, stream)
        ev[2].record(stream)
        plan.mtf_encode_into(chars[:R], ro, mtf, stream)
        ev[3].record(stream)
        plan.vle_encode_into(mtf[:R], ro, table[0], table[1], vle, byte_off, bits, stream)
        ev[4].record(stream)
        torch.cuda.synchronize()
        for i, k in enumerate(names):
            ms[k] += ev[i].elapsed_time(ev[i + 1])
    sampler.end()
    clocks = sampler.stop()
    plan.close()
    vle_bytes = int(byte_off[-1].item())
    stage = {}
    for k, inb in (("bwt", n), ("rle", n), ("mtf", R), ("vle", R)):
        t = ms[k] / args.steps
        stage[k] = {"ms": round(t, 4), "input_bytes": inb, "input_MB_s": round(inb / (t / 1e3) / 1e6, 1)}
    total_ms = sum(ms.values()) / args.steps
    if rank == 0:
        line = {"metric": "BWT -> RLE -> MTF -> VLE pipeline input MB/s on 1 GB300, bit-exact",
                "value": round(n / (total_ms / 1e3) / 1e6, 3), "unit": "MB/s", "n_gpus": 1, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": round(total_ms, 4), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u8",
                "data": "synthetic (seeded generators, no dataset)",
                "config": {"workload": w.name, "blocks": w.num_blocks, "bytes": n, "mode": "stages",
                           "runs": R, "vle_stream_bytes": vle_bytes,
                           "note": "run lengths stay uint32 (not entropy-coded); the VLE stream codes the runs' bytes "
                                   "after move-to-front",
                           "l2": "256 MB flush before every timed step"},
                "clocks": clocks, "stages": stage, "e2e": None, "roofline": None, "cpu_baseline": None}
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    elif args.mode == "inverse":
        inverse_bench(args)
    elif args.mode == "stages":
        stages_bench(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
