"""The N > 1 host logic of bench.py on CPU: two gloo ranks get distinct
batches of the same shape (blocks are independent units, so nothing is
exchanged), and the job's time is the max over ranks."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w = bench.rank_workload(2, 3, rank, world)
    t = bench.reduce_max(10.0 + rank, world)
    out.put((rank, w.seeds, w.sizes, w.sources, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_blocks_and_take_max_time():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, seeds0, sizes0, src0, t0), (r1, seeds1, sizes1, src1, t1) = res
    assert sizes0 == sizes1 and src0 == src1            # same shape per rank (weak scaling)
    assert not set(seeds0) & set(seeds1)                # distinct units
    assert t0 == t1 == 11.0                             # the slowest rank's time
    import bench
    assert np.isclose(bench.job_value(1_000_000, 2, 4, 8.0), 2 * 4 * 1.0 / 0.008)
