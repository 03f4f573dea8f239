"""bwt_forward_batch with BWT_F_GRAPH is stream-ordered and asynchronous: the
call enqueues its work and returns without waiting for the GPU; the device-side
status of the call is read afterwards through bwt_plan_last_status. Outputs
are compared with the oracle byte for byte."""
import numpy as np
import pytest

from paper_1109_2348_gb300 import F_GRAPH, F_LEARNED, Plan, _lib, datagen, model

from gpu_util import assert_matches_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny_model():
    return model.train(datagen.learned_train(num_blocks=2, n=50_000), num_samples=20_000, epochs=2)


@pytest.mark.parametrize("learned", [False, True])
def test_two_calls_back_to_back_without_host_sync(learned, tiny_model):
    """A one-second device sleep goes first on the stream; two forward calls
    with different block layouts, inputs and outputs are enqueued behind it.
    Both calls return while the sleep still runs (neither waited for the GPU),
    and after one synchronisation both outputs equal the oracle's."""
    import torch
    wa = datagen.Workload("a", [datagen.MARKOV3_Z96, datagen.RUNS16, datagen.UNIFORM], [41, 42, 43],
                          [60_000, 33_333, 20_001])
    wb = datagen.Workload("b", [datagen.PERIOD7, datagen.MARKOV3_Z96], [44, 45], [17_000, 90_000])
    flags = F_GRAPH | (F_LEARNED if learned else 0)
    bufs = [w.generate() for w in (wa, wb)]
    with Plan(max_blocks=4, max_total_bytes=120_000, max_block_bytes=90_000, flags=flags) as plan:
        if learned:
            model.install(plan, tiny_model.splitters)
        st = torch.cuda.Stream()
        ins = [torch.from_numpy(b).cuda() for b, _ in bufs]
        Ls = [torch.empty_like(x) for x in ins]
        ps = [torch.empty(off.size - 1, dtype=torch.int32, device="cuda") for _, off in bufs]
        torch.cuda.synchronize()
        done = torch.cuda.Event()
        with torch.cuda.stream(st):
            torch.cuda._sleep(2_000_000_000)  # about a second at 2 GHz
            for i, (b, off) in enumerate(bufs):
                assert plan.forward_into(ins[i], off, Ls[i], ps[i], stream=st) == _lib.BWT_OK
            done.record(st)
        assert not done.query(), "a forward call waited for the GPU"
        st.synchronize()
        assert plan.last_status() == _lib.BWT_OK
        for i, (b, off) in enumerate(bufs):
            assert_matches_oracle(b, off, Ls[i].cpu().numpy(), ps[i].cpu().numpy(), f"call {i}")
        # the first layout again, into the first buffers: the tables are
        # uploaded again and the cached graph of that call is replayed
        Ls[0].zero_()
        plan.forward_into(ins[0], bufs[0][1], Ls[0], ps[0], stream=st)
        st.synchronize()
        assert plan.last_status() == _lib.BWT_OK and plan.stats()["graph_replayed"] == 1
        assert_matches_oracle(bufs[0][0], bufs[0][1], Ls[0].cpu().numpy(), ps[0].cpu().numpy(), "replay")


def test_graph_call_reports_a_device_timeout_through_last_status():
    """A look-back wait that nothing satisfies runs out inside the graph; the
    call itself returned BWT_OK (it only enqueued), bwt_plan_last_status gives
    BWT_ETIMEOUT, and the next call on the plan is exact."""
    import torch
    w = datagen.Workload("t", [datagen.UNIFORM, datagen.MARKOV3_Z96], [1, 2], [20_000, 9_000])
    buf, off = w.generate()
    d_in = torch.from_numpy(buf).cuda()
    with Plan(max_blocks=2, max_total_bytes=buf.size, max_block_bytes=20_000, tile_keys=1024, flags=F_GRAPH) as plan:
        L = torch.empty_like(d_in)
        p = torch.empty(2, dtype=torch.int32, device="cuda")
        plan.debug_waits(2000, True)
        assert plan.forward_into(d_in, off, L, p, raise_on_error=False) == _lib.BWT_OK
        assert plan.last_status() == _lib.BWT_ETIMEOUT
        plan.debug_waits(0, False)
        assert plan.forward_into(d_in, off, L, p) == _lib.BWT_OK
        assert plan.last_status() == _lib.BWT_OK
        assert_matches_oracle(buf, off, L.cpu().numpy(), p.cpu().numpy(), "after the timeout")
