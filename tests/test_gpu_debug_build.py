"""The bounds-checked debug build (-DBWT_DEBUG) on the GPU: in a fresh process
with BWT_DEBUG=1 the library loaded is libbwt_gb300_debug.so, and batches in
every launch mode -- plain host-driven and graph, one launch chain per block,
16-bit digits, learned bucketing with its over-full buckets, and the stages --
must give the oracle's result with no bounds check failing (a failed check
would make the call report BWT_EINTERNAL)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import numpy as np, torch
import oracle
from paper_1109_2348_gb300 import F_GRAPH, F_LEARNED, F_PER_BLOCK_LAUNCH, Plan, _lib, datagen, model
lib = _lib.load()
assert _lib.library_path().name == "libbwt_gb300_debug.so"
w = datagen.Workload("t", [datagen.MARKOV3_Z96, datagen.RUNS16, datagen.UNIFORM, datagen.PERIOD7,
                           datagen.CONST, datagen.FIBONACCI, datagen.UNIFORM],
                     [1, 2, 3, 4, 5, 6, 7], [70_000, 30_001, 20_000, 25_000, 9_999, 33_333, 5])
buf, off = w.generate()
ref_L, ref_p = oracle.bwt_batch(buf, off)
tiny = model.train(datagen.learned_train(num_blocks=2, n=50_000), num_samples=20_000, epochs=2)
d_in = torch.from_numpy(buf).cuda()
cases = [(0, 0), (F_GRAPH, 0), (F_PER_BLOCK_LAUNCH, 0), (F_GRAPH, 16), (F_GRAPH, 11), (F_LEARNED, 0),
         (F_LEARNED | F_GRAPH, 0)]
for flags, rb in cases:
    with Plan(max_blocks=w.num_blocks, max_total_bytes=buf.size, max_block_bytes=70_000, flags=flags,
              radix_bits=rb, tile_keys=1024) as plan:
        if flags & F_LEARNED:
            model.install(plan, tiny.splitters)
        L, p = plan.forward(d_in, off)
        torch.cuda.synchronize()
        st = plan.last_status()
        assert st == 0, (flags, rb, _lib.STATUS_NAMES[st])
        assert np.array_equal(L.cpu().numpy(), ref_L) and np.array_equal(p.cpu().numpy(), ref_p), (flags, rb)
        c, ln, ro = plan.rle_encode(L, off)
        assert torch.equal(plan.rle_decode(c, ln, ro, off), L)
        assert torch.equal(plan.inverse(L, off, p), d_in)
print("debug build: OK", len(cases), "launch modes")
'''


def test_debug_build_runs_clean_against_the_oracle():
    env = dict(os.environ, BWT_DEBUG="1", PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    res = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=900)
    assert res.returncode == 0, res.stdout[-2000:] + res.stderr[-4000:]
    assert "debug build: OK" in res.stdout
