"""Parity at the benchmark's full sizes, in the launch configurations `bench.py` times.

* The large job (4 L0 + 12 L1 tables of 64 MiB, 1 GiB in): the whole output, byte for
  byte, against the oracle's compaction of the same input bytes (built by the oracle's
  own builder), through luda_compact_device with the library's default tuning, as the
  bench's headline leg calls it.
* The 256-job batch (2.2 GB): one batch call and the autotuned plan replay (the bench's
  batched legs); every job's status and entry accounting checked, and a sample of jobs
  (every 16th, plus the largest) compared byte for byte with the oracle.
"""
import numpy as np
import pytest

from helpers import oracle_compact, oracle_inputs
from paper_2004_03054_b300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2004_03054_b300 import autotune  # noqa: E402
from paper_2004_03054_b300 import luda  # noqa: E402
from test_gpu_parity import assert_same, dev  # noqa: E402


def test_large_job_full_size():
    job = W.config3(seed=3, scale=1.0)
    ins = oracle_inputs(job)
    want = oracle_compact(job, ins)
    assert want.status == 0
    got = luda.compact_device([dev(x) for x in ins], job.smallest_snapshot, level=job.level,
                              opts=luda.job_options(job))
    got.tables = [t.cpu().numpy().tobytes() for t in got.tables]
    assert_same(got, want)
    assert sum(len(t) for t in got.tables) > 900 << 20
    del got, ins


def test_batch_full_size_sampled():
    jobs = W.config4(seed=4, scale=1.0, n_jobs=256)
    o = jobs[0]
    ins = [oracle_inputs(j) for j in jobs]
    batch = [([dev(x) for x in xs], j.smallest_snapshot, j.bottommost) for j, xs in zip(jobs, ins)]
    opts = luda.options(o.block_size, o.restart_interval, o.bloom_bits_per_key, o.target_file_size)
    sizes = [sum(len(x) for x in xs) for xs in ins]
    sample = sorted(set(range(0, len(jobs), 16)) | {int(np.argmax(sizes))})
    want = {j: oracle_compact(jobs[j], ins[j]) for j in sample}

    def check(outs):
        for j, g in enumerate(outs):
            assert g.status == 0, (j, g.status, g.detail)
            assert sum(g.n_entries) == g.n_in_entries - g.n_dropped
            if j in want:
                g.tables = [t.cpu().numpy().tobytes() for t in g.tables]
                assert_same(g, want[j])

    rc, outs = luda.batch_compact_device(batch, opts)
    assert rc == 0
    check(outs)
    del outs
    res = autotune.tune(batch, opts, cache_path=None, reps=1)
    plan = luda.Plan(batch, luda.options(o.block_size, o.restart_interval, o.bloom_bits_per_key,
                                         o.target_file_size, tuning=res.tuning))
    plan.run()
    torch.cuda.synchronize()
    check(plan.outputs())
    plan.close()
