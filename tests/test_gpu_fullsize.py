"""Parity at the benchmark's full sizes, in the launch configurations `bench.py` times.

* The large job (4 L0 + 12 L1 tables of 64 MiB, 1 GiB in): the whole output, byte for
  byte, against the oracle's compaction of the same input bytes (built by the oracle's
  own builder), through luda_compact_device with the library's default tuning, as the
  bench's headline leg calls it.
* The 256-job batch (2.2 GB): one batch call and the autotuned plan replay (the bench's
  batched legs); every job's status and entry accounting checked, and a sample of jobs
  (every 16th, plus the largest) compared byte for byte with the oracle.
* The single-job configurations at scale 1.0: the plain job (3 tables, 6 MiB) and the
  LevelDB-default bottommost job (11 tables, 22 MiB), through luda_compact_device and
  luda_compact, and three plain jobs as one luda_batch_compact call (host buffers).
* A served run at the served workload's table size (64 MiB memtables and tables, 4 KiB
  blocks): the write stream through the simulated LSM tree and luda_server with several
  jobs in flight; its first three compaction jobs re-run by the oracle on the same input
  bytes, byte for byte.
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


@pytest.mark.parametrize("cfg,seed", [("config1", 1), ("config2", 2)])
def test_single_job_configs_full_size(cfg, seed):
    job = getattr(W, cfg)(seed=seed, scale=1.0)
    ins = oracle_inputs(job)
    want = oracle_compact(job, ins)
    assert want.status == 0
    assert job.bottommost == (cfg == "config2")
    got = luda.compact_device([dev(x) for x in ins], job.smallest_snapshot, level=job.level,
                              opts=luda.job_options(job))
    got.tables = [t.cpu().numpy().tobytes() for t in got.tables]
    assert_same(got, want)
    host = luda.compact(ins, job.smallest_snapshot, level=job.level, opts=luda.job_options(job))
    assert_same(host, want)
    assert host.ms_h2d > 0 and host.ms_d2h > 0
    assert sum(len(x) for x in ins) > (5 << 20 if cfg == "config1" else 20 << 20)


def test_batch_compact_host_full_size():
    jobs = [W.config1(seed=s, scale=1.0) for s in (1, 11, 12)]
    ins = [oracle_inputs(j) for j in jobs]
    rc, outs = luda.batch_compact([(x, j.smallest_snapshot, j.bottommost) for j, x in zip(jobs, ins)],
                                  luda.job_options(jobs[0]))
    assert rc == 0
    for j, g in enumerate(outs):
        assert_same(g, oracle_compact(jobs[j], ins[j]))
        assert g.ms_h2d > 0 and g.ms_d2h > 0


def test_served_jobs_full_table_size_sampled():
    from paper_2004_03054_b300 import lsm

    kept = []

    def on_complete(rec, out):
        if len(kept) >= 3:
            return
        ins = [luda.device_bytes(t.ptr, t.size).cpu().numpy().tobytes() for t in rec.inputs]
        outs = [luda.device_bytes(out.tables[i].data, out.tables[i].size).cpu().numpy().tobytes()
                for i in range(out.n_tables)]
        kept.append((rec.level, rec.bottommost, ins, outs, int(out.n_in_entries), int(out.n_dropped)))

    stream = W.config5_stream(seed=5, n_memtables=16, write_rate=8e6)
    rep = lsm.serve(stream, n_slots=4, hbm_budget=40 * 10**9, pace=False, on_complete=on_complete)
    assert rep.failed == 0 and rep.jobs >= 2
    assert len(kept) >= 2 and {k[0] for k in kept} >= {0}
    for level, bottom, ins, outs, n_in, n_drop in kept:
        want = oracle.compact(ins, W.MAX_SEQ, bottom, 4096, 16, 10, 64 << 20)
        assert want.status == 0
        assert outs == [t.data for t in want.tables], level
        assert (n_in, n_drop) == (want.n_in_entries, want.n_dropped)
        assert sum(len(x) for x in ins) >= 4 * (50 << 20) or level > 0
