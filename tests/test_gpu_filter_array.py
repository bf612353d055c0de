"""GPU parity for the filter array variant (LUDA_F_FILTER_ARRAY, R10a): table bytes equal
the oracle's on the single-job, batched, graph-plan, ranged and builder paths, including
tables whose blocks share a 2 KiB window, leave windows empty, or hold one entry."""
import numpy as np
import pytest

from helpers import U64MAX, oracle_compact, oracle_inputs
from paper_2004_03054_b300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import sstpy  # noqa: E402
from paper_2004_03054_b300 import luda  # noqa: E402
from test_gpu_parity import assert_same, check_job, dev  # noqa: E402

FA = luda.F_FILTER_ARRAY


@pytest.mark.parametrize("cfg,scale", [(1, 1 / 16), (2, 1 / 16), (3, 1 / 128)])
def test_configs(cfg, scale):
    res = check_job(W.make(cfg, scale=scale), flags=FA)
    r = sstpy.read(res.tables[0])
    assert r["filter_name"] == "filter.luda.bloom2k"
    assert r["filter"] == sstpy.filter_array(r["blocks"], r["handles"]["filter"][0], W.make(cfg, scale=scale)
                                             .bloom_bits_per_key)


@pytest.mark.parametrize("seed", range(30))
def test_small_jobs(seed):
    rng = np.random.default_rng(9100 + seed)
    job = W.tiny_job(rng, n_keys=int(rng.integers(1, 400)), max_versions=4, n_inputs=int(rng.integers(1, 6)),
                     key_len=(0, 20), val_len=(0, 5000))
    job.block_size = int(rng.choice([1, 64, 512, 2048, 4096]))
    job.target_file_size = int(rng.choice([1, 3000, 1 << 20]))
    job.bloom_bits_per_key = int(rng.choice([1, 6, 10, 64]))
    check_job(job, flags=int(rng.choice([FA, FA | luda.F_SHORT_INDEX])))


def test_all_dropped():
    rng = np.random.default_rng(3)
    job = W.tiny_job(rng, n_keys=20, max_versions=1, n_inputs=1, p_del=1.0, snapshot=W.MAX_SEQ, bottommost=True)
    res = check_job(job, flags=FA)
    assert res.tables == []


def test_batch_and_plan():
    jobs = [W.config1(seed=s, scale=1 / 32) for s in (1, 2)] + [W.config2(seed=3, scale=1 / 32)]
    for j in jobs:
        j.block_size, j.restart_interval, j.bloom_bits_per_key, j.target_file_size = 1024, 16, 10, 64 << 10
    ins = [oracle_inputs(j) for j in jobs]
    want = [oracle_compact(j, x, FA) for j, x in zip(jobs, ins)]
    batch = [([dev(b) for b in x], j.smallest_snapshot, j.bottommost) for j, x in zip(jobs, ins)]
    opts = luda.job_options(jobs[0], flags=FA)
    rc, got = luda.batch_compact_device(batch, opts)
    assert rc == 0
    for g, w in zip(got, want):
        g.tables = [t.cpu().numpy().tobytes() for t in g.tables]
        assert_same(g, w)
    plan = luda.Plan(batch, opts)
    for _ in range(2):
        plan.run()
        torch.cuda.synchronize()
        for g, w in zip(plan.outputs(), want):
            g.tables = [t.cpu().numpy().tobytes() for t in g.tables]
            assert_same(g, w)
    plan.close()


def test_ranged_and_subcompaction():
    job = W.config1(seed=5, scale=1 / 32)
    ins = oracle_inputs(job)
    keys = sorted({bytes(r.ukeys[r.ukoff[i]:r.ukoff[i + 1]]) for r in job.inputs for i in range(len(r.seqs))})
    bounds = [keys[len(keys) // 3], keys[2 * len(keys) // 3]]
    want = oracle.subcompact(ins, bounds, smallest_snapshot=job.smallest_snapshot, bottommost=job.bottommost,
                             block_size=job.block_size, restart_interval=job.restart_interval,
                             bloom_bits_per_key=job.bloom_bits_per_key, target_file_size=job.target_file_size,
                             flags=oracle.F_FILTER_ARRAY)
    got = luda.subcompact_device([dev(x) for x in ins], bounds, job.smallest_snapshot,
                                 opts=luda.job_options(job, flags=FA))
    assert got.status == want.status == 0, got.detail
    assert [t.cpu().numpy().tobytes() for t in got.tables] == [t.data for t in want.tables]


@pytest.mark.parametrize("T,vlen", [(4096, 100), (256, 40), (1, 3000), (1, 0)])
def test_builder(T, vlen):
    rng = np.random.default_rng(T + vlen)
    users = sorted({rng.bytes(16) for _ in range(500)})
    n = len(users)
    run = W._make_run(users, np.arange(1, n + 1, dtype=np.uint64), np.ones(n, np.uint8), np.full(n, vlen), rng, 0)
    want = oracle.build_tables(run, T, 16, 10, 200 << 10, flags=oracle.F_FILTER_ARRAY)
    got = luda.build_device(run, luda.options(T, 16, 10, 200 << 10, flags=FA))
    assert got.status == 0, got.detail
    assert [t.cpu().numpy().tobytes() for t in got.tables] == [t.data for t in want.tables]


def test_filter_array_inputs():
    """Tables with filter arrays are inputs like any others."""
    job = W.config1(seed=7, scale=1 / 32)
    fa_ins = []
    for r in job.inputs:
        res = oracle.build_tables(r, job.block_size, job.restart_interval, job.bloom_bits_per_key, U64MAX,
                                  flags=oracle.F_FILTER_ARRAY)
        fa_ins.append(res.tables[0].data)
    check_job(job, fa_ins)
    check_job(job, fa_ins, flags=FA)
