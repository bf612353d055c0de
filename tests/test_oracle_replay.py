"""The oracle's compaction against the brute-force replay of the generated writes."""
import numpy as np
import pytest

import oracle
from helpers import decoded, oracle_compact, oracle_inputs
from paper_2004_03054_b300 import workloads as W
from replay import newest_only, replay


def test_build_roundtrip_python_reader():
    """A table built from one run reads back, through the independent Python reader, as
    exactly the run's entries."""
    job = W.config1(seed=11, scale=1 / 64)
    for run, data in zip(job.inputs, oracle_inputs(job)):
        got = decoded([data], reader="py")
        want = [(run.key(i), int(run.seqs[i]), int(run.types[i]), run.value(i)) for i in range(run.n)]
        assert got == want


@pytest.mark.parametrize("seed", range(400))
def test_tiny_jobs_match_replay(seed):
    rng = np.random.default_rng(1000 + seed)
    job = W.tiny_job(rng, n_keys=int(rng.integers(1, 4)), max_versions=6, n_inputs=3)
    res = oracle_compact(job)
    assert res.status == 0, res.detail
    assert decoded(res.tables, reader="py") == replay(job)
    assert res.n_in_entries == job.n_entries
    assert res.n_in_entries - res.n_dropped == sum(t.n_entries for t in res.tables)


@pytest.mark.parametrize("seed", range(60))
def test_small_random_jobs_match_replay(seed):
    rng = np.random.default_rng(5000 + seed)
    job = W.tiny_job(rng, n_keys=int(rng.integers(5, 60)), max_versions=4, n_inputs=int(rng.integers(1, 6)),
                     key_len=(0, 6), val_len=(0, 40))
    res = oracle_compact(job)
    assert res.status == 0, res.detail
    assert decoded(res.tables, reader="py") == replay(job)


def test_every_snapshot_small_job():
    rng = np.random.default_rng(77)
    job = W.tiny_job(rng, n_keys=3, max_versions=6, n_inputs=3, snapshot=0, bottommost=False)
    max_seq = max(int(s) for r in job.inputs for s in r.seqs)
    inputs = oracle_inputs(job)
    for S in range(0, max_seq + 2):
        for bottom in (False, True):
            job.smallest_snapshot, job.bottommost = S, bottom
            res = oracle_compact(job, inputs)
            assert res.status == 0
            assert decoded(res.tables) == replay(job)


@pytest.mark.parametrize("cfg,scale", [(1, 1 / 16), (2, 1 / 16), (3, 1 / 256)])
def test_configs_match_replay(cfg, scale):
    job = W.make(cfg, scale=scale)
    res = oracle_compact(job)
    assert res.status == 0, res.detail
    got = decoded(res.tables)
    assert got == replay(job)
    assert got == newest_only(job)        # S = max: newest version per key
    assert len({k for k, *_ in got}) == len(got)


def test_config4_job_matches_replay():
    rng = np.random.default_rng(4)
    job = W.config4_job(rng, 300 * 1024, "c4", 4)
    res = oracle_compact(job)
    assert res.status == 0
    assert decoded(res.tables) == replay(job)


def test_all_dropped_gives_no_tables():
    rng = np.random.default_rng(9)
    job = W.tiny_job(rng, n_keys=2, max_versions=1, n_inputs=1, p_del=1.0, snapshot=W.MAX_SEQ, bottommost=True)
    res = oracle_compact(job)
    assert res.status == 0 and res.tables == [] and res.n_dropped == job.n_entries


def test_no_inputs():
    res = oracle.compact([])
    assert res.status == 0 and res.tables == [] and res.n_in_entries == 0
