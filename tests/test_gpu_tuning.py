"""Launch shapes never change the output: every tuning gives the oracle's bytes, alone and
in a plan; luda_autotune times candidates and the tuner's cache returns its choice."""
import ctypes as C

import numpy as np
import pytest

from helpers import oracle_compact, oracle_inputs
from paper_2004_03054_b300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2004_03054_b300 import autotune as AT  # noqa: E402
from paper_2004_03054_b300 import luda  # noqa: E402

T, R, BPK, TARGET = 4096, 16, 10, 64 * 1024

TUNINGS = [
    {"merge_tile": 512},
    {"merge_tile": 2048},
    {"merge_tile": 2048, "merge_ctas_per_sm": 1},
    {"merge_tile": 512, "merge_ctas_per_sm": 32},
    {"decode_warps": 1, "walk_threads": 32},
    {"decode_warps": 16, "walk_threads": 64},
    {"encode_ctas_per_sm": 1},
    {"elem_threads": 64},
    {"elem_threads": 1024},
    {"merge_tile": 512, "merge_ctas_per_sm": 2, "decode_warps": 2, "walk_threads": 96, "encode_ctas_per_sm": 2,
     "elem_threads": 160},
    {"crc_warps": 16, "crc_ctas": 148},
    {"crc_warps": 8, "crc_ctas": 20},
    {"crc_ctas": 1},
]


def _dev(b):
    return torch.frombuffer(bytearray(b), dtype=torch.uint8).cuda()


def _jobs(n, seed):
    rng = np.random.default_rng(seed)
    jobs = []
    for j in range(n):
        if j % 3 == 0:
            job = W.config4_job(rng, int(rng.integers(60_000, 600_000)), f"t{j}", seed)
        elif j % 3 == 1:
            job = W.tiny_job(rng, n_keys=int(rng.integers(5, 400)), max_versions=4, n_inputs=int(rng.integers(1, 7)),
                             key_len=(0, 20), val_len=(0, 400))
        else:
            job = W.config1(seed=seed + j, scale=1 / 128)
        job.block_size, job.restart_interval, job.bloom_bits_per_key, job.target_file_size = T, R, BPK, TARGET
        jobs.append(job)
    return jobs


@pytest.fixture(scope="module")
def batch():
    jobs = _jobs(9, seed=23)
    ins = [oracle_inputs(j) for j in jobs]
    want = [[t.data for t in oracle_compact(j, x).tables] for j, x in zip(jobs, ins)]
    dev = [[_dev(b) for b in x] for x in ins]
    return jobs, dev, want, [(d, j.smallest_snapshot, j.bottommost) for d, j in zip(dev, jobs)]


@pytest.mark.parametrize("tuning", TUNINGS, ids=[str(i) for i in range(len(TUNINGS))])
def test_tuning_keeps_bytes_single_and_plan(batch, tuning):
    jobs, dev, want, b = batch
    opts = luda.options(T, R, BPK, TARGET, tuning=tuning)
    for j in (0, 1, 2, 5):
        o = luda.options(T, R, BPK, TARGET, bottommost=jobs[j].bottommost, tuning=tuning)
        res = luda.compact_device(dev[j], jobs[j].smallest_snapshot, opts=o)
        assert res.status == 0, res.detail
        assert [t.cpu().numpy().tobytes() for t in res.tables] == want[j], j
    plan = luda.Plan(b, opts)
    plan.run()
    for j, r in enumerate(plan.outputs()):
        assert r.status == 0 and [t.cpu().numpy().tobytes() for t in r.tables] == want[j], j
    plan.close()


@pytest.mark.parametrize("tuning", [TUNINGS[1], TUNINGS[-1]], ids=["big_tile", "mixed"])
def test_tuning_large_job(tuning):
    job = W.config3(seed=7, scale=1 / 128)
    ins = oracle_inputs(job)
    want = [t.data for t in oracle_compact(job, ins).tables]
    res = luda.compact_device([_dev(x) for x in ins], job.smallest_snapshot,
                              opts=luda.job_options(job, tuning=tuning))
    assert res.status == 0, res.detail
    assert [t.cpu().numpy().tobytes() for t in res.tables] == want


def test_invalid_tuning_is_rejected(batch):
    jobs, dev, _, _ = batch
    res = luda.compact_device(dev[0], jobs[0].smallest_snapshot,
                              opts=luda.options(T, R, BPK, TARGET, tuning={"merge_tile": 1000}))
    assert res.status == luda.ERR_INVALID_ARG and "merge_tile" in res.detail


def test_autotune_times_candidates(batch, tmp_path):
    _, _, want, b = batch
    opts = luda.options(T, R, BPK, TARGET)
    cands = [AT.DEFAULT, dict(AT.DEFAULT, merge_tile=512), dict(AT.DEFAULT, decode_warps=4, elem_threads=128)]
    js, keep = luda._jobs_array(b)
    arr = (luda.Tuning * 3)(*[luda.Tuning.of(c) for c in cands])
    ms = (C.c_double * 3)()
    best = C.c_uint32(99)
    assert luda.lib().luda_autotune(js, len(b), C.byref(opts), arr, 3, 2, ms, C.byref(best)) == luda.OK
    assert all(m > 0 for m in ms) and best.value == min(range(3), key=lambda i: ms[i])
    arr[1].merge_tile = 300
    assert luda.lib().luda_autotune(js, len(b), C.byref(opts), arr, 3, 2, ms, C.byref(best)) == luda.ERR_INVALID_ARG
    # the tuner: a miss times candidates and fills the cache, the second call hits it
    small = {"merge_tile": (512, 1024), "decode_warps": (4, 8)}
    path = str(tmp_path / "tune.json")
    r1 = AT.tune(b, opts, cache_path=path, reps=2, space=small)
    assert r1.cache == "miss" and len(r1.evaluated) >= 3 and r1.best_ms > 0
    r2 = AT.tune(b, opts, cache_path=path, reps=2, space=small)
    assert r2.cache == "hit" and r2.tuning == r1.tuning
    plan = luda.Plan(b, opts.with_tuning(r2.tuning))
    plan.run()
    assert [[t.cpu().numpy().tobytes() for t in r.tables] for r in plan.outputs()] == want
    plan.close()
    del keep
