"""Batched compaction and graph-captured plans: every job's tables are the same bytes
alone, in a batch, and in a replayed plan, and equal the oracle's."""
import struct

import numpy as np
import pytest

from helpers import oracle_compact, oracle_inputs
from paper_2004_03054_b300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2004_03054_b300 import luda  # noqa: E402

T, R, BPK, TARGET = 4096, 16, 10, 64 * 1024


def _dev(b):
    return torch.frombuffer(bytearray(b), dtype=torch.uint8).cuda()


def _mixed_jobs(n=12, seed=3):
    """Jobs of different shapes sharing one format (a batch shares format options)."""
    rng = np.random.default_rng(seed)
    jobs = []
    for j in range(n):
        kind = j % 3
        if kind == 0:
            job = W.config4_job(rng, int(rng.integers(40_000, 400_000)), f"b{j}", seed)
        elif kind == 1:
            job = W.tiny_job(rng, n_keys=int(rng.integers(5, 300)), max_versions=4, n_inputs=int(rng.integers(1, 6)),
                             key_len=(1, 20), val_len=(0, 500))
        else:
            job = W.config1(seed=seed + j, scale=1 / 128)
        job.block_size, job.restart_interval, job.bloom_bits_per_key, job.target_file_size = T, R, BPK, TARGET
        jobs.append(job)
    return jobs


def _tables(res):
    return [t.cpu().numpy().tobytes() for t in res.tables]


def test_batch_and_plan_equal_oracle_and_alone():
    jobs = _mixed_jobs()
    ins = [oracle_inputs(j) for j in jobs]
    want = [oracle_compact(j, x) for j, x in zip(jobs, ins)]
    dev = [[_dev(b) for b in x] for x in ins]
    opts = luda.options(T, R, BPK, TARGET)
    batch = [(d, j.smallest_snapshot, j.bottommost) for d, j in zip(dev, jobs)]
    rc, got = luda.batch_compact_device(batch, opts)
    assert rc == 0
    plan = luda.Plan(batch, luda.options(T, R, BPK, TARGET))
    for rep in range(2):
        plan.run()
        pl = plan.outputs()
        for j, (w, g, p) in enumerate(zip(want, got, pl)):
            assert g.status == w.status == p.status == 0, (j, g.status, p.status, g.detail, p.detail)
            assert _tables(g) == [t.data for t in w.tables], j
            assert _tables(p) == [t.data for t in w.tables], (j, rep)
            assert g.n_in_entries == p.n_in_entries == w.n_in_entries
            assert g.n_dropped == p.n_dropped == w.n_dropped
    plan.close()
    # alone
    for j in (0, 4, 8):
        alone = luda.compact_device(dev[j], jobs[j].smallest_snapshot,
                                    opts=luda.options(T, R, BPK, TARGET, bottommost=jobs[j].bottommost))
        assert _tables(alone) == [t.data for t in want[j].tables]


def test_corrupt_job_fails_alone_in_batch_and_plan():
    jobs = _mixed_jobs(n=6, seed=9)
    ins = [oracle_inputs(j) for j in jobs]
    want = [oracle_compact(j, x) for j, x in zip(jobs, ins)]
    dev = [[_dev(b) for b in x] for x in ins]
    batch = [(d, j.smallest_snapshot, j.bottommost) for d, j in zip(dev, jobs)]
    plan = luda.Plan(batch, luda.options(T, R, BPK, TARGET))
    # corrupt job 2's first data block in place (same size: the plan stays valid in size)
    st, rt, _ = oracle.read_table(ins[2][0])
    bad = bytearray(ins[2][0])
    bad[rt.blk_off[0] + 5] ^= 0x20
    dev[2][0].copy_(torch.frombuffer(bad, dtype=torch.uint8).cuda())
    rc, got = luda.batch_compact_device(batch, luda.options(T, R, BPK, TARGET))
    assert rc == 0
    plan.run()
    pl = plan.outputs()
    for j in range(len(jobs)):
        if j == 2:
            assert got[j].status == luda.ERR_CORRUPTION and got[j].tables == []
            assert pl[j].status == luda.ERR_CORRUPTION and pl[j].tables == []
        else:
            assert _tables(got[j]) == [t.data for t in want[j].tables]
            assert _tables(pl[j]) == [t.data for t in want[j].tables]
    plan.close()


def test_plan_rejects_changed_block_counts():
    jobs = _mixed_jobs(n=3, seed=5)
    ins = [oracle_inputs(j) for j in jobs]
    dev = [[_dev(b) for b in x] for x in ins]
    batch = [(d, j.smallest_snapshot, j.bottommost) for d, j in zip(dev, jobs)]
    plan = luda.Plan(batch, luda.options(T, R, BPK, TARGET))
    # replace job 0's first input by a different valid table of the same size with a
    # different block count: rebuild it with 1-byte blocks and pad/trim to the same size
    run = jobs[0].inputs[0]
    other = oracle.build_tables(run, 65536, R, BPK, (1 << 64) - 1).tables[0].data
    if len(other) >= len(ins[0][0]):
        pytest.skip("rebuilt table not smaller")
    img = bytearray(ins[0][0])
    img[:] = b"\x00" * len(img)
    img[len(img) - len(other):] = other  # a valid table image ends at the buffer end ... with a new size
    # the footer is read at the end of the buffer, so the table parses with different
    # handles; offsets now point into the zero prefix -> block counts differ from the plan
    dev[0][0].copy_(torch.frombuffer(img, dtype=torch.uint8).cuda())
    plan.run()
    pl = plan.outputs()
    assert pl[0].status in (luda.ERR_PLAN_MISMATCH, luda.ERR_CORRUPTION)
    for j in (1, 2):
        assert pl[j].status == 0
    plan.close()
