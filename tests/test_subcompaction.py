"""R13 ranged compactions and subcompactions in the oracle (CPU): a job split at user-key
bounds gives, range by range, exactly the entries the whole job gives; a ranged compaction
reads only the data blocks that can hold its keys (a corrupt block outside the range goes
unnoticed, one inside fails the job)."""
import struct

import numpy as np
import pytest

import oracle
from helpers import U64MAX, decoded, oracle_compact, oracle_inputs
from paper_2004_03054_b300 import workloads as W


def _opts(job):
    return dict(smallest_snapshot=job.smallest_snapshot, bottommost=job.bottommost, block_size=job.block_size,
                restart_interval=job.restart_interval, bloom_bits_per_key=job.bloom_bits_per_key,
                target_file_size=job.target_file_size)


def _user_keys(job):
    return sorted({bytes(r.ukeys[r.ukoff[i]:r.ukoff[i + 1]]) for r in job.inputs for i in range(len(r.seqs))})


@pytest.mark.parametrize("seed", range(12))
def test_subcompactions_partition_the_job(seed):
    rng = np.random.default_rng(1300 + seed)
    job = W.tiny_job(rng, n_keys=int(rng.integers(10, 500)), max_versions=5, n_inputs=int(rng.integers(1, 6)),
                     key_len=(0, 16), val_len=(0, 200), p_del=0.1)
    job.block_size, job.target_file_size = int(rng.choice([64, 512, 4096])), int(rng.choice([1500, 1 << 20]))
    job.bottommost = bool(rng.integers(0, 2))
    ins = oracle_inputs(job)
    whole = oracle_compact(job, ins)
    assert whole.status == 0
    keys = _user_keys(job)
    # bounds: some of the job's own user keys and some keys between or outside them
    cand = [keys[int(i)] for i in rng.integers(0, len(keys), size=3)] + [rng.bytes(int(rng.integers(0, 6)))
                                                                          for _ in range(2)]
    bounds = sorted(set(cand))
    sub = oracle.subcompact(ins, bounds, **_opts(job))
    assert sub.status == 0
    assert decoded([t.data for t in sub.tables]) == decoded([t.data for t in whole.tables])
    assert sub.n_in_entries - sub.n_dropped == whole.n_in_entries - whole.n_dropped
    # each range's tables hold only keys of the range
    edges = [None] + bounds + [None]
    for lo, hi in zip(edges[:-1], edges[1:]):
        r = oracle.compact(ins, **_opts(job), lo=lo, hi=hi)
        assert r.status == 0
        for uk, _, _, _ in decoded([t.data for t in r.tables]):
            assert (lo is None or uk >= lo) and (hi is None or uk < hi)


def test_empty_and_outside_ranges():
    job = W.config1(seed=3, scale=1 / 64)
    ins = oracle_inputs(job)
    keys = _user_keys(job)
    for lo, hi in ((keys[5], keys[5]), (b"\xff" * 20, None), (None, b""), (keys[-1] + b"\x00", None)):
        r = oracle.compact(ins, **_opts(job), lo=lo, hi=hi)
        assert r.status == 0 and r.tables == [] and r.n_in_entries - r.n_dropped == 0


def test_a_ranged_job_reads_only_its_blocks():
    job = W.config1(seed=9, scale=1 / 32)
    ins = oracle_inputs(job)
    st, rt, _ = oracle.read_table(ins[1])
    assert st == 0 and rt.n_blocks > 10
    # the user key of block 5's last entry, and of block 8's
    last = [rt.keys[rt.blk_last[b]][:-8] for b in range(rt.n_blocks)]
    lo, hi = last[5] + b"\x00", last[8] + b"\x00"   # blocks 6..8 (and 9, whose first key may be below hi)
    bad = bytearray(ins[1])
    bad[rt.blk_off[2] + 3] ^= 0x20                   # a data block far below the range
    r = oracle.compact([ins[0], bytes(bad)] + ins[2:], **_opts(job), lo=lo, hi=hi)
    assert r.status == 0
    full = oracle.compact(ins, **_opts(job), lo=lo, hi=hi)
    assert [t.data for t in r.tables] == [t.data for t in full.tables]
    bad = bytearray(ins[1])
    bad[rt.blk_off[7] + 3] ^= 0x20                   # a data block inside the range
    r = oracle.compact([ins[0], bytes(bad)] + ins[2:], **_opts(job), lo=lo, hi=hi)
    assert r.status == oracle.ERR_CORRUPTION
    # fewer entries decoded than the whole job
    assert full.n_in_entries < oracle.compact(ins, **_opts(job)).n_in_entries
