"""GPU parity: the CUDA path's table bytes equal the oracle's, bit for bit.

Every case goes through the C ABI (libluda.so) via the ctypes binding. Inputs are built
by the oracle's builder from seeded runs; expected outputs come from the oracle only.
"""
import struct

import numpy as np
import pytest

from helpers import U64MAX, oracle_compact, oracle_inputs
from paper_2004_03054_b300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2004_03054_b300 import luda  # noqa: E402


def dev(b: bytes):
    return torch.frombuffer(bytearray(b), dtype=torch.uint8).cuda()


def gpu_compact(job, inputs, flags=0):
    res = luda.compact_device([dev(x) for x in inputs], job.smallest_snapshot,
                              opts=luda.job_options(job, flags=flags))
    res.tables = [t.cpu().numpy().tobytes() for t in res.tables]
    return res


def first_diff(a: bytes, b: bytes):
    n = min(len(a), len(b))
    d = next((i for i in range(n) if a[i] != b[i]), n)
    return f"len {len(a)} vs {len(b)}, first difference at byte {d}"


def assert_same(res, want):
    assert res.status == want.status, (res.status, want.status, res.detail, want.detail)
    assert len(res.tables) == len(want.tables)
    for i, (a, w) in enumerate(zip(res.tables, want.tables)):
        assert a == w.data, f"table {i}: {first_diff(a, w.data)}"
        assert res.smallest[i] == w.smallest and res.largest[i] == w.largest
        assert res.n_entries[i] == w.n_entries
    if want.status == 0:
        assert res.n_in_entries == want.n_in_entries and res.n_dropped == want.n_dropped


def check_job(job, inputs=None, flags=0):
    inputs = oracle_inputs(job) if inputs is None else inputs
    want = oracle_compact(job, inputs, flags)
    res = gpu_compact(job, inputs, flags)
    assert_same(res, want)
    return res


# ---- the builder (pack stages only) ------------------------------------------------------
@pytest.mark.parametrize("T,R,target", [(4096, 16, U64MAX), (1, 1, U64MAX), (64, 3, 900), (16384, 16, 1 << 16)])
def test_build_matches_oracle(T, R, target):
    job = W.config1(seed=3, scale=1 / 32)
    run = job.inputs[0]
    want = oracle.build_tables(run, T, R, 10, target)
    got = luda.build_device(run, luda.options(T, R, 10, target))
    assert got.status == 0, got.detail
    assert [t.cpu().numpy().tobytes() for t in got.tables] == [t.data for t in want.tables]
    host = luda.build(run, luda.options(T, R, 10, target))
    assert host.tables == [t.data for t in want.tables]


def test_build_rejects_unsorted():
    rng = np.random.default_rng(1)
    run = W._make_run([b"b", b"a"], np.array([1, 2], np.uint64), np.array([1, 1], np.uint8), np.array([1, 1]), rng, 0)
    assert luda.build_device(run).status == luda.ERR_INVALID_ARG


# ---- compaction --------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(120))
def test_tiny_jobs(seed):
    rng = np.random.default_rng(1000 + seed)
    job = W.tiny_job(rng, n_keys=int(rng.integers(1, 4)), max_versions=6, n_inputs=3)
    check_job(job)


@pytest.mark.parametrize("seed", range(40))
def test_small_random_jobs(seed):
    rng = np.random.default_rng(5000 + seed)
    job = W.tiny_job(rng, n_keys=int(rng.integers(5, 400)), max_versions=4, n_inputs=int(rng.integers(1, 7)),
                     key_len=(0, 12), val_len=(0, 300))
    check_job(job)


@pytest.mark.parametrize("cfg,scale", [(1, 1 / 16), (2, 1 / 16), (3, 1 / 128)])
def test_configs_reduced(cfg, scale):
    check_job(W.make(cfg, scale=scale))


def test_config4_jobs():
    rng = np.random.default_rng(44)
    for size in (64 * 1024, 300 * 1024, 1 << 20):
        check_job(W.config4_job(rng, size, "c4", 44))


@pytest.mark.parametrize("T,R,target", [(1, 1, 1), (1, 16, 300), (64, 2, 1000), (200, 3, 5000), (777, 5, 20000),
                                        (1 << 20, 16, 1 << 30)])
def test_cut_parameters(T, R, target):
    job = W.config1(seed=5, scale=1 / 64)
    inputs = oracle_inputs(job)
    job.block_size, job.restart_interval, job.target_file_size = T, R, target
    check_job(job, inputs)


def test_keys_longer_than_block_and_empty_values():
    rng = np.random.default_rng(12)
    keys = sorted({rng.bytes(int(rng.integers(100, 3000))) for _ in range(50)})
    run = W._make_run(keys, np.arange(1, 51, dtype=np.uint64), np.ones(50, np.uint8), np.zeros(50, np.int64),
                      rng, 0)
    job = W.Job("long", 0, [run], W.MAX_SEQ, False, 256, 4, 10, 4096)
    check_job(job)


def test_snapshot_and_bottommost_sweep():
    rng = np.random.default_rng(77)
    job = W.tiny_job(rng, n_keys=60, max_versions=6, n_inputs=4, snapshot=0, bottommost=False)
    inputs = oracle_inputs(job)
    max_seq = max(int(s) for r in job.inputs for s in r.seqs)
    for S in sorted({0, 1, max_seq // 3, max_seq // 2, max_seq - 1, max_seq, W.MAX_SEQ}):
        for bottom in (False, True):
            job.smallest_snapshot, job.bottommost = S, bottom
            check_job(job, inputs)


def test_all_dropped_and_no_inputs():
    rng = np.random.default_rng(9)
    job = W.tiny_job(rng, n_keys=30, max_versions=1, n_inputs=2, p_del=1.0, snapshot=W.MAX_SEQ, bottommost=True)
    res = check_job(job)
    assert res.tables == []
    res = luda.compact_device([], opts=luda.options())
    assert res.status == 0 and res.tables == []


def test_duplicates_across_inputs():
    rng = np.random.default_rng(8)
    run = W._make_run([b"k", b"m"], np.array([5, 6], np.uint64), np.array([1, 1], np.uint8), np.array([3, 4]), rng, 0)
    t = oracle.build_tables(run).tables[0].data
    job = W.Job("dup", 0, [run, run], W.MAX_SEQ, False)
    check_job(job, [t, t])
    check_job(job, [t, t], flags=luda.F_STRICT_DUP)


# ---- corruption ----------------------------------------------------------------------------
def _inputs():
    job = W.config1(seed=31, scale=1 / 256)
    return job, oracle_inputs(job)


def test_crc_flip():
    job, ins = _inputs()
    st, rt, _ = oracle.read_table(ins[1])
    bad = bytearray(ins[1])
    bad[rt.blk_off[1] + 7] ^= 0x01
    check_job(job, [ins[0], bytes(bad), ins[2]])


def test_compressed_block():
    job, ins = _inputs()
    st, rt, _ = oracle.read_table(ins[0])
    off, size = rt.blk_off[0], rt.blk_size[0]
    bad = bytearray(ins[0])
    bad[off + size] = 1
    bad[off + size + 1: off + size + 5] = struct.pack("<I", oracle.mask(oracle.crc32c(bytes(bad[off: off + size + 1]))))
    check_job(job, [bytes(bad)] + ins[1:])


@pytest.mark.parametrize("cut", [1, 8, 47, 48, 1000])
def test_truncated(cut):
    job, ins = _inputs()
    check_job(job, [ins[0][:-cut]] + ins[1:])


def test_garbage_input():
    job, ins = _inputs()
    rng = np.random.default_rng(3)
    check_job(job, [rng.bytes(5000)] + ins[1:])
    check_job(job, [b"\x00" * 47] + ins[1:])


def test_out_of_order_input():
    from test_oracle_invariants import _single_block_table
    last = b"a" + struct.pack("<Q", 2 << 8 | 1)
    contents = oracle.encode_block([(b"b" + struct.pack("<Q", 1 << 8 | 1), b"x"), (last, b"y")], 16)
    img = _single_block_table(contents, last)
    job = W.Job("ooo", 0, [], W.MAX_SEQ, False)
    check_job(job, [img])


@pytest.mark.parametrize("index_key", [b"z" * 9, b"b" + struct.pack("<Q", 2 << 8 | 1), b"b" + struct.pack("<Q", 1 << 8 | 1)])
def test_index_key_check(index_key):
    from test_oracle_invariants import _single_block_table
    contents = oracle.encode_block([(b"a" + struct.pack("<Q", 2 << 8 | 1), b"y"),
                                    (b"b" + struct.pack("<Q", 1 << 8 | 1), b"x")], 16)
    job = W.Job("ikey", 0, [], W.MAX_SEQ, False)
    other = oracle_inputs(W.config1(seed=4, scale=1 / 128))
    check_job(job, [_single_block_table(contents, index_key)])
    check_job(job, other + [_single_block_table(contents, index_key)])


# ---- host entry point ----------------------------------------------------------------------
def test_host_entry_point():
    job = W.config2(seed=5, scale=1 / 32)
    inputs = oracle_inputs(job)
    want = oracle_compact(job, inputs)
    res = luda.compact(inputs, job.smallest_snapshot, opts=luda.job_options(job))
    assert_same(res, want)
    assert res.ms_h2d > 0 and res.ms_d2h >= 0


def test_bad_options():
    for kw in (dict(block_size=0), dict(restart_interval=0), dict(bloom_bits_per_key=0), dict(target_file_size=0)):
        res = luda.compact_device([], opts=luda.options(**kw))
        assert res.status == luda.ERR_INVALID_ARG


@pytest.mark.parametrize("seed", range(6))
def test_skewed_runs(seed):
    """Inputs whose key ranges barely overlap (most of one run sorts before the other):
    the merge's co-rank search then finds its split at the far end of the range."""
    rng = np.random.default_rng(700 + seed)
    n_a, n_b = int(rng.integers(3000, 20000)), int(rng.integers(500, 8000))
    keys = np.sort(rng.choice(1 << 30, size=n_a + n_b, replace=False)).astype(np.uint64)
    over = int(rng.integers(0, 40))
    a_keys = keys[:n_a]
    b_keys = np.concatenate([keys[n_a - over:n_a] + np.uint64(1), keys[n_a:]]) if over else keys[n_a:]
    b_keys = np.unique(b_keys)
    runs = []
    for level, ks in ((1, b_keys), (2, a_keys)):
        m = len(ks)
        seqs = rng.permutation(np.arange(1, m + 1, dtype=np.uint64)) + np.uint64(10**6 if level == 1 else 0)
        runs.append(W._make_run(W._fixed_keys(ks), seqs, W._types(rng, m, 0.02), rng.integers(0, 64, size=m), rng,
                                level))
    job = W.Job(f"skew{seed}", seed, runs, W.MAX_SEQ, False, 4096, 16, 10, 1 << 20)
    check_job(job)


# ---- format variant R9s: shortened index keys ------------------------------------------------
@pytest.mark.parametrize("cfg,scale", [(1, 1 / 16), (2, 1 / 16), (3, 1 / 128)])
def test_short_index_configs(cfg, scale):
    job = W.make(cfg, scale=scale)
    check_job(job, flags=luda.F_SHORT_INDEX)


@pytest.mark.parametrize("seed", range(30))
def test_short_index_small_jobs(seed):
    rng = np.random.default_rng(8000 + seed)
    job = W.tiny_job(rng, n_keys=int(rng.integers(5, 400)), max_versions=4, n_inputs=int(rng.integers(1, 6)),
                     key_len=(0, 20), val_len=(0, 300))
    job.block_size = int(rng.choice([1, 64, 512, 4096]))
    job.target_file_size = int(rng.choice([1, 3000, 1 << 20]))
    check_job(job, flags=luda.F_SHORT_INDEX)


def test_short_index_inputs_and_builder():
    """Inputs whose index keys are shortened decode like any others; the device builder
    writes R9s keys as the oracle's builder does."""
    job = W.config1(seed=12, scale=1 / 32)
    short = []
    for r in job.inputs:
        res = oracle.build_tables(r, job.block_size, job.restart_interval, job.bloom_bits_per_key, U64MAX,
                                  flags=oracle.F_SHORT_INDEX)
        short.append(res.tables[0].data)
        got = luda.build_device(r, luda.options(job.block_size, job.restart_interval, job.bloom_bits_per_key,
                                                U64MAX, flags=luda.F_SHORT_INDEX))
        assert got.status == 0 and [t.cpu().numpy().tobytes() for t in got.tables] == [res.tables[0].data]
    check_job(job, short)
    check_job(job, short, flags=luda.F_SHORT_INDEX)


@pytest.mark.parametrize("key0", [b"b" + struct.pack("<Q", 1 << 8 | 1), b"c" + struct.pack("<Q", (1 << 64) - 255),
                                  b"d" + struct.pack("<Q", 1 << 8 | 1), b"d" + struct.pack("<Q", 1 << 8 | 0),
                                  b"e" + struct.pack("<Q", 5 << 8 | 1), b"a" * 9, b"a"])
def test_index_key_interval_check(key0):
    from test_oracle_invariants import _table
    b0 = oracle.encode_block([(b"a" + struct.pack("<Q", 2 << 8 | 1), b"y"), (b"b" + struct.pack("<Q", 1 << 8 | 1), b"x")],
                             16)
    b1 = oracle.encode_block([(b"d" + struct.pack("<Q", 1 << 8 | 1), b"u"), (b"e" + struct.pack("<Q", 1 << 8 | 1), b"v")],
                             16)
    img = _table([(b0, key0), (b1, b"e" + struct.pack("<Q", 1 << 8 | 1))])
    job = W.Job("ikey2", 0, [], W.MAX_SEQ, False)
    check_job(job, [img])
    check_job(job, oracle_inputs(W.config1(seed=4, scale=1 / 128)) + [img])


# ---- R13: ranged jobs and subcompactions -------------------------------------------------------
def _user_keys(job):
    return sorted({bytes(r.ukeys[r.ukoff[i]:r.ukoff[i + 1]]) for r in job.inputs for i in range(len(r.seqs))})


def _oracle_opts(job, flags=0):
    return dict(smallest_snapshot=job.smallest_snapshot, bottommost=job.bottommost, block_size=job.block_size,
                restart_interval=job.restart_interval, bloom_bits_per_key=job.bloom_bits_per_key,
                target_file_size=job.target_file_size, flags=flags)


@pytest.mark.parametrize("seed", range(16))
def test_subcompaction_matches_oracle(seed):
    rng = np.random.default_rng(4400 + seed)
    job = W.tiny_job(rng, n_keys=int(rng.integers(10, 500)), max_versions=5, n_inputs=int(rng.integers(1, 6)),
                     key_len=(0, 16), val_len=(0, 300), p_del=0.1)
    job.block_size, job.target_file_size = int(rng.choice([64, 512, 4096])), int(rng.choice([1500, 1 << 20]))
    job.bottommost = bool(rng.integers(0, 2))
    ins = oracle_inputs(job)
    keys = _user_keys(job)
    bounds = sorted(set([keys[int(i)] for i in rng.integers(0, len(keys), size=int(rng.integers(1, 5)))]
                        + [rng.bytes(int(rng.integers(0, 5)))]))
    flags = int(rng.choice([0, luda.F_SHORT_INDEX]))
    want = oracle.subcompact(ins, bounds, **_oracle_opts(job, flags))
    got = luda.subcompact_device([dev(x) for x in ins], bounds, job.smallest_snapshot,
                                 opts=luda.job_options(job, flags=flags))
    assert got.status == want.status == 0, (got.status, got.detail)
    assert [t.cpu().numpy().tobytes() for t in got.tables] == [t.data for t in want.tables]
    assert got.n_in_entries == want.n_in_entries and got.n_dropped == want.n_dropped
    assert [(s, l) for s, l in zip(got.smallest, got.largest)] == [(t.smallest, t.largest) for t in want.tables]


def test_ranged_jobs_in_a_batch_and_corrupt_blocks_outside_the_range():
    job = W.config1(seed=9, scale=1 / 32)
    ins = oracle_inputs(job)
    st, rt, _ = oracle.read_table(ins[1])
    last = [rt.keys[rt.blk_last[b]][:-8] for b in range(rt.n_blocks)]
    lo, hi = last[5] + b"\x00", last[8] + b"\x00"
    bad_out = bytearray(ins[1])
    bad_out[rt.blk_off[2] + 3] ^= 0x20   # below the range: not read
    bad_in = bytearray(ins[1])
    bad_in[rt.blk_off[7] + 3] ^= 0x20    # inside the range
    cases = [(ins, lo, hi), ([ins[0], bytes(bad_out)] + ins[2:], lo, hi), ([ins[0], bytes(bad_in)] + ins[2:], lo, hi),
             (ins, None, lo), (ins, hi, None), (ins, lo, lo)]
    batch = [([dev(x) for x in c], job.smallest_snapshot, job.bottommost, a, b) for c, a, b in cases]
    rc, got = luda.batch_compact_device(batch, luda.job_options(job))
    assert rc == 0
    for (c, a, b), g in zip(cases, got):
        w = oracle.compact(c, **_oracle_opts(job), lo=a, hi=b)
        assert g.status == w.status, (g.status, w.status, g.detail)
        if w.status == 0:
            assert [t.cpu().numpy().tobytes() for t in g.tables] == [t.data for t in w.tables]
            assert g.n_in_entries == w.n_in_entries and g.n_dropped == w.n_dropped
    assert got[1].status == 0 and got[2].status == luda.ERR_CORRUPTION


def test_subcompaction_bad_bounds_and_plans_reject_ranges():
    job = W.config1(seed=2, scale=1 / 128)
    ins = [dev(x) for x in oracle_inputs(job)]
    assert luda.subcompact_device(ins, [b"b", b"a"]).status == luda.ERR_INVALID_ARG
    assert luda.subcompact_device(ins, [b"a", b"a"]).status == luda.ERR_INVALID_ARG
    with pytest.raises(RuntimeError):
        luda.Plan([(ins, job.smallest_snapshot, job.bottommost, b"a", None)], luda.job_options(job))
