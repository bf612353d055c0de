"""Structural invariants of the oracle's tables, measured from the bytes, and its
error behaviour on corrupted inputs."""
import math
import struct

import numpy as np
import pytest

import oracle
import sstpy
from helpers import oracle_compact, oracle_inputs
from paper_2004_03054_b300 import workloads as W


def _block_cut_facts(contents):
    """(size, size before the last entry was added) of a finished block, from its bytes."""
    (nr,) = struct.unpack_from("<I", contents, len(contents) - 4)
    rstart = len(contents) - 4 - 4 * nr
    restarts = list(struct.unpack_from(f"<{nr}I", contents, rstart))
    pos, last_start = 0, 0
    while pos < rstart:
        last_start = pos
        _, pos = sstpy.varint(contents, pos, rstart)
        nsh, pos = sstpy.varint(contents, pos, rstart)
        vl, pos = sstpy.varint(contents, pos, rstart)
        pos += nsh + vl
    nr_before = nr - 1 if last_start == restarts[-1] else nr
    return len(contents), last_start + 4 * nr_before + 4


def check_cuts(tables, T, target):
    """Greedy cut rules, from the bytes: every block but the job's very last reached T,
    none would have reached it one entry earlier; every file but the last reached the
    target, none reached it one block earlier."""
    for ti, t in enumerate(tables):
        data = t.data
        st, rt, det = oracle.read_table(data)
        assert st == 0, det
        assert rt.layout_ok and rt.index_keys_ok
        flushed = 0
        for b in range(rt.n_blocks):
            contents = data[rt.blk_off[b]: rt.blk_off[b] + rt.blk_size[b]]
            size, before = _block_cut_facts(contents)
            final = ti == len(tables) - 1 and b == rt.n_blocks - 1
            if not final:
                assert size >= T, (ti, b)
            n_in_block = rt.blk_last[b] - (rt.blk_last[b - 1] if b else -1)
            if n_in_block > 1:
                assert before < T, (ti, b)
            flushed += size + 5
            if b < rt.n_blocks - 1:
                assert flushed < target, (ti, b)
        if ti < len(tables) - 1:
            assert flushed >= target, ti


@pytest.mark.parametrize("T,R,target", [(1, 1, 1), (1, 16, 300), (64, 2, 1000), (200, 3, 5000),
                                        (4096, 16, 1 << 20), (777, 5, 20000)])
def test_block_and_file_cuts(T, R, target):
    job = W.config1(seed=5, scale=1 / 128)
    job.block_size, job.restart_interval, job.target_file_size = T, R, target
    res = oracle_compact(job)
    assert res.status == 0
    check_cuts(res.tables, T, target)


def test_config_tables_invariants():
    for cfg, scale in [(1, 1 / 32), (3, 1 / 512)]:
        job = W.make(cfg, scale=scale)
        res = oracle_compact(job)
        check_cuts(res.tables, job.block_size, job.target_file_size)
        prev = None
        for t in res.tables:
            st, rt, _ = oracle.read_table(t.data)
            assert rt.keys[0] == t.smallest and rt.keys[-1] == t.largest
            assert len(rt.keys) == t.n_entries
            if prev is not None:
                assert prev < t.smallest[:-8] or prev == t.smallest[:-8]


def test_bloom_no_false_negatives_and_fp_rate():
    job = W.config1(seed=21, scale=1 / 4)
    job.target_file_size = 1 << 40
    res = oracle_compact(job)
    assert len(res.tables) == 1
    t = res.tables[0]
    st, rt, _ = oracle.read_table(t.data)
    f = rt.filter
    assert f[-1] == 6                                   # k = floor(10 * 0.69)
    n = t.n_entries
    m = (len(f) - 1) * 8
    assert m == max(64, ((n * 10 + 7) // 8) * 8)
    for k in rt.keys:
        assert oracle.bloom_may_contain(f, k[:-8])
    rng = np.random.default_rng(3)
    probes = 200_000
    present = set(k[:-8] for k in rt.keys)
    fp = 0
    for _ in range(probes):
        q = rng.bytes(16)
        if q not in present and oracle.bloom_may_contain(f, q):
            fp += 1
    k = 6
    expect = (1 - math.exp(-k * n / m)) ** k
    assert abs(fp / probes - expect) < 0.3 * expect, (fp / probes, expect)


# ---- errors ----------------------------------------------------------------------------
def _job_and_inputs():
    job = W.config1(seed=31, scale=1 / 256)
    return job, oracle_inputs(job)


def _first_data_block(data):
    st, rt, _ = oracle.read_table(data)
    return rt.blk_off[0], rt.blk_size[0]


def test_crc_flip_is_corruption():
    job, ins = _job_and_inputs()
    off, size = _first_data_block(ins[1])
    bad = bytearray(ins[1])
    bad[off + size // 2] ^= 0x10
    res = oracle_compact(job, [ins[0], bytes(bad), ins[2]])
    assert res.status == oracle.ERR_CORRUPTION and res.tables == []


@pytest.mark.parametrize("typ,status", [(1, oracle.ERR_CORRUPTION), (2, oracle.ERR_NOT_SUPPORTED),
                                        (0xFF, oracle.ERR_NOT_SUPPORTED)])
def test_block_types(typ, status):
    """Type 1 (R4c, Snappy in LevelDB) is read as a compressed stream: raw contents under
    that type do not decode to their announced length. Other types are not supported."""
    job, ins = _job_and_inputs()
    off, size = _first_data_block(ins[0])
    bad = bytearray(ins[0])
    bad[off + size] = typ
    crc = oracle.mask(oracle.crc32c(bytes(bad[off: off + size + 1])))
    bad[off + size + 1: off + size + 5] = struct.pack("<I", crc)
    res = oracle_compact(job, [bytes(bad)] + ins[1:])
    assert res.status == status


@pytest.mark.parametrize("cut", [1, 8, 47, 48])
def test_truncated_or_bad_footer(cut):
    job, ins = _job_and_inputs()
    res = oracle_compact(job, [ins[0][:-cut]] + ins[1:])
    assert res.status == oracle.ERR_CORRUPTION
    res = oracle_compact(job, [b"x" * 10] + ins[1:])
    assert res.status == oracle.ERR_CORRUPTION


def test_out_of_order_input_is_corruption():
    rng = np.random.default_rng(8)
    run = W._make_run([b"b", b"a"], np.array([1, 2], np.uint64), np.array([1, 1], np.uint8),
                      np.array([1, 1]), rng, 0)
    assert oracle.build_tables(run).status == oracle.ERR_INVALID_ARG   # the builder refuses
    last = b"a" + struct.pack("<Q", 2 << 8 | 1)
    contents = oracle.encode_block([(b"b" + struct.pack("<Q", 1 << 8 | 1), b"x"), (last, b"y")], 16)
    res = oracle.compact([_single_block_table(contents, last)])
    assert res.status == oracle.ERR_CORRUPTION and "out of order" in res.detail


def _table(blocks):
    """A minimal table around data blocks [(contents, index_key)] (filter empty-ish, valid
    CRCs); index_key is the block's index entry key."""
    def blk(c):
        return c + b"\x00" + struct.pack("<I", oracle.mask(oracle.crc32c(c + b"\x00")))
    data, handles = b"", []
    for contents, _ in blocks:
        handles.append(oracle.put_varint(len(data)) + oracle.put_varint(len(contents)))
        data += blk(contents)
    filt_c = bytes(8) + b"\x06"
    filt_off = len(data)
    data += blk(filt_c)
    meta_c = oracle.encode_block([(b"filter.luda.bloom", oracle.put_varint(filt_off) + oracle.put_varint(len(filt_c)))], 1)
    meta_off = len(data)
    data += blk(meta_c)
    idx_c = oracle.encode_block([(k, h) for (_, k), h in zip(blocks, handles)], 1)
    idx_off = len(data)
    data += blk(idx_c)
    ft = (oracle.put_varint(meta_off) + oracle.put_varint(len(meta_c)) + oracle.put_varint(idx_off)
          + oracle.put_varint(len(idx_c)))
    ft = ft + bytes(40 - len(ft)) + struct.pack("<Q", 0x4C55444153535431)
    return data + ft


def _single_block_table(contents, index_key):
    """A minimal table around one data block's contents; index_key is its index entry key."""
    return _table([(contents, index_key)])


def _ik(user, seq=1, typ=1):
    return user + struct.pack("<Q", seq << 8 | typ)


def test_hand_made_table_is_valid():
    last = b"b" + struct.pack("<Q", 1 << 8 | 1)
    contents = oracle.encode_block([(b"a" + struct.pack("<Q", 2 << 8 | 1), b"y"), (last, b"x")], 16)
    img = _single_block_table(contents, last)
    res = oracle.compact([img])
    assert res.status == 0 and len(res.tables) == 1
    assert res.tables[0].n_entries == 2


@pytest.mark.parametrize("index_key", [_ik(b"b", 2), b"a" * 9, b"b" * 9, b"a", b""])
def test_index_key_below_last_key_is_corrupt(index_key):
    """R9: an index key below its block's last internal key (or not an internal key at all)
    makes the table corrupt, checksums intact."""
    contents = oracle.encode_block([(_ik(b"a", 2), b"y"), (_ik(b"b", 1), b"x")], 16)
    res = oracle.compact([_single_block_table(contents, index_key)])
    assert res.status == oracle.ERR_CORRUPTION and "index key" in res.detail


@pytest.mark.parametrize("index_key", [_ik(b"b", 1), b"z" * 9, _ik(b"c", oracle.MAX_SEQ), _ik(b"b\x00", 9)])
def test_index_key_at_or_above_last_key_is_valid(index_key):
    """R9: any index key at or above the block's last key is valid for the table's last
    block (shortened index keys are such keys)."""
    contents = oracle.encode_block([(_ik(b"a", 2), b"y"), (_ik(b"b", 1), b"x")], 16)
    res = oracle.compact([_single_block_table(contents, index_key)])
    assert res.status == 0 and res.n_in_entries == 2
    st, rt, _ = oracle.read_table(_single_block_table(contents, index_key))
    assert st == 0 and rt.index_keys_ok and rt.index_keys_exact == (index_key == _ik(b"b", 1))


@pytest.mark.parametrize("key0,ok", [(_ik(b"b", 1), True), (_ik(b"c", oracle.MAX_SEQ), True),
                                     (_ik(b"d", oracle.MAX_SEQ), True), (_ik(b"d", 1), False),
                                     (_ik(b"d", 0), False), (_ik(b"e", 5), False)])
def test_index_key_must_stay_below_next_blocks_first_key(key0, ok):
    """R9: the index key of a block that another block follows must lie below that block's
    first internal key (d@1 here; d@MAX sorts before it, d@1 and d@0 do not)."""
    b0 = oracle.encode_block([(_ik(b"a", 2), b"y"), (_ik(b"b", 1), b"x")], 16)
    b1 = oracle.encode_block([(_ik(b"d", 1), b"u"), (_ik(b"e", 1), b"v")], 16)
    img = _table([(b0, key0), (b1, _ik(b"e", 1))])
    res = oracle.compact([img])
    if ok:
        assert res.status == 0 and res.n_in_entries == 4
    else:
        assert res.status == oracle.ERR_CORRUPTION and "index key" in res.detail
    st, rt, _ = oracle.read_table(img)
    assert st == 0 and rt.index_keys_ok == ok


def test_duplicate_internal_key_across_inputs():
    rng = np.random.default_rng(8)
    run = W._make_run([b"k"], np.array([5], np.uint64), np.array([1], np.uint8), np.array([3]), rng, 0)
    t = oracle.build_tables(run).tables[0].data
    res = oracle.compact([t, t])
    assert res.status == 0 and res.n_dropped == 1         # the later input's copy is dropped
    res = oracle.compact([t, t], flags=oracle.F_STRICT_DUP)
    assert res.status == oracle.ERR_DUPLICATE_KEY


def test_bad_options():
    assert oracle.compact([], block_size=0).status == oracle.ERR_INVALID_ARG
    assert oracle.compact([], restart_interval=0).status == oracle.ERR_INVALID_ARG
    assert oracle.compact([], bloom_bits_per_key=0).status == oracle.ERR_INVALID_ARG
    assert oracle.compact([], target_file_size=0).status == oracle.ERR_INVALID_ARG
