"""Format variant of R10 (LUDA_F_FILTER_ARRAY): LevelDB's filter array, one bloom filter per
2 KiB of data block offsets. The oracle's filter blocks are checked byte for byte against
the independent reader's own construction (its own MurmurHash3, pinned to the published
vectors, and its own bit-at-a-time bloom), against a layout worked out by hand, and by the
query rule (no false negatives)."""
import ast
import os
import struct

import numpy as np
import pytest

import oracle
import sstpy
from helpers import U64MAX, oracle_compact, oracle_inputs
from paper_2004_03054_b300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _vectors():
    out = []
    with open(os.path.join(GOLDEN, "murmur3_vectors.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                msg, seed, want = line.rsplit(None, 2)
                out.append((ast.literal_eval(msg), int(seed, 16), int(want, 16)))
    return out


@pytest.mark.parametrize("msg,seed,want", _vectors())
def test_python_murmur3_published(msg, seed, want):
    assert sstpy.murmur3_32(msg, seed) == want


def _run(n, vlen, seed=3, key_len=16):
    rng = np.random.default_rng(seed)
    users = sorted({rng.bytes(key_len) for _ in range(n)})
    n = len(users)
    return W._make_run(users, np.arange(1, n + 1, dtype=np.uint64), np.ones(n, np.uint8),
                       np.full(n, vlen), rng, 0)


def _filters(contents):
    """(filters, base_lg) of a filter array's contents."""
    lg = contents[-1]
    (arr,) = struct.unpack_from("<I", contents, len(contents) - 5)
    num = (len(contents) - 5 - arr) // 4
    offs = list(struct.unpack_from(f"<{num}I", contents, arr)) + [arr]
    return [contents[offs[i]:offs[i + 1]] for i in range(num)], lg


def test_hand_worked_layout():
    # Three entries, 16-byte keys, 5000-byte values, one entry per block (T = 1): an entry is
    # 1 + 1 + 2 varint bytes + 24 key bytes + 5000 value bytes = 5028; a block adds one
    # restart (4) and the restart count (4), and its trailer 5: 5041 bytes. Blocks start at
    # 0, 5041, 10082 (filter indexes 0, 2, 4); the data ends at 15123, so there are
    # max(15123 >> 11, 4 + 1) = 7 filters, of which 1, 3, 5, 6 are empty.
    res = oracle.build_tables(_run(3, 5000), 1, 16, 10, U64MAX, flags=oracle.F_FILTER_ARRAY)
    assert res.status == 0, res.detail
    (t,) = res.tables
    r = sstpy.read(t.data)
    assert r["filter_name"] == "filter.luda.bloom2k"
    assert [b[0] for b in r["blocks"]] == [0, 5041, 10082]
    assert r["handles"]["filter"][0] == 15123
    fs, lg = _filters(r["filter"])
    assert lg == 11 and len(fs) == 7
    assert [len(f) > 0 for f in fs] == [True, False, True, False, True, False, False]
    # one key each: max(64, 10) bits = 8 bytes, then k = 6
    for i, (off, _, ents) in zip((0, 2, 4), r["blocks"]):
        assert fs[i] == sstpy.bloom([ents[0][0][:-8]], 10) and len(fs[i]) == 9 and fs[i][-1] == 6


@pytest.mark.parametrize("n,vlen,T,R,bpk,target", [
    (400, 100, 4096, 16, 10, U64MAX),    # blocks of 4 KiB: every other filter empty
    (400, 100, 256, 4, 10, U64MAX),      # several blocks per filter
    (300, 3000, 1, 16, 7, U64MAX),       # one big entry per block, runs of empty filters
    (2000, 60, 1024, 16, 10, 32 << 10),  # many tables, the last block's window shared
    (1, 10, 4096, 16, 10, U64MAX),       # a single entry
    (500, 0, 512, 1, 20, U64MAX),        # empty values, restart interval 1
])
def test_filter_array_bytes(n, vlen, T, R, bpk, target):
    run = _run(n, vlen, seed=n + vlen)
    arr = oracle.build_tables(run, T, R, bpk, target, flags=oracle.F_FILTER_ARRAY)
    plain = oracle.build_tables(run, T, R, bpk, target)
    assert arr.status == plain.status == 0
    assert len(arr.tables) == len(plain.tables)
    for ta, tp in zip(arr.tables, plain.tables):
        ra, rp = sstpy.read(ta.data), sstpy.read(tp.data)
        end = ra["handles"]["filter"][0]
        # the data blocks and their cut do not depend on the filter layout
        assert end == rp["handles"]["filter"][0] and ta.data[:end] == tp.data[:end]
        assert ra["entries"] == rp["entries"]
        assert rp["filter"] == sstpy.bloom([e[0][:-8] for e in rp["entries"]], bpk)
        assert ra["filter"] == sstpy.filter_array(ra["blocks"], end, bpk)
        ok, rt, _ = oracle.read_table(ta.data)
        assert ok == 0 and rt.filter_array and rt.filter == ra["filter"]


def test_query_rule():
    run = _run(3000, 40, seed=9)
    res = oracle.build_tables(run, 4096, 16, 10, U64MAX, flags=oracle.F_FILTER_ARRAY)
    (t,) = res.tables
    r = sstpy.read(t.data)
    keys = set()
    for off, _, ents in r["blocks"]:
        for e in ents:
            assert oracle.filter_array_may_contain(r["filter"], off, e[0][:-8])
            keys.add(e[0][:-8])
    # absent keys: the false-positive rate of 10 bits per key and 6 probes (about 0.84%)
    rng = np.random.default_rng(99)
    probes = [rng.bytes(16) for _ in range(4000)]
    hits = sum(oracle.filter_array_may_contain(r["filter"], r["blocks"][i % len(r["blocks"])][0], u)
               for i, u in enumerate(probes) if u not in keys)
    assert hits < 0.03 * len(probes)
    # an offset whose filter is empty holds nothing; one past the array answers "may contain"
    fs, _ = _filters(r["filter"])
    empty = [i for i, f in enumerate(fs) if not f]
    assert empty
    assert not oracle.filter_array_may_contain(r["filter"], empty[0] << 11, next(iter(keys)))
    assert oracle.filter_array_may_contain(r["filter"], len(fs) << 11, b"anything")


@pytest.mark.parametrize("cfg", [1, 2])
def test_compaction_with_filter_array(cfg):
    job = W.config1(seed=4, scale=0.25) if cfg == 1 else W.config2(seed=4, scale=0.25)
    ins = oracle_inputs(job)
    plain = oracle_compact(job, ins)
    arr = oracle_compact(job, ins, flags=oracle.F_FILTER_ARRAY)
    assert plain.status == arr.status == 0
    assert len(plain.tables) == len(arr.tables)
    for ta, tp in zip(arr.tables, plain.tables):
        ra, rp = sstpy.read(ta.data), sstpy.read(tp.data)
        assert ra["entries"] == rp["entries"]
        assert ra["filter"] == sstpy.filter_array(ra["blocks"], ra["handles"]["filter"][0], job.bloom_bits_per_key)
    # tables with filter arrays are valid compaction inputs: the compaction reads no filter
    again = oracle.compact([t.data for t in arr.tables], bottommost=False, block_size=job.block_size,
                           restart_interval=job.restart_interval, bloom_bits_per_key=job.bloom_bits_per_key,
                           target_file_size=job.target_file_size)
    assert again.status == 0
    assert [e for t in again.tables for e in sstpy.read(t.data)["entries"]] == \
        [e for t in plain.tables for e in sstpy.read(t.data)["entries"]]
