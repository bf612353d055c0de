"""Format variant R9s (LUDA_F_SHORT_INDEX): shortened index keys. Pins of the rule on
hand-worked keys, read back by the independent reader; tables written with it decode to
the same entries, and compactions whose inputs and outputs use it keep their entries."""
import struct

import numpy as np
import pytest

import oracle
import sstpy
from helpers import U64MAX, decoded, oracle_compact, oracle_inputs
from paper_2004_03054_b300 import workloads as W

MAXT = oracle.MAX_SEQ << 8 | 1


def _run(users, seqs=None):
    n = len(users)
    rng = np.random.default_rng(1)
    seqs = np.array(seqs if seqs is not None else range(1, n + 1), np.uint64)
    return W._make_run(users, seqs, np.ones(n, np.uint8), np.full(n, 3), rng, 0)


def _index(users, target=U64MAX):
    """Index keys of the tables built with one entry per block (T = 1) and R9s."""
    res = oracle.build_tables(_run(users), 1, 1, 10, target, flags=oracle.F_SHORT_INDEX)
    assert res.status == 0, res.detail
    out = []
    for t in res.tables:
        r = sstpy.read(t.data)
        out.append([(k[:-8], struct.unpack("<Q", k[-8:])[0]) for k in r["index_keys"]])
        assert [e[0][:-8] for e in r["entries"]] == [u for u in users if u in {e[0][:-8] for e in r["entries"]}]
    return out


def test_separator_and_successor_pins():
    users = [b"abcxx", b"abfzz", b"abg", b"abgq", b"b\xff\xff\x01", b"d"]
    (idx,) = _index(users)
    # (user key part, trailer) of each block's index key, worked out by hand:
    want = [(b"abd", MAXT),                # abcxx | abfzz: first difference at 2, c + 1 = d < f
            (b"abfzz", 2 << 8 | 1),        # abfzz | abg: f + 1 = g is not below g: kept
            (b"abg", 3 << 8 | 1),          # abg is a prefix of abgq: kept
            (b"abgq", 4 << 8 | 1),         # abgq | b...: a + 1 = b is not below b: kept
            (b"c", MAXT),                  # b\xff\xff\x01 | d: b + 1 = c < d
            (b"d", 6 << 8 | 1)]            # last key of the table: d + 1 would not be shorter
    assert idx == want


@pytest.mark.parametrize("last,want", [(b"\xff\xffab", (b"\xff\xffb", MAXT)),
                                       (b"\xff\xff", (b"\xff\xff", 1 << 8 | 1)),
                                       (b"q", (b"q", 1 << 8 | 1)),
                                       (b"qrs", (b"r", MAXT))])
def test_successor_of_a_tables_last_key(last, want):
    (idx,) = _index([last])
    assert idx == [want]


def test_same_user_key_across_blocks_is_not_shortened():
    # versions of one user key in consecutive blocks: the separator cannot leave the key
    res = oracle.build_tables(_run([b"kkkk", b"kkkk", b"zz"], [9, 8, 1]), 1, 1, 10, U64MAX,
                              flags=oracle.F_SHORT_INDEX)
    r = sstpy.read(res.tables[0].data)
    assert r["index_keys"][0] == b"kkkk" + struct.pack("<Q", 9 << 8 | 1)


@pytest.mark.parametrize("seed", range(6))
def test_short_index_tables_decode_and_compact_alike(seed):
    rng = np.random.default_rng(300 + seed)
    job = W.tiny_job(rng, n_keys=int(rng.integers(20, 400)), max_versions=4, n_inputs=int(rng.integers(1, 5)),
                     key_len=(0, 24), val_len=(0, 200))
    job.block_size, job.target_file_size = int(rng.choice([64, 256, 1024])), int(rng.choice([2000, 20000]))
    plain = oracle_inputs(job)
    short = []
    for r in job.inputs:
        res = oracle.build_tables(r, job.block_size, job.restart_interval, job.bloom_bits_per_key, U64MAX,
                                  flags=oracle.F_SHORT_INDEX)
        assert res.status == 0
        short.append(res.tables[0].data)
    for a, b in zip(plain, short):
        assert sstpy.read(a)["entries"] == sstpy.read(b)["entries"]
        assert len(b) <= len(a)                 # shorter (or equal) index keys
        st, rt, _ = oracle.read_table(b)
        assert st == 0 and rt.index_keys_ok
    want = oracle_compact(job, plain)
    got = oracle_compact(job, short, flags=oracle.F_SHORT_INDEX)
    assert got.status == want.status == 0
    assert decoded([t.data for t in got.tables]) == decoded([t.data for t in want.tables])
    for t in got.tables:
        sstpy.read(t.data)                      # R9's interval holds in every output table
        st, rt, _ = oracle.read_table(t.data)
        assert st == 0 and rt.index_keys_ok
