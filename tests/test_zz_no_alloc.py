"""luda_check_table_noalloc: the table check for callers that cannot allocate device
memory (inside an allocator callback, engines with all device memory reserved up front,
paths that cannot take an allocation's implicit synchronisation). It must agree with the
compaction entry point on the same tables, call after call (its scratch is a static
device array reused by every call). This file is collected last on purpose, so a run
that stops at the first failure has run every other test first.
"""
import struct

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _dev(b: bytes):
    return torch.frombuffer(bytearray(b), dtype=torch.uint8).cuda()


def test_noalloc_check_matches_compaction_two_calls_in_a_row():
    import oracle
    from helpers import oracle_inputs
    from paper_2004_03054_b300 import luda
    from paper_2004_03054_b300 import workloads as W

    job = W.config1(seed=21, scale=1 / 16)
    inputs = oracle_inputs(job)
    # corrupt variants: a flipped data byte, and a compressed block with a valid CRC
    st, rt, _ = oracle.read_table(inputs[1])
    flip = bytearray(inputs[1])
    flip[rt.blk_off[2] + 11] ^= 0x40
    comp = bytearray(inputs[1])
    off, size = rt.blk_off[0], rt.blk_size[0]
    comp[off + size] = 1
    comp[off + size + 1: off + size + 5] = struct.pack("<I", oracle.mask(oracle.crc32c(bytes(comp[off: off + size + 1]))))
    for x in inputs + [bytes(flip), bytes(comp)]:
        t = _dev(x)
        ref = luda.compact_device([t], job.smallest_snapshot, opts=luda.job_options(job))  # existing entry point
        for _ in range(2):
            got = luda.check_table_noalloc(t)
            torch.cuda.synchronize()
            if x is not inputs[-1] and x == bytes(comp):
                # a type-1 block: the compaction reads it as a compressed stream (raw contents
                # do not decode), the allocation-free check does not decompress
                assert (got.status, ref.status) == (luda.ERR_NOT_SUPPORTED, luda.ERR_CORRUPTION)
                continue
            assert got.status == ref.status, (got.status, ref.status)
            if ref.status == 0:
                assert got.n_entries == ref.n_in_entries
                st, rt, _ = oracle.read_table(x)
                assert got.n_blocks == rt.n_blocks
                assert got.data_bytes == sum(rt.blk_size) + 5 * rt.n_blocks


def test_noalloc_rejects_tables_beyond_its_limit():
    import oracle
    from paper_2004_03054_b300 import luda
    from paper_2004_03054_b300 import workloads as W

    n = 16500  # one entry per block with a 1-byte block size: more blocks than the limit
    rng = np.random.default_rng(2)
    keys = [i.to_bytes(4, "big") for i in range(n)]
    run = W._make_run(keys, np.arange(1, n + 1, dtype=np.uint64), np.ones(n, np.uint8), np.zeros(n, np.int64), rng, 0)
    table = oracle.build_tables(run, 1, 1, 10, (1 << 64) - 1).tables[0].data
    t = _dev(table)
    for _ in range(2):
        got = luda.check_table_noalloc(t)
        assert got.status == luda.ERR_INVALID_ARG
        assert got.n_blocks == 0
        assert "16384" in luda.last_error_detail()
    # a table within the limit still checks fine afterwards
    small = oracle.build_tables(W._make_run(keys[:100], np.arange(1, 101, dtype=np.uint64), np.ones(100, np.uint8),
                                            np.zeros(100, np.int64), rng, 0), 1, 1, 10, (1 << 64) - 1).tables[0].data
    got = luda.check_table_noalloc(_dev(small))
    assert got.status == 0 and got.n_entries == 100 and got.n_blocks == 100
