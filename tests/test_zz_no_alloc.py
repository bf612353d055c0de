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


def test_noalloc_check_does_not_check_key_order():
    """The documented difference: two keys swapped inside a data block, its checksum
    recomputed, pass the allocation-free check (structure and checksums hold) while a
    compaction, which checks the order after decoding the keys, and the oracle reject it."""
    import oracle
    import sstpy
    from helpers import oracle_compact
    from paper_2004_03054_b300 import luda
    from paper_2004_03054_b300 import workloads as W

    job = W.config1(seed=23, scale=1 / 16)
    job.restart_interval = 1  # every key stored whole: equal-size entries can trade places
    run = job.inputs[0]
    table = bytearray(oracle.build_tables(run, job.block_size, 1, job.bloom_bits_per_key, (1 << 64) - 1).tables[0].data)
    st, rt, _ = oracle.read_table(bytes(table))
    assert st == 0
    off, size = rt.blk_off[0], rt.blk_size[0]
    contents = bytes(table[off: off + size])
    n_rest = struct.unpack("<I", contents[-4:])[0]
    end = size - 4 - 4 * n_rest
    spans, pos = [], 0
    while pos < end:
        shared, p = sstpy.varint(contents, pos, end)
        nonshared, p = sstpy.varint(contents, p, end)
        vlen, p = sstpy.varint(contents, p, end)
        assert shared == 0
        spans.append((pos, p + nonshared + vlen))
        pos = p + nonshared + vlen
    # two adjacent entries of equal size, not the block's last (the index key stays right)
    i = next(k for k in range(len(spans) - 2) if spans[k][1] - spans[k][0] == spans[k + 1][1] - spans[k + 1][0])
    (a0, a1), (b0, b1) = spans[i], spans[i + 1]
    swapped = contents[:a0] + contents[b0:b1] + contents[a0:a1] + contents[b1:]
    table[off: off + size] = swapped
    assert table[off + size] == 0  # raw block
    table[off + size + 1: off + size + 5] = struct.pack("<I", oracle.mask(oracle.crc32c(swapped + b"\x00")))
    bad = bytes(table)

    t = _dev(bad)
    for _ in range(2):
        got = luda.check_table_noalloc(t)
        torch.cuda.synchronize()
        assert got.status == 0, luda.last_error_detail()
        assert got.n_entries == len(run.seqs)
    ref = luda.compact_device([t], job.smallest_snapshot, opts=luda.job_options(job))
    assert ref.status == luda.ERR_CORRUPTION and not ref.tables
    assert oracle_compact(job, [bad]).status == oracle.ERR_CORRUPTION


def test_noalloc_rejects_memory_it_cannot_read():
    """A host pointer is refused on the host, before any launch (cudaPointerGetAttributes),
    and the Python wrapper refuses CPU tensors; a device table checks fine afterwards."""
    import ctypes as C

    import oracle
    from paper_2004_03054_b300 import luda
    from paper_2004_03054_b300 import workloads as W

    job = W.config1(seed=24, scale=1 / 64)
    table = oracle.build_tables(job.inputs[0], job.block_size, job.restart_interval, job.bloom_bits_per_key,
                                (1 << 64) - 1).tables[0].data
    host = np.frombuffer(table, dtype=np.uint8).copy()
    pinned = torch.frombuffer(bytearray(table), dtype=torch.uint8).pin_memory()
    for ptr in (host.ctypes.data, pinned.data_ptr()):
        out = luda.TableCheck()
        rc = luda.lib().luda_check_table_noalloc(C.c_void_p(ptr), len(table), luda.current_stream(), C.byref(out))
        assert rc == out.status == luda.ERR_INVALID_ARG
        assert "memory" in luda.last_error_detail() or "pointer" in luda.last_error_detail()
    with pytest.raises(TypeError):
        luda.check_table_noalloc(torch.frombuffer(bytearray(table), dtype=torch.uint8))
    got = luda.check_table_noalloc(_dev(table))
    assert got.status == 0 and got.n_entries == len(job.inputs[0].seqs)
