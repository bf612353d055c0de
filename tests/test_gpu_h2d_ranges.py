"""luda_compact with its transfers overlapped by key ranges (§III-D; luda_tuning.h2d_ranges):
the inputs' data blocks are copied range after range, each range is compacted as soon as
its blocks are on the device and its finished tables go back while later ranges arrive.
The tables, their keys and the entry counts equal the oracle's compaction of the whole job
in one piece, for any number of ranges, from pageable and from pinned host memory, with
every format variant, with user keys whose versions span tables, and on corrupt inputs."""
import ctypes as C

import numpy as np
import pytest

from helpers import oracle_compact, oracle_inputs
from paper_2004_03054_b300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2004_03054_b300 import luda  # noqa: E402
from test_gpu_parity import assert_same  # noqa: E402


def _opts(job, ranges, flags=0):
    return luda.job_options(job, flags=flags, tuning={"h2d_ranges": ranges})


def _pinned_compact(ins, snap, opts):
    """luda_compact from pinned host buffers (copies truly asynchronous)."""
    bufs = []
    arr = (luda.Input * len(ins))()
    for i, b in enumerate(ins):
        t = torch.empty(len(b), dtype=torch.uint8).pin_memory()
        t.numpy()[:] = np.frombuffer(b, dtype=np.uint8)
        bufs.append(t)
        arr[i].data, arr[i].size = t.data_ptr(), len(b)
    out = luda.Outputs()
    rc = luda.lib().luda_compact(arr, len(ins), 1, snap, C.byref(opts), C.byref(out))
    return luda._take(rc, out, device=False)


@pytest.mark.parametrize("cfg,scale,ranges", [("config1", 1.0, 2), ("config1", 1.0, 7), ("config2", 1 / 2, 3),
                                              ("config2", 1 / 2, 16), ("config3", 1 / 16, 5),
                                              ("config3", 1 / 16, 64)])
def test_ranges_give_the_oracle_tables(cfg, scale, ranges):
    job = getattr(W, cfg)(seed=31, scale=scale)
    job.target_file_size = min(job.target_file_size, 256 * 1024)  # several tables per range
    ins = oracle_inputs(job)
    want = oracle_compact(job, ins)
    assert want.status == 0 and len(want.tables) > 2
    got = luda.compact(ins, job.smallest_snapshot, opts=_opts(job, ranges))
    assert_same(got, want)
    assert got.ms_h2d > 0 and got.ms_d2h > 0
    pinned = _pinned_compact(ins, job.smallest_snapshot, _opts(job, ranges))
    assert_same(pinned, want)


@pytest.mark.parametrize("flags", [luda.F_SHORT_INDEX | luda.F_FILTER_ARRAY, luda.F_COMPRESS])
def test_ranges_with_format_variants(flags):
    job = W.config2(seed=32, scale=1 / 4)
    job.target_file_size = 128 * 1024
    ins = oracle_inputs(job)
    want = oracle_compact(job, ins, flags)
    assert want.status == 0
    got = _pinned_compact(ins, job.smallest_snapshot, _opts(job, 6, flags))
    assert_same(got, want)


def test_ranges_with_versions_spanning_tables():
    """Many versions per user key and tiny tables: table boundaries fall inside a user key's
    versions, so the held-back part of a range reaches back past such boundaries."""
    rng = np.random.default_rng(33)
    for trial in range(12):
        job = W.tiny_job(rng, n_keys=int(rng.integers(40, 400)), max_versions=12, n_inputs=int(rng.integers(2, 6)),
                         key_len=(1, 6), val_len=(0, 60))
        job.block_size = int(rng.choice([64, 256, 1024]))
        job.target_file_size = int(rng.choice([1, 200, 700, 3000]))
        ins = oracle_inputs(job)
        want = oracle_compact(job, ins)
        for ranges in (2, 5, 33):
            got = _pinned_compact(ins, job.smallest_snapshot, _opts(job, ranges))
            assert_same(got, want)


def test_one_range_and_the_default_equal_the_ranges():
    job = W.config1(seed=34, scale=1 / 2)
    job.target_file_size = 200 * 1024
    ins = oracle_inputs(job)
    want = oracle_compact(job, ins)
    for ranges in (1, 0, 4):
        assert_same(luda.compact(ins, job.smallest_snapshot, opts=_opts(job, ranges)), want)


def test_corrupt_inputs_fail_with_no_tables():
    job = W.config2(seed=35, scale=1 / 4)
    job.target_file_size = 128 * 1024
    ins = oracle_inputs(job)
    # a data block near the end of the largest input (a late range) and a broken footer
    big = max(range(len(ins)), key=lambda i: len(ins[i]))
    cases = []
    late = bytearray(ins[big])
    late[int(len(late) * 0.6)] ^= 0x10
    cases.append([bytes(late) if i == big else b for i, b in enumerate(ins)])
    foot = bytearray(ins[0])
    foot[-1] ^= 0xFF
    cases.append([bytes(foot)] + ins[1:])
    for bad in cases:
        want = oracle_compact(job, bad)
        assert want.status != 0
        got = _pinned_compact(bad, job.smallest_snapshot, _opts(job, 5))
        assert got.status == want.status and got.tables == []
    # the library is usable afterwards
    assert_same(_pinned_compact(ins, job.smallest_snapshot, _opts(job, 5)), oracle_compact(job, ins))


def test_range_count_is_checked():
    job = W.config1(seed=36, scale=1 / 16)
    ins = oracle_inputs(job)
    got = luda.compact(ins, job.smallest_snapshot, opts=_opts(job, 65))
    assert got.status == luda.ERR_INVALID_ARG


def _varint(n):
    out = bytearray()
    while n >= 0x80:
        out.append((n & 0x7F) | 0x80)
        n >>= 7
    out.append(n)
    return bytes(out)


def test_index_out_of_order_runs_in_one_piece():
    """Two index entries traded (index checksum recomputed): the plan finds the blocks out of
    file order and the call runs in one piece, which rejects the table as the oracle does."""
    import struct

    import sstpy
    job = W.config2(seed=37, scale=1 / 4)
    job.target_file_size = 128 * 1024
    ins = oracle_inputs(job)
    big = max(range(len(ins)), key=lambda i: len(ins[i]))
    t = bytearray(ins[big])
    rd = sstpy.read(bytes(t))
    ioff, isize = rd["handles"]["index"]
    ents = [(k, v) for k, v, _ in sstpy.entries(bytes(t[ioff: ioff + isize]))]
    assert len(ents) > 4
    ents[1], ents[2] = ents[2], ents[1]
    body, starts = bytearray(), []
    for k, v in ents:
        starts.append(len(body))
        body += _varint(0) + _varint(len(k)) + _varint(len(v)) + k + v
    body += b"".join(struct.pack("<I", s) for s in starts) + struct.pack("<I", len(starts))
    assert len(body) == isize
    t[ioff: ioff + isize] = body
    t[ioff + isize + 1: ioff + isize + 5] = struct.pack("<I", oracle.mask(oracle.crc32c(bytes(body) + b"\x00")))
    bad = [bytes(t) if i == big else b for i, b in enumerate(ins)]
    want = oracle_compact(job, bad)
    assert want.status == oracle.ERR_CORRUPTION
    got = _pinned_compact(bad, job.smallest_snapshot, _opts(job, 4))
    assert got.status == luda.ERR_CORRUPTION and got.tables == []


def test_ranges_with_a_callers_allocator_and_failing_allocations():
    """Through the caller's allocator hook: the key-range call gives back every byte it took,
    and whichever allocation fails, the call either returns LUDA_ERR_OOM with no tables or
    (a failure while planning the ranges) runs in one piece with the oracle's tables."""
    from test_gpu_faults import Hook
    job = W.config2(seed=38, scale=1 / 4)
    job.target_file_size = 128 * 1024
    ins = oracle_inputs(job)
    want = [t.data for t in oracle_compact(job, ins).tables]
    L = luda.lib()
    bufs = []
    arr = (luda.Input * len(ins))()
    for i, b in enumerate(ins):
        t = torch.empty(len(b), dtype=torch.uint8).pin_memory()
        t.numpy()[:] = np.frombuffer(b, dtype=np.uint8)
        bufs.append(t)
        arr[i].data, arr[i].size = t.data_ptr(), len(b)

    def run(hook):
        o = hook.options(job)
        o.tuning = C.pointer(luda.Tuning.of({"h2d_ranges": 4}))
        out = luda.Outputs()
        rc = L.luda_compact(arr, len(ins), job.level, job.smallest_snapshot, C.byref(o), C.byref(out))
        torch.cuda.synchronize()
        got = [C.string_at(out.tables[i].data, out.tables[i].size) for i in range(out.n_tables)]
        L.luda_outputs_free(C.byref(out))
        torch.cuda.synchronize()
        return rc, got

    ok = Hook()
    rc, got = run(ok)
    assert rc == 0 and got == want
    assert not ok.live
    n_calls = ok.calls
    assert n_calls > 8
    for k in range(0, n_calls, max(1, n_calls // 24)):
        bad = Hook(fail_at=k)
        rc, got = run(bad)
        assert (rc == luda.ERR_OOM and got == []) or (rc == 0 and got == want), (k, rc)
        assert not bad.live, (k, bad.live)
