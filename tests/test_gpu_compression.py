"""GPU parity for compressed input blocks (R4c): the device decompresses the Snappy-format
data blocks of its inputs and produces the oracle's tables byte for byte; malformed
streams under a valid checksum fail the job as they fail the oracle's."""
import numpy as np
import pytest

from helpers import U64MAX
from paper_2004_03054_b300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import sstpy  # noqa: E402
from paper_2004_03054_b300 import luda  # noqa: E402
from test_compression import _reseal, _run  # noqa: E402
from test_gpu_parity import assert_same, dev  # noqa: E402


def _inputs(n_in, n, vlen, T, seed, compress=(True,)):
    runs = [_run(n, vlen, seed=seed + i) for i in range(n_in)]
    for i, r in enumerate(runs):
        r.seqs[:] = r.seqs + np.uint64(100000 * (n_in - i))   # newer inputs first
    out = []
    for i, r in enumerate(runs):
        flags = oracle.F_COMPRESS if compress[i % len(compress)] else 0
        res = oracle.build_tables(r, T, 16, 10, U64MAX, flags=flags)
        assert res.status == 0 and len(res.tables) == 1
        out.append(res.tables[0].data)
    return out


def _both(ins, T=4096, target=64 << 10, flags=0, snapshot=oracle.MAX_SEQ, bottommost=False):
    want = oracle.compact(ins, snapshot, bottommost, T, 16, 10, target, flags)
    got = luda.compact_device([dev(x) for x in ins], snapshot,
                              opts=luda.options(T, 16, 10, target, bottommost, flags=flags))
    got.tables = [t.cpu().numpy().tobytes() for t in got.tables]
    assert_same(got, want)
    return got


@pytest.mark.parametrize("n_in,n,vlen,T", [(1, 300, 200, 4096), (3, 200, 100, 4096), (4, 150, 40, 256),
                                           (2, 60, 3000, 1), (3, 100, 1000, 16384), (5, 400, 0, 512)])
def test_compressed_inputs(n_in, n, vlen, T):
    ins = _inputs(n_in, n, vlen, T, seed=n + vlen + T)
    if vlen:
        assert any(t == 1 for x in ins for t in sstpy.read(x)["types"])
    _both(ins, T=T)


def test_mixed_compressed_and_raw_inputs():
    ins = _inputs(4, 250, 120, 2048, seed=5, compress=(True, False))
    _both(ins, T=2048, target=32 << 10)
    _both(ins, T=2048, target=32 << 10, flags=luda.F_SHORT_INDEX | luda.F_FILTER_ARRAY)


def test_config_job_with_compressed_inputs():
    job = W.config1(seed=6, scale=1 / 32)
    ins = [oracle.build_tables(r, job.block_size, job.restart_interval, job.bloom_bits_per_key, U64MAX,
                               flags=oracle.F_COMPRESS).tables[0].data for r in job.inputs]
    # random values do not compress: the blocks stay raw, the result is the plain one
    _both(ins, T=job.block_size, target=job.target_file_size, snapshot=job.smallest_snapshot,
          bottommost=job.bottommost)


def test_batched_ranged_and_server():
    ins = _inputs(3, 300, 150, 4096, seed=21)
    keys = sorted({e[0][:-8] for x in ins for e in sstpy.read(x)["entries"]})
    lo, hi = keys[len(keys) // 4], keys[3 * len(keys) // 4]
    opts = luda.options(4096, 16, 10, 64 << 10)
    want_full = oracle.compact(ins, oracle.MAX_SEQ, False, 4096, 16, 10, 64 << 10)
    want_rng = oracle.compact(ins, oracle.MAX_SEQ, False, 4096, 16, 10, 64 << 10, lo=lo, hi=hi)
    batch = [([dev(x) for x in ins], oracle.MAX_SEQ, False), ([dev(x) for x in ins], oracle.MAX_SEQ, False, lo, hi)]
    rc, got = luda.batch_compact_device(batch, opts)
    assert rc == 0
    for g, w in zip(got, [want_full, want_rng]):
        g.tables = [t.cpu().numpy().tobytes() for t in g.tables]
        assert_same(g, w)
    srv = luda.Server(2, 1 << 40, opts)
    t = srv.submit([dev(x) for x in ins], oracle.MAX_SEQ, False)
    res, _ = srv.wait(t, timeout_ms=60_000)
    srv.close()
    assert res.status == 0
    assert [x.cpu().numpy().tobytes() for x in res.tables] == [x.data for x in want_full.tables]


def test_malformed_streams():
    ins = _inputs(2, 80, 300, 4096, seed=31)
    r = sstpy.read(ins[0])
    blocks = [b for b, t in zip(r["blocks"], r["types"]) if t == 1]
    off, size, _ = blocks[0]
    cases = []
    for edit in ("length", "offset", "truncate"):
        bad = bytearray(ins[0])
        if edit == "length":
            bad[off] ^= 0x01                     # announced length off by one
        elif edit == "offset":
            # the first copy element's offset raised beyond the bytes written so far
            s = sstpy.snappy_uncompress(bytes(bad[off:off + size]))
            assert s
            p = off
            while bad[p] & 0x80:
                p += 1
            p += 1
            while True:
                tag = bad[p]
                kind = tag & 3
                if kind == 0:
                    n = tag >> 2
                    nb = n - 59 if n >= 60 else 0
                    n = int.from_bytes(bad[p + 1:p + 1 + nb], "little") if nb else n
                    p += 1 + nb + n + 1
                    continue
                if kind == 1:
                    bad[p] |= 0xE0                # offset high bits 7: beyond the output so far
                    bad[p + 1] = 0xFF
                else:
                    bad[p + 1] = 0xFF
                    bad[p + 2] = 0xFF
                break
        else:
            bad[off + size - 3:off + size] = b"\x00\x00\x00"  # last element's bytes changed
        _reseal(bad, off, size)
        cases.append(bytes(bad))
    for c in cases:
        want = oracle.compact([c, ins[1]], oracle.MAX_SEQ, False, 4096, 16, 10, 64 << 10)
        got = luda.compact_device([dev(c), dev(ins[1])], oracle.MAX_SEQ, opts=luda.options(4096, 16, 10, 64 << 10))
        assert want.status == got.status, (want.status, got.status, want.detail, got.detail)


def test_plan_reports_compressed_inputs_not_supported():
    """Plans are sized once for replays; a job with compressed blocks reports
    NOT_SUPPORTED from its replays (the per-call entry points decompress)."""
    ins = _inputs(2, 100, 200, 4096, seed=41)
    plan = luda.Plan([([dev(x) for x in ins], oracle.MAX_SEQ, False)], luda.options(4096, 16, 10, 64 << 10))
    plan.run()
    torch.cuda.synchronize()
    (out,) = plan.outputs()
    assert out.status == luda.ERR_NOT_SUPPORTED and out.tables == []
    plan.close()


def test_unknown_flags_are_refused():
    ins = _inputs(1, 50, 100, 4096, seed=51)
    res = luda.compact_device([dev(ins[0])], oracle.MAX_SEQ, opts=luda.options(flags=1 << 10))
    assert res.status == luda.ERR_INVALID_ARG


# ---- compressed output (LUDA_F_COMPRESS) ---------------------------------------------------
CZ = luda.F_COMPRESS


@pytest.mark.parametrize("n_in,n,vlen,T,target", [(1, 300, 200, 4096, 64 << 10), (3, 200, 100, 4096, 32 << 10),
                                                  (4, 150, 40, 256, 8 << 10), (2, 60, 3000, 1, 64 << 10),
                                                  (3, 100, 1000, 16384, 1 << 20), (5, 400, 0, 512, 16 << 10),
                                                  (2, 300, 5000, 65536, 1 << 20)])
def test_compressed_output(n_in, n, vlen, T, target):
    ins = _inputs(n_in, n, vlen, T, seed=7 * n + vlen + T, compress=(True, False))
    got = _both(ins, T=T, target=target, flags=CZ)
    if vlen >= 100:
        assert any(t == 1 for x in got.tables for t in sstpy.read(x)["types"])


@pytest.mark.parametrize("flags", [CZ | luda.F_SHORT_INDEX, CZ | luda.F_FILTER_ARRAY,
                                   CZ | luda.F_SHORT_INDEX | luda.F_FILTER_ARRAY])
def test_compressed_output_with_other_variants(flags):
    ins = _inputs(3, 250, 150, 2048, seed=61)
    _both(ins, T=2048, target=24 << 10, flags=flags)


def test_compressed_output_of_incompressible_and_tiny_jobs():
    job = W.config1(seed=8, scale=1 / 32)
    ins = [oracle.build_tables(r, job.block_size, job.restart_interval, job.bloom_bits_per_key, U64MAX).tables[0].data
           for r in job.inputs]
    got = _both(ins, T=job.block_size, target=job.target_file_size, flags=CZ, snapshot=job.smallest_snapshot,
                bottommost=job.bottommost)
    assert all(t == 0 for x in got.tables for t in sstpy.read(x)["types"])   # random values: kept raw
    for seed in range(12):
        rng = np.random.default_rng(700 + seed)
        j = W.tiny_job(rng, n_keys=int(rng.integers(1, 200)), max_versions=3, n_inputs=int(rng.integers(1, 5)),
                       key_len=(0, 20), val_len=(0, 400))
        tins = [oracle.build_tables(r, 256, 4, 10, U64MAX, flags=oracle.F_COMPRESS).tables[0].data
                for r in j.inputs]
        _both(tins, T=int(rng.choice([1, 64, 256, 4096])), target=int(rng.choice([1, 3000, 1 << 20])), flags=CZ,
              snapshot=j.smallest_snapshot, bottommost=j.bottommost)


def test_compressed_builder_batch_and_plan():
    run = _run(500, 300, seed=71)
    want = oracle.build_tables(run, 4096, 16, 10, 64 << 10, flags=oracle.F_COMPRESS)
    got = luda.build_device(run, luda.options(4096, 16, 10, 64 << 10, flags=CZ))
    assert got.status == 0, got.detail
    assert [t.cpu().numpy().tobytes() for t in got.tables] == [t.data for t in want.tables]
    ins = [_inputs(2, 200, 150, 4096, seed=s) for s in (81, 82)]
    wants = [oracle.compact(x, oracle.MAX_SEQ, False, 4096, 16, 10, 32 << 10, oracle.F_COMPRESS) for x in ins]
    batch = [([dev(b) for b in x], oracle.MAX_SEQ, False) for x in ins]
    opts = luda.options(4096, 16, 10, 32 << 10, flags=CZ)
    rc, outs = luda.batch_compact_device(batch, opts)
    assert rc == 0
    for g, w in zip(outs, wants):
        g.tables = [t.cpu().numpy().tobytes() for t in g.tables]
        assert_same(g, w)
    raw_ins = [[oracle.build_tables(_run(200, 150, seed=s + k), 4096, 16, 10, U64MAX).tables[0].data for k in (0, 1)]
               for s in (91, 93)]
    # plans take uncompressed inputs; their output may be compressed
    pw = [oracle.compact(x, oracle.MAX_SEQ, False, 4096, 16, 10, 32 << 10, oracle.F_COMPRESS) for x in raw_ins]
    plan = luda.Plan([([dev(b) for b in x], oracle.MAX_SEQ, False) for x in raw_ins], opts)
    for _ in range(2):
        plan.run()
        torch.cuda.synchronize()
        for g, w in zip(plan.outputs(), pw):
            g.tables = [t.cpu().numpy().tobytes() for t in g.tables]
            assert_same(g, w)
    plan.close()


def test_host_entry_point_and_server_host_jobs_with_compression():
    """luda_compact (host inputs, host outputs) and the server's host-buffer jobs take the
    same decompression and compression paths."""
    ins = _inputs(3, 200, 200, 4096, seed=101, compress=(True, False))
    want = oracle.compact(ins, oracle.MAX_SEQ, False, 4096, 16, 10, 32 << 10, oracle.F_COMPRESS)
    got = luda.compact(ins, oracle.MAX_SEQ, opts=luda.options(4096, 16, 10, 32 << 10, flags=CZ))
    assert got.status == 0, got.detail
    assert [bytes(t) for t in got.tables] == [t.data for t in want.tables]
    host = [torch.frombuffer(bytearray(x), dtype=torch.uint8).pin_memory() for x in ins]
    srv = luda.Server(2, 1 << 40, luda.options(4096, 16, 10, 32 << 10, flags=CZ))
    t = srv.submit(host, oracle.MAX_SEQ, False, host=True)
    res, _ = srv.wait(t, timeout_ms=60_000)
    srv.close()
    assert res.status == 0
    assert [bytes(x) for x in res.tables] == [x.data for x in want.tables]
