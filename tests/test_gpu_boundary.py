"""The host-buffer entry points of the C ABI against the oracle:

* luda_batch_compact: several jobs' host inputs in one call; every job's tables (host
  memory) equal the oracle's, a corrupt job fails alone, and an error that stops the
  batch leaves no tables anywhere.
* luda_compact and the oracle's luda_oracle_compact called with the very same argument
  values (one ctypes input array, one options struct): the same bytes, keys and counts.
"""
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

T, R, BPK, TARGET = 4096, 16, 10, 256 * 1024


def _jobs(n, seed):
    rng = np.random.default_rng(seed)
    jobs = []
    for j in range(n):
        if j % 3 == 0:
            job = W.config4_job(rng, int(rng.integers(200_000, 2_000_000)), f"b{j}", seed)
        elif j % 3 == 1:
            job = W.tiny_job(rng, n_keys=int(rng.integers(5, 300)), max_versions=4, n_inputs=int(rng.integers(1, 6)),
                             key_len=(1, 20), val_len=(0, 400))
        else:
            job = W.config2(seed=seed + j, scale=1 / 16)
        job.block_size, job.restart_interval, job.bloom_bits_per_key, job.target_file_size = T, R, BPK, TARGET
        jobs.append(job)
    return jobs


def test_batch_compact_host_matches_oracle_and_a_corrupt_job_fails_alone():
    jobs = _jobs(7, seed=21)
    ins = [oracle_inputs(j) for j in jobs]
    bad = bytearray(ins[4][0])
    bad[10] ^= 0x40  # inside the first data block: its checksum fails
    ins[4][0] = bytes(bad)
    want = [oracle_compact(j, x) for j, x in zip(jobs, ins)]
    assert want[4].status == oracle.ERR_CORRUPTION
    rc, outs = luda.batch_compact([(x, j.smallest_snapshot, j.bottommost) for j, x in zip(jobs, ins)],
                                  luda.options(T, R, BPK, TARGET))
    assert rc == 0
    for j, (g, w) in enumerate(zip(outs, want)):
        if j == 4:
            assert g.status == luda.ERR_CORRUPTION and not g.tables
        else:
            assert_same(g, w)
    # the same batch again (the library keeps no state between calls)
    rc, again = luda.batch_compact([(x, j.smallest_snapshot, j.bottommost) for j, x in zip(jobs, ins)],
                                   luda.options(T, R, BPK, TARGET))
    assert rc == 0 and [g.tables for g in again] == [g.tables for g in outs]


def test_batch_compact_host_error_stops_the_batch_with_no_tables():
    jobs = _jobs(3, seed=22)
    ins = [oracle_inputs(j) for j in jobs]
    o = luda.options(T, R, BPK, TARGET)
    o.flags = 1 << 30  # unknown flag
    rc, outs = luda.batch_compact([(x, j.smallest_snapshot, j.bottommost) for j, x in zip(jobs, ins)], o)
    assert rc == luda.ERR_INVALID_ARG
    assert all(g.status == luda.ERR_INVALID_ARG and not g.tables for g in outs)
    rc, outs = luda.batch_compact([], luda.options(T, R, BPK, TARGET))
    assert rc == 0 and outs == []


def _oracle_lib():
    L = C.CDLL(oracle.build())
    L.luda_oracle_compact.restype = C.c_int
    L.luda_oracle_compact.argtypes = [C.POINTER(luda.Input), C.c_uint32, C.c_int32, C.c_uint64,
                                      C.POINTER(luda.Options), C.POINTER(luda.Outputs)]
    L.luda_oracle_outputs_free.argtypes = [C.POINTER(luda.Outputs)]
    L.luda_oracle_outputs_free.restype = None
    return L


def _read(out):
    return [(C.string_at(out.tables[i].data, out.tables[i].size), int(out.tables[i].n_entries),
             C.string_at(out.tables[i].smallest, out.tables[i].smallest_len),
             C.string_at(out.tables[i].largest, out.tables[i].largest_len)) for i in range(out.n_tables)]


@pytest.mark.parametrize("cfg,flags", [("config1", 0), ("config2", 0), ("config2", luda.F_SHORT_INDEX),
                                       ("config1", luda.F_FILTER_ARRAY), ("config1", luda.F_COMPRESS)])
def test_luda_compact_and_oracle_compact_take_the_same_arguments(cfg, flags):
    job = getattr(W, cfg)(seed=23, scale=1 / 4)
    ins = oracle_inputs(job)
    arr = (luda.Input * len(ins))()
    bufs = [np.frombuffer(b, dtype=np.uint8) for b in ins]
    for i, b in enumerate(bufs):
        arr[i].data, arr[i].size, arr[i].level = b.ctypes.data, len(b), 0
    o = luda.job_options(job, flags=flags)
    gpu, ora = luda.Outputs(), luda.Outputs()
    rc_g = luda.lib().luda_compact(arr, len(ins), job.level, job.smallest_snapshot, C.byref(o), C.byref(gpu))
    OL = _oracle_lib()
    rc_o = OL.luda_oracle_compact(arr, len(ins), job.level, job.smallest_snapshot, C.byref(o), C.byref(ora))
    assert rc_g == rc_o == 0
    assert _read(gpu) == _read(ora)
    assert (gpu.n_in_entries, gpu.n_dropped) == (ora.n_in_entries, ora.n_dropped)
    assert gpu.ms_h2d > 0 and ora.ms_h2d == 0
    luda.lib().luda_outputs_free(C.byref(gpu))
    OL.luda_oracle_outputs_free(C.byref(ora))
