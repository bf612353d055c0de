"""luda_oracle_compact, the oracle behind luda_compact's signature (include/luda_oracle.h):
its argument structs have the layouts of luda.h's (checked by compiling both headers),
the very same ctypes arguments the binding builds for luda_compact drive it, and its
tables are ora_compact's bytes for every format variant; errors leave no tables."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

import oracle
from helpers import oracle_compact, oracle_inputs
from paper_2004_03054_b300 import luda
from paper_2004_03054_b300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_FIELDS = {
    ("luda_input", "luda_oracle_input"): ["data", "size", "level", "file_number"],
    ("luda_options", "luda_oracle_options"): ["block_size", "restart_interval", "bloom_bits_per_key",
                                              "target_file_size", "bottommost", "flags", "dev_alloc", "dev_free",
                                              "alloc_ctx", "stream", "tuning"],
    ("luda_table", "luda_oracle_table"): ["data", "size", "n_entries", "smallest", "smallest_len", "largest",
                                          "largest_len"],
    ("luda_outputs", "luda_oracle_outputs"): ["tables", "n_tables", "status", "n_in_entries", "n_dropped", "ms_h2d",
                                              "ms_device", "ms_d2h", "stage_ms", "stage_bytes", "_priv"],
}


def test_oracle_abi_structs_have_the_layouts_of_luda_h(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    lines = ["#include <stddef.h>", '#include "luda.h"', '#include "luda_oracle.h"']
    for (a, b), fields in _FIELDS.items():
        lines.append(f"_Static_assert(sizeof({a}) == sizeof({b}), \"size of {a}\");")
        for f in fields:
            lines.append(f"_Static_assert(offsetof({a}, {f}) == offsetof({b}, {f}), \"{a}.{f}\");")
    lines.append("_Static_assert(LUDA_N_STAGES == 8, \"stages\");")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    r = subprocess.run(["gcc", "-std=c11", "-fsyntax-only", "-I", os.path.join(ROOT, "include"), str(src)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def _olib():
    L = C.CDLL(oracle.build())
    L.luda_oracle_compact.restype = C.c_int
    L.luda_oracle_compact.argtypes = [C.POINTER(luda.Input), C.c_uint32, C.c_int32, C.c_uint64,
                                      C.POINTER(luda.Options), C.POINTER(luda.Outputs)]
    L.luda_oracle_outputs_free.argtypes = [C.POINTER(luda.Outputs)]
    L.luda_oracle_outputs_free.restype = None
    return L


def _call(job, ins, flags=0):
    L = _olib()
    arr = (luda.Input * max(1, len(ins)))()
    for i, b in enumerate(ins):
        arr[i].data, arr[i].size = C.cast(C.c_char_p(b), C.c_void_p).value, len(b)
    o = luda.job_options(job, flags=flags)
    out = luda.Outputs()
    rc = L.luda_oracle_compact(arr, len(ins), job.level, job.smallest_snapshot, C.byref(o), C.byref(out))
    tables = [C.string_at(out.tables[i].data, out.tables[i].size) for i in range(out.n_tables)]
    keys = [(C.string_at(out.tables[i].smallest, out.tables[i].smallest_len),
             C.string_at(out.tables[i].largest, out.tables[i].largest_len), int(out.tables[i].n_entries))
            for i in range(out.n_tables)]
    res = (rc, int(out.status), tables, keys, int(out.n_in_entries), int(out.n_dropped), out.ms_device)
    L.luda_oracle_outputs_free(C.byref(out))
    assert out.n_tables == 0 and not out.tables
    return res


@pytest.mark.parametrize("flags", [0, luda.F_SHORT_INDEX, luda.F_FILTER_ARRAY, luda.F_COMPRESS,
                                   luda.F_SHORT_INDEX | luda.F_FILTER_ARRAY | luda.F_TRACE])
@pytest.mark.parametrize("cfg", ["config1", "config2"])
def test_oracle_abi_writes_ora_compacts_bytes(cfg, flags):
    job = getattr(W, cfg)(seed=71, scale=1 / 16)
    ins = oracle_inputs(job)
    want = oracle_compact(job, ins, flags=flags & ~luda.F_TRACE)
    rc, status, tables, keys, n_in, n_drop, ms = _call(job, ins, flags)
    assert rc == 0 and status == 0
    assert tables == [t.data for t in want.tables]
    assert keys == [(t.smallest, t.largest, t.n_entries) for t in want.tables]
    assert (n_in, n_drop) == (want.n_in_entries, want.n_dropped)
    assert ms > 0


def test_oracle_abi_errors_leave_no_tables():
    job = W.config1(seed=72, scale=1 / 32)
    ins = oracle_inputs(job)
    rc, status, tables, *_ = _call(job, ins, flags=32)  # the device-only test flag is not the oracle's
    assert rc == status == luda.ERR_INVALID_ARG and tables == []
    bad = bytearray(ins[0])
    bad[100] ^= 0x40  # inside the first data block: its checksum no longer holds
    rc, status, tables, *_ = _call(job, [bytes(bad)] + ins[1:])
    assert rc == status == luda.ERR_CORRUPTION and tables == []
