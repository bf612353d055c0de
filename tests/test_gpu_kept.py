"""Decoded runs kept on the device (LUDA_F_KEEP_DECODED, §III-D): a compaction whose
inputs are all tables written with the flag takes its records from their kept runs
instead of decoding them, and writes exactly the bytes of the same compaction without the
flag and of the oracle on the same table bytes. A job with one input that has no kept
run decodes all of them as usual; freeing a table's outputs drops its run."""
import ctypes as C

import pytest

from helpers import oracle_inputs
from paper_2004_03054_b300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2004_03054_b300 import luda  # noqa: E402

T, R, BPK, TARGET = 4096, 16, 10, 512 * 1024


def _dev(b):
    return torch.frombuffer(bytearray(b), dtype=torch.uint8).cuda()


def _compact(ptrs, snap, flags, bottommost=False):
    """luda_compact_device on raw (pointer, size) inputs; returns (Outputs, [bytes])."""
    arr = (luda.Input * max(1, len(ptrs)))()
    for i, (p, n) in enumerate(ptrs):
        arr[i].data, arr[i].size = p, n
    o = luda.options(T, R, BPK, TARGET, bottommost=bottommost, flags=flags, stream=luda.current_stream())
    out = luda.Outputs()
    rc = luda.lib().luda_compact_device(arr, len(ptrs), 1, snap, C.byref(o), C.byref(out))
    assert rc == 0, luda.last_error_detail()
    tabs = [luda.device_bytes(out.tables[i].data, out.tables[i].size).cpu().numpy().tobytes()
            for i in range(out.n_tables)]
    return out, tabs


def _ptrs(out):
    return [(out.tables[i].data, out.tables[i].size) for i in range(out.n_tables)]


@pytest.mark.parametrize("fmt_flags", [0, luda.F_SHORT_INDEX | luda.F_FILTER_ARRAY])
def test_kept_runs_give_the_plain_and_oracle_bytes(fmt_flags):
    keep = luda.F_KEEP_DECODED | fmt_flags
    jobs = [W.config1(seed=81, scale=1 / 8), W.config2(seed=82, scale=1 / 8)]
    outs, hosts = [], []
    for job in jobs:
        ins = oracle_inputs(job)
        dev = [_dev(b) for b in ins]
        out, tabs = _compact([(t.data_ptr(), t.numel()) for t in dev], job.smallest_snapshot, keep)
        want = oracle.compact(ins, job.smallest_snapshot, False, T, R, BPK, TARGET, fmt_flags)
        assert tabs == [t.data for t in want.tables]
        outs.append(out)
        hosts.append(tabs)
    # job B: the second job's tables (newer) then the first's; every input has a kept run
    ptrs = _ptrs(outs[1]) + _ptrs(outs[0])
    host_in = hosts[1] + hosts[0]
    u0 = luda.kept_inputs_used()
    kept, kept_tabs = _compact(ptrs, W.MAX_SEQ, keep)
    assert luda.kept_inputs_used() - u0 == len(ptrs)
    u1 = luda.kept_inputs_used()
    plain, plain_tabs = _compact(ptrs, W.MAX_SEQ, fmt_flags)
    assert luda.kept_inputs_used() == u1
    want = oracle.compact(host_in, W.MAX_SEQ, False, T, R, BPK, TARGET, fmt_flags)
    assert want.status == 0
    assert kept_tabs == plain_tabs == [t.data for t in want.tables]
    assert [int(kept.tables[i].n_entries) for i in range(kept.n_tables)] == [t.n_entries for t in want.tables]
    # a second hop from B's kept run, bottommost (tombstones dropped)
    u2 = luda.kept_inputs_used()
    _, hop2 = _compact(_ptrs(kept), W.MAX_SEQ, keep, bottommost=True)
    assert luda.kept_inputs_used() - u2 == kept.n_tables
    want2 = oracle.compact(kept_tabs, W.MAX_SEQ, True, T, R, BPK, TARGET, fmt_flags)
    assert hop2 == [t.data for t in want2.tables]
    for o in (kept, plain, *outs):
        luda.free_outputs(o)


def test_one_input_without_a_kept_run_decodes_all():
    job = W.config1(seed=83, scale=1 / 8)
    ins = oracle_inputs(job)
    dev = [_dev(b) for b in ins]
    out, tabs = _compact([(t.data_ptr(), t.numel()) for t in dev], job.smallest_snapshot, luda.F_KEEP_DECODED)
    extra = W.config1(seed=84, scale=1 / 16)
    extra_in = oracle_inputs(extra)[0]
    ex = _dev(extra_in)
    ptrs = [(ex.data_ptr(), ex.numel())] + _ptrs(out)
    u0 = luda.kept_inputs_used()
    _, got = _compact(ptrs, W.MAX_SEQ, luda.F_KEEP_DECODED)
    assert luda.kept_inputs_used() == u0
    want = oracle.compact([extra_in] + tabs, W.MAX_SEQ, False, T, R, BPK, TARGET)
    assert got == [t.data for t in want.tables]
    luda.free_outputs(out)


def test_freed_tables_drop_their_runs():
    job = W.config1(seed=85, scale=1 / 16)
    ins = oracle_inputs(job)
    dev = [_dev(b) for b in ins]
    out, tabs = _compact([(t.data_ptr(), t.numel()) for t in dev], job.smallest_snapshot, luda.F_KEEP_DECODED)
    # copies of the tables at new addresses have no kept run
    copies = [_dev(t) for t in tabs]
    luda.free_outputs(out)
    u0 = luda.kept_inputs_used()
    _, got = _compact([(t.data_ptr(), t.numel()) for t in copies], W.MAX_SEQ, luda.F_KEEP_DECODED)
    assert luda.kept_inputs_used() == u0
    assert got == [t.data for t in oracle.compact(tabs, W.MAX_SEQ, False, T, R, BPK, TARGET).tables]


def test_served_tree_with_kept_runs_equals_the_plain_tree():
    """The same write stream through the simulated LSM tree with one slot (a deterministic
    schedule), with and without kept runs: the same tables at every level, and most
    compaction inputs served from kept runs."""
    from paper_2004_03054_b300 import lsm as L

    def tree(keep):
        levels = {}

        def grab(t):
            for lv, tabs in enumerate(t.levels):
                levels[lv] = [luda.device_bytes(x.ptr, x.size).cpu().numpy().tobytes() for x in tabs]

        stream = W.config5_stream(seed=9, n_memtables=24, memtable_bytes=1 << 20, write_rate=8e6)
        rep = L.serve(stream, n_slots=1, hbm_budget=1 << 40, pace=False, before_close=grab,
                      lsm_kw={"memtable_bytes": 1 << 20, "target_file": 1 << 20, "keep_decoded": keep})
        return rep, levels

    rep_k, lv_k = tree(True)
    rep_p, lv_p = tree(False)
    assert rep_k.jobs == rep_p.jobs >= 5 and rep_k.failed == rep_p.failed == 0
    assert lv_k == lv_p
    assert rep_p.kept_inputs == 0
    assert rep_k.kept_inputs > 0
