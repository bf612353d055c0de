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


def test_kept_runs_edge_cases():
    """Calls that keep no runs (compressed output, host outputs), a job whose entries are all
    dropped (no tables), ranged jobs (which never take kept runs), and a batch call whose
    tables keep runs that a later job takes."""
    K = luda.F_KEEP_DECODED
    job = W.config1(seed=86, scale=1 / 16)
    ins = oracle_inputs(job)
    dev = [_dev(b) for b in ins]
    ptrs = [(t.data_ptr(), t.numel()) for t in dev]
    # compressed output: tables written, no run kept
    cz, cz_tabs = _compact(ptrs, job.smallest_snapshot, K | luda.F_COMPRESS)
    assert cz_tabs == [t.data for t in oracle.compact(ins, job.smallest_snapshot, False, T, R, BPK, TARGET,
                                                      luda.F_COMPRESS).tables]
    u0 = luda.kept_inputs_used()
    _, again = _compact(_ptrs(cz), W.MAX_SEQ, K)
    assert luda.kept_inputs_used() == u0
    assert again == [t.data for t in oracle.compact(cz_tabs, W.MAX_SEQ, False, T, R, BPK, TARGET).tables]
    luda.free_outputs(cz)
    # host entry point with the flag: the same bytes, nothing kept or used
    host = luda.compact(ins, job.smallest_snapshot, opts=luda.options(T, R, BPK, TARGET, flags=K))
    assert host.status == 0 and host.tables == [t.data for t in oracle.compact(ins, job.smallest_snapshot, False, T, R,
                                                                                BPK, TARGET).tables]
    # every entry dropped: a bottommost job of deletions only writes no table
    import numpy as np
    rng = np.random.default_rng(7)
    keys = [i.to_bytes(4, "big") for i in range(50)]
    run = W._make_run(keys, np.arange(1, 51, dtype=np.uint64), np.zeros(50, np.uint8), np.zeros(50, np.int64), rng, 0)
    dels = oracle.build_tables(run, T, R, BPK, (1 << 64) - 1).tables[0].data
    d = _dev(dels)
    out, tabs = _compact([(d.data_ptr(), d.numel())], W.MAX_SEQ, K, bottommost=True)
    assert out.n_tables == 0 and tabs == []
    luda.free_outputs(out)
    # ranged jobs never take kept runs, and write the oracle's bytes
    kept, kept_tabs = _compact(ptrs, job.smallest_snapshot, K)
    lo = bytes(job.inputs[1].ukeys[:16])
    u1 = luda.kept_inputs_used()
    class Raw:  # the kept tables themselves (their addresses are what the runs are kept under)
        def __init__(self, p, n):
            self.p, self.n = p, n

        def data_ptr(self):
            return self.p

        def numel(self):
            return self.n

    rc, outs = luda.batch_compact_device([([Raw(p, n) for p, n in _ptrs(kept)], W.MAX_SEQ, False, lo, None)],
                                         luda.options(T, R, BPK, TARGET, flags=K))
    assert rc == 0 and luda.kept_inputs_used() == u1
    want = oracle.compact(kept_tabs, W.MAX_SEQ, False, T, R, BPK, TARGET, lo=lo)
    assert [t.cpu().numpy().tobytes() for t in outs[0].tables] == [t.data for t in want.tables]
    luda.free_outputs(kept)
    # a batch call keeps the runs of all its jobs' tables; a later job takes them
    jobs2 = [W.config1(seed=s, scale=1 / 16) for s in (87, 88)]
    ins2 = [oracle_inputs(j) for j in jobs2]
    rc, bouts = luda.batch_compact_device([([_dev(b) for b in x], j.smallest_snapshot, False) for j, x in
                                           zip(jobs2, ins2)], luda.options(T, R, BPK, TARGET, flags=K),
                                          copy_out=False)
    assert rc == 0
    bptrs = _ptrs(bouts[1]) + _ptrs(bouts[0])
    host_in = [luda.device_bytes(p, n).cpu().numpy().tobytes() for p, n in bptrs]
    u2 = luda.kept_inputs_used()
    _, got = _compact(bptrs, W.MAX_SEQ, K)
    assert luda.kept_inputs_used() - u2 == len(bptrs)
    assert got == [t.data for t in oracle.compact(host_in, W.MAX_SEQ, False, T, R, BPK, TARGET).tables]
    for o in bouts:
        luda.free_outputs(o)
