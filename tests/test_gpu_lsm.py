"""The simulated LSM tree under host-side fault injection and across a snapshot: a failed
compaction leaves its input tables in the tree and its retry gives the same bytes as the
job run alone; a tree written by snapshot() and read back by restore() holds the same
tables and the same newest version of every key."""
import numpy as np
import pytest

from helpers import decoded
from paper_2004_03054_b300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2004_03054_b300 import lsm as L  # noqa: E402
from paper_2004_03054_b300 import luda  # noqa: E402

MIB = 1 << 20
T, R, BPK = 4096, 16, 10
KW = dict(memtable_bytes=2 * MIB, target_file=2 * MIB, fanout=3, value_pool_bytes=64 * MIB)


def _stream(n=16, seed=33):
    return list(W.config5_stream(seed=seed, n_memtables=n, memtable_bytes=2 * MIB, write_rate=4e6,
                                 universe_bits=16))


def _newest_written(stream):
    newest = {}
    for mt in stream:
        for hi, lo, s in zip(mt.hi.tolist(), mt.lo.tolist(), mt.seqs.tolist()):
            newest[hi.to_bytes(8, "big") + lo.to_bytes(8, "big")] = s
    return newest


def _tree_newest(lsm):
    """Newest sequence number of every user key in the tree (level 0 newest table first)."""
    newest = {}
    for lv in range(L.N_LEVELS):
        tabs = sorted(lsm.levels[lv], key=lambda t: -t.number) if lv == 0 else lsm.levels[lv]
        for t in tabs:
            data = luda.device_bytes(t.ptr, t.size).cpu().numpy().tobytes()
            for uk, seq, typ, _ in decoded([data]):
                if uk not in newest:
                    newest[uk] = seq
    return newest


class _Ptr:
    def __init__(self, p, n):
        self._p, self._n = p, n

    def data_ptr(self):
        return self._p

    def numel(self):
        return self._n


def test_failed_jobs_keep_inputs_and_retry_gives_the_same_bytes():
    stream = _stream()
    hit = {0, 2, 3}
    checked = []

    def check(rec, out):
        # the (retried) job's tables equal the same inputs compacted alone
        o = luda.options(T, R, BPK, 2 * MIB, bottommost=rec.bottommost)
        alone = luda.compact_device([_Ptr(t.ptr, t.size) for t in rec.inputs], W.MAX_SEQ, opts=o)
        assert alone.status == 0
        got = [luda.device_bytes(out.tables[i].data, out.tables[i].size).cpu().numpy().tobytes()
               for i in range(out.n_tables)]
        assert [t.cpu().numpy().tobytes() for t in alone.tables] == got
        checked.append(rec.level)

    final = {}
    rep = L.serve(stream, n_slots=3, hbm_budget=1 << 40, pace=False, on_complete=check,
                  lsm_kw=dict(KW, fault=lambda i, level: i in hit),
                  before_close=lambda lsm: final.update(_tree_newest(lsm)))
    assert rep.failed == len(hit) and rep.retried == len(hit)
    assert rep.jobs == len(checked) + len(hit)
    assert final == _newest_written(stream)


def test_snapshot_restore_round_trip(tmp_path):
    stream = _stream(12, seed=34)
    saved = {}

    def snap(lsm):
        saved["manifest"] = lsm.snapshot(str(tmp_path))
        saved["newest"] = _tree_newest(lsm)
        saved["bytes"] = {t.number: luda.device_bytes(t.ptr, t.size).cpu().numpy().tobytes()
                          for lv in lsm.levels for t in lv}

    L.serve(stream, n_slots=2, hbm_budget=1 << 40, pace=False, lsm_kw=dict(KW), before_close=snap)
    assert saved["newest"] == _newest_written(stream)
    opts = luda.options(T, R, BPK, 2 * MIB)
    srv = luda.Server(2, 1 << 40, opts)
    lsm = L.LSM(srv, **KW)
    try:
        lsm.restore(str(tmp_path))
        assert [[t.number for t in lv] for lv in lsm.levels] == \
            [[e["number"] for e in lv] for lv in saved["manifest"]["levels"]]
        assert {t.number: luda.device_bytes(t.ptr, t.size).cpu().numpy().tobytes()
                for lv in lsm.levels for t in lv} == saved["bytes"]
        assert _tree_newest(lsm) == saved["newest"]
        # the restored tree keeps working: one more memtable, then every job it triggers
        more = list(W.config5_stream(seed=35, n_memtables=2, memtable_bytes=2 * MIB, write_rate=4e6,
                                     universe_bits=16, first_seq=10**9))
        for mt in more:
            lsm.flush(mt)
            torch.cuda.synchronize()
            lsm.schedule()
        while lsm.jobs:
            lsm.complete(srv.next(60_000))
            lsm.schedule()
        want = dict(saved["newest"])
        want.update(_newest_written(more))
        assert _tree_newest(lsm) == want
        with pytest.raises(RuntimeError):
            lsm.restore(str(tmp_path))  # not empty
    finally:
        lsm.close()
        srv.close()
