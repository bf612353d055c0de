"""Serving (luda_server): jobs that run together under an HBM budget produce the same
bytes as alone and as the oracle; a corrupt job fails alone; the simulated LSM tree keeps
every key's newest write."""
import numpy as np
import pytest

from helpers import decoded, oracle_compact, oracle_inputs
from paper_2004_03054_b300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2004_03054_b300 import luda  # noqa: E402

T, R, BPK, TARGET = 4096, 16, 10, 64 * 1024


def _dev(b):
    return torch.frombuffer(bytearray(b), dtype=torch.uint8).cuda()


def _jobs(n, seed):
    rng = np.random.default_rng(seed)
    jobs = []
    for j in range(n):
        if j % 3 == 0:
            job = W.config4_job(rng, int(rng.integers(100_000, 1_500_000)), f"s{j}", seed)
        elif j % 3 == 1:
            job = W.tiny_job(rng, n_keys=int(rng.integers(5, 400)), max_versions=4, n_inputs=int(rng.integers(1, 6)),
                             key_len=(1, 20), val_len=(0, 500))
        else:
            job = W.config1(seed=seed + j, scale=1 / 64)
        job.block_size, job.restart_interval, job.bloom_bits_per_key, job.target_file_size = T, R, BPK, TARGET
        jobs.append(job)
    return jobs


def _tables(res):
    return [t.cpu().numpy().tobytes() for t in res.tables]


@pytest.mark.parametrize("n_slots,budget,prewarm", [(4, 1 << 40, 0), (4, 24 << 20, 0), (1, 1 << 40, 0), (8, 1, 0),
                                                    (3, 1 << 40, 1 << 30)])
def test_server_mix_equals_alone_and_oracle(n_slots, budget, prewarm):
    jobs = _jobs(15, seed=11)
    ins = [oracle_inputs(j) for j in jobs]
    want = [oracle_compact(j, x) for j, x in zip(jobs, ins)]
    dev = [[_dev(b) for b in x] for x in ins]
    torch.cuda.synchronize()
    srv = luda.Server(n_slots, budget, luda.options(T, R, BPK, TARGET), prewarm_bytes=prewarm)
    tickets = [srv.submit(d, j.smallest_snapshot, j.bottommost) for d, j in zip(dev, jobs)]
    seen = set()
    for _ in tickets:
        t = srv.next(60_000)
        assert t is not None
        seen.add(t)
    assert seen == set(tickets)
    stats = []
    for j, t in enumerate(tickets):
        res, st = srv.wait(t)
        assert res.status == want[j].status == 0, (j, res.status, res.detail)
        assert _tables(res) == [x.data for x in want[j].tables], j
        assert res.n_in_entries == want[j].n_in_entries and res.n_dropped == want[j].n_dropped
        assert st.latency_ms >= st.run_ms >= 0 and st.input_bytes == sum(len(b) for b in ins[j])
        stats.append(st)
    ss = srv.stats()
    srv.close()
    assert ss.submitted == ss.completed == len(jobs) and ss.failed == 0
    assert 1 <= ss.running_peak <= n_slots
    if n_slots > 1 and budget >= 1 << 40:
        assert ss.running_peak > 1  # jobs did run on the device together
    if budget >= 1 << 40:
        assert ss.budget_peak <= budget
    else:
        # every admission either fit the budget or ran alone
        for st in stats:
            assert st.reserved_bytes <= budget or st.running_at_admit == 1
    # alone, same stream discipline as a user call
    for j in (0, 1, 2, 3):
        alone = luda.compact_device(dev[j], jobs[j].smallest_snapshot,
                                    opts=luda.options(T, R, BPK, TARGET, bottommost=jobs[j].bottommost))
        assert _tables(alone) == [x.data for x in want[j].tables]


def test_server_corrupt_job_fails_alone():
    jobs = _jobs(6, seed=5)
    ins = [oracle_inputs(j) for j in jobs]
    bad = bytearray(ins[3][0])
    bad[10] ^= 0x40                      # inside the first data block: CRC mismatch
    ins[3][0] = bytes(bad)
    dev = [[_dev(b) for b in x] for x in ins]
    torch.cuda.synchronize()
    srv = luda.Server(3, 1 << 40, luda.options(T, R, BPK, TARGET))
    tickets = [srv.submit(d, j.smallest_snapshot, j.bottommost) for d, j in zip(dev, jobs)]
    for j, t in enumerate(tickets):
        res, _ = srv.wait(t, timeout_ms=60_000)
        if j == 3:
            assert res.status == luda.ERR_CORRUPTION and not res.tables
            assert "offset" in res.detail
        else:
            assert res.status == 0
            assert _tables(res) == [x.data for x in oracle_compact(jobs[j], ins[j]).tables]
    assert srv.stats().failed == 1
    srv.close()


def test_server_wait_timeout_and_unknown_ticket():
    srv = luda.Server(1, 1 << 40, luda.options(T, R, BPK, TARGET))
    assert srv.next(0) is None
    with pytest.raises(KeyError):
        srv.wait(12345)
    # the C entry point itself rejects an unknown ticket
    out, st = luda.Outputs(), luda.JobStats()
    assert luda.lib().luda_server_wait(srv.handle, 12345, 0, luda.C.byref(out), luda.C.byref(st)) == luda.ERR_INVALID_ARG
    srv.close()


def test_lsm_served_tree_keeps_newest_writes():
    """A small served LSM run (2 MiB memtables, 24 flushes, fanout 3, 3 slots): each job is
    also re-run alone through luda_compact_device and must give the same bytes; at the end
    the newest version of every written key is the one the tree returns."""
    from paper_2004_03054_b300 import lsm as L
    mib = 1 << 20
    stream = list(W.config5_stream(seed=21, n_memtables=24, memtable_bytes=2 * mib, write_rate=4e6,
                                   universe_bits=16))
    checked = []

    def check(rec, out):
        d = [(t.ptr, t.size) for t in rec.inputs]
        o = luda.options(T, R, BPK, 2 * mib, bottommost=rec.bottommost)
        alone = luda.compact_device([_ptr_tensor(p, n) for p, n in d], W.MAX_SEQ, opts=o)
        mix = [luda.device_bytes(out.tables[i].data, out.tables[i].size).cpu().numpy().tobytes()
               for i in range(out.n_tables)]
        assert alone.status == 0
        assert _tables(alone) == mix
        checked.append(rec.level)

    captured = {}
    rep = _serve_and_capture(L, stream, check, mib, captured)
    assert rep.failed == 0 and rep.jobs == len(checked) and rep.jobs >= 5
    assert max(checked) >= 1                      # jobs below level 0 ran as well
    newest = {}
    for mt in stream:
        for hi, lo, s in zip(mt.hi.tolist(), mt.lo.tolist(), mt.seqs.tolist()):
            newest[hi.to_bytes(8, "big") + lo.to_bytes(8, "big")] = s
    got = captured["newest"]
    assert got == newest


class _ptr_tensor:
    """Minimal stand-in for a CUDA tensor over (device pointer, size)."""

    def __init__(self, ptr, n):
        self._p, self._n = ptr, n

    def data_ptr(self):
        return self._p

    def numel(self):
        return self._n


def _serve_and_capture(L, stream, check, mib, captured):
    """serve() with a hook that reads the final tree back before it is freed."""
    orig_close = L.LSM.close

    def close(self):
        newest = {}
        for lv in range(L.N_LEVELS):
            tabs = sorted(self.levels[lv], key=lambda t: -t.number) if lv == 0 else self.levels[lv]
            for t in tabs:
                data = luda.device_bytes(t.ptr, t.size).cpu().numpy().tobytes()
                for uk, seq, typ, _ in decoded([data]):
                    if uk not in newest:
                        newest[uk] = seq
        captured["newest"] = newest
        orig_close(self)

    L.LSM.close = close
    try:
        return L.serve(stream, n_slots=3, hbm_budget=1 << 40, pace=False, on_complete=check,
                       lsm_kw=dict(memtable_bytes=2 * mib, target_file=2 * mib, fanout=3, value_pool_bytes=64 * mib))
    finally:
        L.LSM.close = orig_close


@pytest.mark.parametrize("n_slots", [1, 3])
def test_server_host_jobs_equal_oracle(n_slots):
    """Jobs with host-memory inputs: copied in, compacted and copied back by the slots;
    the tables equal the oracle's and those of the device path."""
    jobs = _jobs(9, seed=17)
    ins = [oracle_inputs(j) for j in jobs]
    want = [oracle_compact(j, x) for j, x in zip(jobs, ins)]
    host = [[torch.frombuffer(bytearray(b), dtype=torch.uint8).pin_memory() for b in x] for x in ins]
    srv = luda.Server(n_slots, 1 << 40, luda.options(T, R, BPK, TARGET))
    tickets = [srv.submit(h, j.smallest_snapshot, j.bottommost, host=True) for h, j in zip(host, jobs)]
    for j, t in enumerate(tickets):
        res, st = srv.wait(t, timeout_ms=60_000)
        assert res.status == want[j].status == 0, (j, res.status, res.detail)
        assert res.tables == [x.data for x in want[j].tables], j
        assert st.reserved_bytes >= sum(len(b) for b in ins[j])
    srv.close()
