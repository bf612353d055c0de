"""A simulated LSM tree whose tables live in device memory, served by luda_server.

The paper runs LUDA inside LevelDB: the store flushes memtables into level-0 tables and
hands compaction jobs (a table of one level plus the overlapping tables of the next) to
the GPU (§II-A, §III-A). This module is the host side of that loop for the served
workload: a 7-level tree with a level-0 trigger of 4 tables, fanout 10, 64 MiB memtables
and 64 MiB output tables. Every table stays resident in HBM as the exact bytes a disk
would hold; memtables are packed on the GPU by luda_build_device; compaction jobs go to a
luda.Server, which runs several at once under an HBM budget (continuous batching).

Policy (LevelDB's, with concurrent jobs on disjoint tables):
  * score(L0) = tables / 4; score(Li) = bytes / (640 MiB * 10^(i-1)) for i >= 1.
  * an L0 job takes every idle L0 table (newest first) plus the overlapping L1 tables;
    an Li job takes the next idle table after the level's compaction pointer plus the
    overlapping Li+1 tables. A job starts only if none of its tables is busy; jobs keep
    starting while the level's bytes, less those already being compacted out of it, exceed
    its target.
  * a job is bottommost when no deeper level holds a table overlapping its key range;
    there are no snapshots (smallest snapshot = newest sequence number).
  * writes stall while L0 holds 12 tables (LevelDB's stop trigger).

Failures: a job is all-or-nothing (its outputs depend only on its inputs and options), so
a failed job leaves its input tables in the tree untouched and the policy simply starts it
again; the same tables failing three times in a row is an error. For tests, `fault`
injects failures on the host: a job it selects gets one extra, corrupted input table.

Checkpoint: snapshot() writes the tree (every table's bytes plus a JSON manifest of levels,
key ranges, table numbers and compaction pointers) to a directory; restore() rebuilds the
tree on the device from it. A compaction in flight is not part of a snapshot (it would be
redone).
"""
from __future__ import annotations

import ctypes as C
import json
import os
import time
from dataclasses import dataclass, field

import numpy as np

from . import luda
from . import workloads as W

MiB = 1 << 20
N_LEVELS = 7


class _Owner:
    """Keeps one luda_outputs (device tables of a finished job) alive until every table
    cut from it has left the tree."""

    def __init__(self, out: luda.Outputs, n: int):
        self.out = out
        self.refs = n

    def release(self):
        self.refs -= 1
        if self.refs == 0:
            luda.lib().luda_outputs_free(C.byref(self.out))


@dataclass(eq=False)
class SST:
    number: int
    ptr: int
    size: int
    smallest: bytes          # user keys
    largest: bytes
    n_entries: int
    owner: object = None     # _Owner or a torch tensor
    busy: str = ""           # "" idle, "upper" or "lower" input of a running job

    def release(self):
        if isinstance(self.owner, _Owner):
            self.owner.release()
        self.owner = None


@dataclass
class JobRecord:
    ticket: int
    level: int
    inputs: list
    bottommost: bool
    submitted: float
    stats: object = None
    in_bytes: int = 0
    out_bytes: int = 0
    extra: object = None     # an injected corrupt input (kept alive until the job ends)


@dataclass
class ServeReport:
    wall_s: float = 0.0
    jobs: int = 0
    failed: int = 0
    compaction_in_bytes: int = 0
    compaction_out_bytes: int = 0
    written_bytes: int = 0
    latencies_ms: list = field(default_factory=list)
    run_ms: list = field(default_factory=list)
    admit_wait_ms: list = field(default_factory=list)
    running_peak: int = 0
    budget_peak: int = 0
    stall_s: float = 0.0
    level_bytes: list = field(default_factory=list)
    flushes: int = 0
    retried: int = 0         # jobs started again after a failure
    kept_inputs: int = 0     # input tables whose records came from kept decoded runs

    def pct(self, p: float) -> float:
        if not self.latencies_ms:
            return 0.0
        v = sorted(self.latencies_ms)
        return v[min(len(v) - 1, int(p * len(v)))]


def _overlaps(a: SST, lo: bytes, hi: bytes) -> bool:
    return not (a.largest < lo or a.smallest > hi)


class LSM:
    def __init__(self, server: luda.Server, memtable_bytes: int = 64 * MiB, l0_trigger: int = 4,
                 l0_stop: int = 12, fanout: int = 10, target_file: int = 64 * MiB, block_size: int = 4096,
                 restart_interval: int = 16, bloom_bits_per_key: int = 10, value_pool_bytes: int = 256 * MiB,
                 seed: int = 5, on_complete=None, fault=None, keep_decoded: bool = False):
        import torch
        self.server = server
        self.fault = fault            # fault(job_index, level) -> True: corrupt that job
        self.submitted = 0
        self.fail_count = {}          # table numbers of a failed job -> failures in a row
        self.l0_trigger, self.l0_stop, self.fanout = l0_trigger, l0_stop, fanout
        self.l1_target = fanout * memtable_bytes
        self.levels = [[] for _ in range(N_LEVELS)]
        self.pointer = [b""] * N_LEVELS
        self.next_number = 1
        self.jobs = {}
        self.on_complete = on_complete
        self.fmt = (block_size, restart_interval, bloom_bits_per_key)
        # keep_decoded: flushes and compactions keep their tables' decoded runs on the device,
        # and a compaction whose inputs all have one skips decoding them (§III-D)
        self.build_opts = luda.options(block_size, restart_interval, bloom_bits_per_key, (1 << 64) - 1,
                                       flags=luda.F_KEEP_DECODED if keep_decoded else 0)
        self.report = ServeReport()
        g = torch.Generator(device="cuda")
        g.manual_seed(seed)
        # value bytes: slices of one random pool on the device (values are opaque to the method)
        self.pool = torch.randint(0, 256, (value_pool_bytes,), dtype=torch.uint8, device="cuda", generator=g)
        self.rng = np.random.default_rng(seed)

    # ---- tree ----------------------------------------------------------------------------
    def target(self, level: int) -> float:
        return self.l1_target * (self.fanout ** (level - 1))

    def level_bytes(self, level: int, idle_only: bool = False) -> int:
        return sum(t.size for t in self.levels[level] if not (idle_only and t.busy))

    def _insert(self, level: int, tables: list):
        if level == 0:
            self.levels[0].extend(tables)          # oldest first
        else:
            self.levels[level].extend(tables)
            self.levels[level].sort(key=lambda t: t.smallest)

    # ---- memtable flush ------------------------------------------------------------------
    def flush(self, mt: W.Memtable) -> SST:
        """Sort the memtable (user key ascending, sequence descending; the skiplist's order)
        and pack it into one level-0 table on the GPU."""
        import torch
        order = np.lexsort((~mt.seqs, mt.lo, mt.hi))
        km = np.empty((mt.n, 2), dtype=">u8")
        km[:, 0] = mt.hi[order]
        km[:, 1] = mt.lo[order]
        n = mt.n
        vbytes = n * mt.value_len
        off = int(self.rng.integers(0, (self.pool.numel() - vbytes) // 256 + 1)) * 256
        host = [km.view(np.uint8).reshape(-1), np.arange(n + 1, dtype=np.uint64) * np.uint64(16),
                mt.seqs[order], np.ones(n, np.uint8), None,
                np.arange(n + 1, dtype=np.uint64) * np.uint64(mt.value_len)]
        dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda(non_blocking=False) if a is not None else None
               for a in host]
        ra = luda.RunArrays(dev[0].data_ptr(), dev[1].data_ptr(), dev[2].data_ptr(), dev[3].data_ptr(),
                            self.pool.data_ptr() + off, dev[5].data_ptr(), n)
        o = luda.Options.from_buffer_copy(self.build_opts)
        o.stream = luda.current_stream()
        out = luda.Outputs()
        rc = luda.lib().luda_build_device(C.byref(ra), C.byref(o), C.byref(out))
        if rc != 0 or out.n_tables != 1:
            raise RuntimeError(f"memtable flush failed: {luda.strerror(rc)} {luda.last_error_detail()}")
        t = out.tables[0]
        sst = SST(self.next_number, t.data, t.size, C.string_at(t.smallest, t.smallest_len)[:-8],
                  C.string_at(t.largest, t.largest_len)[:-8], int(t.n_entries), _Owner(out, 1))
        self.next_number += 1
        self._insert(0, [sst])
        self.report.flushes += 1
        self.report.written_bytes += n * (16 + mt.value_len)
        return sst

    # ---- compaction picking --------------------------------------------------------------
    def _bottommost(self, out_level: int, lo: bytes, hi: bytes) -> bool:
        return not any(_overlaps(t, lo, hi) for lv in range(out_level + 1, N_LEVELS) for t in self.levels[lv])

    def _submit(self, level: int, upper: list, lower: list):
        inputs = upper + lower
        lo = min(t.smallest for t in inputs)
        hi = max(t.largest for t in inputs)
        for t in upper:
            t.busy = "upper"
        for t in lower:
            t.busy = "lower"
        bottom = self._bottommost(level + 1, lo, hi)
        extra = None
        if self.fault is not None and self.fault(self.submitted, level):
            extra = luda.device_bytes(inputs[0].ptr, inputs[0].size)
            extra[min(10, extra.numel() - 1)] ^= 0x40  # inside the first data block: its checksum fails
        self.submitted += 1
        pairs = ([(extra.data_ptr(), extra.numel())] if extra is not None else []) + [(t.ptr, t.size) for t in inputs]
        ticket = self.server.submit(pairs, W.MAX_SEQ, bottom, level + 1)
        rec = JobRecord(ticket, level, inputs, bottom, time.perf_counter(), in_bytes=sum(t.size for t in inputs),
                        extra=extra)
        self.jobs[ticket] = rec
        return rec

    def schedule(self) -> int:
        """Start every job the policy allows now; returns how many were started."""
        started = 0
        # level 0
        idle0 = [t for t in self.levels[0] if not t.busy]
        if len(self.levels[0]) >= self.l0_trigger and len(idle0) == len(self.levels[0]):
            lo = min(t.smallest for t in idle0)
            hi = max(t.largest for t in idle0)
            lower = [t for t in self.levels[1] if _overlaps(t, lo, hi)]
            if not any(t.busy for t in lower):
                self._submit(0, list(reversed(idle0)), lower)
                started += 1
        # levels 1..5
        for lv in range(1, N_LEVELS - 1):
            # tables already leaving this level (upper inputs of running jobs) do not count
            excess = sum(t.size for t in self.levels[lv] if t.busy != "upper") - self.target(lv)
            if excess <= 0:
                continue
            cand = [t for t in self.levels[lv] if not t.busy]
            # round robin from the compaction pointer
            cand.sort(key=lambda t: (t.smallest <= self.pointer[lv], t.smallest))
            for t in cand:
                if excess <= 0:
                    break
                lower = [u for u in self.levels[lv + 1] if _overlaps(u, t.smallest, t.largest)]
                if any(u.busy for u in lower):
                    continue
                self._submit(lv, [t], lower)
                self.pointer[lv] = t.largest
                excess -= t.size
                started += 1
        return started

    # ---- completion ----------------------------------------------------------------------
    def complete(self, ticket: int):
        rec = self.jobs.pop(ticket)
        out, stats = self.server.wait(ticket, copy_out=False)
        rec.stats = stats
        r = self.report
        r.jobs += 1
        r.latencies_ms.append(stats.latency_ms)
        r.run_ms.append(stats.run_ms)
        r.admit_wait_ms.append(stats.admit_wait_ms)
        r.compaction_in_bytes += rec.in_bytes
        rec.extra = None
        if out.status != 0:
            # all or nothing: the inputs stay in the tree and the policy starts the job again
            r.failed += 1
            for t in rec.inputs:
                t.busy = ""
            key = frozenset(t.number for t in rec.inputs)
            n = self.fail_count.get(key, 0) + 1
            self.fail_count[key] = n
            if n >= 3:
                raise RuntimeError(f"compaction job failed three times: {luda.strerror(out.status)}")
            r.retried += 1
            return
        self.fail_count.pop(frozenset(t.number for t in rec.inputs), None)
        if self.on_complete is not None:
            self.on_complete(rec, out)
        owner = _Owner(out, out.n_tables) if out.n_tables else None
        if owner is None:
            luda.lib().luda_outputs_free(C.byref(out))
        new = []
        for i in range(out.n_tables):
            t = out.tables[i]
            new.append(SST(self.next_number, t.data, t.size, C.string_at(t.smallest, t.smallest_len)[:-8],
                           C.string_at(t.largest, t.largest_len)[:-8], int(t.n_entries), owner))
            self.next_number += 1
            rec.out_bytes += t.size
        r.compaction_out_bytes += rec.out_bytes
        gone = set(id(t) for t in rec.inputs)
        for lv in (rec.level, rec.level + 1):
            self.levels[lv] = [t for t in self.levels[lv] if id(t) not in gone]
        for t in rec.inputs:
            t.release()
        self._insert(rec.level + 1, new)

    def close(self):
        for lv in self.levels:
            for t in lv:
                t.release()
            lv.clear()

    # ---- checkpoint ------------------------------------------------------------------------
    def snapshot(self, path: str) -> dict:
        """Write every table (its bytes, <number>.sst) and manifest.json to directory
        `path`; returns the manifest. Call with no job running."""
        if self.jobs:
            raise RuntimeError("snapshot with compaction jobs running")
        os.makedirs(path, exist_ok=True)
        levels = []
        for lv in self.levels:
            entries = []
            for t in lv:
                name = f"{t.number:06d}.sst"
                luda.device_bytes(t.ptr, t.size).cpu().numpy().tofile(os.path.join(path, name))
                entries.append({"number": t.number, "file": name, "size": t.size, "smallest": t.smallest.hex(),
                                "largest": t.largest.hex(), "n_entries": t.n_entries})
            levels.append(entries)
        manifest = {"levels": levels, "pointer": [p.hex() for p in self.pointer], "next_number": self.next_number,
                    "format": list(self.fmt), "l0_trigger": self.l0_trigger, "l0_stop": self.l0_stop,
                    "fanout": self.fanout, "l1_target": self.l1_target}
        tmp = os.path.join(path, "manifest.json.tmp")
        with open(tmp, "w") as f:
            json.dump(manifest, f, indent=1)
        os.replace(tmp, os.path.join(path, "manifest.json"))
        return manifest

    def restore(self, path: str) -> None:
        """Replace this (empty) tree with the one snapshot() wrote to `path`."""
        import torch
        if any(self.levels) or self.jobs:
            raise RuntimeError("restore into a tree that is not empty")
        with open(os.path.join(path, "manifest.json")) as f:
            m = json.load(f)
        if tuple(m["format"]) != tuple(self.fmt):
            raise ValueError(f"snapshot format {m['format']} differs from this tree's {list(self.fmt)}")
        for lv, entries in enumerate(m["levels"]):
            for e in entries:
                data = np.fromfile(os.path.join(path, e["file"]), dtype=np.uint8)
                if data.size != e["size"]:
                    raise ValueError(f"{e['file']}: {data.size} bytes, manifest says {e['size']}")
                dev = torch.from_numpy(data).cuda()
                self.levels[lv].append(SST(e["number"], dev.data_ptr(), int(e["size"]), bytes.fromhex(e["smallest"]),
                                           bytes.fromhex(e["largest"]), int(e["n_entries"]), dev))
        self.pointer = [bytes.fromhex(p) for p in m["pointer"]]
        self.next_number = int(m["next_number"])


def serve(stream, n_slots: int = 4, hbm_budget: int = 40 * 10**9, pace: bool = True, on_complete=None,
          lsm_kw: dict | None = None, before_close=None, prewarm_bytes: int = 0) -> ServeReport:
    """Feed a write stream (workloads.config5_stream) into a simulated LSM tree served by a
    luda.Server with `n_slots` slots: memtables are flushed when the stream time says they
    are full (wall clock, if `pace`), compactions start as soon as the policy allows and
    are installed as they complete. Returns latencies and byte counts; every submitted job
    has completed when it returns."""
    import torch
    kw = dict(lsm_kw or {})
    opts = luda.options(kw.get("block_size", 4096), kw.get("restart_interval", 16), kw.get("bloom_bits_per_key", 10),
                        kw.get("target_file", 64 * MiB),
                        flags=luda.F_KEEP_DECODED if kw.get("keep_decoded") else 0)
    server = luda.Server(n_slots, hbm_budget, opts, prewarm_bytes=prewarm_bytes)
    lsm = LSM(server, on_complete=on_complete, **kw)
    torch.cuda.synchronize()
    mts = list(stream)
    kept0 = luda.kept_inputs_used()
    t0 = time.perf_counter()
    k = 0
    try:
        while k < len(mts) or lsm.jobs:
            now = time.perf_counter() - t0
            if k < len(mts) and (not pace or now >= mts[k].t_full):
                if len(lsm.levels[0]) >= lsm.l0_stop:
                    if not lsm.jobs and not lsm.schedule():
                        raise RuntimeError("level 0 is full and no compaction can start")
                    ts = time.perf_counter()
                    ticket = server.next(-1)
                    lsm.report.stall_s += time.perf_counter() - ts
                    lsm.complete(ticket)
                    lsm.schedule()
                    continue
                lsm.flush(mts[k])
                torch.cuda.current_stream().synchronize()
                k += 1
                lsm.schedule()
                continue
            wait_ms = -1
            if k < len(mts):
                wait_ms = max(0, int((mts[k].t_full - now) * 1e3))
            ticket = server.next(wait_ms) if (lsm.jobs or wait_ms >= 0) else None
            if ticket is not None:
                lsm.complete(ticket)
                lsm.schedule()
        rep = lsm.report
        rep.wall_s = time.perf_counter() - t0
        rep.kept_inputs = luda.kept_inputs_used() - kept0
        st = server.stats()
        rep.running_peak, rep.budget_peak = int(st.running_peak), int(st.budget_peak)
        rep.level_bytes = [lsm.level_bytes(i) for i in range(N_LEVELS)]
        if before_close is not None:
            before_close(lsm)
        return rep
    finally:
        lsm.close()
        server.close()
