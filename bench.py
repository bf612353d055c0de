#!/usr/bin/env python
"""Benchmark: SSTable compaction throughput (compaction input MiB/s) on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--scale S]

One step = one full compaction job through libluda's C ABI: decode and verify every
input data block, merge, drop rule, block/file cut, encode with CRC trailers, bloom
filter, index/metaindex/footer of every new table. The workload is the large job: 4
overlapping 64 MiB L0 tables + 12 L1 tables (~1 GiB of input, 8-64 B keys sharing 0-24 B
prefixes, 1 KiB values, 10% overwrites, 3% deletions, 16 KiB blocks, restart interval 16,
10 bits/key bloom, 64 MiB target files), synthetic and seeded. Its input tables are built
on the GPU by the library's own table builder and stay resident in HBM; at 1 GiB they
are far larger than the 126 MB L2, so no flush is needed between steps.

`value` is device-resident input MiB/s over all ranks; `e2e` is the same metric through
luda_compact with pinned host buffers (host-to-device copy of the inputs and
device-to-host copy of the new tables inside the timed region). Multi-GPU is replicas
only: each rank compacts its own copy of the job; nothing is exchanged.

`--impl reference` times the CPU oracle (the plain single-threaded C compactor used by
the tests, pinned to one host core) on the same workload; it is the baseline arm.
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import os
import shutil
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MiB = float(1 << 20)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _max_over_ranks(values, ws):
    """Element-wise maximum of `values` over all ranks (an all-reduce on the process group
    the replicas share), or `values` themselves on one rank."""
    if ws <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6400.0)), "measured"
    return 6400.0, "fallback"


# ---- clocks during the timed region -------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append((time.time(), ln.strip()))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0: float, t1: float) -> dict:
        sm, mx, reasons = [], [], set()
        for ts, ln in self.lines:
            if not (t0 - 0.15 <= ts <= t1 + 0.15):
                continue
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"),
                                 parts[4:8]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# DRAM bytes (read + write) of one compaction call on the large job: all its kernels, and
# the kernels the roofline lists, from an ncu capture of one call of the same job at
# quarter scale (dram__bytes_read.sum + dram__bytes_write.sum per launch) times 4 (the
# traffic grows with the entries; profiles/dram_traffic_cfg3_quarter.md), with the SHA-256
# of the CUDA sources at the time: once a source changes the numbers no longer describe
# the call and the bench reports null.
_CALL_TRAFFIC = (4 * 1.0593e9, "f171ab9115b1b6f779606a52e994da5852aa9405bd6f4e1743bc4f254ab10a35")
_KERNEL_TRAFFIC = {"k_encode_stg": 4 * 475.8e6, "k_unpack": 4 * 268.0e6, "k_keys": 4 * 43.8e6}


def _sources_digest():
    import hashlib
    src = os.path.join(ROOT, "paper_2004_03054_b300", "csrc")
    h = hashlib.sha256()
    for f in sorted(os.listdir(src)):
        if f.endswith((".cu", ".cuh")):
            with open(os.path.join(src, f), "rb") as fh:
                h.update(f.encode() + b"\0" + fh.read())
    return h.hexdigest()


def _recorded_traffic(scale, kernel=None):
    try:
        digest = _sources_digest()
    except OSError:
        return None
    if digest != _CALL_TRAFFIC[1] or scale != 1.0:
        return None
    return _CALL_TRAFFIC[0] if kernel is None else _KERNEL_TRAFFIC.get(kernel)


# ---- our arm ------------------------------------------------------------------------------
def run_ours(args, ws, rank, local):
    import torch
    from paper_2004_03054_b300 import luda
    from paper_2004_03054_b300 import workloads as W

    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    L = luda.lib()
    # the clock sampler starts before the inputs are built, so that the GPU goes from the
    # input build straight into the warm-up steps (an idle GPU takes a while to come back
    # to full speed)
    props = torch.cuda.get_device_properties(local)
    uuid = getattr(props, "uuid", None)
    sampler = ClockSampler(f"GPU-{uuid}" if uuid else str(local))
    sampler.start()
    job = W.config3(seed=3, scale=args.scale)
    # inputs: the library's own builder packs each run into one table, kept on the device
    inputs = []
    for r in job.inputs:
        res = luda.build_device(r, luda.options(job.block_size, job.restart_interval, job.bloom_bits_per_key,
                                                (1 << 64) - 1))
        if res.status != 0 or len(res.tables) != 1:
            raise RuntimeError(f"input build failed: {res.status} {res.detail}")
        inputs.append(res.tables[0])
    in_bytes = sum(t.numel() for t in inputs)
    ins = (luda.Input * len(inputs))()
    for i, t in enumerate(inputs):
        ins[i].data, ins[i].size = t.data_ptr(), t.numel()
    stream = torch.cuda.current_stream()
    opts = luda.job_options(job, flags=luda.F_TRACE, stream=C.c_void_p(stream.cuda_stream))

    def step():
        out = luda.Outputs()
        rc = L.luda_compact_device(ins, len(inputs), job.level, job.smallest_snapshot, C.byref(opts),
                                   C.byref(out))
        if rc != 0:
            raise RuntimeError(f"compaction failed: {rc} {luda.last_error_detail()}")
        info = (sum(out.tables[i].size for i in range(out.n_tables)), out.n_tables, list(out.stage_ms),
                list(out.stage_bytes), int(out.n_in_entries), int(out.n_dropped))
        L.luda_outputs_free(C.byref(out))
        return info

    for _ in range(args.warmup):
        out_bytes, n_tables, *_ = step()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    l0 = luda.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.time()
    torch.cuda.nvtx.range_push("timed")
    e0.record(stream)
    stages, sbytes = [], []
    for _ in range(args.steps):
        out_bytes, n_tables, sm, sb, n_in, n_drop = step()
        stages.append(sm)
        sbytes.append(sb)
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    t1 = time.time()
    if ws > 1:
        torch.distributed.barrier()
    launches = luda.launch_count() - l0
    ms = e0.elapsed_time(e1) / args.steps
    ms = _max_over_ranks([ms], ws)[0]
    value = ws * in_bytes / MiB / (ms / 1e3)

    # roofline of the whole call: algorithmic bytes (every input table read once, every new
    # table written once) over the time per call; the kernels that take more than a tenth of
    # the call beside it, each with its own algorithmic bytes and its CUDA-event time (stage
    # events on the stream it runs on)
    peak, peak_kind = _peaks()
    avg = [statistics.mean(s[i] for s in stages) for i in range(8)]
    path_bytes = in_bytes + out_bytes
    path_gbs = path_bytes / (ms / 1e3) / 1e9
    kernels = []
    for name, idx, what in (("k_encode_stg", 5, "data blocks written + survivors' keys and values read"),
                            ("k_unpack (checksum pass, second stream, 56 SMs)", 1, "input data blocks read"),
                            ("k_keys", 2, "records and keys (latency-bound; key deltas and entry tables read)")):
        if avg[idx] <= 0 or avg[idx] < 0.1 * ms:
            continue
        b = sbytes[-1][idx]
        k = {"kernel": name, "ms_per_launch": round(avg[idx], 4), "share_of_call": round(avg[idx] / ms, 3),
             "traffic": _recorded_traffic(args.scale, name.split()[0])}
        if b:
            k.update({"bytes_per_launch": b, "algorithmic_bytes": what,
                      "achieved": round(b / (avg[idx] / 1e3) / 1e9, 1), "frac": round(b / (avg[idx] / 1e3) / 1e9 / peak, 4)})
        kernels.append(k)
    roofline = {"bound": "hbm", "scope": "whole compaction call (all kernels; input + output table bytes)",
                "achieved": round(path_gbs, 1), "peak": peak, "unit": "GB/s", "frac": round(path_gbs / peak, 4),
                "peak_source": f"{peak_kind} hbm_gbs", "bytes_per_call": path_bytes, "ms_per_call": round(ms, 4),
                "traffic": args.traffic if args.traffic is not None else _recorded_traffic(args.scale),
                "kernels": kernels}
    stage_names = ["sizing", "unpack_checksums", "keys", "sort", "gc_cut_layout", "encode", "meta", "device_span"]

    # end to end: luda_compact with pinned host inputs, new tables back in pinned host memory
    e2e = None
    if not args.no_e2e:
        host = [torch.empty(t.numel(), dtype=torch.uint8, pin_memory=True) for t in inputs]
        for h, t in zip(host, inputs):
            h.copy_(t)
        hins = (luda.Input * len(host))()
        for i, h in enumerate(host):
            hins[i].data, hins[i].size = h.data_ptr(), h.numel()
        hopts = luda.job_options(job, stream=C.c_void_p(stream.cuda_stream))
        d2h = 0

        def hstep():
            out = luda.Outputs()
            rc = L.luda_compact(hins, len(host), job.level, job.smallest_snapshot, C.byref(hopts), C.byref(out))
            if rc != 0:
                raise RuntimeError(f"host compaction failed: {rc} {luda.last_error_detail()}")
            n = sum(out.tables[i].size for i in range(out.n_tables))
            L.luda_outputs_free(C.byref(out))
            return n

        for _ in range(2):
            d2h = hstep()
        torch.cuda.synchronize()
        ke = max(3, args.steps // 10)
        ts = time.perf_counter()
        for _ in range(ke):
            d2h = hstep()
        torch.cuda.synchronize()
        te_single = (time.perf_counter() - ts) / ke
        # the same call with its transfers in one piece (one copy in, compaction, one copy out)
        hopts_one = luda.job_options(job, stream=C.c_void_p(stream.cuda_stream), tuning={"h2d_ranges": 1})
        hopts_ranged = hopts
        hopts = hopts_one
        hstep()
        torch.cuda.synchronize()
        ts = time.perf_counter()
        for _ in range(ke):
            hstep()
        torch.cuda.synchronize()
        te_one = (time.perf_counter() - ts) / ke
        hopts = hopts_ranged

        # the same jobs through a three-slot server (luda_server_submit_host), three jobs in
        # flight: one job's inputs go in while another computes and a third's tables come
        # out (the server lets one job at a time copy in each direction)
        depth = 3
        srv = luda.Server(depth, 1 << 46, luda.job_options(job))

        def pipelined(k):
            pending = []
            nbytes = 0
            for _ in range(k):
                pending.append(srv.submit(host, job.smallest_snapshot, job.bottommost, host=True))
                if len(pending) == depth:
                    out, _ = srv.wait(pending.pop(0), copy_out=False)
                    if out.status != 0:
                        raise RuntimeError(f"served host job failed: {out.status}")
                    nbytes = sum(out.tables[i].size for i in range(out.n_tables))
                    L.luda_outputs_free(C.byref(out))
            for t in pending:
                out, _ = srv.wait(t, copy_out=False)
                nbytes = sum(out.tables[i].size for i in range(out.n_tables))
                L.luda_outputs_free(C.byref(out))
            return nbytes

        pipelined(2 * depth)
        torch.cuda.synchronize()
        ts = time.perf_counter()
        d2h = pipelined(ke)
        torch.cuda.synchronize()
        te = (time.perf_counter() - ts) / ke
        srv.close()
        te, te_single, te_one = _max_over_ranks([te, te_single, te_one], ws)
        e2e = {"value": round(ws * in_bytes / MiB / te_single, 1), "unit": "MiB/s", "h2d_bytes_per_step": in_bytes,
               "d2h_bytes_per_step": d2h, "ms_per_step": round(te_single * 1e3, 3), "steps": ke,
               "api": "luda_compact (pinned host inputs in, new tables out to pinned host memory, one call at a time; "
                      "copies in and out overlapped by key ranges inside the call, default range count)",
               "one_piece": {"value": round(ws * in_bytes / MiB / te_one, 1), "unit": "MiB/s",
                             "ms_per_step": round(te_one * 1e3, 3), "steps": ke,
                             "api": "luda_compact with luda_tuning.h2d_ranges = 1 (copy in, compact, copy out)"},
               "pipelined": {"value": round(ws * in_bytes / MiB / te, 1), "unit": "MiB/s",
                             "ms_per_step": round(te * 1e3, 3), "steps": ke,
                             "api": f"luda_server_submit_host, {depth} slots, {depth} jobs in flight "
                                    "(one job's copies in and another's copies out overlap)"}}
    sampler.stop()
    clocks = sampler.summary(t0, t1)

    if rank != 0:
        return
    line = {
        "metric": "compaction input MiB/s (large job, device-resident inputs)",
        "value": round(value, 1), "unit": "MiB/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u8", "data": "synthetic (seeded, shaped like the paper's workloads)",
        "config": {"workload": "cfg3_large: 4 L0 + 12 L1 tables of 64 MiB, 8-64 B keys (0-24 B shared prefixes), "
                               "1 KiB values, 10% overwrites, 3% deletes, 16 KiB blocks, R=16, bpk=10, 64 MiB files",
                   "scale": args.scale, "input_bytes": in_bytes, "output_bytes": out_bytes, "tables_out": n_tables,
                   "entries_in": n_in, "entries_dropped": n_drop,
                   "l2": "inputs (1 GiB) larger than the 126 MB L2; no flush", "parallelism": f"replicas x{ws}"},
        "roofline": roofline,
        "stage_ms": {n: round(v, 4) for n, v in zip(stage_names, avg)},
        "gpu_launches": launches,
        "clocks": clocks,
        "e2e": e2e,
    }
    if not args.no_variants:
        line["variants"] = variants(job, inputs, in_bytes, stream, scale=args.scale)
    if not args.no_batched:
        line["batched"] = batched(args, stream)
    if not args.no_served:
        line["served"] = served(args)
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline(args)
        if "batched" in line:
            line["batched"]["cpu_baseline"] = batched_cpu_baseline(args)
    print(json.dumps(line), flush=True)


def variants(job, inputs, in_bytes, stream, scale=1.0, steps=5):
    """The same large job with the format variants (shortened index keys R9s, the 2 KiB
    filter array R10a, both, compressed output R4c) and as four range subcompactions (R13,
    split at the first user keys of the lower level's tables at its quartiles), and the
    same job shape with compressible values whose inputs are stored compressed (read, and
    read + written compressed): device ms per call (CUDA events around `steps` calls after
    two warm-up calls) and input MiB/s (stored input bytes)."""
    import torch
    from paper_2004_03054_b300 import luda
    from paper_2004_03054_b300 import workloads as W

    L = luda.lib()
    ins = (luda.Input * len(inputs))()
    for i, t in enumerate(inputs):
        ins[i].data, ins[i].size = t.data_ptr(), t.numel()
    lower = [r for r in job.inputs if r.level == max(x.level for x in job.inputs)]
    picks = sorted({len(lower) * k // 4 for k in (1, 2, 3)} - {0})
    bounds = [bytes(lower[i].ukeys[int(lower[i].ukoff[0]):int(lower[i].ukoff[1])]) for i in picks]
    bufs = [C.create_string_buffer(b, max(1, len(b))) for b in bounds]
    keys = (luda.Key * len(bounds))()
    for i, (b, buf) in enumerate(zip(bounds, bufs)):
        keys[i].data, keys[i].len = C.cast(buf, C.c_void_p), len(b)

    def timed(call):
        def once():
            out = luda.Outputs()
            rc = call(out)
            if rc != 0:
                raise RuntimeError(f"variant failed: {rc} {luda.last_error_detail()}")
            n = sum(out.tables[i].size for i in range(out.n_tables))
            L.luda_outputs_free(C.byref(out))
            return n
        for _ in range(2):
            once()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            nout = once()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        return {"ms_per_step": round(ms, 4), "value": round(in_bytes / MiB / (ms / 1e3), 1), "unit": "MiB/s",
                "output_bytes": nout}

    res = {}
    for name, flags in (("default", 0), ("short_index", luda.F_SHORT_INDEX), ("filter_array", luda.F_FILTER_ARRAY),
                        ("short_index+filter_array", luda.F_SHORT_INDEX | luda.F_FILTER_ARRAY),
                        ("compress_output", luda.F_COMPRESS)):
        o = luda.job_options(job, flags=flags, stream=C.c_void_p(stream.cuda_stream))
        res[name] = timed(lambda out, o=o: L.luda_compact_device(ins, len(inputs), job.level, job.smallest_snapshot,
                                                                 C.byref(o), C.byref(out)))
    o = luda.job_options(job, stream=C.c_void_p(stream.cuda_stream))
    res["subcompactions_4"] = timed(lambda out: L.luda_subcompact_device(ins, len(inputs), job.level,
                                                                         job.smallest_snapshot, keys, len(bounds),
                                                                         C.byref(o), C.byref(out)))
    res["subcompactions_4"]["bounds"] = "first user keys of the lower level's tables at its quartiles"
    res["compress_output"]["note"] = "random values: blocks are compressed, then kept raw (no eighth saved)"

    # LUDA_F_KEEP_DECODED: the job keeping its tables' decoded runs, and the same job when
    # every input table already has a kept run (the inputs built with the flag and kept
    # alive), which skips the footer, index, walk, checksum and key kernels
    kf = luda.F_KEEP_DECODED
    o = luda.job_options(job, flags=kf, stream=C.c_void_p(stream.cuda_stream))
    res["keep_outputs"] = timed(lambda out: L.luda_compact_device(ins, len(inputs), job.level, job.smallest_snapshot,
                                                                  C.byref(o), C.byref(out)))
    kouts, kins = [], (luda.Input * len(job.inputs))()
    for i, r in enumerate(job.inputs):
        ra, keep_arrays = luda._run_arrays(r, device=True)
        bo = luda.options(job.block_size, job.restart_interval, job.bloom_bits_per_key, (1 << 64) - 1, flags=kf,
                          stream=C.c_void_p(stream.cuda_stream))
        out = luda.Outputs()
        if L.luda_build_device(C.byref(ra), C.byref(bo), C.byref(out)) != 0 or out.n_tables != 1:
            raise RuntimeError(f"kept input build failed: {luda.last_error_detail()}")
        del keep_arrays
        kouts.append(out)
        kins[i].data, kins[i].size = out.tables[0].data, out.tables[0].size
    u0 = luda.kept_inputs_used()
    res["kept_inputs"] = timed(lambda out: L.luda_compact_device(kins, len(kouts), job.level, job.smallest_snapshot,
                                                                 C.byref(o), C.byref(out)))
    res["kept_inputs"]["inputs_from_kept_runs"] = luda.kept_inputs_used() - u0
    for out in kouts:
        L.luda_outputs_free(C.byref(out))

    # R4c on compressible data: the same job shape with values drawn from a word vocabulary
    # (about half compressible), its input tables built compressed on the device
    cjob = W.with_compressible_values(W.config3(seed=3, scale=scale))
    cins = []
    for r in cjob.inputs:
        b = luda.build_device(r, luda.options(cjob.block_size, cjob.restart_interval, cjob.bloom_bits_per_key,
                                              (1 << 64) - 1, flags=luda.F_COMPRESS))
        if b.status != 0 or len(b.tables) != 1:
            raise RuntimeError(f"compressed input build failed: {b.status} {b.detail}")
        cins.append(b.tables[0])
    del cjob
    cin = (luda.Input * len(cins))()
    for i, t in enumerate(cins):
        cin[i].data, cin[i].size = t.data_ptr(), t.numel()
    stored = sum(t.numel() for t in cins)
    for name, flags in (("compressed_inputs", 0), ("compressed_inputs+compress_output", luda.F_COMPRESS)):
        o = luda.job_options(job, flags=flags, stream=C.c_void_p(stream.cuda_stream))
        r = timed(lambda out, o=o: L.luda_compact_device(cin, len(cins), job.level, job.smallest_snapshot,
                                                         C.byref(o), C.byref(out)))
        r["value"] = round(stored / MiB / (r["ms_per_step"] / 1e3), 1)
        r["input_bytes_stored"] = stored
        r["workload"] = "cfg3_large shape, values from a 256-word vocabulary of 8-byte words, inputs stored compressed"
        res[name] = r
    return res


def batched(args, stream):
    """The batched workload: 256 independent jobs (per-job input lognormal 256 KiB-64 MiB,
    16-32 B keys, 32 B-4 KiB values, 4 KiB blocks, 2 MiB tables), run three ways on the
    same device-resident inputs: one luda_compact_device call per job (the plain per-job
    launch), one luda_batch_compact_device call for all jobs, and a plan (sized once,
    captured in one CUDA graph) replayed. Reports input MiB/s for each and, for the
    per-job launch, p50/p99 job latency."""
    import torch
    from paper_2004_03054_b300 import luda
    from paper_2004_03054_b300 import workloads as W

    L = luda.lib()
    jobs = W.config4(seed=4, scale=args.batch_scale, n_jobs=args.batch_jobs)
    o = jobs[0]
    dev_jobs = []
    for job in jobs:
        ins = []
        for r in job.inputs:
            res = luda.build_device(r, luda.options(o.block_size, o.restart_interval, o.bloom_bits_per_key,
                                                    (1 << 64) - 1))
            if res.status != 0 or len(res.tables) != 1:
                raise RuntimeError(f"input build failed: {res.status} {res.detail}")
            ins.append(res.tables[0])
        dev_jobs.append((ins, job.smallest_snapshot, job.bottommost))
    in_bytes = sum(t.numel() for ins, _, _ in dev_jobs for t in ins)
    opts = luda.options(o.block_size, o.restart_interval, o.bloom_bits_per_key, o.target_file_size,
                        stream=C.c_void_p(stream.cuda_stream))
    arrays = []
    for ins, _, _ in dev_jobs:
        a = (luda.Input * len(ins))()
        for i, t in enumerate(ins):
            a[i].data, a[i].size = t.data_ptr(), t.numel()
        arrays.append(a)

    def per_job(lat=None):
        for j, (ins, snap, bottom) in enumerate(dev_jobs):
            if lat is not None:
                ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ev[0].record(stream)
            out = luda.Outputs()
            jo = luda.Options.from_buffer_copy(opts)
            jo.bottommost = int(bool(bottom))
            rc = L.luda_compact_device(arrays[j], len(ins), o.level, snap, C.byref(jo), C.byref(out))
            if rc != 0:
                raise RuntimeError(f"job {j}: {rc} {luda.last_error_detail()}")
            L.luda_outputs_free(C.byref(out))
            if lat is not None:
                ev[1].record(stream)
                lat.append(ev)

    js, keep = luda._jobs_array(dev_jobs)
    outs = (luda.Outputs * len(dev_jobs))()

    def batch():
        rc = L.luda_batch_compact_device(js, len(dev_jobs), C.byref(opts), outs)
        if rc != 0:
            raise RuntimeError(f"batch: {rc} {luda.last_error_detail()}")
        for j in range(len(dev_jobs)):
            if outs[j].status != 0:
                raise RuntimeError(f"batch job {j}: {outs[j].status}")
            L.luda_outputs_free(C.byref(outs[j]))

    def timed(fn, k):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    k, w = args.batch_steps, max(1, args.batch_warmup)
    l0 = luda.launch_count()
    for _ in range(w):
        per_job()
    lat = []
    ms_job = timed(lambda: per_job(lat), k)
    lat_ms = sorted(a.elapsed_time(b) for a, b in lat)
    for _ in range(w):
        batch()
    ms_batch = timed(batch, k)
    def plan_leg(o):
        plan = luda.Plan(dev_jobs, o)
        for _ in range(w):
            plan.run(C.c_void_p(stream.cuda_stream))
        c0 = luda.launch_count()
        ms = timed(lambda: plan.run(C.c_void_p(stream.cuda_stream)), k)
        launches = (luda.launch_count() - c0) // k
        pouts = plan.outputs(copy_out=False)
        bad = [j for j in range(len(dev_jobs)) if pouts[j].status != 0]
        plan.close()
        if bad:
            raise RuntimeError(f"plan jobs failed: {bad[:5]}")
        return ms, launches

    ms_plan_default, _ = plan_leg(opts)
    tuned = None
    if not args.no_autotune:
        from paper_2004_03054_b300 import autotune as AT
        res = AT.tune(dev_jobs, opts, reps=3)
        tuned = {"tuning": res.tuning, "cache": res.cache, "candidates_timed": len(res.evaluated),
                 "search_s": round(res.seconds, 2), "tuner_best_ms": round(res.best_ms, 3),
                 "tuner_default_ms": round(res.default_ms, 3) if res.default_ms else None,
                 "method": "coordinate descent over luda_tuning; each candidate a plan timed by luda_autotune"}
        ms_plan, plan_launches = plan_leg(opts.with_tuning(res.tuning))
    else:
        ms_plan, plan_launches = plan_leg(opts)
    del keep

    def q(p):
        return round(lat_ms[min(len(lat_ms) - 1, int(p * len(lat_ms)))], 3)

    mib = in_bytes / MiB
    return {"workload": f"cfg4_batched: {len(dev_jobs)} jobs, input lognormal 256 KiB-64 MiB per job "
                        "(16-32 B keys, 32 B-4 KiB values, 4 KiB blocks, 2 MiB tables)",
            "jobs": len(dev_jobs), "input_bytes": in_bytes, "steps": k, "warmup": w,
            "per_job": {"value": round(mib / (ms_job / 1e3), 1), "unit": "MiB/s", "ms_per_step": round(ms_job, 3),
                        "job_latency_ms": {"p50": q(0.50), "p99": q(0.99), "max": round(lat_ms[-1], 3)}},
            "batch_call": {"value": round(mib / (ms_batch / 1e3), 1), "unit": "MiB/s",
                           "ms_per_step": round(ms_batch, 3)},
            "plan_replay": {"value": round(mib / (ms_plan / 1e3), 1), "unit": "MiB/s",
                            "ms_per_step": round(ms_plan, 3), "gpu_launches_per_replay": plan_launches,
                            "tuning": "autotuned" if tuned else "default"},
            "plan_replay_default_tuning": {"value": round(mib / (ms_plan_default / 1e3), 1), "unit": "MiB/s",
                                           "ms_per_step": round(ms_plan_default, 3)},
            "autotune": tuned,
            "gpu_launches_total": luda.launch_count() - l0}


def served(args):
    """The served workload: a simulated 7-level LSM tree (L0 trigger 4, fanout 10, 4 KiB
    blocks) fed by a seeded Poisson write stream (16 B keys, half uniform and half
    zipf(0.99), 256 B values). Compaction jobs go to a luda_server with continuous
    batching under a 40 GB HBM budget; the same stream is then served by a one-slot server
    (the plain per-job launch, first in first out). Two sizes: 64 MiB memtables and tables
    (the paper's table size, a few dozen jobs), and 4 MiB memtables and tables (hundreds of
    jobs, so that p99 is a percentile rather than the maximum). Reports compaction input
    MiB/s over the run's wall time and p50/p99 job latency."""
    from paper_2004_03054_b300 import lsm as L
    from paper_2004_03054_b300 import workloads as W

    def run(name, slots, n_memtables, table_bytes, seed, keep=False):
        stream = W.config5_stream(seed=seed, n_memtables=n_memtables, memtable_bytes=table_bytes,
                                  write_rate=args.serve_rate)
        rep = L.serve(stream, n_slots=slots, hbm_budget=40 * 10**9, pace=True, prewarm_bytes=16 << 30,
                      lsm_kw={"memtable_bytes": table_bytes, "target_file": table_bytes, "keep_decoded": keep})
        return {"slots": slots, "jobs": rep.jobs, "failed": rep.failed, "inputs_from_kept_runs": rep.kept_inputs,
                "value": round(rep.compaction_in_bytes / MiB / rep.wall_s, 1), "unit": "MiB/s",
                "wall_s": round(rep.wall_s, 3), "compaction_in_bytes": rep.compaction_in_bytes,
                "written_bytes": rep.written_bytes,
                "job_latency_ms": {"p50": round(rep.pct(0.5), 3), "p99": round(rep.pct(0.99), 3),
                                   "max": round(max(rep.latencies_ms, default=0), 3)},
                "admit_wait_ms_p99": round(sorted(rep.admit_wait_ms)[int(0.99 * (len(rep.admit_wait_ms) - 1))]
                                           if rep.admit_wait_ms else 0, 3),
                "running_peak": rep.running_peak, "budget_peak_bytes": rep.budget_peak,
                "write_stall_s": round(rep.stall_s, 3),
                "level_bytes": rep.level_bytes}

    out = {"workload": f"cfg5_served: {args.serve_memtables} memtables of 64 MiB, Poisson writes at "
                       f"{args.serve_rate:.0f}/s, 16 B keys (50% uniform, 50% zipf 0.99), 256 B values, "
                       "L0 trigger 4, fanout 10, 64 MiB tables, 40 GB budget"}
    for name, slots in (("continuous", args.serve_slots), ("per_job_fifo", 1)):
        out[name] = run(name, slots, args.serve_memtables, 64 * (1 << 20), 5)
    if args.serve_small_memtables:
        small = {"workload": f"cfg5_served with 4 MiB memtables and tables: {args.serve_small_memtables} memtables, "
                             f"the same stream shape and rate"}
        for name, slots in (("continuous", args.serve_slots), ("per_job_fifo", 1)):
            small[name] = run(name, slots, args.serve_small_memtables, 4 * (1 << 20), 6)
        # the same, every table keeping its decoded run (flushes and compactions)
        small["continuous_kept_runs"] = run("continuous_kept_runs", args.serve_slots, args.serve_small_memtables,
                                            4 * (1 << 20), 6, keep=True)
        out["tables_4mib"] = small
    return out


def cpu_baseline(args):
    """The oracle as it stands on the same job: three runs in a child process pinned to one
    host core (taskset -c 0, else sched_setaffinity), median of the three compaction times."""
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-baseline-child", "--cpu-scale", str(args.cpu_scale)]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    if shutil.which("taskset"):
        cmd = ["taskset", "-c", "0"] + cmd
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError(f"cpu baseline failed: {r.stderr[-2000:]}")
    return json.loads(r.stdout.strip().splitlines()[-1])


def _cpu_baseline_child(args):
    import oracle
    from paper_2004_03054_b300 import workloads as W
    try:
        os.sched_setaffinity(0, {sorted(os.sched_getaffinity(0))[0]})
    except (AttributeError, OSError):
        pass
    scale = args.cpu_scale
    job = W.config3(seed=3, scale=scale)
    ins = [oracle.build_tables(r, job.block_size, job.restart_interval, job.bloom_bits_per_key,
                               (1 << 64) - 1).tables[0].data for r in job.inputs]
    nbytes = sum(len(x) for x in ins)
    secs = []
    for _ in range(3):
        timing = {}
        res = oracle.compact(ins, job.smallest_snapshot, job.bottommost, job.block_size, job.restart_interval,
                             job.bloom_bits_per_key, job.target_file_size, timing=timing)
        if res.status != 0:
            raise RuntimeError("oracle failed")
        secs.append(timing["seconds"])
    sec = statistics.median(secs)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else 1
    print(json.dumps({"value": round(nbytes / MiB / sec, 2), "unit": "MiB/s", "cores": cores, "kind": "oracle",
                      "sample": f"cfg3 job at scale {scale} ({nbytes / MiB:.0f} MiB of input), median of 3 runs "
                                f"({', '.join(f'{x:.2f}' for x in secs)} s) on one pinned core",
                      "cpu": _cpu_model(), "host_cores": os.cpu_count()}), flush=True)


def _oracle_job_seconds(job):
    """Oracle builder for the job's inputs, then its compaction timed alone (one worker)."""
    import oracle
    ins = [oracle.build_tables(r, job.block_size, job.restart_interval, job.bloom_bits_per_key,
                               (1 << 64) - 1).tables[0].data for r in job.inputs]
    timing = {}
    res = oracle.compact(ins, job.smallest_snapshot, job.bottommost, job.block_size, job.restart_interval,
                         job.bloom_bits_per_key, job.target_file_size, timing=timing)
    if res.status != 0:
        raise RuntimeError("oracle failed")
    return sum(len(x) for x in ins), timing["seconds"]


def batched_cpu_baseline(args):
    """The batched workload's 256 jobs through the oracle, job-parallel over all host cores
    (a spawned process pool: this process has used the GPU). Each worker builds a job's
    inputs and times its compaction alone; the value is the input bytes over the busy time
    spread over the workers (sum of compaction seconds / workers)."""
    import multiprocessing as mp
    from paper_2004_03054_b300 import workloads as W
    jobs = W.config4(seed=4, scale=args.batch_scale, n_jobs=args.batch_jobs)
    workers = os.cpu_count() or 1
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(workers) as pool:
        res = pool.map(_oracle_job_seconds, jobs, chunksize=1)
    wall = time.perf_counter() - t0
    nbytes = sum(r[0] for r in res)
    busy = sum(r[1] for r in res)
    return {"value": round(nbytes / MiB / (busy / workers), 1), "unit": "MiB/s", "cores": workers,
            "kind": "oracle", "sample": f"all {len(jobs)} jobs ({nbytes / MiB:.0f} MiB), {busy:.1f} s of "
                                        f"compaction over {workers} workers ({wall:.1f} s wall with input builds)"}


def _cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


# ---- reference arm: the oracle ------------------------------------------------------------
def run_reference(args, ws, rank):
    if rank != 0:
        return
    import oracle
    from paper_2004_03054_b300 import workloads as W
    try:  # one host core, like the cpu baseline
        os.sched_setaffinity(0, {sorted(os.sched_getaffinity(0))[0]})
    except (AttributeError, OSError):
        pass
    scale = args.ref_scale
    job = W.config3(seed=3, scale=scale)
    ins = [oracle.build_tables(r, job.block_size, job.restart_interval, job.bloom_bits_per_key,
                               (1 << 64) - 1).tables[0].data for r in job.inputs]
    nbytes = sum(len(x) for x in ins)

    def step():
        timing = {}
        res = oracle.compact(ins, job.smallest_snapshot, job.bottommost, job.block_size, job.restart_interval,
                             job.bloom_bits_per_key, job.target_file_size, timing=timing)
        if res.status != 0:
            raise RuntimeError("oracle failed")
        return timing["seconds"]

    for _ in range(args.warmup):
        step()
    secs = [step() for _ in range(args.steps)]
    sec = sum(secs) / len(secs)
    value = nbytes / MiB / sec
    sample = f"cfg3 job at scale {scale} ({nbytes / MiB:.0f} MiB of input) per step"
    line = {"impl": "reference", "metric": "compaction input MiB/s (large job, device-resident inputs)",
            "value": round(value, 2), "unit": "MiB/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(sec * 1e3, 2), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u8", "data": "synthetic (seeded, shaped like the paper's workloads)",
            "config": {"workload": "cfg3_large: 4 L0 + 12 L1 tables of 64 MiB, 8-64 B keys (0-24 B shared prefixes), "
                                   "1 KiB values, 10% overwrites, 3% deletes, 16 KiB blocks, R=16, bpk=10, 64 MiB files"
                                   + ("" if scale == 1.0 else f" (bounded sample at scale {scale})"),
                       "scale": scale, "input_bytes": nbytes},
            "cpu_baseline": {"value": round(value, 2), "unit": "MiB/s", "cores": 1, "kind": "oracle",
                             "sample": sample, "cpu": _cpu_model()},
            "e2e": {"value": round(value, 2), "unit": "MiB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--cpu-scale", type=float, default=1.0)
    ap.add_argument("--ref-scale", type=float, default=1.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="batched leg: plan with the default launch shapes")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--no-variants", action="store_true", help="skip the format-variant and subcompaction timings")
    ap.add_argument("--serve-memtables", type=int, default=40)
    ap.add_argument("--serve-rate", type=float, default=8e6, help="writes per second of the served stream")
    ap.add_argument("--serve-slots", type=int, default=6)
    ap.add_argument("--serve-small-memtables", type=int, default=400,
                    help="memtables of the 4 MiB served run (0: skip it)")
    ap.add_argument("--batch-jobs", type=int, default=256)
    ap.add_argument("--batch-scale", type=float, default=1.0)
    ap.add_argument("--batch-steps", type=int, default=5)
    ap.add_argument("--batch-warmup", type=int, default=3)
    ap.add_argument("--traffic", type=float, default=None,
                    help="dram bytes per launch of the dominant kernel from an ncu capture (default: the "
                         "recorded capture while the encoder's source is unchanged)")
    ap.add_argument("--cpu-baseline-child", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.cpu_baseline_child:
        _cpu_baseline_child(args)
        return
    ws, rank, local = _dist()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
