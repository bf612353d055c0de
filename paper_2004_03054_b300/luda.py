"""ctypes binding of libluda.so (argument marshalling only; every step runs in the
library's CUDA kernels).

The library must have been built (``python -m paper_2004_03054_b300.build``); loading
fails loudly otherwise. PyTorch is used for device memory and the current stream only.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libluda.so")

OK = 0
ERR_INVALID_ARG = -1
ERR_CORRUPTION = -2
ERR_NOT_SUPPORTED = -3
ERR_OOM = -4
ERR_CUDA = -5
ERR_TIMEOUT = -6
ERR_DUPLICATE_KEY = -7
ERR_PLAN_MISMATCH = -8
F_STRICT_DUP = 1
F_TRACE = 2
F_SHORT_INDEX = 4  # shortened index keys (format variant R9s)
F_FILTER_ARRAY = 8  # one bloom filter per 2 KiB of data block offsets (format variant R10a)
F_COMPRESS = 16  # data blocks written compressed when that saves an eighth (format variant R4c)
F_TEST_WAIT0 = 32  # test only: the encoder's copy-slot waits give up at once (LUDA_ERR_TIMEOUT, no tables)
F_KEEP_DECODED = 64  # keep the new tables' decoded runs on the device; take kept runs for inputs (§III-D)
MAX_SEQ = (1 << 56) - 1


class Input(C.Structure):
    _fields_ = [("data", C.c_void_p), ("size", C.c_uint64), ("level", C.c_int32), ("file_number", C.c_uint64)]


class Tuning(C.Structure):
    """luda_tuning: launch shapes (0 = default); they never change the output bytes."""
    _fields_ = [("merge_tile", C.c_uint32), ("merge_ctas_per_sm", C.c_uint32), ("decode_warps", C.c_uint32),
                ("walk_threads", C.c_uint32), ("encode_ctas_per_sm", C.c_uint32), ("elem_threads", C.c_uint32),
                ("crc_ctas", C.c_uint32), ("crc_warps", C.c_uint32),
                ("h2d_ranges", C.c_uint32)]
    KNOBS = ("merge_tile", "merge_ctas_per_sm", "decode_warps", "walk_threads", "encode_ctas_per_sm",
             "elem_threads", "crc_ctas", "crc_warps", "h2d_ranges")

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k in self.KNOBS}

    @classmethod
    def of(cls, d: dict) -> "Tuning":
        t = cls()
        for k, v in d.items():
            setattr(t, k, int(v))
        return t


class Options(C.Structure):
    _fields_ = [("block_size", C.c_uint32), ("restart_interval", C.c_uint32), ("bloom_bits_per_key", C.c_uint32),
                ("target_file_size", C.c_uint64), ("bottommost", C.c_int32), ("flags", C.c_uint32),
                ("dev_alloc", C.c_void_p), ("dev_free", C.c_void_p), ("alloc_ctx", C.c_void_p),
                ("stream", C.c_void_p), ("tuning", C.POINTER(Tuning))]

    def with_tuning(self, t: "Tuning | dict | None") -> "Options":
        """A copy of these options with launch shapes t (None: defaults); the copy keeps t alive."""
        o = Options.from_buffer_copy(self)
        if isinstance(t, dict):
            t = Tuning.of(t)
        o._tuning_ref = t
        o.tuning = C.pointer(t) if t is not None else None
        return o


class Table(C.Structure):
    _fields_ = [("data", C.c_void_p), ("size", C.c_uint64), ("n_entries", C.c_uint64),
                ("smallest", C.c_void_p), ("smallest_len", C.c_uint32),
                ("largest", C.c_void_p), ("largest_len", C.c_uint32)]


class Outputs(C.Structure):
    _fields_ = [("tables", C.POINTER(Table)), ("n_tables", C.c_uint32), ("status", C.c_int32),
                ("n_in_entries", C.c_uint64), ("n_dropped", C.c_uint64), ("ms_h2d", C.c_double),
                ("ms_device", C.c_double), ("ms_d2h", C.c_double), ("stage_ms", C.c_double * 8),
                ("stage_bytes", C.c_uint64 * 8), ("_priv", C.c_void_p)]


class Job(C.Structure):
    _fields_ = [("inputs", C.POINTER(Input)), ("n_inputs", C.c_uint32), ("level", C.c_int32),
                ("smallest_snapshot", C.c_uint64), ("bottommost", C.c_int32),
                ("range_lo", C.c_void_p), ("range_lo_len", C.c_uint32),
                ("range_hi", C.c_void_p), ("range_hi_len", C.c_uint32)]


class Key(C.Structure):
    _fields_ = [("data", C.c_void_p), ("len", C.c_uint32)]


class ServerConfig(C.Structure):
    _fields_ = [("n_slots", C.c_uint32), ("hbm_budget", C.c_uint64), ("opts", Options),
                ("prewarm_bytes", C.c_uint64)]


class JobStats(C.Structure):
    _fields_ = [("queue_ms", C.c_double), ("admit_wait_ms", C.c_double), ("run_ms", C.c_double),
                ("latency_ms", C.c_double), ("reserved_bytes", C.c_uint64), ("input_bytes", C.c_uint64),
                ("slot", C.c_uint32), ("running_at_admit", C.c_uint32)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("failed", C.c_uint64),
                ("budget_peak", C.c_uint64), ("running_peak", C.c_uint32), ("pad", C.c_uint32)]


class TableCheck(C.Structure):
    _fields_ = [("status", C.c_int32), ("n_blocks", C.c_uint32), ("n_entries", C.c_uint64),
                ("data_bytes", C.c_uint64), ("bad_offset", C.c_uint64)]


class RunArrays(C.Structure):
    _fields_ = [("ukeys", C.c_void_p), ("ukoff", C.c_void_p), ("seqs", C.c_void_p), ("types", C.c_void_p),
                ("vals", C.c_void_p), ("voff", C.c_void_p), ("n", C.c_uint64)]


_lib = None


def lib():
    """Load libluda.so; raises if it is missing (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"libluda.so not built ({_LIB_PATH}); run python -m paper_2004_03054_b300.build")
        L = C.CDLL(_LIB_PATH)
        st = C.c_int
        L.luda_options_default.argtypes = [C.POINTER(Options)]
        L.luda_compact.restype = st
        L.luda_compact.argtypes = [C.POINTER(Input), C.c_uint32, C.c_int32, C.c_uint64, C.POINTER(Options),
                                   C.POINTER(Outputs)]
        L.luda_compact_device.restype = st
        L.luda_compact_device.argtypes = L.luda_compact.argtypes
        L.luda_batch_compact_device.restype = st
        L.luda_batch_compact_device.argtypes = [C.POINTER(Job), C.c_uint32, C.POINTER(Options), C.POINTER(Outputs)]
        L.luda_batch_compact.restype = st
        L.luda_batch_compact.argtypes = L.luda_batch_compact_device.argtypes
        L.luda_build.restype = st
        L.luda_build.argtypes = [C.POINTER(RunArrays), C.POINTER(Options), C.POINTER(Outputs)]
        L.luda_build_device.restype = st
        L.luda_build_device.argtypes = L.luda_build.argtypes
        L.luda_outputs_free.argtypes = [C.POINTER(Outputs)]
        L.luda_strerror.restype = C.c_char_p
        L.luda_strerror.argtypes = [C.c_int]
        L.luda_last_error_detail.restype = C.c_char_p
        L.luda_version.restype = C.c_char_p
        L.luda_launch_count.restype = C.c_uint64
        L.luda_kept_inputs_used.restype = C.c_uint64
        L.luda_check_table_noalloc.restype = st
        L.luda_check_table_noalloc.argtypes = [C.c_void_p, C.c_uint64, C.c_void_p, C.POINTER(TableCheck)]
        for name in ("luda_plan_create", "luda_plan_run", "luda_plan_outputs"):
            getattr(L, name).restype = st
        L.luda_plan_create.argtypes = [C.POINTER(Job), C.c_uint32, C.POINTER(Options), C.POINTER(C.c_void_p)]
        L.luda_plan_run.argtypes = [C.c_void_p, C.c_void_p]
        L.luda_plan_outputs.argtypes = [C.c_void_p, C.POINTER(Outputs)]
        L.luda_plan_destroy.argtypes = [C.c_void_p]
        L.luda_plan_destroy.restype = None
        L.luda_tuning_default.argtypes = [C.POINTER(Tuning)]
        L.luda_tuning_default.restype = None
        L.luda_tuning_check.argtypes = [C.POINTER(Tuning)]
        L.luda_tuning_check.restype = st
        L.luda_autotune.argtypes = [C.POINTER(Job), C.c_uint32, C.POINTER(Options), C.POINTER(Tuning), C.c_uint32,
                                    C.c_uint32, C.POINTER(C.c_double), C.POINTER(C.c_uint32)]
        L.luda_autotune.restype = st
        L.luda_subcompact_device.restype = st
        L.luda_subcompact_device.argtypes = [C.POINTER(Input), C.c_uint32, C.c_int32, C.c_uint64, C.POINTER(Key),
                                             C.c_uint32, C.POINTER(Options), C.POINTER(Outputs)]
        L.luda_server_create.restype = st
        L.luda_server_create.argtypes = [C.POINTER(ServerConfig), C.POINTER(C.c_void_p)]
        L.luda_server_submit.restype = st
        L.luda_server_submit.argtypes = [C.c_void_p, C.POINTER(Job), C.POINTER(C.c_uint64)]
        L.luda_server_submit_host.restype = st
        L.luda_server_submit_host.argtypes = [C.c_void_p, C.POINTER(Job), C.POINTER(C.c_uint64)]
        L.luda_server_next.restype = st
        L.luda_server_next.argtypes = [C.c_void_p, C.c_int64, C.POINTER(C.c_uint64)]
        L.luda_server_wait.restype = st
        L.luda_server_wait.argtypes = [C.c_void_p, C.c_uint64, C.c_int64, C.POINTER(Outputs), C.POINTER(JobStats)]
        L.luda_server_stats_get.restype = st
        L.luda_server_stats_get.argtypes = [C.c_void_p, C.POINTER(ServerStats)]
        L.luda_server_destroy.restype = None
        L.luda_server_destroy.argtypes = [C.c_void_p]
        _lib = L
    return _lib


def options(block_size=4096, restart_interval=16, bloom_bits_per_key=10, target_file_size=2 << 20,
            bottommost=False, flags=0, stream=None, tuning=None) -> Options:
    o = Options()
    lib().luda_options_default(C.byref(o))
    o.block_size, o.restart_interval, o.bloom_bits_per_key = block_size, restart_interval, bloom_bits_per_key
    o.target_file_size, o.bottommost, o.flags = target_file_size, int(bool(bottommost)), flags
    o.stream = stream
    return o.with_tuning(tuning) if tuning is not None else o


def job_options(job, **kw) -> Options:
    """Options of a workloads.Job."""
    return options(job.block_size, job.restart_interval, job.bloom_bits_per_key, job.target_file_size,
                   job.bottommost, **kw)


def launch_count() -> int:
    """Kernels libluda has launched in this process."""
    return int(lib().luda_launch_count())


def kept_inputs_used() -> int:
    """Input tables whose records came from kept decoded runs in this process."""
    return int(lib().luda_kept_inputs_used())


def strerror(s: int) -> str:
    return lib().luda_strerror(s).decode()


def last_error_detail() -> str:
    return lib().luda_last_error_detail().decode(errors="replace")


def current_stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


@dataclass
class Result:
    status: int
    tables: list = field(default_factory=list)      # bytes (host) or torch uint8 tensors (device)
    smallest: list = field(default_factory=list)
    largest: list = field(default_factory=list)
    n_entries: list = field(default_factory=list)
    n_in_entries: int = 0
    n_dropped: int = 0
    ms_h2d: float = 0.0
    ms_device: float = 0.0
    ms_d2h: float = 0.0
    stage_ms: list = field(default_factory=list)
    stage_bytes: list = field(default_factory=list)
    detail: str = ""


class _CudaView:
    """Exposes a device byte range through __cuda_array_interface__ (zero copy)."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "|u1", "data": (ptr, False), "version": 3,
                                         "strides": None}


def device_bytes(ptr: int, n: int):
    """A torch uint8 CUDA tensor copy of n bytes at device address ptr."""
    import torch
    if n == 0:
        return torch.empty(0, dtype=torch.uint8, device="cuda")
    return torch.as_tensor(_CudaView(ptr, n), device="cuda").clone()


def _take(rc: int, out: Outputs, device: bool) -> Result:
    res = Result(int(out.status) if rc == OK else rc, detail=last_error_detail() if rc or out.status else "")
    res.n_in_entries, res.n_dropped = int(out.n_in_entries), int(out.n_dropped)
    res.ms_h2d, res.ms_device, res.ms_d2h = out.ms_h2d, out.ms_device, out.ms_d2h
    res.stage_ms, res.stage_bytes = list(out.stage_ms), [int(x) for x in out.stage_bytes]
    if rc == OK and out.status == OK:
        for i in range(out.n_tables):
            t = out.tables[i]
            if device:
                res.tables.append(device_bytes(t.data, t.size))
            else:
                res.tables.append(C.string_at(t.data, t.size))
            res.smallest.append(C.string_at(t.smallest, t.smallest_len))
            res.largest.append(C.string_at(t.largest, t.largest_len))
            res.n_entries.append(int(t.n_entries))
    lib().luda_outputs_free(C.byref(out))
    return res


def _u8(b) -> np.ndarray:
    if isinstance(b, np.ndarray):
        return np.ascontiguousarray(b, dtype=np.uint8)
    return np.frombuffer(bytes(b), dtype=np.uint8)


def compact(inputs, smallest_snapshot: int = MAX_SEQ, level: int = 1, opts: Options | None = None) -> Result:
    """Host entry point: inputs are host byte strings / uint8 arrays (listed newest first)."""
    arrs = [_u8(x) for x in inputs]
    ins = (Input * max(1, len(arrs)))()
    for i, a in enumerate(arrs):
        ins[i].data, ins[i].size = a.ctypes.data, len(a)
    o = opts or options()
    out = Outputs()
    rc = lib().luda_compact(ins, len(arrs), level, smallest_snapshot, C.byref(o), C.byref(out))
    return _take(rc, out, device=False)


def compact_device(inputs, smallest_snapshot: int = MAX_SEQ, level: int = 1, opts: Options | None = None,
                   copy_out: bool = True):
    """Device entry point: inputs are torch uint8 CUDA tensors. Returns a Result whose
    tables are torch CUDA tensors (copies); with copy_out=False returns (rc, Outputs) and
    the caller must call free_outputs."""
    ins = (Input * max(1, len(inputs)))()
    for i, t in enumerate(inputs):
        ins[i].data, ins[i].size = t.data_ptr(), t.numel()
    o = opts or options()
    if o.stream is None:
        o.stream = current_stream()
    out = Outputs()
    rc = lib().luda_compact_device(ins, len(inputs), level, smallest_snapshot, C.byref(o), C.byref(out))
    if not copy_out:
        return rc, out
    return _take(rc, out, device=True)


def free_outputs(out: Outputs) -> None:
    lib().luda_outputs_free(C.byref(out))


def batch_compact_device(jobs, opts: Options | None = None, copy_out: bool = True):
    """jobs: list of (inputs: [torch CUDA uint8 tensors], smallest_snapshot, bottommost)."""
    js, keep = _jobs_array(jobs)
    o = opts or options()
    if o.stream is None:
        o.stream = current_stream()
    outs = (Outputs * max(1, len(jobs)))()
    rc = lib().luda_batch_compact_device(js, len(jobs), C.byref(o), outs)
    del keep
    if not copy_out:
        return rc, outs
    return rc, [_take(rc, outs[j], device=True) for j in range(len(jobs))]


def batch_compact(jobs, opts: Options | None = None):
    """luda_batch_compact: jobs as for batch_compact_device, but each job's inputs are host
    byte strings / uint8 arrays. Returns (rc, [Result]) with host tables."""
    js, keep = _jobs_array(jobs)
    o = opts or options()
    outs = (Outputs * max(1, len(jobs)))()
    rc = lib().luda_batch_compact(js, len(jobs), C.byref(o), outs)
    del keep
    return rc, [_take(rc, outs[j], device=False) for j in range(len(jobs))]


def subcompact_device(inputs, bounds, smallest_snapshot: int = MAX_SEQ, level: int = 1,
                      opts: Options | None = None, copy_out: bool = True):
    """R13 subcompactions of one job (inputs: torch uint8 CUDA tensors) at the strictly
    increasing user keys `bounds`: one Result with the ranges' tables in key order."""
    ins = (Input * max(1, len(inputs)))()
    for i, t in enumerate(inputs):
        ins[i].data, ins[i].size = t.data_ptr(), t.numel()
    bufs = [C.create_string_buffer(bytes(b), max(1, len(b))) for b in bounds]
    keys = (Key * max(1, len(bounds)))()
    for i, (b, buf) in enumerate(zip(bounds, bufs)):
        keys[i].data, keys[i].len = C.cast(buf, C.c_void_p), len(b)
    o = Options.from_buffer_copy(opts or options())
    if o.stream is None:
        o.stream = current_stream()
    out = Outputs()
    rc = lib().luda_subcompact_device(ins, len(inputs), level, smallest_snapshot, keys, len(bounds), C.byref(o),
                                      C.byref(out))
    if not copy_out:
        return rc, out
    return _take(rc, out, device=True)


def _jobs_array(jobs):
    """jobs: list of (inputs: [torch CUDA uint8 tensors], smallest_snapshot, bottommost), or
    of (inputs, smallest_snapshot, bottommost, lo, hi) for ranged jobs (R13; bytes or None)."""
    keep = []
    js = (Job * max(1, len(jobs)))()
    for j, job in enumerate(jobs):
        inputs, snap, bottom = job[:3]
        lo, hi = (job[3], job[4]) if len(job) > 3 else (None, None)
        ins = (Input * max(1, len(inputs)))()
        for i, t in enumerate(inputs):
            if hasattr(t, "data_ptr"):
                ins[i].data, ins[i].size = t.data_ptr(), t.numel()
            else:  # host bytes (luda_batch_compact)
                a = _u8(t)
                keep.append(a)
                ins[i].data, ins[i].size = a.ctypes.data, len(a)
        keep.append(ins)
        js[j].inputs = C.cast(ins, C.POINTER(Input))
        js[j].n_inputs, js[j].smallest_snapshot, js[j].bottommost = len(inputs), snap, int(bool(bottom))
        for name, key in (("lo", lo), ("hi", hi)):
            if key is not None:
                buf = C.create_string_buffer(bytes(key), max(1, len(key)))
                keep.append(buf)
                setattr(js[j], "range_" + name, C.cast(buf, C.c_void_p))
                setattr(js[j], "range_" + name + "_len", len(key))
    return js, keep


class Plan:
    """A batch of jobs sized once and captured in a CUDA graph (luda_plan_*). The input
    tensors must stay alive and unchanged in size while the plan exists."""

    def __init__(self, jobs, opts: Options | None = None):
        self._js, self._keep = _jobs_array(jobs)
        self._inputs = [t for job in jobs for t in job[0]]
        self.n_jobs = len(jobs)
        self.opts = opts or options()
        self.handle = C.c_void_p()
        rc = lib().luda_plan_create(self._js, len(jobs), C.byref(self.opts), C.byref(self.handle))
        if rc != OK:
            raise RuntimeError(f"luda_plan_create: {strerror(rc)}: {last_error_detail()}")

    def run(self, stream=None) -> None:
        rc = lib().luda_plan_run(self.handle, stream if stream is not None else current_stream())
        if rc != OK:
            raise RuntimeError(f"luda_plan_run: {strerror(rc)}: {last_error_detail()}")

    def outputs(self, copy_out: bool = True):
        outs = (Outputs * max(1, self.n_jobs))()
        rc = lib().luda_plan_outputs(self.handle, outs)
        if rc != OK:
            raise RuntimeError(f"luda_plan_outputs: {strerror(rc)}: {last_error_detail()}")
        if not copy_out:
            return outs
        return [_take(OK, outs[j], device=True) for j in range(self.n_jobs)]

    def close(self) -> None:
        if self.handle:
            lib().luda_plan_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous batching of compaction jobs (luda_server_*): up to n_slots jobs run at
    once, each on its own stream, admitted under an HBM budget. Input tables are CUDA
    uint8 tensors (or (device pointer, size) pairs) that must stay alive until their job
    completes; the server keeps a reference to tensors until the job is collected."""

    def __init__(self, n_slots: int, hbm_budget: int, opts: Options | None = None, prewarm_bytes: int = 0):
        cfg = ServerConfig()
        cfg.n_slots, cfg.hbm_budget, cfg.prewarm_bytes = n_slots, hbm_budget, prewarm_bytes
        cfg.opts = opts or options()
        self.handle = C.c_void_p()
        rc = lib().luda_server_create(C.byref(cfg), C.byref(self.handle))
        if rc != OK:
            raise RuntimeError(f"luda_server_create: {strerror(rc)}: {last_error_detail()}")
        self._keep = {}

    def submit(self, inputs, smallest_snapshot: int = MAX_SEQ, bottommost: bool = False, level: int = 1,
               host: bool = False) -> int:
        """inputs: CUDA uint8 tensors or (device pointer, size) pairs; with host=True, host
        tensors (pinned for the fastest copies), numpy uint8 arrays or (host pointer, size)
        pairs, and the job's tables come back in host memory."""
        ins = (Input * max(1, len(inputs)))()
        for i, t in enumerate(inputs):
            if isinstance(t, tuple):
                ins[i].data, ins[i].size = t
            elif isinstance(t, np.ndarray):
                ins[i].data, ins[i].size = t.ctypes.data, t.nbytes
            else:
                ins[i].data, ins[i].size = t.data_ptr(), t.numel()
        job = Job()
        job.inputs = C.cast(ins, C.POINTER(Input))
        job.n_inputs, job.level = len(inputs), level
        job.smallest_snapshot, job.bottommost = smallest_snapshot, int(bool(bottommost))
        ticket = C.c_uint64()
        fn = lib().luda_server_submit_host if host else lib().luda_server_submit
        rc = fn(self.handle, C.byref(job), C.byref(ticket))
        if rc != OK:
            raise RuntimeError(f"luda_server_submit: {strerror(rc)}: {last_error_detail()}")
        self._keep[ticket.value] = (list(inputs), host)
        return ticket.value

    def next(self, timeout_ms: int = -1):
        """Ticket of a completed, not yet announced job, or None on timeout."""
        t = C.c_uint64()
        rc = lib().luda_server_next(self.handle, timeout_ms, C.byref(t))
        if rc == ERR_TIMEOUT:
            return None
        if rc != OK:
            raise RuntimeError(f"luda_server_next: {strerror(rc)}")
        return t.value

    def wait(self, ticket: int, timeout_ms: int = -1, copy_out: bool = True):
        """(Result or raw Outputs, JobStats) of a job; the ticket is then gone."""
        if ticket not in self._keep:
            raise KeyError(f"unknown or already collected ticket {ticket}")
        out, stats = Outputs(), JobStats()
        rc = lib().luda_server_wait(self.handle, ticket, timeout_ms, C.byref(out), C.byref(stats))
        if rc == ERR_TIMEOUT:
            raise TimeoutError(f"ticket {ticket} not done")
        _, host = self._keep.pop(ticket, (None, False))
        if not copy_out:
            out.status = rc
            return out, stats
        return _take(rc, out, device=not host), stats

    def stats(self) -> ServerStats:
        st = ServerStats()
        lib().luda_server_stats_get(self.handle, C.byref(st))
        return st

    def close(self) -> None:
        if self.handle:
            lib().luda_server_destroy(self.handle)
            self.handle = C.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _run_arrays(run, device: bool):
    # an empty array (no key or value bytes at all) still gets a buffer: the C ABI wants
    # every array of a non-empty run non-NULL, and reads none of its bytes
    arrs = [np.ascontiguousarray(a) if np.asarray(a).size else np.zeros(1, np.asarray(a).dtype)
            for a in (run.ukeys, run.ukoff, run.seqs, run.types, run.vals, run.voff)]
    if device:
        import torch
        keep = [torch.from_numpy(a).cuda() for a in arrs]
        ptrs = [t.data_ptr() for t in keep]
    else:
        keep = arrs
        ptrs = [a.ctypes.data for a in keep]
    ra = RunArrays(*ptrs, run.n)
    return ra, keep


def check_table_noalloc(table, stream=None) -> TableCheck:
    """Check one table (torch uint8 CUDA tensor) with the entry point that allocates no
    device memory; returns the filled luda_table_check. The call runs with the tensor's
    device current (on that device's current stream unless `stream` is given)."""
    import torch
    if not isinstance(table, torch.Tensor) or not table.is_cuda:
        raise TypeError("check_table_noalloc takes a CUDA tensor")
    if table.dtype != torch.uint8 or not table.is_contiguous():
        raise TypeError("check_table_noalloc takes a contiguous uint8 tensor")
    out = TableCheck()
    with torch.cuda.device(table.device):
        lib().luda_check_table_noalloc(C.c_void_p(table.data_ptr()), table.numel(),
                                       stream if stream is not None else current_stream(), C.byref(out))
    return out


def build(run, opts: Options | None = None) -> Result:
    """Pack one sorted run (a workloads.Run) into tables; host arrays in, bytes out."""
    ra, keep = _run_arrays(run, device=False)
    o = opts or options(target_file_size=(1 << 64) - 1)
    out = Outputs()
    rc = lib().luda_build(C.byref(ra), C.byref(o), C.byref(out))
    del keep
    return _take(rc, out, device=False)


def build_device(run, opts: Options | None = None) -> Result:
    """Pack one sorted run on the device; tables come back as torch CUDA tensors."""
    ra, keep = _run_arrays(run, device=True)
    o = opts or options(target_file_size=(1 << 64) - 1)
    if o.stream is None:
        o.stream = current_stream()
    out = Outputs()
    rc = lib().luda_build_device(C.byref(ra), C.byref(o), C.byref(out))
    del keep
    return _take(rc, out, device=True)
