"""Autotuner for the launch shapes of the batched pipeline (luda_tuning).

A tuning decides how the pipeline's kernels split their work over CTAs: records per merge
tile, merge CTAs per SM, key-rebuild warps per CTA, block-walk CTA size, staged-encoder CTAs per
SM, the CTA size of the per-record kernels and the SMs given to the checksum kernels (which
run beside the other stages). No tuning changes an output byte, so the tuner is free to
pick whichever is fastest for a batch.

The search is coordinate descent over a small grid (one knob at a time, the others held at
the best values so far): every candidate of one knob is timed by the library itself
(luda_autotune builds a plan per candidate and times its CUDA-graph replays between CUDA
events), the fastest value is kept, and the next knob follows. The winner is cached in a
JSON file keyed by the GPU's name and SM count and a signature of the batch (format
options, log2 of the job count and of the input bytes), so that later batches of the same
kind reuse it without timing.
"""
from __future__ import annotations

import ctypes as C
import json
import math
import os
import time
from dataclasses import dataclass, field

from . import luda

# Values tried per knob; 0 means the library's default (for encode_ctas_per_sm: as many
# CTAs per SM as shared memory allows).
SPACE: dict[str, tuple[int, ...]] = {
    "merge_tile": (512, 1024, 2048),
    "merge_ctas_per_sm": (4, 8, 16),
    "decode_warps": (2, 4, 8),
    "walk_threads": (64, 128, 256),
    "encode_ctas_per_sm": (1, 2, 0),
    "elem_threads": (128, 256, 512),
    "crc_ctas": (100, 74, 64, 56),
    "crc_warps": (32, 16),
}
# The library's defaults, resolved.
DEFAULT = {"merge_tile": 512, "merge_ctas_per_sm": 16, "decode_warps": 4, "walk_threads": 256,
           "encode_ctas_per_sm": 0, "elem_threads": 256, "crc_ctas": 56, "crc_warps": 32}


@dataclass
class Result:
    tuning: dict
    best_ms: float
    default_ms: float | None
    evaluated: list = field(default_factory=list)  # (tuning dict, ms) in the order timed
    seconds: float = 0.0
    cache: str = "miss"                              # "hit", "miss" or "off"
    key: str = ""


def coordinate_search(measure, space: dict | None = None, start: dict | None = None, sweeps: int = 1):
    """Coordinate descent. measure(list of tuning dicts) -> list of ms (negative = failed).
    Each knob's candidates are measured together; a tuning already measured is not
    measured again. Returns (best tuning, its ms, [(tuning, ms), ...])."""
    space = space or SPACE
    best = dict(start or DEFAULT)
    seen: dict[tuple, float] = {}
    log = []

    def key(t):
        return tuple(sorted(t.items()))

    def run(cands):
        todo = [c for c in cands if key(c) not in seen]
        if todo:
            for c, ms in zip(todo, measure(todo)):
                seen[key(c)] = ms
                log.append((dict(c), ms))
        return [seen[key(c)] for c in cands]

    best_ms = run([best])[0]
    for _ in range(max(1, sweeps)):
        changed = False
        for knob, values in space.items():
            cands = [dict(best, **{knob: v}) for v in values]
            ms = run(cands)
            for c, m in zip(cands, ms):
                if m >= 0 and (best_ms < 0 or m < best_ms):
                    best, best_ms, changed = c, m, True
        if not changed:
            break
    return best, best_ms, log


def signature(jobs, opts: luda.Options) -> str:
    """What the cached tuning depends on: the format options and the batch's rough size."""
    n_jobs = max(1, len(jobs))
    nbytes = max(1, sum(int(t.numel()) for job in jobs for t in job[0]))
    return (f"T{opts.block_size}-R{opts.restart_interval}-bpk{opts.bloom_bits_per_key}-"
            f"tgt{opts.target_file_size}-jobs2^{round(math.log2(n_jobs))}-bytes2^{round(math.log2(nbytes))}")


def device_key() -> str:
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}|{p.multi_processor_count}sm"


def default_cache_path() -> str:
    return os.environ.get("LUDA_TUNE_CACHE") or os.path.join(
        os.environ.get("XDG_CACHE_HOME") or os.path.expanduser("~/.cache"), "luda", "tuning.json")


def load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(path: str, data: dict) -> None:
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def measure_fn(jobs, opts: luda.Options, reps: int = 3):
    """A measure() for coordinate_search: times candidates through luda_autotune."""
    L = luda.lib()
    js, keep = luda._jobs_array(jobs)

    def measure(cands):
        arr = (luda.Tuning * len(cands))(*[luda.Tuning.of(c) for c in cands])
        ms = (C.c_double * len(cands))()
        best = C.c_uint32()
        rc = L.luda_autotune(js, len(jobs), C.byref(opts), arr, len(cands), reps, ms, C.byref(best))
        if rc not in (luda.OK,) and all(m < 0 for m in ms):
            raise RuntimeError(f"luda_autotune: {luda.strerror(rc)}: {luda.last_error_detail()}")
        _ = keep
        return [float(m) for m in ms]

    return measure


def tune(jobs, opts: luda.Options, cache_path: str | None = "", reps: int = 3, sweeps: int = 1,
         refresh: bool = False, space: dict | None = None) -> Result:
    """The tuning for a batch. jobs: [(inputs: [CUDA uint8 tensors], snapshot, bottommost)].
    cache_path "" = the default cache file, None = no cache. A cached entry for the same GPU
    and batch signature is returned without timing unless refresh is set."""
    path = default_cache_path() if cache_path == "" else cache_path
    key = f"{device_key()}|{signature(jobs, opts)}"
    cache = load_cache(path) if path else {}
    if path and not refresh and key in cache:
        e = cache[key]
        return Result(dict(DEFAULT, **e["tuning"]), e.get("ms", -1.0), e.get("default_ms"), [], 0.0, "hit", key)
    t0 = time.perf_counter()
    best, best_ms, log = coordinate_search(measure_fn(jobs, opts, reps), space=space, sweeps=sweeps)
    secs = time.perf_counter() - t0
    default_ms = next((ms for t, ms in log if t == DEFAULT), None)
    if path:
        cache = load_cache(path)
        cache[key] = {"tuning": best, "ms": best_ms, "default_ms": default_ms, "candidates": len(log),
                      "when": time.strftime("%Y-%m-%dT%H:%M:%S")}
        save_cache(path, cache)
    return Result(best, best_ms, default_ms, log, secs, "miss" if path else "off", key)
