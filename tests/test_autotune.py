"""The autotuner's host logic (no GPU): coordinate descent, the cache, the tuning ABI and
its range check in the library."""
import ctypes as C
import itertools
import json

import pytest

from paper_2004_03054_b300 import autotune as AT
from paper_2004_03054_b300 import luda


def _cost(t):
    """A separable cost with a known minimum per knob (in ms)."""
    best = {"merge_tile": 2048, "merge_ctas_per_sm": 4, "decode_warps": 8, "walk_threads": 128,
            "encode_ctas_per_sm": 1, "elem_threads": 512, "crc_ctas": 64, "crc_warps": 16}
    return 10.0 + sum(abs(AT.SPACE[k].index(t[k]) - AT.SPACE[k].index(best[k])) for k in AT.SPACE), best


def test_coordinate_search_finds_separable_minimum_and_times_each_candidate_once():
    calls = []

    def measure(cands):
        calls.extend(tuple(sorted(c.items())) for c in cands)
        return [_cost(c)[0] for c in cands]

    best, ms, log = AT.coordinate_search(measure, sweeps=2)
    assert best == _cost(best)[1] and ms == 10.0
    assert len(calls) == len(set(calls))                       # nothing timed twice
    assert len(log) == len(calls) and log[0][0] == AT.DEFAULT   # the default is timed first
    # exhaustive check on the same cost: the grid minimum is the one found
    grid = [dict(zip(AT.SPACE, v)) for v in itertools.product(*AT.SPACE.values())]
    assert min(_cost(g)[0] for g in grid) == ms


def test_coordinate_search_skips_failed_candidates():
    def measure(cands):
        return [-1.0 if c["merge_tile"] == 2048 else (5.0 if c["merge_tile"] == 512 else 6.0) for c in cands]

    best, ms, _ = AT.coordinate_search(measure)
    assert best["merge_tile"] == 512 and ms == 5.0


def test_cache_round_trip_and_hit(tmp_path, monkeypatch):
    class FakeT:
        def __init__(self, n):
            self.n = n

        def numel(self):
            return self.n

    jobs = [([FakeT(1 << 20), FakeT(3 << 20)], 1, False)] * 5
    opts = luda.options(4096, 16, 10, 2 << 20)
    monkeypatch.setattr(AT, "device_key", lambda: "FakeGPU|148sm")
    key = f"FakeGPU|148sm|{AT.signature(jobs, opts)}"
    path = tmp_path / "t.json"
    want = dict(AT.DEFAULT, merge_tile=512)
    AT.save_cache(str(path), {key: {"tuning": want, "ms": 3.5, "default_ms": 4.0}})
    assert json.loads(path.read_text())[key]["tuning"] == want

    def boom(*a, **k):
        raise AssertionError("a cache hit must not time anything")

    monkeypatch.setattr(AT, "measure_fn", boom)
    res = AT.tune(jobs, opts, cache_path=str(path))
    assert res.cache == "hit" and res.tuning == want and res.best_ms == 3.5 and res.key == key
    # another batch size is another entry
    assert AT.signature(jobs * 8, opts) != AT.signature(jobs, opts)
    assert AT.load_cache(str(tmp_path / "missing.json")) == {}


def test_tuning_struct_layout():
    assert C.sizeof(luda.Tuning) == 36  # nine uint32 fields, as luda.h declares
    assert luda.Options.tuning.offset == luda.Options.stream.offset + 8
    t = luda.Tuning.of({"merge_tile": 512, "elem_threads": 128})
    assert t.as_dict()["merge_tile"] == 512 and t.as_dict()["decode_warps"] == 0
    o = luda.options().with_tuning({"decode_warps": 4})
    assert o.tuning.contents.decode_warps == 4
    assert not luda.options().tuning


def test_library_checks_tuning_ranges():
    L = luda.lib()
    for combo in [dict(AT.DEFAULT)] + [dict(AT.DEFAULT, **{k: v}) for k, vs in AT.SPACE.items() for v in vs]:
        assert L.luda_tuning_check(C.byref(luda.Tuning.of(combo))) == luda.OK, combo
    t0 = luda.Tuning()
    L.luda_tuning_default(C.byref(t0))
    assert L.luda_tuning_check(C.byref(t0)) == luda.OK
    for bad in ({"merge_tile": 768}, {"merge_tile": 4096}, {"merge_ctas_per_sm": 33}, {"decode_warps": 17},
                {"walk_threads": 48}, {"walk_threads": 512}, {"encode_ctas_per_sm": 9}, {"elem_threads": 32},
                {"elem_threads": 100}, {"elem_threads": 2048}, {"crc_ctas": 149},
                {"crc_warps": 4}, {"crc_warps": 20}, {"crc_warps": 40}, {"h2d_ranges": 65}):
        assert L.luda_tuning_check(C.byref(luda.Tuning.of(bad))) == luda.ERR_INVALID_ARG, bad
        assert list(bad)[0] in luda.last_error_detail()
    assert L.luda_tuning_check(None) == luda.ERR_INVALID_ARG
