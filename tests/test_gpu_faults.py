"""Host-side fault injection through the allocator hook: whichever device allocation of a
call fails, the call returns LUDA_ERR_OOM with empty outputs and gives back every byte it
took; the same call then succeeds with the oracle's bytes (a failed job is simply redone)."""
import ctypes as C

import pytest

from helpers import oracle_compact, oracle_inputs
from paper_2004_03054_b300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2004_03054_b300 import luda  # noqa: E402

ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class Hook:
    """A device allocator over PyTorch's caching allocator that can fail on call k."""

    def __init__(self, fail_at=-1):
        self.fail_at, self.calls, self.live = fail_at, 0, {}
        self._alloc, self._free = ALLOC(self.alloc), FREE(self.free)

    def alloc(self, n, ctx, stream):
        k = self.calls
        self.calls += 1
        if k == self.fail_at:
            return None
        p = torch.cuda.caching_allocator_alloc(n, stream=torch.cuda.current_stream())
        self.live[p] = n
        return p

    def free(self, p, ctx, stream):
        torch.cuda.caching_allocator_delete(p)
        del self.live[p]

    def options(self, job):
        o = luda.job_options(job)
        o.dev_alloc = C.cast(self._alloc, C.c_void_p)
        o.dev_free = C.cast(self._free, C.c_void_p)
        return o


def _dev(b):
    return torch.frombuffer(bytearray(b), dtype=torch.uint8).cuda()


@pytest.mark.parametrize("host", [False, True])
def test_every_failing_allocation_is_clean_and_the_retry_matches(host):
    job = W.config1(seed=61, scale=1 / 32)
    ins = oracle_inputs(job)
    want = [t.data for t in oracle_compact(job, ins).tables]
    dev = [_dev(b) for b in ins]
    L = luda.lib()

    def run(hook):
        arr = (luda.Input * len(ins))()
        for i, (b, d) in enumerate(zip(ins, dev)):
            if host:
                arr[i].data, arr[i].size = C.cast(C.c_char_p(b), C.c_void_p).value, len(b)
            else:
                arr[i].data, arr[i].size = d.data_ptr(), d.numel()
        out = luda.Outputs()
        o = hook.options(job)
        fn = L.luda_compact if host else L.luda_compact_device
        rc = fn(arr, len(ins), job.level, job.smallest_snapshot, C.byref(o), C.byref(out))
        torch.cuda.synchronize()
        return rc, out

    ok = Hook()
    rc, out = run(ok)
    assert rc == 0
    n_calls = ok.calls
    got = [C.string_at(out.tables[i].data, out.tables[i].size) if host else
           luda.device_bytes(out.tables[i].data, out.tables[i].size).cpu().numpy().tobytes()
           for i in range(out.n_tables)]
    assert got == want
    L.luda_outputs_free(C.byref(out))
    assert not ok.live and n_calls >= 3
    for k in range(n_calls):
        bad = Hook(fail_at=k)
        rc, out = run(bad)
        assert rc == luda.ERR_OOM, (k, rc)
        assert out.n_tables == 0 and not out.tables
        assert not bad.live, (k, bad.live)       # everything taken was given back
    # the redone job
    again = Hook()
    rc, out = run(again)
    assert rc == 0 and out.n_tables == len(want)
    L.luda_outputs_free(C.byref(out))
    assert not again.live


@pytest.mark.parametrize("host,flags", [(False, 0), (True, 0), (False, luda.F_COMPRESS)])
def test_encoder_wait_that_runs_out_fails_cleanly_and_the_next_call_matches(host, flags):
    """The staged encoder's bounded waits for its copy slots, made to run out at once by the
    test-only flag: the call returns LUDA_ERR_TIMEOUT with no tables, the copies already in
    flight are drained (the device stays usable), and the same call without the flag then
    writes the oracle's bytes."""
    job = W.config1(seed=62, scale=1 / 8)
    ins = oracle_inputs(job)
    want = [t.data for t in oracle_compact(job, ins, flags=flags).tables]
    dev = [_dev(b) for b in ins]
    L = luda.lib()

    def run(extra):
        arr = (luda.Input * len(ins))()
        for i, (b, d) in enumerate(zip(ins, dev)):
            if host:
                arr[i].data, arr[i].size = C.cast(C.c_char_p(b), C.c_void_p).value, len(b)
            else:
                arr[i].data, arr[i].size = d.data_ptr(), d.numel()
        out = luda.Outputs()
        o = luda.job_options(job, flags=flags | extra)
        fn = L.luda_compact if host else L.luda_compact_device
        rc = fn(arr, len(ins), job.level, job.smallest_snapshot, C.byref(o), C.byref(out))
        torch.cuda.synchronize()
        return rc, out

    for _ in range(2):
        rc, out = run(luda.F_TEST_WAIT0)
        assert rc == luda.ERR_TIMEOUT, luda.last_error_detail()
        assert out.n_tables == 0
        assert out.status == luda.ERR_TIMEOUT
        L.luda_outputs_free(C.byref(out))
    rc, out = run(0)
    assert rc == 0, luda.last_error_detail()
    got = [C.string_at(out.tables[i].data, out.tables[i].size) if host else
           luda.device_bytes(out.tables[i].data, out.tables[i].size).cpu().numpy().tobytes()
           for i in range(out.n_tables)]
    L.luda_outputs_free(C.byref(out))
    assert got == want
