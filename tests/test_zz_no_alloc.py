"""The allocation-free trace check gives the same races as the context-based one.

hr_check_trace_noalloc is for callers that cannot allocate device memory:
code that runs while another component owns the device memory budget (a
framework's caching allocator or a fixed pool) and latency-critical paths
where cudaMalloc/cudaFree would synchronise the device.  The tests own every
buffer they hand over (trace, shadow, race buffer, result block) and call the
entry point through the C-ABI.  Two calls in a row on different traces are
each compared with hr_check_trace on the same trace and with the CPU oracle:
same race keys, same count, no error.  Race reports are integer data, so the
comparison is exact.  Further cases: a second call on a shadow that an earlier
call left dirty (each call is a fresh check), an empty trace, more waves than
the built-in scratch holds (HR_ERR_CAPACITY, nothing checked) and a race
buffer smaller than the race count (exact count, truncated flag).

This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

RESULT_DT = np.dtype([("n_races", "<u8"), ("error", "<u4"), ("flags", "<u4")])
MAX_WAVES = 4096          # HR_NOALLOC_MAX_WAVES in include/hirace.h


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2401_04701_gb300 import hirace
    lib = hirace.load_library()
    fn = lib.hr_check_trace_noalloc
    P, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
    fn.argtypes = [P, u64, P, u64, u32, u32, P, u64, P, P]
    fn.restype = ctypes.c_int
    return hirace, fn


def _traces():
    from paper_2401_04701_gb300 import tracegen as tg
    a, ia = tg.gen_global_mix(tg.seed_for(2, 7), inject=True, n_blocks=8)
    b, ib = tg.gen_tree_reduction(tg.seed_for(1, 7), inject=True, segments=8, reps=3)
    return [(a, ia["n_words"], ia["block_dim"]), (b, ib["n_words"], ib["block_dim"])]


def _dev(trace):
    import torch
    return torch.from_numpy(np.ascontiguousarray(trace).view(np.uint8)).cuda()


def _call(env, d_trace, n, shadow, n_words, block_dim, cap):
    """One call through the C-ABI with caller-owned buffers; (rc, result, races)."""
    import torch
    hirace, fn = env
    races = torch.zeros(max(cap, 1) * 16, dtype=torch.uint8, device="cuda")
    result = torch.full((16,), 0xAB, dtype=torch.uint8, device="cuda")   # stale bytes on purpose
    stream = torch.cuda.current_stream()
    rc = fn(d_trace.data_ptr() if n else None, n, shadow.data_ptr(), n_words, block_dim, 32, races.data_ptr(),
            cap, result.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    res = result.cpu().numpy().view(RESULT_DT)[0]
    got = races.cpu().numpy().view(hirace.RACE_DTYPE)[:min(cap, int(res["n_races"]))]
    return rc, res, got


def test_noalloc_equals_context_check_on_consecutive_calls(env, oracle_mod):
    import torch
    hirace, _ = env
    cap = 1 << 16
    for trace, n_words, block_dim in _traces():
        d_trace = _dev(trace)
        with hirace.Checker([dict(n_words=n_words, block_dim=block_dim)], report_capacity=cap) as ck:
            ck.check_trace(0, d_trace)
            want, status, want_total, _ = ck.report(0)
        assert status == hirace.HR_OK and want_total > 0
        oracle_keys = oracle_mod.race_keys(oracle_mod.bruteforce(trace, block_dim))
        assert hirace.race_keys(want) == oracle_keys

        shadow = torch.zeros(n_words, dtype=torch.int64, device="cuda")
        rc, res, got = _call(env, d_trace, len(trace), shadow, n_words, block_dim, cap)
        assert rc == 0
        assert int(res["error"]) == 0 and int(res["flags"]) == 0
        assert int(res["n_races"]) == want_total
        assert hirace.race_keys(got) == hirace.race_keys(want) == oracle_keys


def test_dirty_shadow_from_an_earlier_call_does_not_leak(env, oracle_mod):
    """Trace B run after trace A on the same shadow buffer (same kernel
    ordinals, no zeroing in between) gives B's races alone."""
    import torch
    hirace, _ = env
    from paper_2401_04701_gb300 import tracegen as tg
    a, info = tg.gen_global_mix(tg.seed_for(2, 12), inject=True, n_blocks=8)
    b, _ = tg.gen_global_mix(tg.seed_for(2, 13), inject=True, n_blocks=8)
    n_words = info["n_words"]
    want_b = oracle_mod.race_keys(oracle_mod.bruteforce(b, 256))
    shadow = torch.full((n_words,), -1, dtype=torch.int64, device="cuda")     # garbage on entry
    for tr in (a, b):
        rc, res, got = _call(env, _dev(tr), len(tr), shadow, n_words, 256, 1 << 16)
        assert rc == 0 and int(res["error"]) == 0
    assert hirace.race_keys(got) == want_b and int(res["n_races"]) == len(want_b)


def test_empty_trace_writes_a_zero_result(env):
    import torch
    shadow = torch.zeros(16, dtype=torch.int64, device="cuda")
    rc, res, _ = _call(env, shadow, 0, shadow, 16, 32, 4)
    assert rc == 0
    assert int(res["n_races"]) == 0 and int(res["error"]) == 0 and int(res["flags"]) == 0


def test_more_waves_than_the_scratch_holds(env):
    """MAX_WAVES + 1 block epochs: HR_ERR_CAPACITY in the result, nothing checked."""
    import torch
    hirace, _ = env
    from paper_2401_04701_gb300 import tracegen as tg
    # two threads of one block write word 0 in every epoch: a race if it were checked
    prog = [("W", 0), ("ST",)] * MAX_WAVES + [("W", 0)]
    tr = tg.build_trace([{0: prog, 1: prog}])
    assert len(np.unique(tg.wave_keys(tr))) == MAX_WAVES + 1
    shadow = torch.zeros(4, dtype=torch.int64, device="cuda")
    rc, res, _ = _call(env, _dev(tr), len(tr), shadow, 4, 32, 16)
    assert rc == 0
    assert hirace.STATUS[int(res["error"])] == "HR_ERR_CAPACITY"
    assert int(res["n_races"]) == 0


def test_race_buffer_smaller_than_the_race_count(env, oracle_mod):
    import torch
    hirace, _ = env
    trace, n_words, block_dim = _traces()[0]
    want = oracle_mod.race_keys(oracle_mod.bruteforce(trace, block_dim))
    assert len(want) > 10
    shadow = torch.zeros(n_words, dtype=torch.int64, device="cuda")
    rc, res, got = _call(env, _dev(trace), len(trace), shadow, n_words, block_dim, 10)
    assert rc == 0 and int(res["error"]) == 0
    assert int(res["n_races"]) == len(want)
    assert int(res["flags"]) & hirace.FLAG_TRUNCATED
    assert len(got) == 10 and hirace.race_keys(got) <= want
