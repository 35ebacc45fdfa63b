"""The allocation-free trace check gives the same races as the context-based one.

hr_check_trace_noalloc is for callers that cannot allocate device memory:
code that runs while another component owns the device memory budget (a
framework's caching allocator or a fixed pool) and latency-critical paths
where cudaMalloc/cudaFree would synchronise the device.  The test owns every
buffer it hands over (trace, shadow, race buffer, result block), calls the
entry point through the C-ABI twice in a row on different traces, and
compares each call with hr_check_trace on the same trace: same race keys,
same count, no error.  Race reports are integer data, so the comparison is
exact.

This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

RESULT_DT = np.dtype([("n_races", "<u8"), ("error", "<u4"), ("flags", "<u4")])


def _traces():
    from paper_2401_04701_gb300 import tracegen as tg
    a, ia = tg.gen_global_mix(tg.seed_for(2, 7), inject=True, n_blocks=8)
    b, ib = tg.gen_tree_reduction(tg.seed_for(1, 7), inject=True, segments=8, reps=3)
    return [(a, ia["n_words"], ia["block_dim"]), (b, ib["n_words"], ib["block_dim"])]


def test_noalloc_equals_context_check_on_consecutive_calls():
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
    cap = 1 << 16
    stream = torch.cuda.current_stream()
    for trace, n_words, block_dim in _traces():
        d_trace = torch.from_numpy(trace.view(np.uint8)).cuda()
        with hirace.Checker([dict(n_words=n_words, block_dim=block_dim)], report_capacity=cap) as ck:
            ck.check_trace(0, d_trace)
            want, status, want_total, _ = ck.report(0)
        assert status == hirace.HR_OK and want_total > 0

        shadow = torch.zeros(n_words, dtype=torch.int64, device="cuda")
        races = torch.zeros(cap * 16, dtype=torch.uint8, device="cuda")
        result = torch.full((16,), 0xAB, dtype=torch.uint8, device="cuda")   # stale bytes on purpose
        rc = fn(d_trace.data_ptr(), len(trace), shadow.data_ptr(), n_words, block_dim, 32, races.data_ptr(), cap,
                result.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        assert rc == 0
        res = result.cpu().numpy().view(RESULT_DT)[0]
        assert int(res["error"]) == 0 and int(res["flags"]) == 0
        assert int(res["n_races"]) == want_total
        got = races.cpu().numpy().view(hirace.RACE_DTYPE)[:want_total]
        assert hirace.race_keys(got) == hirace.race_keys(want)
