"""Selective monitoring (hr_set_filter) == the oracle on the filtered trace.

The filter's meaning is plain: the checker reports exactly the races among the
accesses it monitors.  So the expected set is the brute force over the trace
with the unmonitored access records removed (barrier records stay: they only
carry clocks).
"""
import numpy as np
import pytest

from paper_2401_04701_gb300 import tracegen as tg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2401_04701_gb300 import hirace
    return hirace


def to_dev(trace):
    import torch
    return torch.from_numpy(np.ascontiguousarray(trace).view(np.uint8)).cuda()


def keep_mask(trace, block_dim, warp=32, word_lo=0, word_hi=0, block_lo=0, block_hi=0, lane_mask=0xFFFFFFFF):
    acc = trace["op"] <= tg.OP_A
    w = trace["word"].astype(np.int64)
    tid = trace["tid"].astype(np.int64)
    blk, lane = tid // block_dim, (tid % block_dim) % warp
    ok = np.ones(len(trace), bool)
    if word_hi:
        ok &= (w >= word_lo) & (w < word_hi)
    if block_hi:
        ok &= (blk >= block_lo) & (blk < block_hi)
    ok &= ((lane_mask >> lane) & 1).astype(bool)
    return ~acc | ok


FILTERS = [dict(word_lo=1 << 19, word_hi=3 << 19), dict(block_lo=3, block_hi=9), dict(lane_mask=0x11111111),
           dict(word_lo=65536, word_hi=65536 * 9, block_lo=2, block_hi=14, lane_mask=0x0000FFFF)]


@pytest.mark.parametrize("aggregate", [True, False])
@pytest.mark.parametrize("fi", range(len(FILTERS)))
def test_filters_on_global_mix(oracle_mod, hr, fi, aggregate):
    f = FILTERS[fi]
    tr, info = tg.gen_global_mix(tg.seed_for(2, 5), inject=True, n_blocks=16)
    kept = tr[keep_mask(tr, 256, **f)]
    want = oracle_mod.race_keys(oracle_mod.bruteforce(kept, 256, 32))
    assert want  # every filter keeps some injected races
    n_words = (f["word_hi"] - f["word_lo"]) if f.get("word_hi") else info["n_words"]
    with hr.Checker([dict(n_words=n_words, block_dim=256)], report_capacity=1 << 20) as ck:
        ck.set_filter(0, **f)
        ck.check_trace(0, to_dev(tr), aggregate=aggregate)
        races, status, n_total, _ = ck.report(0)
        assert status == hr.HR_OK and hr.race_keys(races) == want and n_total == len(want)
        if not f.get("word_hi"):  # without a window the same region can monitor everything again
            ck.clear_filter(0)
            ck.reset(0)
            ck.check_trace(0, to_dev(tr), aggregate=aggregate)
            races, status, n_total, _ = ck.report(0)
            assert hr.race_keys(races) == oracle_mod.race_keys(oracle_mod.bruteforce(tr, 256, 32))


def test_filter_on_compact_shadow(oracle_mod, hr):
    f = dict(word_lo=1 << 18, word_hi=5 << 18, lane_mask=0xF0F0F0F0)
    tr, info = tg.gen_global_mix(tg.seed_for(2, 6), inject=True, n_blocks=16)
    want = oracle_mod.race_keys(oracle_mod.bruteforce(tr[keep_mask(tr, 256, **f)], 256, 32))
    reg = dict(n_words=4 << 18, block_dim=256, shadow_bytes=4, tid_bits=18)
    with hr.Checker([reg], report_capacity=1 << 20) as ck:
        ck.set_filter(0, **f)
        ck.check_trace(0, to_dev(tr))
        races, status, n_total, _ = ck.report(0)
    assert status == hr.HR_OK and hr.race_keys(races) == want and n_total == len(want)


def test_filter_on_inline_kernel(oracle_mod, hr):
    """hr_access honours the view's filter (word window, blocks, lanes) in a stencil."""
    import torch
    hr.load_workloads()
    n = 1 << 18
    # input words from 30000 up, blocks 100..699, all lanes but 15 and 31 of each warp
    f = dict(word_lo=30000, word_hi=n, block_lo=100, block_hi=700, lane_mask=0x7FFF7FFF)
    prog = tg.stencil_program(n, 7)
    want = oracle_mod.race_keys(oracle_mod.bruteforce(prog[keep_mask(prog, 256, **f)], 256, 32))
    assert want
    d_in = torch.rand(n, device="cuda")
    d_out = torch.zeros(n, device="cuda")
    with hr.Checker([dict(n_words=n - 30000, block_dim=256)]) as ck:
        ck.set_filter(0, **f)
        hr.run_stencil(ck.device_view(0), d_in, d_out, racy_stride=7)
        races, status, n_total, _ = ck.report(0)
    assert status == hr.HR_OK and hr.race_keys(races) == want and n_total == len(want)


@pytest.mark.parametrize("bad", [dict(word_lo=5, word_hi=5), dict(word_lo=0, word_hi=1 << 30), dict(word_lo=3),
                                 dict(block_lo=9, block_hi=3), dict(lane_mask=0)])
def test_filter_validation(hr, bad):
    with hr.Checker([dict(n_words=1024, block_dim=256)]) as ck:
        with pytest.raises(hr.HiRaceError):
            ck.set_filter(0, **bad)
