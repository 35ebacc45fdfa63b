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


# ---------------------------------------------------------------------------
# Symmetric work groups: members folded onto a representative block
# ---------------------------------------------------------------------------

def fold_trace(trace, block_dim, sym_lo, sym_hi, stride, word_lo=0, word_hi=0):
    """The accesses the checker applies under a symmetric group, written out:
    an access of thread t of block sym_lo + m (0 < m < sym_hi - sym_lo) to word
    w becomes thread t - m * block_dim's access to w - m * stride (dropped if
    w < m * stride), then the word window keeps [word_lo, word_hi).  Barrier
    records are dropped (they carry only clocks, which every record has)."""
    acc = trace[trace["op"] <= tg.OP_A].copy()
    tid = acc["tid"].astype(np.int64)
    w = acc["word"].astype(np.int64)
    m = tid // block_dim - sym_lo
    member = (m > 0) & (tid // block_dim < sym_hi)
    shift = np.where(member, m * stride, 0)
    keep = w >= shift
    w = w - shift
    tid = tid - np.where(member, m * block_dim, 0)
    if word_hi:
        keep &= (w >= word_lo) & (w < word_hi)
    out = acc[keep]
    out["word"] = w[keep]
    out["tid"] = tid[keep]
    return out


def symmetric_program(rng, n_members, block_dim, stride, n_acc=3000):
    """One block's random program (reads, writes, atomics on `stride` words,
    a few barriers) run by n_members blocks, member b on words shifted up by
    b * stride: (trace, the representative block's trace alone)."""
    from tests import _cases as C
    base = C.random_program(rng, n_threads=block_dim, block_dim=block_dim, n_words=stride, n_acc=n_acc,
                            n_st=3, n_sw=2, n_kernels=1)[0]
    progs = {}
    for b in range(n_members):
        for t, ev in base.items():
            progs[b * block_dim + t] = [(e[0], e[1] + b * stride) + tuple(e[2:]) if e[0] in ("R", "W", "A") else e
                                        for e in ev]
    return tg.build_trace([progs]), tg.build_trace([base])


@pytest.mark.parametrize("variant", ["plain", "aggregated", "binned"])
def test_symmetric_group_equals_its_representative(oracle_mod, hr, variant):
    """Exactly symmetric members: the folded check on a shadow of one member's
    words reports the representative block's races (the same races every
    member has, Sec. IV-A's representative tracking), and equals the oracle
    on the folded trace."""
    rng = np.random.default_rng(31)
    bd, stride, G = 64, 97, 12
    tr, rep = symmetric_program(rng, G, bd, stride)
    want_rep = oracle_mod.race_keys(oracle_mod.bruteforce(rep, bd, 32))
    assert want_rep
    folded = fold_trace(tr, bd, 0, G, stride, 0, stride)
    assert oracle_mod.race_keys(oracle_mod.bruteforce_parallel(folded, bd, stride, threads=1)) == want_rep
    with hr.Checker([dict(n_words=stride, block_dim=bd)], report_capacity=1 << 16) as ck:
        if variant == "binned":
            ck.set_variant(hr.binned_variant())
        ck.set_filter(0, word_lo=0, word_hi=stride, sym_lo=0, sym_hi=G, sym_stride=stride)
        ck.check_trace(0, to_dev(tr), aggregate=variant == "aggregated")
        races, status, n_total, _ = ck.report(0)
    assert status == hr.HR_OK and hr.race_keys(races) == want_rep and n_total == len(want_rep)


@pytest.mark.parametrize("variant", ["plain", "aggregated", "binned"])
def test_symmetric_group_on_global_mix(oracle_mod, hr, variant):
    """Members that are not symmetric (the global mix: random words shared by
    all blocks): the checker applies exactly the folded accesses, with a word
    window, blocks outside the group unchanged."""
    tr, info = tg.gen_global_mix(tg.seed_for(2, 14), inject=True, n_blocks=16)
    f = dict(sym_lo=3, sym_hi=11, sym_stride=65536, word_lo=65536, word_hi=65536 * 9)
    folded = fold_trace(tr, 256, 3, 11, 65536, 65536, 65536 * 9)
    want = oracle_mod.race_keys(oracle_mod.bruteforce_parallel(folded, 256, info["n_words"], threads=1))
    assert want
    with hr.Checker([dict(n_words=65536 * 8, block_dim=256)], report_capacity=1 << 20) as ck:
        if variant == "binned":
            ck.set_variant(hr.binned_variant())
        ck.set_filter(0, **f)
        ck.check_trace(0, to_dev(tr), aggregate=variant == "aggregated")
        races, status, n_total, _ = ck.report(0)
    assert status == hr.HR_OK and hr.race_keys(races) == want and n_total == len(want)


def test_symmetric_group_validation(hr):
    with hr.Checker([dict(n_words=1024, block_dim=256)]) as ck:
        with pytest.raises(hr.HiRaceError):
            ck.set_filter(0, sym_lo=5, sym_hi=5)
        with pytest.raises(hr.HiRaceError):
            ck.set_filter(0, sym_lo=6, sym_hi=2)
