"""Binned checker (per-segment shadow in shared memory) == CPU oracle.

The binned checker moves every access into a (shadow segment, wave) bucket
and applies each segment's buckets in wave order on a shared-memory copy of
the segment.  Its results must be the oracle's race keys exactly, on the same
cases as the per-wave kernel: golden listings, the exhaustive toy universe,
random programs with many kernels (shadow clears at kernel-tag group changes),
a trace with more than the binned limit of waves (the per-wave kernel then
takes the check), segment and chunk boundaries, chunked calls that carry the shadow from
one call to the next, the compact shadow, filters and every error status.
"""
import numpy as np
import pytest

from paper_2401_04701_gb300 import tracegen as tg
from tests import _cases as C

pytestmark = pytest.mark.gpu

SEG = 4096          # shadow words per segment
CHUNK = 2048        # bucketed accesses a thread group stages in shared memory at a time (4-byte form)
MAX_WAVES = 256     # waves of a check the binned checker takes


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


def n_waves(trace):
    k = tg.wave_keys(trace)
    return int(np.count_nonzero(np.r_[True, k[1:] != k[:-1]])) if len(k) else 0


def bin_check(hr, trace, reg, chunks=None, filt=None, kernel_bases=(0,), cap=1 << 20):
    with hr.Checker([reg], report_capacity=cap) as ck:
        ck.set_variant(hr.binned_variant())
        if filt:
            ck.set_filter(0, **filt)
        for kb in kernel_bases:
            if chunks is None:
                ck.check_trace(0, to_dev(trace), kernel_base=kb)
            else:
                for a, b in zip(chunks[:-1], chunks[1:]):
                    if b > a:
                        ck.check_trace(0, to_dev(trace[a:b]), kernel_base=kb)
        races, status, n_total, _ = ck.report(0)
        cnt = ck.counters(0)
    return races, status, n_total, cnt


def assert_parity(O, hr, trace, n_words, block_dim, warp_size=32, **kw):
    bf = O.bruteforce(trace, block_dim, warp_size)
    reg = dict(n_words=n_words, block_dim=block_dim, warp_size=warp_size)
    races, status, n_total, cnt = bin_check(hr, trace, reg, **kw)
    assert status == hr.HR_OK, hr.STATUS[status]
    assert n_total == len(races) == len(bf)
    assert hr.race_keys(races) == O.race_keys(bf)
    ops = {(int(k), int(w)): int(m) for k, w, m in zip(bf["kernel"], bf["word"], bf["ops_mask"])}
    for k, w, op in zip(races["kernel"], races["word"], races["op"]):
        assert (ops[(int(k), int(w))] >> int(op)) & 1
    return races, cnt


def test_variant_is_listed(hr):
    v = hr.binned_variant()
    assert dict(hr.variants())[v] == dict(aggregate=False, records_per_lane=0, consumer_warps=0, binned=True)


@pytest.mark.parametrize("name", ["listing1_no_sync", "listing2_block_sync", "listing2_one_block",
                                  "listing3_multi_read"])
def test_listings(oracle_mod, hr, name):
    g = C.load_golden(name)
    races, _ = assert_parity(oracle_mod, hr, C.golden_trace(g), g["n_words"], g["block_dim"], g["warp_size"])
    assert hr.race_keys(races) == {tuple(x) for x in g["expected_races"]}


@pytest.mark.parametrize("k", [1, 2, 3])
def test_exhaustive_universe(oracle_mod, hr, k):
    rng = np.random.default_rng(150 + k)
    cases = C.exhaustive_cases(k, C.PHASES4)
    base = C.combined_trace(cases, C.PHASES4)
    for tr in (base, tg.shuffle_within_waves(base, rng)):
        assert_parity(oracle_mod, hr, tr, len(cases), C.TOY_BLOCK_DIM, C.TOY_WARP)


def test_random_programs_across_segments(oracle_mod, hr):
    """Words spread over several segments (region sizes not a multiple of the
    segment) and up to 20 kernels in one trace (shadow clears when the kernel
    tag wraps)."""
    rng = np.random.default_rng(161)
    seen = 0
    for it in range(24):
        bd = int(rng.choice([3, 16, 40, 64, 256]))   # 16 with warp 32: one warp per block
        ws = int(rng.choice([2, 32]))
        n_words = int(rng.choice([16, SEG + 1, 3 * SEG + 5, 20000]))
        kernels = C.random_program(rng, n_threads=int(rng.integers(2, 700)), block_dim=bd, n_words=n_words,
                                   n_acc=int(rng.integers(1, 6000)), n_st=int(rng.integers(0, 5)),
                                   n_sw=int(rng.integers(0, 5)), n_kernels=int(rng.integers(1, 21)))
        tr = tg.build_trace(kernels)
        if len(tr) == 0:
            continue
        seen += n_waves(tr) <= MAX_WAVES
        assert_parity(oracle_mod, hr, tr, n_words, bd, ws)
    assert seen >= 20


def test_many_waves_fall_back(oracle_mod, hr):
    """More waves than the binned limit: the per-wave kernel does the check."""
    kernels = [{t: [("W", t % 7), ("ST",), ("R", (t + 1) % 7)] for t in range(64)} for _ in range(150)]
    tr = tg.build_trace(kernels)
    assert n_waves(tr) > MAX_WAVES
    races, _ = assert_parity(oracle_mod, hr, tr, 7, 32, 32)
    assert len(races) > 0


def test_segment_edges(oracle_mod, hr):
    """Races on the first and last word of segments and of the region, and a
    clean word next to each; a region whose last segment is partial."""
    n_words = 3 * SEG + 5
    edges = [0, SEG - 1, SEG, 2 * SEG - 1, 2 * SEG, 3 * SEG, n_words - 1]
    threads = {}
    for i, w in enumerate(edges):
        a, b = 2 * i, 64 + 2 * i                      # two blocks of 64 threads
        threads.setdefault(a, []).append(("W", w))
        threads.setdefault(b, []).append(("R", w))
        nb = w + 1 if w + 1 < n_words else w - 1      # neighbour: one writer only
        threads.setdefault(a + 1, []).append(("W", nb))
    tr = tg.build_trace([threads])
    races, _ = assert_parity(oracle_mod, hr, tr, n_words, 64, 32)
    assert set(races["word"].tolist()) == set(edges)


def test_buckets_longer_than_a_chunk(oracle_mod, hr):
    """Buckets of several thousand accesses (one segment, few waves) are staged
    in pieces; the pieces of one wave and of consecutive waves stay ordered."""
    rng = np.random.default_rng(170)
    kernels = C.random_program(rng, n_threads=2048, block_dim=256, n_words=300, n_acc=3 * CHUNK * 4,
                               n_st=2, n_sw=1, n_kernels=2)
    tr = tg.build_trace(kernels)
    assert n_waves(tr) <= MAX_WAVES and len(tr) > 4 * CHUNK
    _, cnt = assert_parity(oracle_mod, hr, tr, 300, 256, 32)
    assert cnt["accesses"] == int(np.count_nonzero(tr["op"] <= tg.OP_A))


def test_wide_tids_and_clocks(oracle_mod, hr):
    """Thread ids of 17 bits (8-byte bucketed accesses, 4-byte working shadow),
    of 23 bits and block clocks too wide for the 4-byte working shadow (both
    then take the 8-byte working shadow), and a check that continues a kernel
    (nothing fresh: the stored shadow is read)."""
    tr, info = tg.gen_global_mix(tg.seed_for(2, 22), inject=True, n_blocks=300, tile_words=4096, epochs=2,
                                 slots=2)
    assert tr["tid"].max() >= 1 << 16
    races, _ = assert_parity(oracle_mod, hr, tr, info["n_words"], info["block_dim"])
    assert set(races["word"].tolist()) == set(info["injected"].tolist())
    base = 1 << 23
    wide = tg.build_trace([{base + t: [("W", t % 5), ("ST",), ("R", (t + 1) % 5)] for t in range(0, 512, 7)}])
    assert_parity(oracle_mod, hr, wide, 5, 256, 32)
    deep = tg.build_trace([{(1 << 17) + t: ([("R", t % 9)] + [("ST",)] * 40 + [("W", (t * 3) % 9)])
                            for t in range(96)}])
    assert_parity(oracle_mod, hr, deep, 9, 64, 32)
    rng = np.random.default_rng(171)
    kernels = C.random_program(rng, n_threads=600, block_dim=64, n_words=SEG + 77, n_acc=5000, n_st=3, n_sw=2,
                               n_kernels=1)
    tr = tg.build_trace(kernels)
    cuts = [0, len(tr) // 3, 2 * len(tr) // 3, len(tr)]
    assert_parity(oracle_mod, hr, tr, SEG + 77, 64, 32, chunks=cuts)


def test_skewed_large_check_falls_back(oracle_mod, hr):
    """A check of at least 2^22 accesses whose largest segment holds more than
    1/256 of them (here the hub words of a power-law graph: segment 0 holds
    over a third) is handed to the per-wave checker by the skew guard; the
    races are still the oracle's."""
    tr, info = tg.gen_powerlaw_push(tg.seed_for(3, 22), log2_vertices=17, sweeps=2)
    assert np.count_nonzero(tr["op"] <= 2) >= 1 << 22
    seg0 = np.count_nonzero((tr["op"] <= 2) & (tr["word"] < 4096))
    assert seg0 * 256 > len(tr)
    assert_parity(oracle_mod, hr, tr, info["n_words"], info["block_dim"])


def test_workloads(oracle_mod, hr):
    tr, info = tg.gen_global_mix(tg.seed_for(2, 21), inject=True, n_blocks=16)
    races, _ = assert_parity(oracle_mod, hr, tr, info["n_words"], info["block_dim"])
    assert set(races["word"].tolist()) == set(info["injected"].tolist())
    tr, info = tg.gen_tree_reduction(tg.seed_for(1, 21), inject=True)
    assert_parity(oracle_mod, hr, tr, info["n_words"], info["block_dim"])
    tr, info = tg.gen_powerlaw_push(tg.seed_for(3, 21), log2_vertices=14, sweeps=2)
    assert_parity(oracle_mod, hr, tr, info["n_words"], info["block_dim"])


def test_chunked_calls_and_kernel_bases(oracle_mod, hr):
    """Calls that cut waves in two carry the shadow from one call to the next;
    rebased kernel ordinals that cross a kernel-tag group (6..9) clear it."""
    tr, info = tg.gen_global_mix(tg.seed_for(2, 22), inject=True, n_blocks=8)
    rng = np.random.default_rng(22)
    cuts = np.sort(rng.integers(0, len(tr), 9))
    chunks = [0] + cuts.tolist() + [len(tr)]
    assert_parity(oracle_mod, hr, tr, info["n_words"], info["block_dim"], chunks=chunks)
    want = oracle_mod.race_keys(oracle_mod.bruteforce(tr, info["block_dim"]))
    reg = dict(n_words=info["n_words"], block_dim=info["block_dim"])
    races, status, n_total, _ = bin_check(hr, tr, reg, kernel_bases=(6, 7, 8, 9))
    assert status == hr.HR_OK and n_total == 4 * len(want)
    assert hr.race_keys(races) == {(kb, w, e) for kb in (6, 7, 8, 9) for (_, w, e) in want}


def test_compact_shadow(oracle_mod, hr):
    tr, info = tg.gen_global_mix(tg.seed_for(2, 23), inject=True, n_blocks=16)
    want = oracle_mod.race_keys(oracle_mod.bruteforce(tr, 256))
    reg = dict(n_words=info["n_words"], block_dim=256, shadow_bytes=4, tid_bits=16)
    races, status, n_total, _ = bin_check(hr, tr, reg)
    assert status == hr.HR_OK and hr.race_keys(races) == want and n_total == len(want)
    # a thread id wider than the packing stops the check
    reg = dict(n_words=info["n_words"], block_dim=256, shadow_bytes=4, tid_bits=8)
    _, status, _, _ = bin_check(hr, tr, reg)
    assert hr.STATUS[status] == "HR_ERR_CLOCK_OVERFLOW"


def test_filters(oracle_mod, hr):
    from tests.test_gpu_filter import FILTERS, keep_mask
    tr, info = tg.gen_global_mix(tg.seed_for(2, 24), inject=True, n_blocks=16)
    for f in FILTERS:
        want = oracle_mod.race_keys(oracle_mod.bruteforce(tr[keep_mask(tr, 256, **f)], 256, 32))
        n_words = (f["word_hi"] - f["word_lo"]) if f.get("word_hi") else info["n_words"]
        races, status, n_total, _ = bin_check(hr, tr, dict(n_words=n_words, block_dim=256), filt=f)
        assert status == hr.HR_OK and hr.race_keys(races) == want and n_total == len(want), f


def test_error_statuses(hr):
    tr, info = tg.gen_global_mix(tg.seed_for(2, 25), inject=True, n_blocks=8)
    reg = dict(n_words=info["n_words"], block_dim=256)
    bad = tr.copy()
    bad[[100, len(bad) - 100]] = bad[[len(bad) - 100, 100]]
    assert hr.STATUS[bin_check(hr, bad, reg)[1]] == "HR_ERR_ORDER"
    assert hr.STATUS[bin_check(hr, tr, dict(reg, n_words=1 << 10))[1]] == "HR_ERR_RANGE"
    bad = tr.copy()
    sw = np.flatnonzero(bad["op"] == tg.OP_SYNCWARP)[5]
    bad["flags"][sw] = tg.FLAG_PARTIAL_MASK
    assert hr.STATUS[bin_check(hr, bad, reg)[1]] == "HR_ERR_UNSUPPORTED"
