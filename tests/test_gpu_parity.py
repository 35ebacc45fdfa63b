"""GPU checker == CPU oracle, through the C-ABI.

Race keys (kernel, word, epoch) must match bit for bit; the reported op must be
one the oracle says can complete the first racy pair (several are possible
inside one wave).  Every case runs the warp-aggregated and the plain kernel.
"""
import os

import numpy as np
import pytest

from paper_2401_04701_gb300 import tracegen as tg
from tests import _cases as C

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


def gpu_check(hr, trace, n_words, block_dim, warp_size=32, aggregate=True, chunks=None, cap=1 << 20):
    with hr.Checker([dict(n_words=n_words, block_dim=block_dim, warp_size=warp_size)], report_capacity=cap) as ck:
        if chunks is None:
            ck.check_trace(0, to_dev(trace), aggregate=aggregate)
        else:
            for a, b in zip(chunks[:-1], chunks[1:]):
                if b > a:
                    ck.check_trace(0, to_dev(trace[a:b]), aggregate=aggregate)
        races, status, n_total, flags = ck.report(0)
        cnt = ck.counters(0)
    return races, status, n_total, flags, cnt


def assert_parity(O, hr, trace, n_words, block_dim, warp_size=32, aggregate=True, chunks=None):
    bf = O.bruteforce(trace, block_dim, warp_size)
    races, status, n_total, flags, _ = gpu_check(hr, trace, n_words, block_dim, warp_size, aggregate, chunks)
    assert status == hr.HR_OK, hr.STATUS[status]
    assert n_total == len(races) == len(bf)
    assert hr.race_keys(races) == O.race_keys(bf)
    ops = {(int(k), int(w)): int(m) for k, w, m in zip(bf["kernel"], bf["word"], bf["ops_mask"])}
    for k, w, op in zip(races["kernel"], races["word"], races["op"]):
        assert (ops[(int(k), int(w))] >> int(op)) & 1
    return races


@pytest.mark.parametrize("aggregate", [True, False])
@pytest.mark.parametrize("name", ["listing1_no_sync", "listing2_block_sync", "listing2_one_block",
                                  "listing3_multi_read"])
def test_listings(oracle_mod, hr, name, aggregate):
    g = C.load_golden(name)
    tr = C.golden_trace(g)
    races = assert_parity(oracle_mod, hr, tr, g["n_words"], g["block_dim"], g["warp_size"], aggregate)
    assert hr.race_keys(races) == {tuple(x) for x in g["expected_races"]}


@pytest.mark.parametrize("aggregate", [True, False])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_exhaustive_universe(oracle_mod, hr, k, aggregate):
    rng = np.random.default_rng(50 + k)
    cases = C.exhaustive_cases(k, C.PHASES4)
    base = C.combined_trace(cases, C.PHASES4)
    for tr in (base, tg.shuffle_within_waves(base, rng)):
        assert_parity(oracle_mod, hr, tr, len(cases), C.TOY_BLOCK_DIM, C.TOY_WARP, aggregate)


@pytest.mark.parametrize("aggregate", [True, False])
def test_random_deep_and_multi_kernel(oracle_mod, hr, aggregate):
    rng = np.random.default_rng(60)
    cases = C.random_cases(rng, 20000, 10, C.PHASES4)
    assert_parity(oracle_mod, hr, C.combined_trace(cases, C.PHASES4), len(cases), C.TOY_BLOCK_DIM, C.TOY_WARP,
                  aggregate)
    for _ in range(10):
        bd = int(rng.choice([3, 40, 64, 256]))
        ws = int(rng.choice([2, 32]))
        kernels = C.random_program(rng, n_threads=int(rng.integers(2, 600)), block_dim=bd, n_words=16,
                                   n_acc=int(rng.integers(1, 3000)), n_st=int(rng.integers(0, 4)),
                                   n_sw=int(rng.integers(0, 4)), n_kernels=int(rng.integers(1, 20)))
        tr = tg.build_trace(kernels)
        assert_parity(oracle_mod, hr, tr, 16, bd, ws, aggregate)


@pytest.mark.parametrize("aggregate", [True, False])
def test_tree_reduction_workload(oracle_mod, hr, aggregate):
    tr, info = tg.gen_tree_reduction(tg.seed_for(1), inject=False)
    races, status, n_total, _, _ = gpu_check(hr, tr, info["n_words"], info["block_dim"], aggregate=aggregate)
    assert status == hr.HR_OK and n_total == 0
    tr, info = tg.gen_tree_reduction(tg.seed_for(1), inject=True)
    assert_parity(oracle_mod, hr, tr, info["n_words"], info["block_dim"], aggregate=aggregate)


@pytest.mark.parametrize("aggregate", [True, False])
def test_global_mix_small(oracle_mod, hr, aggregate):
    tr, info = tg.gen_global_mix(tg.seed_for(2, 1), inject=True, n_blocks=16)
    races = assert_parity(oracle_mod, hr, tr, info["n_words"], info["block_dim"], aggregate=aggregate)
    assert set(races["word"].tolist()) == set(info["injected"].tolist())


def test_global_mix_full_size(oracle_mod, hr):
    """The benchmark workload at full size (1024 x 256 threads, 2^26 words, 75.2M
    records) in the configuration bench.py times: the autotuner's variant, and
    the trace checked as a later kernel launch (rebased kernel ordinal)."""
    tr, info = tg.gen_global_mix(tg.seed_for(2), inject=True)
    bf = oracle_mod.bruteforce(tr, info["block_dim"])
    want = oracle_mod.race_keys(bf)
    assert len(want) == len(info["injected"]) == 67108
    d = to_dev(tr)
    with hr.Checker([dict(n_words=info["n_words"], block_dim=256)], report_capacity=1 << 22) as ck:
        best, _ = ck.autotune(0, d)
        ck.check_trace(0, d)
        races, status, n_total, _ = ck.report(0)
        assert status == hr.HR_OK and hr.race_keys(races) == want and n_total == len(want)
        ck.reset(0)
        for kb in (3, 4):
            ck.check_trace(0, d, kernel_base=kb)
        races, status, n_total, _ = ck.report(0)
        assert status == hr.HR_OK and n_total == 2 * len(want)
        assert hr.race_keys(races) == {(kb, w, e) for kb in (3, 4) for (_, w, e) in want}


def test_chunked_calls_equal_one_call(oracle_mod, hr):
    tr, info = tg.gen_global_mix(tg.seed_for(2, 2), inject=True, n_blocks=8)
    rng = np.random.default_rng(3)
    cuts = np.sort(rng.integers(0, len(tr), 9))      # cuts land inside waves too
    chunks = [0] + cuts.tolist() + [len(tr)]
    assert_parity(oracle_mod, hr, tr, info["n_words"], info["block_dim"], chunks=chunks)


def test_many_tiny_waves_and_ragged_tail(oracle_mod, hr):
    # 2000 block epochs of a few records each; lengths not multiples of a tile
    rng = np.random.default_rng(4)
    progs = {}
    for t in range(70):
        ev = []
        for e in range(2000):
            if rng.random() < 0.3:
                ev.append(("RWA"[int(rng.integers(0, 3))], int(rng.integers(0, 50))))
            ev.append(("ST",))
        progs[t] = ev
    tr = tg.build_trace([progs])
    assert_parity(oracle_mod, hr, tr, 50, 70, 32)


def test_empty_and_single_record(oracle_mod, hr):
    import torch
    with hr.Checker([dict(n_words=4, block_dim=32)]) as ck:
        ck.check_trace(0, torch.zeros(0, dtype=torch.uint8, device="cuda"))
        one = tg.build_trace([{0: [("W", 3)]}])
        ck.check_trace(0, to_dev(one))
        races, status, n_total, _ = ck.report(0)
        assert status == hr.HR_OK and n_total == 0


def test_kernel_base_and_sync(oracle_mod, hr):
    tr = tg.build_trace([{0: [("W", 1)], 40: [("W", 1)]}])        # one race per launch
    with hr.Checker([dict(n_words=4, block_dim=32)]) as ck:
        for kb in range(0, 20):
            ck.check_trace(0, to_dev(tr), kernel_base=kb)
        races, status, n_total, _ = ck.report(0)
        assert status == hr.HR_OK
        assert hr.race_keys(races) == {(kb, 1, 0) for kb in range(20)}
        ck.sync(0)                       # kernel 19 ended: kernel 19 again is out of order
        ck.check_trace(0, to_dev(tr), kernel_base=19)
        _, status, _, _ = ck.report(0)
        assert hr.STATUS[status] == "HR_ERR_ORDER"


def test_errors_are_reported_not_faulted(hr):
    good = tg.build_trace([{0: [("W", 1), ("ST",), ("R", 1)], 1: [("ST",), ("R", 2)]}])
    cases = {}
    bad = good.copy()
    bad["word"][-1] = 100
    cases["HR_ERR_RANGE"] = bad
    cases["HR_ERR_ORDER"] = good[::-1].copy()
    partial = tg.build_trace([{0: [("SW", tg.FLAG_PARTIAL_MASK), ("R", 1)]}])
    cases["HR_ERR_UNSUPPORTED"] = partial
    over = tg.build_trace([{0: [("R", 1)]}])
    over["wc"] = 300
    cases["HR_ERR_CLOCK_OVERFLOW"] = over
    badop = good.copy()
    badop["op"][0] = 9
    cases["HR_ERR_UNSUPPORTED "] = badop
    for want, tr in cases.items():
        with hr.Checker([dict(n_words=4, block_dim=32)]) as ck:
            ck.check_trace(0, to_dev(tr))
            _, status, _, _ = ck.report(0)
            assert hr.STATUS[status] == want.strip(), want


def test_report_ring_overflow_keeps_exact_count(oracle_mod, hr):
    tr, info = tg.gen_global_mix(tg.seed_for(2, 3), inject=True, n_blocks=8)
    n_expected = len(oracle_mod.bruteforce(tr, 256))
    with hr.Checker([dict(n_words=info["n_words"], block_dim=256, report_capacity=100)]) as ck:
        ck.check_trace(0, to_dev(tr))
        races, status, n_total, flags = ck.report(0)
    assert status == hr.HR_OK and n_total == n_expected and len(races) == 100
    assert flags & hr.FLAG_TRUNCATED


def test_wave_capacity_error(hr, monkeypatch):
    monkeypatch.setenv("HR_MAX_WAVES", "8")
    tr = tg.build_trace([{t: [("R", t), ("ST",)] * 20 for t in range(4)}])
    with hr.Checker([dict(n_words=8, block_dim=4)]) as ck:
        ck.check_trace(0, to_dev(tr))
        _, status, _, _ = ck.report(0)
    assert hr.STATUS[status] == "HR_ERR_CAPACITY"


@pytest.mark.parametrize("aggregate", [True, False])
def test_powerlaw_push_small(oracle_mod, hr, aggregate):
    tr, info = tg.gen_powerlaw_push(tg.seed_for(3, 1), log2_vertices=15, sweeps=3)
    races = assert_parity(oracle_mod, hr, tr, info["n_words"], info["block_dim"], aggregate=aggregate)
    assert len(races) > 0
    clean, _ = tg.gen_powerlaw_push(tg.seed_for(3, 1), log2_vertices=15, sweeps=3, inject=False)
    _, status, n_total, _, cnt = gpu_check(hr, clean, info["n_words"], info["block_dim"], aggregate=aggregate)
    assert status == hr.HR_OK and n_total == 0
    if aggregate:
        assert cnt["merged"] > 0          # repeated dist[src] reads fold into one update


@pytest.fixture(scope="module")
def powerlaw_full(oracle_mod):
    """The power-law push workload at full size (2^22 vertices, 2^26 edges, 4
    sweeps: 536,870,912 records) and the oracle's complete race set, computed
    by the brute force on disjoint word ranges over all host cores."""
    tr, info = tg.gen_powerlaw_push(tg.seed_for(3))
    bf = oracle_mod.bruteforce_parallel(tr, info["block_dim"], info["n_words"])
    return tr, info, oracle_mod.race_keys(bf)


@pytest.mark.slow
def test_powerlaw_push_full_size(oracle_mod, hr, powerlaw_full):
    """Every racy (kernel, word, epoch) of the full trace, hub words included,
    for the autotuned variant (as bench.py runs it), the plain kernel and the
    warp-aggregated kernel."""
    tr, info, want = powerlaw_full
    assert len(want) > 0
    d = to_dev(tr)
    with hr.Checker([dict(n_words=info["n_words"], block_dim=info["block_dim"])], report_capacity=1 << 24) as ck:
        ck.autotune(0, d)
        for agg in (None, True, False):
            ck.reset(0)
            if agg is None:
                ck.check_trace(0, d)
            else:
                ck.check_trace(0, d, aggregate=agg)
            races, status, n_total, _ = ck.report(0)
            assert status == hr.HR_OK and n_total == len(races) == len(want), agg
            assert hr.race_keys(races) == want, agg


@pytest.mark.slow
def test_powerlaw_push_full_size_sampled(oracle_mod, hr, powerlaw_full):
    """The same trace, checked against the oracle run on a sample of words
    (every injected word's records plus random words) on their own: a word's
    result depends on its records alone."""
    tr, info, want_all = powerlaw_full
    races, status, n_total, _, _ = gpu_check(hr, tr, info["n_words"], info["block_dim"], cap=1 << 24)
    assert status == hr.HR_OK and n_total == len(races)
    rng = np.random.default_rng(9)
    inj_words = np.unique(tr["word"][info["injected"]])
    sample = np.unique(np.concatenate([rng.choice(inj_words, 3000, replace=False),
                                       rng.integers(0, info["n_words"], 3000)]))
    keep = np.isin(tr["word"], sample)
    sub = tr[keep]
    want = oracle_mod.race_keys(oracle_mod.bruteforce(sub, info["block_dim"]))
    words = set(sample.tolist())
    got = {k for k in hr.race_keys(races) if k[1] in words}
    assert got == want == {k for k in want_all if k[1] in words}
    assert len(want) > 0


def test_bounded_wait_reports_timeout_and_context_recovers(oracle_mod, hr):
    """A stage dependency that nothing satisfies: the wait runs out after its
    bound, the region reports HR_ERR_TIMEOUT, and the next check is exact."""
    import time
    tr, info = tg.gen_global_mix(tg.seed_for(2, 8), inject=True, n_blocks=4)
    want = oracle_mod.race_keys(oracle_mod.bruteforce(tr, 256))
    with hr.Checker([dict(n_words=info["n_words"], block_dim=256)]) as ck:
        ck.set_limits(wait_ns=200_000_000, test_flags=1)
        t0 = time.perf_counter()
        ck.check_trace(0, to_dev(tr))
        _, status, _, _ = ck.report(0)
        took = time.perf_counter() - t0
        assert hr.STATUS[status] == "HR_ERR_TIMEOUT"
        assert took < 5.0
        ck.set_limits()
        ck.reset(0)
        ck.check_trace(0, to_dev(tr))
        races, status, _, _ = ck.report(0)
        assert status == hr.HR_OK and hr.race_keys(races) == want


def test_cas_retry_cap_reports_contention(hr):
    """Zero retries allowed and 64K threads of 256 blocks writing one word in one
    wave: some CAS loses and the region reports HR_ERR_CONTENTION."""
    n = 1 << 16
    tr = np.zeros(n, tg.RECORD)
    tr["tid"] = np.arange(n)
    tr["op"] = tg.OP_W
    with hr.Checker([dict(n_words=1, block_dim=256)]) as ck:
        ck.set_limits(cas_retry_cap=0)
        ck.check_trace(0, to_dev(tr), aggregate=False)
        _, status, _, _ = ck.report(0)
        assert hr.STATUS[status] == "HR_ERR_CONTENTION"
        ck.set_limits()
        ck.reset(0)
        ck.check_trace(0, to_dev(tr), aggregate=False)
        races, status, n_total, _ = ck.report(0)
        assert status == hr.HR_OK and n_total == 1


@pytest.fixture(scope="module")
def variant_cases():
    cases = []
    g = C.load_golden("listing2_block_sync")
    cases.append((C.golden_trace(g), g["n_words"], g["block_dim"], g["warp_size"]))
    ex = C.exhaustive_cases(3, C.PHASES4)
    cases.append((C.combined_trace(ex, C.PHASES4), len(ex), C.TOY_BLOCK_DIM, C.TOY_WARP))
    tr, info = tg.gen_global_mix(tg.seed_for(2, 9), inject=True, n_blocks=8)
    cases.append((tr, info["n_words"], 256, 32))
    tr, info = tg.gen_powerlaw_push(tg.seed_for(3, 9), log2_vertices=14, sweeps=2)
    cases.append((tr, info["n_words"], 256, 32))
    tr, info = tg.gen_tree_reduction(tg.seed_for(1, 9), segments=8, reps=3)
    cases.append((tr, info["n_words"], 256, 32))
    return cases


def test_every_kernel_variant_matches_oracle(oracle_mod, hr, variant_cases):
    for v, desc in hr.variants():
        for tr, nw, bd, ws in variant_cases:
            with hr.Checker([dict(n_words=nw, block_dim=bd, warp_size=ws)]) as ck:
                ck.set_variant(v)
                ck.check_trace(0, to_dev(tr))
                races, status, n_total, _ = ck.report(0)
            want = oracle_mod.race_keys(oracle_mod.bruteforce(tr, bd, ws))
            assert status == hr.HR_OK and hr.race_keys(races) == want, (v, desc)


def test_autotune_keeps_the_fastest(oracle_mod, hr):
    tr, info = tg.gen_global_mix(tg.seed_for(2, 10), inject=True, n_blocks=16)
    want = oracle_mod.race_keys(oracle_mod.bruteforce(tr, 256))
    with hr.Checker([dict(n_words=info["n_words"], block_dim=256)]) as ck:
        d = to_dev(tr)
        best, ms = ck.autotune(0, d)
        assert ck.variant() == best and ms[best] == min(ms) and all(t > 0 for t in ms)
        ck.check_trace(0, d)
        races, status, _, _ = ck.report(0)
    assert status == hr.HR_OK and hr.race_keys(races) == want


@pytest.mark.parametrize("chunk", [0, 4096, 100_003])
def test_check_from_host_memory(oracle_mod, hr, chunk):
    """hr_check_trace_host: chunks copied through two staging buffers while the
    previous chunk is checked give the oracle's races, pinned or pageable."""
    import torch
    tr, info = tg.gen_global_mix(tg.seed_for(2, 11), inject=True, n_blocks=8)
    want = oracle_mod.race_keys(oracle_mod.bruteforce(tr, info["block_dim"]))
    pinned = torch.from_numpy(tr.view(np.uint8)).pin_memory()
    with hr.Checker([dict(n_words=info["n_words"], block_dim=256)], report_capacity=1 << 20) as ck:
        for host in (pinned, np.ascontiguousarray(tr)):
            ck.reset(0)
            ck.check_trace_host(0, host, chunk_records=chunk)
            races, status, n_total, _ = ck.report(0)
            assert status == hr.HR_OK and hr.race_keys(races) == want and n_total == len(want)
