"""Batched checks: many traces, each on its own region, in one persistent launch.

Per region the races equal the oracle's and equal a single-trace check of the
same trace; a job that fails validation leaves the others untouched; a
CUDA-graph capture of (reset, batch) replays with the same results.
"""
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


def mixed_jobs():
    """(trace, n_words, block_dim, warp_size) for a varied set of traces."""
    rng = np.random.default_rng(21)
    jobs = []
    for name in ("listing1_no_sync", "listing2_block_sync", "listing2_one_block", "listing3_multi_read"):
        g = C.load_golden(name)
        jobs.append((C.golden_trace(g), g["n_words"], g["block_dim"], g["warp_size"]))
    for k in (2, 3):
        cases = C.exhaustive_cases(k, C.PHASES4)
        jobs.append((C.combined_trace(cases, C.PHASES4), len(cases), C.TOY_BLOCK_DIM, C.TOY_WARP))
    tr, info = tg.gen_tree_reduction(tg.seed_for(1, 3), segments=8, reps=4)
    jobs.append((tr, info["n_words"], info["block_dim"], 32))
    tr, info = tg.gen_global_mix(tg.seed_for(2, 5), n_blocks=4)
    jobs.append((tr, info["n_words"], info["block_dim"], 32))
    tr, info = tg.gen_powerlaw_push(tg.seed_for(3, 5), log2_vertices=12, sweeps=3)
    jobs.append((tr, info["n_words"], info["block_dim"], 32))
    for _ in range(20):
        bd = int(rng.choice([3, 40, 64, 256]))
        kernels = C.random_program(rng, n_threads=int(rng.integers(2, 400)), block_dim=bd, n_words=8,
                                   n_acc=int(rng.integers(1, 2000)), n_st=int(rng.integers(0, 4)),
                                   n_sw=int(rng.integers(0, 3)), n_kernels=int(rng.integers(1, 12)))
        jobs.append((tg.build_trace(kernels), 8, bd, 32))
    return jobs


def test_batch_equals_oracle_and_single(oracle_mod, hr):
    jobs = mixed_jobs()
    regions = [dict(n_words=nw, block_dim=bd, warp_size=ws) for _, nw, bd, ws in jobs]
    dev = [to_dev(tr) for tr, _, _, _ in jobs]
    with hr.Checker(regions) as batch, hr.Checker(regions) as single:
        batch.check_batch([(i, d) for i, d in enumerate(dev)])
        for i, d in enumerate(dev):
            single.check_trace(i, d)
        for i, (tr, nw, bd, ws) in enumerate(jobs):
            want = oracle_mod.race_keys(oracle_mod.bruteforce(tr, bd, ws))
            rb, sb, nb, _ = batch.report(i)
            rs, ss, ns, _ = single.report(i)
            assert sb == hr.HR_OK and ss == hr.HR_OK
            assert hr.race_keys(rb) == want == hr.race_keys(rs), i
            assert nb == ns == len(want)


def test_batch_failing_job_is_isolated(oracle_mod, hr):
    good, info = tg.gen_global_mix(tg.seed_for(2, 6), n_blocks=4)
    bad = good.copy()
    bad["word"][len(bad) // 2] = info["n_words"] + 5           # out of range
    unsorted = good[::-1].copy()
    regions = [dict(n_words=info["n_words"], block_dim=256)] * 3
    with hr.Checker(regions) as ck:
        ck.check_batch([(0, to_dev(good)), (1, to_dev(bad)), (2, to_dev(unsorted))])
        r0, s0, n0, _ = ck.report(0)
        _, s1, _, _ = ck.report(1)
        _, s2, _, _ = ck.report(2)
    assert s0 == hr.HR_OK
    assert hr.race_keys(r0) == oracle_mod.race_keys(oracle_mod.bruteforce(good, 256))
    assert hr.STATUS[s1] == "HR_ERR_RANGE" and hr.STATUS[s2] == "HR_ERR_ORDER"


def test_batch_rejects_duplicate_regions(hr):
    tr = tg.build_trace([{0: [("W", 1)]}])
    with hr.Checker([dict(n_words=4, block_dim=32)] * 2) as ck:
        d = to_dev(tr)
        with pytest.raises(hr.HiRaceError):
            ck.check_batch([(0, d), (0, d)])


def test_batch_in_cuda_graph(oracle_mod, hr):
    import torch
    jobs = mixed_jobs()[4:10]
    regions = [dict(n_words=nw, block_dim=bd, warp_size=ws) for _, nw, bd, ws in jobs]
    dev = [to_dev(tr) for tr, _, _, _ in jobs]
    want = [oracle_mod.race_keys(oracle_mod.bruteforce(tr, bd, ws)) for tr, _, bd, ws in jobs]
    with hr.Checker(regions) as ck:
        ck.batch_reserve(len(jobs), 1 << 16)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):                       # warm-up outside capture
            for i in range(len(jobs)):
                ck.reset(i, stream=s)
            ck.check_batch(list(enumerate(dev)), stream=s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            for i in range(len(jobs)):
                ck.reset(i, stream=s)
            ck.check_batch(list(enumerate(dev)), stream=s)
        for _ in range(3):
            g.replay()
            torch.cuda.synchronize()
            for i in range(len(jobs)):
                races, status, n_total, _ = ck.report(i)
                assert status == hr.HR_OK and hr.race_keys(races) == want[i]


def test_uneven_batch_workload(oracle_mod, hr):
    """64 traces of the batch workload (lengths 1K..200K, shared and global kinds)."""
    jobs = tg.gen_batch(tg.seed_for(4, 1), n_traces=64, min_len=1000, max_len=200_000)
    regions = [dict(n_words=info["n_words"], block_dim=info["block_dim"]) for _, info in jobs]
    dev = [to_dev(tr) for tr, _ in jobs]
    with hr.Checker(regions, report_capacity=1 << 16) as ck:
        ck.check_batch(list(enumerate(dev)))
        for i, (tr, info) in enumerate(jobs):
            want = oracle_mod.race_keys(oracle_mod.bruteforce(tr, info["block_dim"]))
            races, status, n_total, _ = ck.report(i)
            assert status == hr.HR_OK and hr.race_keys(races) == want, i


@pytest.mark.slow
def test_full_batch_workload_equals_oracle(oracle_mod, hr):
    """The batch workload at full size: 512 traces (lengths log-uniform 10K..10M,
    600.6M records, 60% shared-memory and 40% global-memory traces) in one
    batched launch, the way bench.py times it; every trace's race set equals the
    oracle's brute force on that trace, and one launch per trace gives the same."""
    from concurrent.futures import ThreadPoolExecutor
    jobs = tg.gen_batch(tg.seed_for(4))
    assert len(jobs) == 512
    with ThreadPoolExecutor(len(__import__("os").sched_getaffinity(0))) as ex:
        want = list(ex.map(lambda j: oracle_mod.race_keys(oracle_mod.bruteforce(j[0], j[1]["block_dim"])), jobs))
    regions = [dict(n_words=info["n_words"], block_dim=info["block_dim"]) for _, info in jobs]
    dev = [to_dev(tr) for tr, _ in jobs]
    del jobs
    with hr.Checker(regions, report_capacity=1 << 18) as ck:
        ck.batch_reserve(len(dev), 1 << 18)
        ck.check_batch(list(enumerate(dev)))
        for i in range(len(dev)):
            races, status, n_total, _ = ck.report(i)
            assert status == hr.HR_OK and n_total == len(want[i]) and hr.race_keys(races) == want[i], i
        for i in range(len(dev)):
            ck.reset(i)
        for i, d in enumerate(dev):
            ck.check_trace(i, d)
        for i in range(len(dev)):
            races, status, n_total, _ = ck.report(i)
            assert status == hr.HR_OK and hr.race_keys(races) == want[i], i
    assert sum(len(x) for x in want) > 0


def test_batch_job_completion_times(hr):
    """hr_batch_job_times: one device-clock completion time per job of the last
    batch; an empty trace reads 0; no job ends after the batch's own span, and
    the last one ends late in it (stages interleave wave-major, so the job with
    the most waves tends to end last, not the longest)."""
    import torch
    jobs = mixed_jobs()
    big, info = tg.gen_global_mix(tg.seed_for(2, 13), n_blocks=64)
    regions = [dict(n_words=nw, block_dim=bd, warp_size=ws) for _, nw, bd, ws in jobs]
    regions.append(dict(n_words=info["n_words"], block_dim=256))
    regions.append(dict(n_words=8, block_dim=32))
    dev = [to_dev(tr) for tr, _, _, _ in jobs] + [to_dev(big), to_dev(big[:0])]
    with hr.Checker(regions) as ck:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        ck.check_batch(list(enumerate(dev)))
        b.record()
        torch.cuda.synchronize()
        span_ns = a.elapsed_time(b) * 1e6
        t = ck.batch_job_times(len(dev))
        for i in range(len(dev) - 1):
            assert ck.report(i)[1] == hr.HR_OK
    assert t[-1] == 0                                  # the empty trace
    assert (t[:-1] > 0).all() and t[:-1].max() <= span_ns
    assert t[:-1].max() >= 0.5 * span_ns
