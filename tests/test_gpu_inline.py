"""Inline device path: kernels instrumented by hand with hr_access() find
exactly the races the oracle finds on the same access program.

The access program of each synthetic kernel is rebuilt on the host as a trace
(paper_2401_04701_gb300.tracegen.*_program) and checked by the oracle.  These
kernels' races are either inside one block or between blocks with no barrier
in between, so even the epoch of each race is schedule-independent and the
whole (kernel, word, epoch) key is compared.
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
    hirace.load_workloads()
    return hirace


def oracle_keys(O, trace, n_words, block=256):
    assert O.validate(trace) == (0, 0)
    return O.race_keys(O.bruteforce(trace, block, 32))


@pytest.mark.parametrize("racy", [0, 7, 1000])
def test_stencil(oracle_mod, hr, racy):
    import torch
    n = 1 << 20
    d_in = torch.rand(n, device="cuda")
    d_out = torch.zeros(n, device="cuda")
    with hr.Checker([dict(n_words=2 * n, block_dim=256)]) as ck:
        hr.run_stencil(ck.device_view(0), d_in, d_out, racy_stride=racy)
        races, status, n_total, _ = ck.report(0)
    assert status == hr.HR_OK
    want = oracle_keys(oracle_mod, tg.stencil_program(n, racy), 2 * n)
    assert hr.race_keys(races) == want and n_total == len(want)
    if racy == 0:
        assert n_total == 0


def test_stencil_instrumentation_keeps_results(hr):
    import torch
    n = 1 << 16
    d_in = torch.rand(n, device="cuda")
    a, b = torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    with hr.Checker([dict(n_words=2 * n, block_dim=256)]) as ck:
        hr.run_stencil(ck.device_view(0), d_in, a)
        hr.run_stencil(None, d_in, b)
        torch.cuda.synchronize()
    assert torch.equal(a, b)


@pytest.mark.parametrize("racy", [0, 13])
def test_histogram(oracle_mod, hr, racy):
    import torch
    n, n_bins = 1 << 20, 4096
    keys = np.random.default_rng(5).integers(0, n_bins, n).astype(np.uint32)
    d_keys = torch.from_numpy(keys.view(np.int32)).cuda()
    d_bins = torch.zeros(n_bins, dtype=torch.int32, device="cuda")
    with hr.Checker([dict(n_words=n_bins, block_dim=256)]) as ck:
        hr.run_histogram(ck.device_view(0), d_keys, d_bins, racy_stride=racy)
        races, status, n_total, _ = ck.report(0)
    assert status == hr.HR_OK
    want = oracle_keys(oracle_mod, tg.histogram_program(keys, racy), n_bins)
    assert hr.race_keys(races) == want and n_total == len(want)


@pytest.mark.parametrize("drop", [-1, 0, 4, 7])
def test_reduction(oracle_mod, hr, drop):
    import torch
    n = 1 << 20
    d = torch.rand(n, device="cuda")
    with hr.Checker([dict(n_words=n, block_dim=256)]) as ck:
        hr.run_reduce(ck.device_view(0), d, drop_level=drop)
        races, status, n_total, _ = ck.report(0)
    assert status == hr.HR_OK
    want = oracle_keys(oracle_mod, tg.reduce_program(n, 256, drop), n)
    assert hr.race_keys(races) == want and n_total == len(want)
    if drop < 0:
        assert n_total == 0


def test_kernel_end_between_launches(oracle_mod, hr):
    """hr_sync between two instrumented launches: each launch is checked on its own."""
    import torch
    n = 1 << 16
    d_in = torch.rand(n, device="cuda")
    d_out = torch.zeros(n, device="cuda")
    want = oracle_keys(oracle_mod, tg.stencil_program(n, 5), 2 * n)
    with hr.Checker([dict(n_words=2 * n, block_dim=256)]) as ck:
        for k in range(10):                      # crosses a kernel-tag group of 8
            hr.run_stencil(ck.device_view(0), d_in, d_out, racy_stride=5 if k % 2 else 0)
            ck.sync(0)
        races, status, n_total, _ = ck.report(0)
    assert status == hr.HR_OK
    got = hr.race_keys(races)
    assert got == {(k, w, e) for k in range(1, 10, 2) for (_, w, e) in want}


@pytest.mark.parametrize("drop", [-1, 0, 3, 7])
def test_shared_memory_shadow(oracle_mod, hr, drop):
    """Block reduction through __shared__ memory: the shadow in shared memory
    (hr_access_shared) and the region's global shadow (hr_access) report the
    oracle's races on the per-block word numbering, and the sums are unchanged."""
    import torch
    n, block = 1 << 18, 256
    d_in = torch.rand(n, device="cuda")
    grid = n // block
    want = oracle_keys(oracle_mod, tg.smem_reduce_program(n, block, drop), n)
    if drop < 0:
        assert not want
    outs = []
    for mode in (1, 2):
        out = torch.zeros(grid, device="cuda")
        with hr.Checker([dict(n_words=n, block_dim=block)]) as ck:
            hr.run_smem_reduce(ck.device_view(0), d_in, out, mode, block, drop)
            races, status, n_total, _ = ck.report(0)
        assert status == hr.HR_OK
        assert hr.race_keys(races) == want and n_total == len(want)
        outs.append(out)
    plain = torch.zeros(grid, device="cuda")
    hr.run_smem_reduce(None, d_in, plain, 0, block, drop)
    torch.cuda.synchronize()
    if drop < 0:
        assert torch.equal(outs[0], plain) and torch.equal(outs[1], plain)
