"""Every-epoch reporting (report_mode REPORT_EVERY_EPOCH) == the oracle's
every-racy-epoch brute force.

In this mode RACE is not absorbing: each (kernel, word, epoch) in which some
access completes a racy pair is reported once, with the op of an access that
completes one.
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


def every_check(hr, trace, n_words, block_dim, warp_size=32, aggregate=True, variant=None):
    reg = dict(n_words=n_words, block_dim=block_dim, warp_size=warp_size, report_mode=hr.REPORT_EVERY_EPOCH)
    with hr.Checker([reg], report_capacity=1 << 21) as ck:
        if variant is not None:
            ck.set_variant(variant)
        ck.check_trace(0, to_dev(trace), aggregate=aggregate)
        return ck.report(0)


def assert_parity(O, hr, trace, n_words, block_dim, warp_size=32, aggregate=True, variant=None):
    want = O.bruteforce_epochs(trace, block_dim, warp_size)
    races, status, n_total, _ = every_check(hr, trace, n_words, block_dim, warp_size, aggregate, variant)
    assert status == hr.HR_OK, hr.STATUS[status]
    assert n_total == len(races) == len(want)
    assert hr.race_keys(races) == O.race_keys(want)
    ops = {(int(k), int(w), int(e)): int(m) for k, w, e, m in zip(want["kernel"], want["word"], want["epoch"],
                                                                    want["ops_mask"])}
    for k, w, e, op in zip(races["kernel"], races["word"], races["epoch"], races["op"]):
        assert (ops[(int(k), int(w), int(e))] >> int(op)) & 1
    return races


@pytest.mark.parametrize("name", ["listing1_no_sync", "listing2_block_sync", "listing3_multi_read"])
def test_listings(oracle_mod, hr, name):
    g = C.load_golden(name)
    assert_parity(oracle_mod, hr, C.golden_trace(g), g["n_words"], g["block_dim"], g["warp_size"])


@pytest.mark.parametrize("aggregate", [True, False])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_exhaustive_universe(oracle_mod, hr, k, aggregate):
    rng = np.random.default_rng(90 + k)
    cases = C.exhaustive_cases(k, C.PHASES4)
    base = C.combined_trace(cases, C.PHASES4)
    for tr in (base, tg.shuffle_within_waves(base, rng)):
        assert_parity(oracle_mod, hr, tr, len(cases), C.TOY_BLOCK_DIM, C.TOY_WARP, aggregate)


def test_random_programs(oracle_mod, hr):
    rng = np.random.default_rng(91)
    cases = C.random_cases(rng, 20000, 10, C.PHASES4)
    assert_parity(oracle_mod, hr, C.combined_trace(cases, C.PHASES4), len(cases), C.TOY_BLOCK_DIM, C.TOY_WARP)
    for _ in range(10):
        bd = int(rng.choice([3, 40, 64, 256]))
        ws = int(rng.choice([2, 32]))
        kernels = C.random_program(rng, n_threads=int(rng.integers(2, 600)), block_dim=bd, n_words=16,
                                   n_acc=int(rng.integers(1, 3000)), n_st=int(rng.integers(0, 4)),
                                   n_sw=int(rng.integers(0, 4)), n_kernels=int(rng.integers(1, 20)))
        assert_parity(oracle_mod, hr, tg.build_trace(kernels), 16, bd, ws)


def test_tree_reduction(oracle_mod, hr):
    tr, info = tg.gen_tree_reduction(tg.seed_for(1), inject=True)
    assert_parity(oracle_mod, hr, tr, info["n_words"], info["block_dim"])


@pytest.mark.parametrize("variant", [0, 3])
def test_global_mix_small(oracle_mod, hr, variant):
    """Injected cross-block writes race in several epochs: more reports than racy words."""
    tr, info = tg.gen_global_mix(tg.seed_for(2, 8), inject=True, n_blocks=16)
    races = assert_parity(oracle_mod, hr, tr, info["n_words"], info["block_dim"], variant=variant)
    assert len(races) > len(set(races["word"].tolist()))


def test_with_filter(oracle_mod, hr):
    """Every-epoch mode behind a word window and a block range."""
    tr, info = tg.gen_global_mix(tg.seed_for(2, 9), inject=True, n_blocks=16)
    lo, hi = 1 << 19, 3 << 19
    w = tr["word"].astype(np.int64)
    blk = tr["tid"].astype(np.int64) // 256
    keep = (tr["op"] > tg.OP_A) | ((w >= lo) & (w < hi) & (blk >= 2) & (blk < 12))
    want = oracle_mod.race_keys(oracle_mod.bruteforce_epochs(tr[keep], 256, 32))
    reg = dict(n_words=hi - lo, block_dim=256, report_mode=hr.REPORT_EVERY_EPOCH)
    with hr.Checker([reg], report_capacity=1 << 20) as ck:
        ck.set_filter(0, word_lo=lo, word_hi=hi, block_lo=2, block_hi=12)
        ck.check_trace(0, to_dev(tr))
        races, status, n_total, _ = ck.report(0)
    assert status == hr.HR_OK and hr.race_keys(races) == want and n_total == len(want)


@pytest.mark.parametrize("drop", [-1, 3])
def test_inline_kernels(oracle_mod, hr, drop):
    """hr_access through a view in every-epoch mode: stencil and tree reduction."""
    import torch
    hr.load_workloads()
    n = 1 << 18
    d_in = torch.rand(n, device="cuda")
    d_out = torch.zeros(n, device="cuda")
    want = oracle_mod.race_keys(oracle_mod.bruteforce_epochs(tg.stencil_program(n, 5), 256, 32))
    with hr.Checker([dict(n_words=2 * n, block_dim=256, report_mode=hr.REPORT_EVERY_EPOCH)]) as ck:
        hr.run_stencil(ck.device_view(0), d_in, d_out, racy_stride=5)
        races, status, n_total, _ = ck.report(0)
    assert status == hr.HR_OK and hr.race_keys(races) == want and n_total == len(want)
    d = torch.rand(1 << 16, device="cuda")
    want = oracle_mod.race_keys(oracle_mod.bruteforce_epochs(tg.reduce_program(1 << 16, 256, drop), 256, 32))
    with hr.Checker([dict(n_words=1 << 16, block_dim=256, report_mode=hr.REPORT_EVERY_EPOCH)]) as ck:
        hr.run_reduce(ck.device_view(0), d, drop_level=drop)
        races, status, n_total, _ = ck.report(0)
    assert status == hr.HR_OK and hr.race_keys(races) == want and n_total == len(want)


def test_mode_validation(hr):
    with pytest.raises(hr.HiRaceError):
        hr.Checker([dict(n_words=64, block_dim=32, report_mode=hr.REPORT_EVERY_EPOCH, shadow_bytes=4)])
    with pytest.raises(hr.HiRaceError):
        hr.Checker([dict(n_words=64, block_dim=32, report_mode=2)])


def test_cas_retry_cap_reports_contention(hr):
    """Every-epoch mode with zero retries allowed: 64K threads of 256 blocks
    writing one word in one wave make some summary CAS lose, and the region
    reports HR_ERR_CONTENTION; with the default cap the same trace gives the
    one racy (word, kernel, epoch)."""
    n = 1 << 16
    tr = np.zeros(n, tg.RECORD)
    tr["tid"] = np.arange(n)
    tr["op"] = tg.OP_W
    reg = dict(n_words=1, block_dim=256, report_mode=hr.REPORT_EVERY_EPOCH)
    with hr.Checker([reg]) as ck:
        ck.set_limits(cas_retry_cap=0)
        ck.check_trace(0, to_dev(tr))
        _, status, _, _ = ck.report(0)
        assert hr.STATUS[status] == "HR_ERR_CONTENTION"
        ck.set_limits()
        ck.reset(0)
        ck.check_trace(0, to_dev(tr))
        races, status, n_total, _ = ck.report(0)
        assert status == hr.HR_OK and n_total == 1
