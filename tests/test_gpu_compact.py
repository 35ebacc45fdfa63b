"""Compact 4-byte shadow (tid_bits-wide tid, narrow clocks) == CPU oracle.

The compact word is only a storage form of the 8-byte shadow value, so every
trace whose thread ids and clocks fit the packing must give the oracle's race
keys exactly; one that does not fit must stop with HR_ERR_CLOCK_OVERFLOW.
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


def compact_check(hr, trace, n_words, block_dim, warp_size=32, tid_bits=16, aggregate=True, kernel_base=0):
    reg = dict(n_words=n_words, block_dim=block_dim, warp_size=warp_size, shadow_bytes=4, tid_bits=tid_bits)
    with hr.Checker([reg], report_capacity=1 << 20) as ck:
        ck.check_trace(0, to_dev(trace), aggregate=aggregate, kernel_base=kernel_base)
        races, status, n_total, _ = ck.report(0)
    return races, status, n_total


def assert_parity(O, hr, trace, n_words, block_dim, warp_size=32, tid_bits=16, aggregate=True):
    bf = O.bruteforce(trace, block_dim, warp_size)
    races, status, n_total = compact_check(hr, trace, n_words, block_dim, warp_size, tid_bits, aggregate)
    assert status == hr.HR_OK, hr.STATUS[status]
    assert n_total == len(races) == len(bf)
    assert hr.race_keys(races) == O.race_keys(bf)
    ops = {(int(k), int(w)): int(m) for k, w, m in zip(bf["kernel"], bf["word"], bf["ops_mask"])}
    for k, w, op in zip(races["kernel"], races["word"], races["op"]):
        assert (ops[(int(k), int(w))] >> int(op)) & 1
    return races


@pytest.mark.parametrize("aggregate", [True, False])
@pytest.mark.parametrize("name", ["listing1_no_sync", "listing2_block_sync", "listing3_multi_read"])
def test_listings(oracle_mod, hr, name, aggregate):
    g = C.load_golden(name)
    races = assert_parity(oracle_mod, hr, C.golden_trace(g), g["n_words"], g["block_dim"], g["warp_size"], 8,
                          aggregate)
    assert hr.race_keys(races) == {tuple(x) for x in g["expected_races"]}


@pytest.mark.parametrize("aggregate", [True, False])
def test_exhaustive_universe(oracle_mod, hr, aggregate):
    cases = C.exhaustive_cases(3, C.PHASES4)
    tr = C.combined_trace(cases, C.PHASES4)
    assert_parity(oracle_mod, hr, tr, len(cases), C.TOY_BLOCK_DIM, C.TOY_WARP, 4, aggregate)


def test_random_multi_kernel(oracle_mod, hr):
    """More than 8 kernels (the tag wraps and the compact shadow is cleared by bytes)."""
    rng = np.random.default_rng(61)
    for _ in range(6):
        bd = int(rng.choice([3, 40, 64, 256]))
        kernels = C.random_program(rng, n_threads=int(rng.integers(2, 600)), block_dim=bd, n_words=37,
                                   n_acc=int(rng.integers(1, 3000)), n_st=int(rng.integers(0, 4)),
                                   n_sw=int(rng.integers(0, 4)), n_kernels=int(rng.integers(9, 20)))
        assert_parity(oracle_mod, hr, tg.build_trace(kernels), 37, bd, 32, 12)


def test_tree_reduction(oracle_mod, hr):
    tr, info = tg.gen_tree_reduction(tg.seed_for(1), inject=True)
    assert_parity(oracle_mod, hr, tr, info["n_words"], info["block_dim"], tid_bits=8)


@pytest.mark.parametrize("aggregate", [True, False])
def test_global_mix_small(oracle_mod, hr, aggregate):
    """18-bit tids leave 3 bits each for bc (8 epochs) and wc (4 sub-epochs)."""
    tr, info = tg.gen_global_mix(tg.seed_for(2, 1), inject=True, n_blocks=16)
    races = assert_parity(oracle_mod, hr, tr, info["n_words"], info["block_dim"], tid_bits=18, aggregate=aggregate)
    assert set(races["word"].tolist()) == set(info["injected"].tolist())


def test_tid_overflow(hr):
    """Thread 300 does not fit 8 tid bits: the check stops with HR_ERR_CLOCK_OVERFLOW."""
    rec = np.zeros(2, tg.RECORD)
    rec["word"] = [5, 5]
    rec["tid"] = [3, 300]
    rec["op"] = [tg.OP_R, tg.OP_W]
    races, status, n_total = compact_check(hr, rec, 16, 256, tid_bits=9)
    assert status == hr.HR_OK and n_total == 1          # 300 < 2^9
    races, status, n_total = compact_check(hr, rec, 16, 256, tid_bits=8)
    assert hr.STATUS[status] == "HR_ERR_CLOCK_OVERFLOW"


def test_clock_overflow(hr):
    """tid_bits 20 leaves 2 bits each for bc and wc: bc 4 does not fit."""
    rec = np.zeros(3, tg.RECORD)
    rec["word"] = [1, 1, 1]
    rec["tid"] = [0, 1, 2]
    rec["bc"] = [0, 3, 4]
    rec["op"] = [tg.OP_W, tg.OP_W, tg.OP_W]
    races, status, n_total = compact_check(hr, rec[:2], 4, 4, tid_bits=20)
    assert status == hr.HR_OK
    races, status, n_total = compact_check(hr, rec, 4, 4, tid_bits=20)
    assert hr.STATUS[status] == "HR_ERR_CLOCK_OVERFLOW"


def test_inline_stencil_and_reduction(oracle_mod, hr):
    """Hand-instrumented kernels on compact views: the same races as the oracle."""
    import torch
    hr.load_workloads()
    n = 1 << 18
    d_in = torch.rand(n, device="cuda")
    d_out = torch.zeros(n, device="cuda")
    with hr.Checker([dict(n_words=2 * n, block_dim=256, shadow_bytes=4, tid_bits=18)]) as ck:
        hr.run_stencil(ck.device_view(0), d_in, d_out, racy_stride=7)
        races, status, n_total, _ = ck.report(0)
    assert status == hr.HR_OK
    want = oracle_mod.race_keys(oracle_mod.bruteforce(tg.stencil_program(n, 7), 256, 32))
    assert hr.race_keys(races) == want and n_total == len(want)
    n = 1 << 16
    d = torch.rand(n, device="cuda")
    with hr.Checker([dict(n_words=n, block_dim=256, shadow_bytes=4, tid_bits=15)]) as ck:
        hr.run_reduce(ck.device_view(0), d, drop_level=4)
        races, status, n_total, _ = ck.report(0)
    assert status == hr.HR_OK
    want = oracle_mod.race_keys(oracle_mod.bruteforce(tg.reduce_program(n, 256, 4), 256, 32))
    assert hr.race_keys(races) == want and n_total == len(want)


def test_batch_mixes_shadow_sizes(oracle_mod, hr):
    """One batched launch over an 8-byte and a 4-byte region."""
    import torch
    t1, i1 = tg.gen_tree_reduction(tg.seed_for(1), inject=True)
    t2, i2 = tg.gen_global_mix(tg.seed_for(2, 2), inject=True, n_blocks=8)
    regs = [dict(n_words=i1["n_words"], block_dim=256),
            dict(n_words=i2["n_words"], block_dim=256, shadow_bytes=4, tid_bits=18)]
    with hr.Checker(regs, report_capacity=1 << 20) as ck:
        ck.check_batch([(0, to_dev(t1)), (1, to_dev(t2))])
        got = [ck.report(r) for r in (0, 1)]
    for (races, status, n_total, _), (tr, info) in zip(got, [(t1, i1), (t2, i2)]):
        assert status == hr.HR_OK
        assert hr.race_keys(races) == oracle_mod.race_keys(oracle_mod.bruteforce(tr, 256, 32))


@pytest.mark.parametrize("shadow_bytes", [8, 4])
def test_caller_owned_buffers(oracle_mod, hr, shadow_bytes):
    """hr_init_with_buffers: the checker works in tensors the caller allocated,
    finds the oracle's races, and leaves the tensors to the caller."""
    import torch
    tr, info = tg.gen_global_mix(tg.seed_for(2, 3), inject=True, n_blocks=8)
    n = info["n_words"]
    shadow = torch.full((n * shadow_bytes // 4,), -1, dtype=torch.int32, device="cuda")  # garbage: init clears it
    ring = torch.zeros((1 << 16) * 4, dtype=torch.int32, device="cuda")
    reg = dict(n_words=n, block_dim=256, shadow_bytes=shadow_bytes, tid_bits=18 if shadow_bytes == 4 else 0,
               report_capacity=1 << 16)
    ck = hr.Checker([reg], buffers=[(shadow, ring)])
    ck.check_trace(0, to_dev(tr))
    races, status, n_total, _ = ck.report(0)
    ck.close()
    assert status == hr.HR_OK
    assert hr.race_keys(races) == oracle_mod.race_keys(oracle_mod.bruteforce(tr, 256, 32))
    torch.cuda.synchronize()
    assert int((shadow != 0).sum()) > 0            # the checker's state lives in the caller's tensor
    shadow.zero_()                                   # still the caller's to use after hr_destroy
    ring.zero_()
    torch.cuda.synchronize()
