"""The product's flat FSM table, applied on the CPU exactly as the device step
applies it (kernel-tag check, compareTids, checkSync, one lookup, canonical
packing), equals the oracle's race definition on the exhaustive universes.

This checks the table and the packing rules without a GPU; the CUDA kernels
are checked against the oracle in the GPU parity tests.
"""
import numpy as np
import pytest

from paper_2401_04701_gb300 import tracegen as tg
from tests import _cases as C

U = np.uint64


@pytest.fixture(scope="module")
def table():
    from paper_2401_04701_gb300 import build, hirace
    build.build()
    t, n = hirace.fsm_table()
    return t, n


def emulate(trace, table, block_dim, warp_size):
    """Apply the table to every access in trace order; returns {(kernel, word, epoch): op}."""
    acc = trace[trace["op"] <= tg.OP_A]
    order = np.argsort(acc["word"], kind="stable")
    acc = acc[order]
    words, starts, counts = np.unique(acc["word"], return_index=True, return_counts=True)
    shadow = np.zeros(len(words), U)
    last_kernel = np.zeros(len(words), np.int64)
    raced_at = {}
    bd, ws = U(block_dim), U(warp_size)
    for j in range(int(counts.max()) if len(counts) else 0):
        sel = np.flatnonzero(counts > j)
        rec = acc[starts[sel] + j]
        o = shadow[sel]
        # the device clears the whole shadow when the kernel ordinal enters a new group of 8
        kern = rec["kernel"].astype(np.int64)
        o = np.where((kern >> 3) != (last_kernel[sel] >> 3), U(0), o)
        last_kernel[sel] = kern
        tid = rec["tid"].astype(U)
        op = rec["op"].astype(U)
        bc = rec["bc"].astype(U)
        wc = rec["wc"].astype(U)
        ktag = (rec["kernel"].astype(U) & U(7))
        os_ = o >> U(59)
        stale = (os_ != 0) & (((o >> U(56)) & U(7)) != ktag)
        os_ = np.where(stale, U(0), os_)
        blk = tid // bd
        loc = tid - blk * bd
        warp = loc // ws
        lane = loc - warp * ws
        otid = o & U(0xFFFFFFFF)
        oblk = otid // bd
        owarp = (otid - oblk * bd) // ws
        trel = np.where(otid == tid, U(0), np.where(oblk != blk, U(3), np.where(owarp == warp, U(1), U(2))))
        obc = (o >> U(40)) & U(0xFFFF)
        owc = (o >> U(32)) & U(0xFF)
        srel = np.where(bc != obc, U(2), np.where(wc != owc, U(1), U(0)))
        e = table[((os_ << U(6)) | (op << U(4)) | (trel << U(2)) | srel).astype(np.int64)].astype(U)
        assert np.all(e != 0xFF), "unused table entry reached"
        ns = e & U(31)
        lvl = e >> U(5)
        n = (ns << U(59)) | (ktag << U(56))
        n = np.where(lvl == 1, n | (bc << U(40)) | (wc << U(32)) | tid, n)
        n = np.where(lvl == 2, n | (bc << U(40)) | (wc << U(32)) | (tid - lane), n)
        n = np.where(lvl == 3, n | (bc << U(40)) | (tid - loc), n)
        raced = (ns == 31) & (os_ != 31)
        for i in np.flatnonzero(raced):
            raced_at[(int(rec["kernel"][i]), int(words[sel[i]]), int(bc[i]))] = int(op[i])
        shadow[sel] = n
    return raced_at


def test_state_count(table):
    t, n = table
    # Sec. IV-B: the state fits in 5 bits (the paper's own machine has 25 states)
    assert 2 <= n <= 32
    assert t[0] != 0xFF


@pytest.mark.parametrize("k,phases", [(1, C.PHASES4), (2, C.PHASES4), (3, C.PHASES4)])
def test_table_equals_bruteforce_exhaustive(oracle_mod, table, k, phases):
    O = oracle_mod
    rng = np.random.default_rng(k)
    cases = C.exhaustive_cases(k, phases)
    base = C.combined_trace(cases, phases)
    bf = O.bruteforce(base, C.TOY_BLOCK_DIM, C.TOY_WARP)
    keys = O.race_keys(bf)
    ops = {(int(a), int(b)): int(m) for a, b, m in zip(bf["kernel"], bf["word"], bf["ops_mask"])}
    tr = base
    for _ in range(4):
        got = emulate(tr, table[0], C.TOY_BLOCK_DIM, C.TOY_WARP)
        assert set(got) == keys
        for (kk, w, e), op in got.items():
            assert (ops[(kk, w)] >> op) & 1
        tr = tg.shuffle_within_waves(base, rng)


def test_table_equals_bruteforce_random_deep(oracle_mod, table):
    O = oracle_mod
    rng = np.random.default_rng(11)
    cases = C.random_cases(rng, 20000, 10, C.PHASES4)
    tr = C.combined_trace(cases, C.PHASES4)
    keys = O.race_keys(O.bruteforce(tr, C.TOY_BLOCK_DIM, C.TOY_WARP))
    assert set(emulate(tr, table[0], C.TOY_BLOCK_DIM, C.TOY_WARP)) == keys


def test_kernel_tag_wraps_after_eight_kernels(oracle_mod, table):
    # a write in kernel 0 and a read by another thread in kernel 8 (same 3-bit tag)
    kernels = [{0: [("W", 0)]}] + [{}] * 7 + [{1: [("R", 0)]}, {2: [("W", 1)], 3: [("W", 1)]}]
    tr = tg.build_trace(kernels)
    keys = oracle_mod.race_keys(oracle_mod.bruteforce(tr, 64, 32))
    assert keys == {(9, 1, 0)}
    assert set(emulate(tr, table[0], 64, 32)) == keys


def test_table_multi_kernel_and_wide_blocks(oracle_mod, table):
    O = oracle_mod
    rng = np.random.default_rng(12)
    for _ in range(30):
        bd = int(rng.choice([3, 4, 40, 64]))
        ws = int(rng.choice([2, 32]))
        kernels = C.random_program(rng, n_threads=int(rng.integers(2, 100)), block_dim=bd, n_words=4,
                                   n_acc=int(rng.integers(1, 60)), n_st=int(rng.integers(0, 3)),
                                   n_sw=int(rng.integers(0, 3)), n_kernels=int(rng.integers(1, 11)))
        tr = tg.build_trace(kernels)
        keys = O.race_keys(O.bruteforce(tr, bd, ws))
        assert set(emulate(tr, table[0], bd, ws)) == keys
