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


def _step_pow2(t, o, tid, op, bc, wc, ktag, bd_shift, ws_shift):
    """One transition of a packed shadow value, power-of-two geometry, the way
    the device applies the table (kernel-tag check, compareTids, checkSync,
    lookup, canonical packing)."""
    ohi = o >> 32
    os_ = ohi >> 27
    if os_ != 0 and ((ohi >> 24) & 7) != ktag:
        os_ = 0
    x = tid ^ (o & 0xFFFFFFFF)
    trel = 0 if x == 0 else (3 if x >> bd_shift else (2 if x >> ws_shift else 1))
    obc, owc = (ohi >> 8) & 0xFFFF, ohi & 0xFF
    srel = 2 if bc != obc else (1 if wc != owc else 0)
    e = int(t[(os_ << 6) | (op << 4) | (trel << 2) | srel])
    assert e != 0xFF
    ns, lvl = e & 31, e >> 5
    hi, lo = (ns << 27) | (ktag << 24), 0
    if 1 <= lvl <= 3:
        low = 0 if lvl == 1 else (min(ws_shift, bd_shift) if lvl == 2 else bd_shift)
        lo = tid & ~((1 << low) - 1)
        hi |= (bc << 8) | (0 if lvl == 3 else wc)
    return (hi << 32) | lo


@pytest.mark.slow
def test_an_applied_access_stays_absorbed(table):
    """Warp aggregation drops an access that repeats another lane's (same word,
    thread, op, wave), whatever else reaches the word in between.  That needs
    two facts of the table, checked here on every shadow value reachable in a
    2-block x 2-warp x 2-thread grid over several clock pairs and two kernel
    tags: re-applying an access is a no-op (step(step(S, a), a) ==
    step(S, a)), and once a is absorbed it stays absorbed under any access b
    of the same wave (step(S, a) == S implies step(step(S, b), a) ==
    step(S, b))."""
    t, _ = table
    bd, ws = 2, 1
    clocks = [(0, 0), (0, 1), (1, 0), (1, 1), (2, 0)]
    accs = [(tid, op) for tid in range(8) for op in range(3)]
    seen, frontier = {0}, [0]
    while frontier:
        nxt = []
        for s in frontier:
            for ktag in (0, 1):
                for bc, wc in clocks:
                    for tid, op in accs:
                        n = _step_pow2(t, s, tid, op, bc, wc, ktag, bd, ws)
                        if n not in seen:
                            seen.add(n)
                            nxt.append(n)
        frontier = nxt
    assert len(seen) > 300
    for s in seen:
        for ktag in (0, 1):
            for bc, wc in clocks:
                st = {a: _step_pow2(t, s, *a, bc, wc, ktag, bd, ws) for a in accs}
                for a in accs:
                    sa = st[a]
                    assert _step_pow2(t, sa, *a, bc, wc, ktag, bd, ws) == sa, (hex(s), a)
                    if sa != s:
                        continue
                    for b in accs:
                        sb = st[b]
                        assert _step_pow2(t, sb, *a, bc, wc, ktag, bd, ws) == sb, (hex(s), a, b)
