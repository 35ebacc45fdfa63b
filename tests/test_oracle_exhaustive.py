"""The three oracle statements agree with each other on small universes.

* Every multiset of up to 3 accesses to one word on the Fig. 3 grid
  (2 blocks x 2 warps x 2 threads, warp size 2), over four barrier phases,
  and of 4 accesses over three phases, in many within-wave orders: the serial
  FSM equals the pairwise brute force key for key, and the access it reports
  can complete the first racy pair.
* Random tiny programs (several words, kernels, random barrier skeletons):
  the C brute force equals happens-before reachability.
* Big groups: the count form equals the pairwise form.
"""
import numpy as np
import pytest

from paper_2401_04701_gb300 import tracegen as tg
from tests import _cases as C


def _fsm_vs_bruteforce(O, trace, n_words, block_dim, warp_size, rng, n_orders):
    bf = O.bruteforce(trace, block_dim, warp_size)
    keys = O.race_keys(bf)
    ops_of = {(int(k), int(w)): int(m) for k, w, m in zip(bf["kernel"], bf["word"], bf["ops_mask"])}
    tr = trace
    for _ in range(n_orders):
        rep = O.serial_fsm(tr, block_dim, n_words, warp_size)
        assert O.race_keys(rep) == keys
        assert len(rep) == len(keys)
        for k, w, op in zip(rep["kernel"], rep["word"], rep["op"]):
            assert (ops_of[(int(k), int(w))] >> int(op)) & 1
        tr = tg.shuffle_within_waves(trace, rng)
    return keys


def test_exhaustive_up_to_three_accesses(oracle_mod):
    rng = np.random.default_rng(1)
    for k in (1, 2, 3):
        cases = C.exhaustive_cases(k, C.PHASES4)
        tr = C.combined_trace(cases, C.PHASES4)
        keys = _fsm_vs_bruteforce(oracle_mod, tr, len(cases), C.TOY_BLOCK_DIM, C.TOY_WARP, rng, 6)
        if k == 1:
            assert not keys
        else:
            assert 0 < len(keys) < len(cases)


@pytest.mark.slow
def test_exhaustive_four_accesses(oracle_mod):
    rng = np.random.default_rng(2)
    cases = C.exhaustive_cases(4, C.PHASES3)
    tr = C.combined_trace(cases, C.PHASES3)
    _fsm_vs_bruteforce(oracle_mod, tr, len(cases), C.TOY_BLOCK_DIM, C.TOY_WARP, rng, 3)


def test_random_deep_cases(oracle_mod):
    rng = np.random.default_rng(3)
    cases = C.random_cases(rng, 20000, 10, C.PHASES4)
    tr = C.combined_trace(cases, C.PHASES4)
    _fsm_vs_bruteforce(oracle_mod, tr, len(cases), C.TOY_BLOCK_DIM, C.TOY_WARP, rng, 4)


@pytest.mark.parametrize("seed", range(4))
def test_bruteforce_equals_happens_before(oracle_mod, seed):
    O = oracle_mod
    rng = np.random.default_rng(100 + seed)
    for _ in range(60):
        bd = int(rng.choice([2, 3, 4, 6]))
        ws = int(rng.choice([1, 2, 4]))
        kernels = C.random_program(rng, n_threads=int(rng.integers(2, 9)), block_dim=bd, n_words=3,
                                   n_acc=int(rng.integers(1, 9)), n_st=int(rng.integers(0, 3)),
                                   n_sw=int(rng.integers(0, 3)), n_kernels=int(rng.integers(1, 3)))
        tr = tg.build_trace(kernels)
        assert O.validate(tr) == (0, 0)
        bf = O.race_keys(O.bruteforce(tr, bd, ws))
        hb = {(k, w, e) for (k, w), e in O.hb_races(tr, bd, ws).items()}
        assert bf == hb
        fsm = O.race_keys(O.serial_fsm(tr, bd, 3, ws))
        assert fsm == bf


def test_count_form_equals_pairwise(oracle_mod):
    O = oracle_mod
    rng = np.random.default_rng(7)
    for trial in range(40):
        bd = int(rng.choice([4, 8, 64]))
        ws = int(rng.choice([2, 4, 32]))
        kernels = C.random_program(rng, n_threads=int(rng.integers(2, 130)), block_dim=bd, n_words=1,
                                   n_acc=int(rng.integers(2, 300)), n_st=int(rng.integers(0, 3)),
                                   n_sw=int(rng.integers(0, 3)))
        tr = tg.build_trace(kernels)
        idx = np.flatnonzero(tr["op"] <= tg.OP_A)
        a = O.group_check(tr, idx, bd, ws, use_counts=False)
        b = O.group_check(tr, idx, bd, ws, use_counts=True)
        assert (a is None) == (b is None)
        if a is not None:
            assert (a["epoch"], a["ops_mask"]) == (b["epoch"], b["ops_mask"])
    # the public entry point switches forms by group size
    tr = tg.build_trace(C.random_program(np.random.default_rng(9), 64, 8, 2, 2000, 2, 1))
    assert O.race_keys(O.bruteforce(tr, 8, 4, pair_limit=1)) == O.race_keys(O.bruteforce(tr, 8, 4))


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_word_partitioned_serial_fsm_equals_serial(oracle_mod, threads):
    """Word-range partitions run the same per-word FSM: identical report set."""
    from paper_2401_04701_gb300 import tracegen as tg
    tr, info = tg.gen_global_mix(tg.seed_for(2, 4), inject=True, n_blocks=4)
    a = oracle_mod.serial_fsm(tr, info["block_dim"], info["n_words"])
    b = oracle_mod.serial_fsm_parallel(tr, info["block_dim"], info["n_words"], threads=threads)
    key = lambda r: {(int(k), int(w), int(e), int(t), int(o))
                     for k, w, e, t, o in zip(r["kernel"], r["word"], r["epoch"], r["tid"], r["op"])}
    assert len(a) == len(b) and key(a) == key(b)
    rng = np.random.default_rng(7)
    cases = C.random_cases(rng, 3000, 6, C.PHASES4)
    tr = C.combined_trace(cases, C.PHASES4)
    a = oracle_mod.serial_fsm(tr, C.TOY_BLOCK_DIM, len(cases), C.TOY_WARP)
    b = oracle_mod.serial_fsm_parallel(tr, C.TOY_BLOCK_DIM, len(cases), C.TOY_WARP, threads=threads)
    assert key(a) == key(b)


# --------------------------------------------- every racy epoch (report mode 1)

def test_every_epoch_hand_built(oracle_mod):
    """Two blocks race in epoch 0 and again in epoch 1 (blocks are never ordered);
    two lanes of one warp race in epoch 0 only (the barrier orders what follows)."""
    O = oracle_mod
    cross = [{0: [("W", 0), ("ST",), ("W", 0)], 4: [("R", 0), ("ST",)]}]
    tr = tg.build_trace(cross)
    assert O.race_keys(O.bruteforce_epochs(tr, 4, 2)) == {(0, 0, 0), (0, 0, 1)}
    assert O.race_keys(O.bruteforce(tr, 4, 2)) == {(0, 0, 0)}
    local = [{0: [("W", 0), ("ST",), ("R", 0)], 1: [("W", 0), ("ST",)]}]
    tr = tg.build_trace(local)
    assert O.race_keys(O.bruteforce_epochs(tr, 4, 2)) == {(0, 0, 0)}
    later = [{0: [("R", 0), ("ST",), ("W", 0)], 1: [("R", 0), ("ST",), ("R", 0)]}]
    tr = tg.build_trace(later)  # reads race-free in epoch 0, W/R of two lanes in epoch 1
    assert O.race_keys(O.bruteforce_epochs(tr, 4, 2)) == {(0, 0, 1)}
    assert O.race_keys(O.bruteforce(tr, 4, 2)) == {(0, 0, 1)}


@pytest.mark.parametrize("seed", range(3))
def test_every_epoch_equals_happens_before(oracle_mod, seed):
    """The every-epoch brute force against reachability; its first epoch per
    word is the absorbing report set."""
    O = oracle_mod
    rng = np.random.default_rng(300 + seed)
    for _ in range(60):
        bd = int(rng.choice([2, 3, 4, 6]))
        ws = int(rng.choice([1, 2, 4]))
        kernels = C.random_program(rng, n_threads=int(rng.integers(2, 9)), block_dim=bd, n_words=3,
                                   n_acc=int(rng.integers(1, 12)), n_st=int(rng.integers(0, 4)),
                                   n_sw=int(rng.integers(0, 3)), n_kernels=int(rng.integers(1, 3)))
        tr = tg.build_trace(kernels)
        ep = O.race_keys(O.bruteforce_epochs(tr, bd, ws))
        assert ep == O.hb_races(tr, bd, ws, every_epoch=True)
        first = {}
        for k, w, e in ep:
            first[(k, w)] = min(e, first.get((k, w), e))
        assert {(k, w, e) for (k, w), e in first.items()} == O.race_keys(O.bruteforce(tr, bd, ws))


def test_every_epoch_count_form_equals_pairwise(oracle_mod):
    O = oracle_mod
    rng = np.random.default_rng(77)
    cases = C.random_cases(rng, 4000, 8, C.PHASES4)
    tr = C.combined_trace(cases, C.PHASES4)
    a = O.bruteforce_epochs(tr, C.TOY_BLOCK_DIM, C.TOY_WARP)
    b = O.bruteforce_epochs(tr, C.TOY_BLOCK_DIM, C.TOY_WARP, pair_limit=1)
    assert O.race_keys(a) == O.race_keys(b)
    assert (a["ops_mask"] == b["ops_mask"]).all()
    # injected cross-block writes race with reads of later epochs too: more rows than racy words
    tr, info = tg.gen_global_mix(tg.seed_for(2, 7), inject=True, n_blocks=4)
    a = O.bruteforce_epochs(tr, info["block_dim"])
    b = O.bruteforce_epochs(tr, info["block_dim"], pair_limit=1)
    assert O.race_keys(a) == O.race_keys(b) and len(a) > len(O.bruteforce(tr, info["block_dim"]))


@pytest.mark.parametrize("threads", [1, 4, 7])
def test_word_partitioned_bruteforce_equals_bruteforce(oracle_mod, threads):
    """Word ranges split the (kernel, word) groups: the same rows as one run."""
    O = oracle_mod
    tr, info = tg.gen_global_mix(tg.seed_for(2, 15), inject=True, n_blocks=4)
    a = O.bruteforce(tr, 256)
    b = O.bruteforce_parallel(tr, 256, info["n_words"], threads=threads)
    assert len(a) == len(b) and O.race_keys(a) == O.race_keys(b)
    key = lambda r: sorted(zip(r["kernel"].tolist(), r["word"].tolist(), r["ops_mask"].tolist()))
    assert key(a) == key(b)
