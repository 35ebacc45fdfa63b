"""Pins of the CPU oracle to what the paper and the definitions fix.

Each expected value here is derived by hand from the paper (the listings'
marked race lines, the scenario state names, the race definition of
Sec. II-A and the barrier semantics of Sec. II-B), never from the oracle or
the CUDA checker.  Every case runs through all three oracle statements: the
pairwise brute force (C), the happens-before reachability checker (Python)
and the serial FSM (C).
"""
import numpy as np
import pytest

from paper_2401_04701_gb300 import tracegen as tg
from tests._cases import golden_trace, load_golden

OPS = {"R": tg.OP_R, "W": tg.OP_W, "A": tg.OP_A}


def all_three(O, trace, block_dim, warp_size, n_words):
    assert O.validate(trace) == (0, 0)
    bf = O.race_keys(O.bruteforce(trace, block_dim, warp_size))
    hb = {(k, w, e) for (k, w), e in O.hb_races(trace, block_dim, warp_size).items()}
    fsm = O.race_keys(O.serial_fsm(trace, block_dim, n_words, warp_size))
    return bf, hb, fsm


def expect(O, kernels, block_dim, warp_size, n_words, expected):
    tr = tg.build_trace(kernels)
    bf, hb, fsm = all_three(O, tr, block_dim, warp_size, n_words)
    assert bf == set(expected), "brute force"
    assert hb == set(expected), "happens-before reachability"
    assert fsm == set(expected), "serial FSM"


@pytest.mark.parametrize("name", ["listing1_no_sync", "listing2_block_sync", "listing2_one_block",
                                  "listing3_multi_read"])
def test_listing_verdicts(oracle_mod, name):
    g = load_golden(name)
    tr = golden_trace(g)
    bf, hb, fsm = all_three(oracle_mod, tr, g["block_dim"], g["warp_size"], g["n_words"])
    exp = {tuple(x) for x in g["expected_races"]}
    assert bf == exp and hb == exp and fsm == exp


def test_scenario_state_names(oracle_mod):
    """Sec. III-A Scenarios 1 and 2: the named states after each step."""
    O = oracle_mod
    g = load_golden("scenarios")
    for seq in g["sequences"]:
        rec = np.zeros(len(seq["steps"]), tg.RECORD)
        for i, (tid, op, bc) in enumerate(seq["steps"]):
            rec[i] = (0, tid, 0, bc, 0, OPS[op], 0)
        _, names = O.serial_fsm(rec, g["block_dim"], 1, g["warp_size"], names=True)
        got = [O.STATE_NAMES[x] for x in names]
        assert got == seq["names"], seq["what"]


# --- hand-built races (Sec. II-A definition, Sec. II-B barrier semantics) ---

def test_write_write_and_read_write_same_epoch(oracle_mod):
    # two warps of one block, no barrier between them: concurrent
    expect(oracle_mod, [{0: [("W", 5)], 32: [("W", 5)]}], 64, 32, 8, [(0, 5, 0)])
    expect(oracle_mod, [{0: [("R", 5)], 40: [("W", 5)]}], 64, 32, 8, [(0, 5, 0)])


def test_read_read_never_races(oracle_mod):
    expect(oracle_mod, [{0: [("R", 5)], 40: [("R", 5)], 70: [("R", 5)]}], 64, 32, 8, [])


def test_syncthreads_orders_a_block(oracle_mod):
    expect(oracle_mod, [{0: [("W", 5), ("ST",)], 40: [("ST",), ("R", 5)]}], 64, 32, 8, [])


def test_missing_syncthreads(oracle_mod):
    # both after the first barrier, nothing between them: race in epoch 1
    expect(oracle_mod, [{0: [("ST",), ("W", 5)], 40: [("ST",), ("R", 5)]}], 64, 32, 8, [(0, 5, 1)])


def test_cross_block_race_despite_barrier(oracle_mod):
    # __syncthreads does not order two blocks; epoch = max of the two block clocks
    expect(oracle_mod, [{0: [("W", 5), ("ST",)], 32: [("ST",), ("R", 5)]}], 32, 32, 8, [(0, 5, 1)])


def test_epoch_is_min_over_racy_pairs(oracle_mod):
    # block 0 writes at bc 2; block 1 reads at bc 0 and bc 3: pairs give 2 and 3
    k = {0: [("ST",), ("ST",), ("W", 5), ("ST",)],
         64: [("R", 5), ("ST",), ("ST",), ("ST",), ("R", 5)]}
    expect(oracle_mod, [k], 64, 32, 8, [(0, 5, 2)])


def test_syncwarp_orders_a_warp_only(oracle_mod):
    expect(oracle_mod, [{0: [("W", 5), ("SW",)], 1: [("SW",), ("R", 5)]}], 32, 32, 8, [])
    expect(oracle_mod, [{0: [("W", 5)], 1: [("R", 5)]}], 32, 32, 8, [(0, 5, 0)])
    # lanes of two different warps: __syncwarp does not order them
    expect(oracle_mod, [{0: [("W", 5), ("SW",)], 33: [("SW",), ("R", 5)]}], 64, 32, 8, [(0, 5, 0)])


def test_syncthreads_resets_warp_clock(oracle_mod):
    # same warp, same bc, same wc (0) after the block barrier: concurrent again
    k = {0: [("SW",), ("W", 5), ("ST",), ("R", 6)], 1: [("SW",), ("ST",), ("W", 6)]}
    expect(oracle_mod, [k], 32, 32, 8, [(0, 6, 1)])


def test_warp_index_is_within_block(oracle_mod):
    # blockDim 40: tids 60 and 70 are lanes 20 and 30 of warp 0 of block 1
    expect(oracle_mod, [{60: [("W", 5), ("SW",)], 70: [("SW",), ("R", 5)]}], 40, 32, 8, [])
    # tids 39 and 41 are in different blocks
    expect(oracle_mod, [{39: [("W", 5), ("SW",)], 41: [("SW",), ("R", 5)]}], 40, 32, 8, [(0, 5, 0)])


def test_atomics(oracle_mod):
    O = oracle_mod
    expect(O, [{0: [("A", 5)], 40: [("A", 5)], 70: [("A", 5)]}], 64, 32, 8, [])        # A-A
    expect(O, [{0: [("A", 5)], 40: [("W", 5)]}], 64, 32, 8, [(0, 5, 0)])                # A-W
    expect(O, [{0: [("A", 5)], 40: [("R", 5)]}], 64, 32, 8, [(0, 5, 0)])                # A-R
    expect(O, [{0: [("A", 5), ("ST",)], 40: [("ST",), ("R", 5)]}], 64, 32, 8, [])      # ordered
    expect(O, [{0: [("A", 5), ("ST",)], 64: [("ST",), ("R", 5)]}], 64, 32, 8, [(0, 5, 1)])  # blocks


def test_same_thread_never_races(oracle_mod):
    expect(oracle_mod, [{7: [("R", 5), ("W", 5), ("A", 5), ("R", 5), ("W", 5)]}], 64, 32, 8, [])


def test_kernel_end_orders_everything(oracle_mod):
    expect(oracle_mod, [{0: [("W", 5)]}, {1: [("R", 5)]}], 64, 32, 8, [])
    expect(oracle_mod, [{0: [("W", 5)]}, {1: [("R", 5)], 100: [("W", 5)]}], 64, 32, 8, [(1, 5, 0)])


def test_race_is_once_per_word_and_kernel(oracle_mod):
    O = oracle_mod
    k = {0: [("W", 5), ("ST",), ("W", 5)], 40: [("W", 5), ("ST",), ("W", 5)]}
    tr = tg.build_trace([k, k])
    rep = O.serial_fsm(tr, 64, 8, 32)
    assert sorted(O.race_keys(rep)) == [(0, 5, 0), (1, 5, 0)]
    assert len(rep) == 2


def test_validate_rejects_bad_traces(oracle_mod):
    O = oracle_mod
    tr = tg.build_trace([{0: [("W", 5), ("ST",), ("R", 5)], 1: [("ST",)]}])
    assert O.validate(tr) == (0, 0)
    bad = tr.copy()
    bad["bc"][-1] = 2                      # clock that no barrier explains
    assert O.validate(bad)[0] in (1, 2)
    # thread 1's barrier record ahead of thread 0's epoch-0 write: clocks fine, order not
    two = tg.build_trace([{0: [("W", 5)], 1: [("ST",)]}])
    assert O.validate(two) == (0, 0)
    assert O.validate(two[::-1].copy()) == (1, 1)
    partial = tg.build_trace([{0: [("SW", tg.FLAG_PARTIAL_MASK), ("R", 1)]}])
    assert O.validate(partial)[0] == 3
    badop = tr.copy()
    badop["op"][0] = 9
    assert O.validate(badop)[0] == 4


def test_reported_op_is_the_completing_access(oracle_mod):
    O = oracle_mod
    # a read waits in an earlier wave; the completing access is the write
    tr = tg.build_trace([{0: [("R", 5), ("ST",)], 64: [("ST",), ("W", 5)]}])
    bf = O.bruteforce(tr, 64, 32)
    assert bf["ops_mask"][0] == 1 << tg.OP_W
    assert bf["kinds_mask"][0] == 1 << 0          # R-W
    rep = O.serial_fsm(tr, 64, 8, 32)
    assert rep["op"][0] == tg.OP_W and rep["tid"][0] == 64
