"""Test-side trace builders: small exhaustive universes and random tiny programs.

Input construction only (like the generator module): nothing here decides
whether accesses race.
"""
import itertools
import json
import os

import numpy as np

from paper_2401_04701_gb300 import tracegen as tg

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

# Fig. 3 grid: 2 blocks x 2 warps x 2 threads
TOY_BLOCK_DIM = 4
TOY_WARP = 2
TOY_THREADS = 8

# barrier structure shared by every thread: phase p has clocks PHASES[p]
PHASES4 = [(0, 0), (0, 1), (1, 0), (1, 1)]
PHASES3 = [(0, 0), (0, 1), (1, 0)]


def load_golden(name):
    with open(os.path.join(GOLDEN, name + ".json")) as f:
        return json.load(f)


def golden_trace(g):
    kernels = [{int(t): [tuple(ev) for ev in evs] for t, evs in k.items()} for k in g["kernels"]]
    return tg.build_trace(kernels)


def _sync_records(phases, n_threads, kernel=0):
    out = []
    for tid in range(n_threads):
        for p in range(1, len(phases)):
            bc, wc = phases[p]
            op = tg.OP_SYNCTHREADS if wc == 0 else tg.OP_SYNCWARP
            out.append((0, tid, wc, bc, kernel, op, 0))
    return out


def combined_trace(cases, phases, n_threads=TOY_THREADS, kernel=0):
    """One trace holding many independent small cases: case c lives on word c.

    ``cases`` is an int array (n_cases, k, 3) of (tid, op, phase); entries with
    tid < 0 are absent.  Every thread runs the same barrier sequence, so all
    cases share the sync records.
    """
    cases = np.asarray(cases, dtype=np.int64)
    n_cases, k, _ = cases.shape
    word = np.repeat(np.arange(n_cases), k)
    flat = cases.reshape(-1, 3)
    keep = flat[:, 0] >= 0
    word, flat = word[keep], flat[keep]
    ph = np.asarray(phases, dtype=np.int64)
    acc = np.zeros(len(flat), tg.RECORD)
    acc["word"] = word
    acc["tid"] = flat[:, 0]
    acc["op"] = flat[:, 1]
    acc["bc"] = ph[flat[:, 2], 0]
    acc["wc"] = ph[flat[:, 2], 1]
    acc["kernel"] = kernel
    syn = np.array(_sync_records(phases, n_threads, kernel), dtype=tg.RECORD)
    allr = np.concatenate([syn, acc])
    sub = np.r_[np.zeros(len(syn)), np.ones(len(acc))]
    order = np.lexsort((np.arange(len(allr)), sub, allr["wc"], allr["bc"], allr["kernel"]))
    return allr[order]


def exhaustive_cases(k, phases, n_threads=TOY_THREADS):
    """Every multiset of k accesses (tid, op, phase) on one word."""
    syms = [(t, o, p) for t in range(n_threads) for o in (tg.OP_R, tg.OP_W, tg.OP_A)
            for p in range(len(phases))]
    combos = np.array(list(itertools.combinations_with_replacement(range(len(syms)), k)), dtype=np.int64)
    table = np.array(syms, dtype=np.int64)
    return table[combos]


def random_cases(rng, n_cases, k_max, phases, n_threads=TOY_THREADS):
    """Random cases of 1..k_max accesses (padding rows have tid = -1)."""
    out = np.full((n_cases, k_max, 3), -1, dtype=np.int64)
    ks = rng.integers(1, k_max + 1, n_cases)
    for c in range(n_cases):
        kk = ks[c]
        out[c, :kk, 0] = rng.integers(0, n_threads, kk)
        out[c, :kk, 1] = rng.integers(0, 3, kk)
        out[c, :kk, 2] = rng.integers(0, len(phases), kk)
    return out


def random_program(rng, n_threads, block_dim, n_words, n_acc, n_st, n_sw, n_kernels=1):
    """Random per-thread programs with a uniform barrier skeleton per kernel.

    Returns the ``kernels`` structure of ``tracegen.build_trace``.
    """
    kernels = []
    for _ in range(n_kernels):
        # skeleton: a list of slots; barrier slots are shared by all threads
        skel = ["ST"] * n_st + ["SW"] * n_sw
        rng.shuffle(skel)
        progs = {t: [] for t in range(n_threads)}
        slots = len(skel) + 1
        acc_at = {}
        for _a in range(n_acc):
            t = int(rng.integers(0, n_threads))
            s = int(rng.integers(0, slots))
            op = "RWA"[int(rng.integers(0, 3))]
            w = int(rng.integers(0, n_words))
            acc_at.setdefault((t, s), []).append((op, w))
        for t in range(n_threads):
            for s in range(slots):
                progs[t].extend(acc_at.get((t, s), []))
                if s < len(skel):
                    progs[t].append((skel[s],))
        kernels.append(progs)
    return kernels
