"""CPU oracle for the race check (TEST INFRASTRUCTURE ONLY).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  The product path never does, and the
oracle never imports the product package: it reads the documented 16-byte
trace record layout on its own.

* ``validate``     - clocks recomputed from each thread's barrier records.
* ``bruteforce``   - the race definition (Sec. II-A, II-B), every pair of
                     accesses per (kernel, word); C code in ``hr_oracle.c``.
                     ``bruteforce_epochs`` keeps every racy epoch of a word
                     instead of the first (the non-absorbing report mode).
* ``serial_fsm``   - a serial restatement of the parallel FSM (Sec. III,
                     Algorithm 1) in C, one record at a time;
                     ``serial_fsm_parallel`` runs it on disjoint word ranges,
                     one host thread each (the CPU baseline on all cores).
* ``hb_races``     - a second, pure-Python statement of the definition for
                     tiny traces: happens-before is *reachability* over
                     program order and barrier edges (the textbook relation
                     of Sec. II-A, built from Sec. II-B's barrier semantics),
                     not a comparison of clock fields.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hr_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libhroracle.so")

# the oracle's own view of the 16-byte record layout
_REC = np.dtype([("word", "<u4"), ("tid", "<u4"), ("wc", "<u2"), ("bc", "<u2"),
                 ("kernel", "<u2"), ("op", "u1"), ("flags", "u1")])
R, W, A, SYNCTHREADS, SYNCWARP = 0, 1, 2, 3, 4

RACE_DT = np.dtype([("word", "<u4"), ("kernel", "<u2"), ("epoch", "<u2"), ("ops_mask", "u1"),
                    ("kinds_mask", "u1"), ("method", "u1"), ("pad", "u1"), ("pad2", "<u4")])
REPORT_DT = np.dtype([("word", "<u4"), ("tid", "<u4"), ("kernel", "<u2"), ("epoch", "<u2"),
                      ("op", "u1"), ("pad", "u1", (3,))])
assert RACE_DT.itemsize == 16 and REPORT_DT.itemsize == 16

VALIDATE_ERRORS = {0: "ok", 1: "unsorted", 2: "clock mismatch", 3: "partial-mask __syncwarp",
                   4: "unknown op"}
STATE_NAMES = ["INIT", "READ", "WRITE", "ATOMIC", "WREAD", "WATOMIC", "BREAD", "BATOMIC",
               "GREAD", "GATOMIC", "RACE"]

_lib_handle = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (plain -O2, portable C99)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _lib():
    global _lib_handle
    if _lib_handle is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        u64, u32, i64 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64
        lib.hro_validate.argtypes = [P, u64, ctypes.POINTER(u64)]
        lib.hro_validate.restype = ctypes.c_int
        lib.hro_bruteforce.argtypes = [P, u64, u32, u32, u64, P, u64]
        lib.hro_bruteforce.restype = i64
        lib.hro_bruteforce_range.argtypes = [P, u64, u32, u32, u64, u64, u64, P, u64]
        lib.hro_bruteforce_range.restype = i64
        lib.hro_bruteforce_epochs.argtypes = [P, u64, u32, u32, u64, P, u64]
        lib.hro_bruteforce_epochs.restype = i64
        lib.hro_group_check.argtypes = [P, P, u64, u32, u32, ctypes.c_int, P]
        lib.hro_group_check.restype = ctypes.c_int
        lib.hro_serial_fsm.argtypes = [P, u64, u32, u32, u64, P, u64, P]
        lib.hro_serial_fsm.restype = i64
        lib.hro_serial_fsm_range.argtypes = [P, u64, u32, u32, u64, u64, u64, P, P, u64]
        lib.hro_serial_fsm_range.restype = i64
        lib.hro_word_bytes.argtypes = []
        lib.hro_word_bytes.restype = u64
        _lib_handle = lib
    return _lib_handle


def _as_records(trace) -> np.ndarray:
    a = np.ascontiguousarray(trace)
    if a.dtype.itemsize != 16:
        raise ValueError("records must be 16 bytes")
    return a.view(_REC)


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a.size else ctypes.c_void_p(0)


def validate(trace):
    """(code, index): 0 when every record's clocks equal the clocks recomputed
    from that thread's own barrier records and the trace is wave-sorted."""
    rec = _as_records(trace)
    bad = ctypes.c_uint64(0)
    rc = _lib().hro_validate(_ptr(rec), len(rec), ctypes.byref(bad))
    return rc, int(bad.value)


def bruteforce(trace, block_dim: int, warp_size: int = 32, pair_limit: int = 4096) -> np.ndarray:
    """Racy (kernel, word) groups with their epoch e*, sorted by (kernel, word)."""
    rec = _as_records(trace)
    rc, idx = validate(rec)
    if rc:
        raise ValueError("invalid trace: %s at record %d" % (VALIDATE_ERRORS[rc], idx))
    cap = 1 << 16
    while True:
        out = np.zeros(cap, RACE_DT)
        n = _lib().hro_bruteforce(_ptr(rec), len(rec), block_dim, warp_size, pair_limit, _ptr(out), cap)
        if n <= cap:
            return out[:n]
        cap = int(n)


def bruteforce_parallel(trace, block_dim: int, n_words: int, warp_size: int = 32, pair_limit: int = 4096,
                        threads: int = 0) -> np.ndarray:
    """bruteforce over `threads` disjoint word ranges at once (one host thread
    each; the C calls release the GIL).  The same rows as bruteforce, in range
    order.  threads=0: every core this process may run on.  The trace is not
    validated here (bruteforce does that)."""
    from concurrent.futures import ThreadPoolExecutor
    rec = _as_records(trace)
    if threads <= 0:
        threads = len(os.sched_getaffinity(0))
    threads = max(1, min(threads, n_words))
    bounds = [n_words * i // threads for i in range(threads + 1)]

    def run(i):
        cap = 1 << 12
        while True:
            out = np.zeros(cap, RACE_DT)
            n = _lib().hro_bruteforce_range(_ptr(rec), len(rec), block_dim, warp_size, pair_limit, bounds[i],
                                            bounds[i + 1], _ptr(out), cap)
            if n <= cap:
                return out[:n]
            cap = int(n)

    _lib()
    with ThreadPoolExecutor(threads) as ex:
        parts = list(ex.map(run, range(threads)))
    return np.concatenate(parts) if parts else np.zeros(0, RACE_DT)


def bruteforce_epochs(trace, block_dim: int, warp_size: int = 32, pair_limit: int = 4096) -> np.ndarray:
    """Every racy (kernel, word, epoch): one row per distinct epoch max(bc_a, bc_b)
    over the racy pairs of each (kernel, word), sorted by (kernel, word, epoch).
    The report set of the every-epoch mode (RACE not absorbing)."""
    rec = _as_records(trace)
    rc, idx = validate(rec)
    if rc:
        raise ValueError("invalid trace: %s at record %d" % (VALIDATE_ERRORS[rc], idx))
    cap = 1 << 16
    while True:
        out = np.zeros(cap, RACE_DT)
        n = _lib().hro_bruteforce_epochs(_ptr(rec), len(rec), block_dim, warp_size, pair_limit, _ptr(out), cap)
        if n <= cap:
            return out[:n]
        cap = int(n)


def group_check(trace, group_idx, block_dim: int, warp_size: int, use_counts: bool):
    """One (kernel, word) group through the pairwise or the count form."""
    rec = _as_records(trace)
    g = np.ascontiguousarray(group_idx, dtype=np.uint64)
    out = np.zeros(1, RACE_DT)
    racy = _lib().hro_group_check(_ptr(rec), _ptr(g), len(g), block_dim, warp_size, int(use_counts),
                                  _ptr(out))
    return out[0] if racy else None


def serial_fsm(trace, block_dim: int, n_words: int, warp_size: int = 32, names: bool = False):
    """Reports (word, tid, kernel, epoch, op) in the order words enter RACE.
    With names=True also returns the named state after every record."""
    rec = _as_records(trace)
    cap = 1 << 16
    nm = np.zeros(len(rec), np.uint8) if names else None
    while True:
        out = np.zeros(cap, REPORT_DT)
        n = _lib().hro_serial_fsm(_ptr(rec), len(rec), block_dim, warp_size, n_words, _ptr(out), cap,
                                  _ptr(nm) if names else ctypes.c_void_p(0))
        if n == -1:
            raise ValueError("word index out of range")
        if n < 0:
            raise MemoryError("oracle could not allocate the word summaries")
        if n <= cap:
            return (out[:n], nm) if names else out[:n]
        cap = int(n)


def serial_fsm_parallel(trace, block_dim: int, n_words: int, warp_size: int = 32, threads: int = 0):
    """serial_fsm over `threads` disjoint word ranges at once (one host thread
    each; the C calls release the GIL).  Same report set as serial_fsm, in
    range order.  threads=0: every core this process may run on."""
    from concurrent.futures import ThreadPoolExecutor
    rec = _as_records(trace)
    if threads <= 0:
        threads = len(os.sched_getaffinity(0))
    threads = max(1, min(threads, n_words))
    bounds = [n_words * i // threads for i in range(threads + 1)]
    # one zeroed array of word summaries, written once here so the threads do
    # not take its page faults one at a time
    wb = int(_lib().hro_word_bytes())
    summaries = np.empty(n_words * wb, np.uint8)
    summaries.fill(0)

    def run(i):
        cap = 1 << 12
        sh = summaries[bounds[i] * wb:]
        while True:
            out = np.zeros(cap, REPORT_DT)
            sh[:(bounds[i + 1] - bounds[i]) * wb].fill(0)
            n = _lib().hro_serial_fsm_range(_ptr(rec), len(rec), block_dim, warp_size, bounds[i], bounds[i + 1],
                                            n_words, _ptr(sh), _ptr(out), cap)
            if n == -1:
                raise ValueError("word index out of range")
            if n < 0:
                raise MemoryError("oracle could not allocate the word summaries")
            if n <= cap:
                return out[:n]
            cap = int(n)

    _lib()
    with ThreadPoolExecutor(threads) as ex:
        parts = list(ex.map(run, range(threads)))
    return np.concatenate(parts) if parts else np.zeros(0, REPORT_DT)


def race_keys(arr) -> set:
    """{(kernel, word, epoch)} of an oracle or checker result array."""
    return {(int(k), int(w), int(e)) for k, w, e in zip(arr["kernel"], arr["word"], arr["epoch"])}


# ---------------------------------------------------------------------------
# Pure-Python happens-before statement of the definition (tiny traces only)
# ---------------------------------------------------------------------------

def hb_races(trace, block_dim: int, warp_size: int = 32, every_epoch: bool = False):
    """{(kernel, word): epoch} computed from happens-before reachability (with
    every_epoch: the set of (kernel, word, epoch) over all racy pairs).

    Happens-before (Sec. II-A) is the transitive closure of
    * program order of each thread (its records in trace order), and
    * barrier edges (Sec. II-B): the k-th __syncthreads of every thread of a
      block is one barrier instance; everything a participant did before it
      happens before everything any participant does after it.  The m-th
      __syncwarp of the lanes of one warp is one warp barrier instance.
    Different kernels never race.  Clock *fields* are not read: each record's
    block clock (for the epoch) is the count of its thread's earlier
    __syncthreads records.
    """
    rec = _as_records(trace)
    n = len(rec)
    recs = [tuple(int(rec[f][i]) for f in ("word", "tid", "kernel", "op")) for i in range(n)]
    warps_per_block = -(-block_dim // warp_size)
    # node ids: records 0..n-1, then one node per barrier instance
    succ = [set() for _ in range(n)]
    barrier_node = {}
    last_of_thread = {}
    st_count = {}
    sw_count = {}
    bc_of = [0] * n
    for i, (word, tid, kern, op) in enumerate(recs):
        key = (kern, tid)
        if key in last_of_thread:
            succ[last_of_thread[key]].add(i)          # program order
        bc_of[i] = st_count.get(key, 0) + (1 if op == SYNCTHREADS else 0)
        if op in (SYNCTHREADS, SYNCWARP):
            blk = tid // block_dim
            if op == SYNCTHREADS:
                k = st_count.get(key, 0) + 1
                st_count[key] = k
                inst = ("B", kern, blk, k)
            else:
                m = sw_count.get(key, 0) + 1
                sw_count[key] = m
                inst = ("W", kern, blk * warps_per_block + (tid % block_dim) // warp_size, m)
            if inst not in barrier_node:
                barrier_node[inst] = len(succ)
                succ.append(set())
            b = barrier_node[inst]
            if key in last_of_thread:
                succ[last_of_thread[key]].add(b)      # before the barrier -> barrier
            succ[b].add(i)                            # barrier -> the thread's sync record
        last_of_thread[key] = i
    # reachability bitsets over the DAG, filled in reverse topological order (Kahn)
    total = len(succ)
    indeg = [0] * total
    for v in range(total):
        for s in succ[v]:
            indeg[s] += 1
    topo = [v for v in range(total) if indeg[v] == 0]
    for v in topo:
        for s in succ[v]:
            indeg[s] -= 1
            if indeg[s] == 0:
                topo.append(s)
    if len(topo) != total:
        raise ValueError("synchronization edges form a cycle")
    reach = [0] * total
    for v in reversed(topo):
        r = 0
        for s in succ[v]:
            r |= (1 << s) | reach[s]
        reach[v] = r

    def ordered(i, j):
        return bool((reach[i] >> j) & 1) or bool((reach[j] >> i) & 1)

    def conflict(a, b):
        return (a in (W, A) or b in (W, A)) and not (a == A and b == A)

    wave = [(recs[i][2], bc_of[i]) for i in range(n)]
    acc = [i for i in range(n) if recs[i][3] <= A]
    best = {}
    for x in range(len(acc)):
        for y in range(x + 1, len(acc)):
            i, j = acc[x], acc[y]
            wi, ti, ki, oi = recs[i]
            wj, tj, kj, oj = recs[j]
            if wi != wj or ki != kj or ti == tj or not conflict(oi, oj) or ordered(i, j):
                continue
            e = max(bc_of[i], bc_of[j])
            if every_epoch:
                best[(ki, wi, e)] = e
                continue
            cur = best.get((ki, wi))
            if cur is None or e < cur:
                best[(ki, wi)] = e
    if every_epoch:
        return set(best)
    return {key: e for key, e in best.items()}
