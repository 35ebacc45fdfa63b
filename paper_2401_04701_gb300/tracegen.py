"""Seeded synthetic access traces: the input side of the race checker.

This module only *builds* inputs.  It holds no race arithmetic: it never
decides whether two accesses conflict or are ordered.  Both the CUDA checker
(through its tests and benchmarks) and the CPU oracle consume what it makes.

Trace format (one 16-byte little-endian record per event, array-of-structs):

    offset  size  field    meaning
    0       4     word     word index inside the checked region (access records)
    4       4     tid      global thread id = blockIdx * blockDim + threadIdx
    8       2     wc       warp clock: full-warp __syncwarp() since the last __syncthreads()
    10      2     bc       block clock: __syncthreads() executed so far in this kernel
    12      2     kernel   launch ordinal of the traced kernel
    14      1     op       0 read, 1 write, 2 atomic, 3 __syncthreads, 4 __syncwarp
    15      1     flags    bit 0: the atomic is an atomic load (informational)
                           bit 1: __syncwarp with a partial mask (unsupported)

The (bc, wc) pair of an access is the thread-private clock of the paper's
shadow record (Section III, Fig. 2 / Algorithm 1 inputs `bc`, `wc`).  A sync
record carries the clocks the thread holds *after* the barrier.  A trace is
sorted by its wave key (kernel, bc, wc); inside a wave each thread's records
keep program order.  The bytes at offsets 8..13 read as a little-endian u64,
masked to 48 bits, are exactly that key.
"""
from __future__ import annotations

import numpy as np

RECORD = np.dtype([("word", "<u4"), ("tid", "<u4"), ("wc", "<u2"), ("bc", "<u2"),
                   ("kernel", "<u2"), ("op", "u1"), ("flags", "u1")])
assert RECORD.itemsize == 16

OP_R, OP_W, OP_A, OP_SYNCTHREADS, OP_SYNCWARP = 0, 1, 2, 3, 4
FLAG_ATOMIC_LOAD = 1
FLAG_PARTIAL_MASK = 2

SEED_BASE = 0x48695261

_OPS = {"R": OP_R, "W": OP_W, "A": OP_A}


def seed_for(config: int, trial: int = 0) -> int:
    """Seed of a workload: fixed base + 1000 * workload number + trial."""
    return SEED_BASE + config * 1000 + trial


def wave_keys(trace: np.ndarray) -> np.ndarray:
    """(kernel, bc, wc) packed into one integer per record (sort key of a trace)."""
    return ((trace["kernel"].astype(np.int64) << 32) | (trace["bc"].astype(np.int64) << 16)
            | trace["wc"].astype(np.int64))


def is_sorted(trace: np.ndarray) -> bool:
    k = wave_keys(trace)
    return bool(np.all(k[1:] >= k[:-1])) if len(k) > 1 else True


# --------------------------------------------------------------------------
# Hand-written programs (litmus tests, small exhaustive universes)
# --------------------------------------------------------------------------

def build_trace(kernels, kernel_base: int = 0) -> np.ndarray:
    """Trace of small hand-written per-thread programs.

    ``kernels`` is a list (one entry per launch) of ``{tid: [event, ...]}``.
    An event is ``("R"|"W"|"A", word)``, ``("A", word, FLAG_ATOMIC_LOAD)``,
    ``("ST",)`` for __syncthreads or ``("SW",)`` / ``("SW", FLAG_PARTIAL_MASK)``
    for __syncwarp.  Each thread's clocks are counted from its own barriers
    (a thread's clocks restart at every launch).  Records are ordered by wave,
    then by program step, then by tid: the order a SIMT tracer logging one
    instruction for all lanes at a time would produce.
    """
    rows = []
    for k, threads in enumerate(kernels):
        for tid, events in threads.items():
            bc = wc = 0
            for step, ev in enumerate(events):
                kind = ev[0]
                if kind == "ST":
                    bc += 1
                    wc = 0
                    rows.append((0, tid, wc, bc, kernel_base + k, OP_SYNCTHREADS, 0, step))
                elif kind == "SW":
                    wc += 1
                    fl = ev[1] if len(ev) > 1 else 0
                    rows.append((0, tid, wc, bc, kernel_base + k, OP_SYNCWARP, fl, step))
                else:
                    fl = ev[2] if len(ev) > 2 else 0
                    rows.append((ev[1], tid, wc, bc, kernel_base + k, _OPS[kind], fl, step))
    if not rows:
        return np.zeros(0, RECORD)
    a = np.array(rows, dtype=np.int64)
    order = np.lexsort((a[:, 1], a[:, 7], a[:, 2], a[:, 3], a[:, 4]))
    a = a[order]
    out = np.zeros(len(a), RECORD)
    for i, name in enumerate(("word", "tid", "wc", "bc", "kernel", "op", "flags")):
        out[name] = a[:, i]
    return out


def shuffle_within_waves(trace: np.ndarray, rng: np.random.Generator) -> np.ndarray:
    """Another valid interleaving: records permuted inside each wave while
    every thread keeps its own program order."""
    if len(trace) == 0:
        return trace.copy()
    keys = wave_keys(trace)
    starts = np.flatnonzero(np.r_[True, keys[1:] != keys[:-1]])
    ends = np.r_[starts[1:], len(trace)]
    out = trace.copy()
    for s, e in zip(starts, ends):
        seg = trace[s:e]
        perm = rng.permutation(e - s)
        shuffled = seg[perm]
        # restore per-thread program order on the positions each thread now holds
        for tid in np.unique(seg["tid"]):
            pos = np.flatnonzero(shuffled["tid"] == tid)
            shuffled[pos] = seg[seg["tid"] == tid]
        out[s:e] = shuffled
    return out


# --------------------------------------------------------------------------
# Workload 1: shared-memory tree reduction, one block
# --------------------------------------------------------------------------

def gen_tree_reduction(seed: int, inject: bool = True, segments: int = 48, block_dim: int = 256,
                       reps: int = 28, p_unit: float = 0.01, force: bool = True):
    """One block of ``block_dim`` threads over ``segments`` x ``block_dim`` shared words.

    Epoch k (k = 0..log2(block_dim)-1) has stride s = block_dim/2 >> k; thread t < s
    reads words t and t+s of every segment and writes word t, ``reps`` times per
    epoch, with a __syncthreads() between epochs.  Injection: each (segment, epoch)
    unit draws a doubled active bound (t < 2s, partner index mod block_dim) with
    probability ``p_unit``; each barrier draws "dropped" with the same probability;
    when ``force`` and a kind drew nothing, one unit of that kind is forced.

    Returns (trace, info) with info = dict(n_words, block_dim, n_threads, doubled, dropped).
    """
    rng = np.random.default_rng(seed)
    n_epochs = int(np.log2(block_dim))
    n_words = segments * block_dim
    doubled = np.zeros((segments, n_epochs), bool)
    dropped = np.zeros(n_epochs - 1, bool)
    if inject:
        doubled = rng.random((segments, n_epochs)) < p_unit
        dropped = rng.random(n_epochs - 1) < p_unit
        if force and not doubled.any():
            doubled[rng.integers(segments), rng.integers(n_epochs)] = True
        if force and not dropped.any():
            dropped[rng.integers(n_epochs - 1)] = True
    # block clock of each epoch after dropped barriers are removed
    bc_of_epoch = np.zeros(n_epochs, np.int64)
    for k in range(1, n_epochs):
        bc_of_epoch[k] = bc_of_epoch[k - 1] + (0 if dropped[k - 1] else 1)

    # Records in SIMT log order: epoch by epoch, its barrier records (thread
    # order) first, then its accesses ordered by warp, instruction (rep, seg,
    # j) and lane; built directly in that order, block_dim a multiple of 32
    # (else lane-major inside one ragged warp, the same order).
    t_all = np.arange(block_dim)
    nwarp = -(-block_dim // 32)
    wl = np.arange(nwarp * 32).reshape(nwarp, 32)           # thread id of (warp, lane)
    parts = []
    for k in range(n_epochs):
        s = (block_dim // 2) >> k
        bc = bc_of_epoch[k]
        if k > 0 and not dropped[k - 1]:
            sync = np.zeros(block_dim, RECORD)
            sync["tid"] = t_all
            sync["bc"] = bc
            sync["op"] = OP_SYNCTHREADS
            parts.append(sync)
        # grid over (warp, rep, seg, j, lane), kept where t < the unit's active bound
        shape = (nwarp, reps, segments, 3, 32)
        t = np.broadcast_to(wl.reshape(nwarp, 1, 1, 1, 32), shape)
        seg = np.broadcast_to(np.arange(segments).reshape(1, 1, -1, 1, 1), shape)
        j = np.broadcast_to(np.arange(3).reshape(1, 1, 1, 3, 1), shape)
        bound = np.where(doubled[:, k], 2 * s, s).reshape(1, 1, -1, 1, 1)
        keep = (t < bound) & (t < block_dim)
        t, seg, j = t[keep], seg[keep], j[keep]
        idx = np.where(j == 1, (t + s) % block_dim, t)
        rec = np.zeros(len(t), RECORD)
        rec["word"] = seg * block_dim + idx
        rec["tid"] = t
        rec["bc"] = bc
        rec["op"] = np.where(j == 2, OP_W, OP_R)
        parts.append(rec)
    trace = np.concatenate(parts) if parts else np.zeros(0, RECORD)
    info = dict(n_words=n_words, block_dim=block_dim, n_threads=block_dim,
                doubled=[(int(a), int(b)) for a, b in zip(*np.nonzero(doubled))],
                dropped=[int(x) for x in np.flatnonzero(dropped)])
    return trace, info


# --------------------------------------------------------------------------
# Workload 2: global memory, owned tiles + random shared words
# --------------------------------------------------------------------------

def gen_global_mix(seed: int, inject: bool = True, n_blocks: int = 1024, block_dim: int = 256,
                   tile_words: int = 65536, epochs: int = 8, subs: int = 4, slots: int = 8,
                   inject_frac: float = 0.001):
    """Grid of ``n_blocks`` x ``block_dim`` threads over ``n_blocks * tile_words`` words.

    Every thread makes ``epochs * subs * slots`` accesses: ``slots`` per warp
    sub-epoch, a __syncwarp() between sub-epochs and a __syncthreads() between
    epochs.  Each access draws its class: 45% read of a random read-only word,
    5% atomic on a random atomic-only word (both anywhere in the array), 25%
    read and 25% write of the block's own tile.  Tile words split by offset:
    the first quarter is owned (block-strided rows; in epoch e, slot i uses row
    e*slots+i, column (warp+e) mod warps, lane (lane+sub) mod 32), the next
    sixteenth is atomic-only, the rest read-only.  Injection retargets
    ``inject_frac * n_words`` random-class accesses, as writes, to distinct
    words that a thread of another block touches.

    Returns (trace, info) with info = dict(n_words, block_dim, n_threads, injected).
    """
    assert block_dim % 32 == 0
    nwarp = block_dim // 32
    ow = tile_words // 4
    assert epochs * slots * block_dim <= ow, "tile too small for the owned rows"
    at_lo, at_hi = ow, ow + tile_words // 16
    ro_lo, ro_hi = at_hi, tile_words
    n_words = n_blocks * tile_words
    rng = np.random.default_rng(seed)

    # full grid in wave order: (epoch, sub, block, warp, slot[0 = sync], lane)
    shape = (epochs, subs, n_blocks, nwarp, slots + 1, 32)
    n_all = int(np.prod(shape))
    e = np.arange(epochs, dtype=np.int64).reshape(-1, 1, 1, 1, 1, 1)
    w = np.arange(subs, dtype=np.int64).reshape(1, -1, 1, 1, 1, 1)
    b = np.arange(n_blocks, dtype=np.int64).reshape(1, 1, -1, 1, 1, 1)
    v = np.arange(nwarp, dtype=np.int64).reshape(1, 1, 1, -1, 1, 1)
    i = np.arange(slots + 1, dtype=np.int64).reshape(1, 1, 1, 1, -1, 1)
    ln = np.arange(32, dtype=np.int64).reshape(1, 1, 1, 1, 1, -1)

    rec = np.zeros(n_all, RECORD)
    rec["tid"] = np.broadcast_to(b * block_dim + v * 32 + ln, shape).ravel()
    rec["bc"] = np.broadcast_to(e, shape).ravel()
    rec["wc"] = np.broadcast_to(w, shape).ravel()
    is_sync = np.broadcast_to(i == 0, shape).ravel()
    sync_op = np.broadcast_to(np.where(w == 0, OP_SYNCTHREADS, OP_SYNCWARP), shape).ravel()

    u = rng.random(n_all, dtype=np.float32)
    rand_tile = rng.integers(0, n_blocks, n_all, dtype=np.int64)
    ro_off = rng.integers(ro_lo, ro_hi, n_all, dtype=np.int64)
    at_off = rng.integers(at_lo, at_hi, n_all, dtype=np.int64)
    strided = np.broadcast_to(
        b * tile_words + (e * slots + (i - 1)) * block_dim + ((v + e) % nwarp) * 32 + (ln + w) % 32,
        shape).ravel()

    cls = np.where(u < 0.45, 0, np.where(u < 0.50, 1, np.where(u < 0.75, 2, 3))).astype(np.int8)
    word = np.where(cls == 0, rand_tile * tile_words + ro_off,
                    np.where(cls == 1, rand_tile * tile_words + at_off, strided))
    del u, rand_tile, ro_off, at_off, strided
    op = np.where(cls == 0, OP_R, np.where(cls == 1, OP_A, np.where(cls == 2, OP_R, OP_W)))
    rec["word"] = np.where(is_sync, 0, word)
    rec["op"] = np.where(is_sync, sync_op, op)
    del word, op
    cls = np.where(is_sync, -1, cls)

    keep = ~(is_sync & (rec["bc"] == 0) & (rec["wc"] == 0))
    rec = rec[keep]
    cls = cls[keep]

    injected = np.zeros(0, np.int64)
    if inject:
        random_idx = np.flatnonzero((cls == 0) | (cls == 1))
        # short traces have fewer random accesses than the word-based count asks for
        n_inj = min(int(inject_frac * n_words), len(random_idx) // 2)
        source_pool = np.flatnonzero((cls == 0) | (cls >= 2))
        carriers = rng.choice(random_idx, size=n_inj, replace=False)
        carrier_mask = np.zeros(len(rec), bool)
        carrier_mask[carriers] = True
        source_pool = source_pool[~carrier_mask[source_pool]]
        cblock = rec["tid"][carriers] // block_dim
        targets = np.full(n_inj, -1, np.int64)
        taken = set()
        todo = np.arange(n_inj)
        while len(todo):
            src = rng.choice(source_pool, size=len(todo))
            cand = rec["word"][src].astype(np.int64)
            ok = (rec["tid"][src] // block_dim) != cblock[todo]
            nxt = []
            for j, c, good in zip(todo, cand, ok):
                if good and c not in taken:
                    taken.add(int(c))
                    targets[j] = c
                else:
                    nxt.append(j)
            todo = np.array(nxt, dtype=np.int64)
        rec["word"][carriers] = targets
        rec["op"][carriers] = OP_W
        rec["flags"][carriers] = 0
        injected = np.sort(targets)
    info = dict(n_words=n_words, block_dim=block_dim, n_threads=n_blocks * block_dim,
                injected=injected)
    return rec, info


# --------------------------------------------------------------------------
# Access programs of the hand-instrumented kernels (same accesses, as traces)
# --------------------------------------------------------------------------

def _pack(word, tid, bc, op, step):
    """Records from per-access columns, ordered by (bc, step, tid)."""
    word, tid, bc, op, step = (np.asarray(x, dtype=np.int64) for x in (word, tid, bc, op, step))
    order = np.lexsort((tid, step, bc))
    rec = np.zeros(len(order), RECORD)
    rec["word"] = word[order]
    rec["tid"] = tid[order]
    rec["bc"] = bc[order]
    rec["op"] = op[order]
    return rec


def stencil_program(n: int, racy_stride: int = 0) -> np.ndarray:
    """Thread i reads in[i], in[i-1], in[i+1] (words i-1..i+1) and writes out[i]
    (word n+i); with racy_stride, threads i % racy_stride == 0 also write in[i]."""
    i = np.arange(n, dtype=np.int64)
    cols = [(i, i, np.zeros(n), np.full(n, OP_R), np.zeros(n))]
    m = i > 0
    cols.append((i[m] - 1, i[m], np.zeros(m.sum()), np.full(m.sum(), OP_R), np.ones(m.sum())))
    m = i + 1 < n
    cols.append((i[m] + 1, i[m], np.zeros(m.sum()), np.full(m.sum(), OP_R), np.full(m.sum(), 2)))
    cols.append((n + i, i, np.zeros(n), np.full(n, OP_W), np.full(n, 3)))
    if racy_stride:
        m = i % racy_stride == 0
        cols.append((i[m], i[m], np.zeros(m.sum()), np.full(m.sum(), OP_W), np.full(m.sum(), 4)))
    return _pack(*(np.concatenate([c[j] for c in cols]) for j in range(5)))


def histogram_program(keys: np.ndarray, racy_stride: int = 0) -> np.ndarray:
    """Thread i does atomicAdd(bins[keys[i]]); with racy_stride, threads
    i % racy_stride == 0 do a plain read then write of that bin instead."""
    keys = np.asarray(keys, dtype=np.int64)
    n = len(keys)
    i = np.arange(n, dtype=np.int64)
    racy = (i % racy_stride == 0) if racy_stride else np.zeros(n, bool)
    a = ~racy
    cols = [(keys[a], i[a], np.zeros(a.sum()), np.full(a.sum(), OP_A), np.zeros(a.sum())),
            (keys[racy], i[racy], np.zeros(racy.sum()), np.full(racy.sum(), OP_R), np.zeros(racy.sum())),
            (keys[racy], i[racy], np.zeros(racy.sum()), np.full(racy.sum(), OP_W), np.ones(racy.sum()))]
    return _pack(*(np.concatenate([c[j] for c in cols]) for j in range(5)))


def reduce_program(n: int, block: int, drop_level: int = -1) -> np.ndarray:
    """Per block b, a tree reduction over data[2*block*b ...]: at level L (stride
    s = block >> L) thread t < s reads t and t+s and writes t, then a barrier
    (removed after level drop_level)."""
    grid = -(-n // (2 * block))
    parts = []
    bc = 0
    level = 0
    s = block
    b = np.arange(grid, dtype=np.int64).reshape(-1, 1)
    while s > 0:
        t = np.arange(block, dtype=np.int64).reshape(1, -1)
        base = 2 * block * b
        ok = (t < s) & (base + t + s < n)
        tid = np.broadcast_to(b * block + t, ok.shape)[ok]
        w0 = np.broadcast_to(base + t, ok.shape)[ok]
        w1 = np.broadcast_to(base + t + s, ok.shape)[ok]
        k = len(tid)
        step = 3 * level
        parts.append((w0, tid, np.full(k, bc), np.full(k, OP_R), np.full(k, step)))
        parts.append((w1, tid, np.full(k, bc), np.full(k, OP_R), np.full(k, step + 1)))
        parts.append((w0, tid, np.full(k, bc), np.full(k, OP_W), np.full(k, step + 2)))
        if level != drop_level:
            bc += 1
            every = (b * block + t).ravel()
            parts.append((np.zeros(len(every)), every, np.full(len(every), bc),
                          np.full(len(every), OP_SYNCTHREADS), np.full(len(every), step + 2.5)))
        s >>= 1
        level += 1
    word, tid, bcs, op, step = (np.concatenate([p[j] for p in parts]) for j in range(5))
    order = np.lexsort((tid, step, bcs))
    rec = np.zeros(len(order), RECORD)
    rec["word"] = word[order].astype(np.int64)
    rec["tid"] = tid[order]
    rec["bc"] = bcs[order]
    rec["op"] = op[order]
    return rec


def smem_reduce_program(n: int, block: int, drop_level: int = -1) -> np.ndarray:
    """Access program of a block reduction through a __shared__ buffer of
    ``block`` words per block (word = block index * block + t): every thread
    writes its word, a barrier, then at level L threads t < s = block >> (L+1)
    read t and t+s and write t, each level followed by a barrier (except after
    level drop_level); finally thread 0 reads word 0."""
    grid = -(-n // block)
    b = np.arange(grid, dtype=np.int64).reshape(-1, 1)
    t = np.arange(block, dtype=np.int64).reshape(1, -1)
    every_tid = (b * block + t).ravel()
    parts = []

    def add(mask, word, op, bc, step):
        tid = np.broadcast_to(b * block + t, mask.shape)[mask]
        w = np.broadcast_to(word, mask.shape)[mask]
        parts.append((w, tid, np.full(len(tid), bc), np.full(len(tid), op), np.full(len(tid), step)))

    full = np.ones((grid, block), bool)
    add(full, b * block + t, OP_W, 0, 0.0)
    bc = 1
    parts.append((np.zeros(len(every_tid)), every_tid, np.full(len(every_tid), bc),
                  np.full(len(every_tid), OP_SYNCTHREADS), np.full(len(every_tid), 0.5)))
    level, s = 0, block >> 1
    while s > 0:
        act = np.broadcast_to(t < s, (grid, block))
        step = 1.0 + 3 * level
        add(act, b * block + t, OP_R, bc, step)
        add(act, b * block + t + s, OP_R, bc, step + 1)
        add(act, b * block + t, OP_W, bc, step + 2)
        if level != drop_level:
            bc += 1
            parts.append((np.zeros(len(every_tid)), every_tid, np.full(len(every_tid), bc),
                          np.full(len(every_tid), OP_SYNCTHREADS), np.full(len(every_tid), step + 2.5)))
        s >>= 1
        level += 1
    add(np.broadcast_to(t == 0, (grid, block)), b * block, OP_R, bc, 1.0 + 3 * level)
    word, tid, bcs, op, step = (np.concatenate([p[j] for p in parts]) for j in range(5))
    order = np.lexsort((tid, step, bcs))
    rec = np.zeros(len(order), RECORD)
    rec["word"] = word[order].astype(np.int64)
    rec["tid"] = tid[order]
    rec["bc"] = bcs[order]
    rec["op"] = op[order]
    return rec


# --------------------------------------------------------------------------
# Workload 3: power-law graph, push-style relaxation
# --------------------------------------------------------------------------

def _sample_cdf(cdf: np.ndarray, u: np.ndarray, n: int) -> np.ndarray:
    """Inverse-CDF sampling: the index i with cdf[i-1] <= u < cdf[i], capped at
    n - 1; the lookups run in chunks on host threads (same result as one call)."""
    from concurrent.futures import ThreadPoolExecutor
    chunks = np.array_split(u, max(1, min(64, len(u) >> 16)))
    with ThreadPoolExecutor(min(16, len(chunks))) as ex:
        parts = list(ex.map(lambda c: np.searchsorted(cdf, c, side="right"), chunks))
    out = np.concatenate(parts).astype(np.int64) if parts else np.zeros(0, np.int64)
    np.minimum(out, n - 1, out=out)
    return out


def gen_powerlaw_push(seed: int, log2_vertices: int = 22, avg_degree: int = 16, sweeps: int = 4,
                      gamma: float = 2.1, block_dim: int = 256, inject_frac: float = 0.0005,
                      inject: bool = True):
    """Push-style relaxation over a Chung-Lu power-law graph.

    Vertex weights are proportional to (i+1)^(-1/(gamma-1)); both endpoints of
    each of the n*avg_degree edges are drawn with those weights, so in- and
    out-degrees follow a power law with exponent gamma.  Thread v owns vertex v
    (block_dim threads per block) and, in each of ``sweeps`` kernel launches,
    visits its out-edges in CSR order: an atomic load of dist[v] (op A, flag
    atomic-load) then an atomicMin of dist[u] (op A).  There are no barriers,
    so each launch is one wave; a thread's records are contiguous (the order
    a per-thread trace buffer produces).  Injection turns ``inject_frac`` of
    the atomicMins into plain writes.

    Returns (trace, info) with info = dict(n_words, block_dim, n_threads,
    injected (indices of the injected records), edges).
    """
    rng = np.random.default_rng(seed)
    n = 1 << log2_vertices
    m = n * avg_degree
    w = (np.arange(1, n + 1, dtype=np.float64)) ** (-1.0 / (gamma - 1.0))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    src = _sample_cdf(cdf, rng.random(m), n)
    dst = _sample_cdf(cdf, rng.random(m), n)
    # CSR order: edges stably sorted by source (the key src * 2^k + edge index
    # is unique, so an unstable sort of it is the stable order by source)
    kbits = max(1, int(m - 1).bit_length())
    key = (src.astype(np.uint64) << np.uint64(kbits)) | np.arange(m, dtype=np.uint64)
    key.sort()
    order = (key & np.uint64((1 << kbits) - 1)).astype(np.int64)
    del key
    src = src[order].astype(np.uint32)
    dst = dst[order].astype(np.uint32)
    del order
    per = 2 * m
    trace = np.zeros(per * sweeps, RECORD)
    first = trace[:per]
    first["tid"][0::2] = src
    first["tid"][1::2] = src
    first["word"][0::2] = src
    first["word"][1::2] = dst
    first["op"] = OP_A
    first["flags"][0::2] = FLAG_ATOMIC_LOAD
    for k in range(1, sweeps):
        trace[k * per:(k + 1) * per] = first
        trace["kernel"][k * per:(k + 1) * per] = k
    injected = np.zeros(0, np.int64)
    if inject:
        n_inj = int(inject_frac * m * sweeps)
        picks = rng.choice(m * sweeps, size=n_inj, replace=False)
        injected = np.sort((picks // m) * per + 2 * (picks % m) + 1)
        trace["op"][injected] = OP_W
    info = dict(n_words=n, block_dim=block_dim, n_threads=n, injected=injected, edges=m)
    return trace, info


# --------------------------------------------------------------------------
# Workload 4: a batch of independent traces of uneven length
# --------------------------------------------------------------------------

def gen_batch(seed: int, n_traces: int = 512, min_len: int = 10_000, max_len: int = 10_000_000,
              shared_frac: float = 0.6, max_rate: float = 0.01):
    """``n_traces`` independent traces with lengths log-uniform in [min_len, max_len].

    A ``shared_frac`` share are shared-memory tree reductions (block size 64..1024
    in steps of 32, a 4..48 KB array of 4-byte words, repetitions set to reach
    the drawn length); the rest are global-memory traces shaped like
    ``gen_global_mix`` over a 1..64 MB region (log-uniform), with the per-thread
    access count scaled toward the drawn length.  Each trace draws its race
    injection rate uniformly in [0, max_rate].

    Returns a list of (trace, info) with info = dict(n_words, block_dim, kind, target).
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_traces):
        target = int(np.exp(rng.uniform(np.log(min_len), np.log(max_len))))
        rate = float(rng.uniform(0.0, max_rate))
        sub = int(rng.integers(0, 2**31))
        if rng.random() < shared_frac:
            block = int(rng.integers(2, 33)) * 32
            kb = int(rng.integers(4, 49))
            segments = max(1, (kb * 256) // block)
            n_epochs = int(np.log2(block))
            per_rep = segments * 3 * sum((block // 2) >> k for k in range(n_epochs))
            reps = max(1, target // max(1, per_rep))
            trace, info = gen_tree_reduction(sub, inject=rate > 0, segments=segments, block_dim=block, reps=reps,
                                             p_unit=rate, force=False)
            info = dict(n_words=info["n_words"], block_dim=block, kind="shared", target=target)
        else:
            mb = float(np.exp(rng.uniform(0.0, np.log(64.0))))
            n_blocks = max(1, int(mb * 262144) // 65536)
            threads = n_blocks * 256
            per_thread = max(1, target // threads)
            epochs = int(np.clip(per_thread // 32, 1, 8))
            slots = int(np.clip(per_thread // (4 * epochs), 1, 8))
            trace, info = gen_global_mix(sub, inject=rate > 0, n_blocks=n_blocks, epochs=epochs, slots=slots,
                                         inject_frac=rate)
            info = dict(n_words=info["n_words"], block_dim=256, kind="global", target=target)
        out.append((trace, info))
    return out
