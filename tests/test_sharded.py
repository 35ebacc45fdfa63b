"""Word-range sharded checking: the routed partition gives the single-rank race set.

A trace spread over ranks that each own a word range is partitioned by owner,
exchanged with one all-to-all, merged per rank and checked per rank; the union
of the ranks' races (words shifted back) must equal the races of the whole
trace on one rank.  On the CPU, two gloo ranks run the orchestration
(``sharded.sharded_check``) with host stand-ins for the three device steps,
written out here, and the CPU oracle as each rank's checker; the device
partition and merge are compared with the same stand-ins in
``test_gpu_sharded.py``.
"""
import os
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def host_partition(trace, bounds):
    """Accesses by owner rank, words rebased to the owner's range, each
    destination's records in trace order; barrier records are not routed."""
    rec = np.ascontiguousarray(trace)
    acc = rec[(rec["op"] <= 2) & (rec["word"] < bounds[-1])]
    owner = np.searchsorted(np.asarray(bounds), acc["word"], side="right") - 1
    blocks, counts = [], []
    for d in range(len(bounds) - 1):
        b = acc[owner == d].copy()
        b["word"] -= np.uint32(bounds[d])
        blocks.append(b)
        counts.append(len(b))
    return blocks, counts


def host_merge(blocks):
    """One wave-sorted trace from wave-sorted blocks: stable by wave key, so
    equal keys keep block order."""
    from paper_2401_04701_gb300 import tracegen as tg
    cat = np.concatenate(blocks) if blocks else np.zeros(0, tg.RECORD)
    return cat[np.argsort(tg.wave_keys(cat), kind="stable")]


class HostOps:
    """The three device steps on the host (uint8 CPU tensors), checked by the oracle."""

    def __init__(self, block_dim):
        self.block_dim = block_dim

    def partition(self, trace_u8, bounds):
        import torch
        from paper_2401_04701_gb300 import tracegen as tg
        tr = trace_u8.numpy().view(tg.RECORD)
        blocks, counts = host_partition(tr, bounds)
        flat = np.concatenate(blocks) if blocks else np.zeros(0, tg.RECORD)
        return torch.from_numpy(flat.view(np.uint8).copy()), counts

    def merge(self, recv_u8, counts):
        import torch
        from paper_2401_04701_gb300 import tracegen as tg
        rec = recv_u8.numpy().view(tg.RECORD)
        starts = np.concatenate([[0], np.cumsum(counts)])
        return torch.from_numpy(host_merge([rec[a:b] for a, b in zip(starts[:-1], starts[1:])]).view(np.uint8).copy())

    def check(self, trace_u8, n_local_words):
        from oracle import oracle
        from paper_2401_04701_gb300 import hirace, tracegen as tg
        tr = trace_u8.numpy().view(tg.RECORD)
        bf = oracle.bruteforce_parallel(tr, self.block_dim, max(1, n_local_words), threads=1)
        out = np.zeros(len(bf), hirace.RACE_DTYPE)
        for f in ("word", "kernel", "epoch"):
            out[f] = bf[f]
        return out


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2401_04701_gb300 import sharded, tracegen as tg
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    tr, info = tg.gen_global_mix(tg.seed_for(2, 30), inject=True, n_blocks=16, tile_words=8192, epochs=2, slots=4)
    # each rank holds a contiguous part of the trace (wave-sorted, like any prefix/suffix of it)
    cut = [0, len(tr) // 3, len(tr)][rank:rank + 2]
    local = torch.from_numpy(np.ascontiguousarray(tr[cut[0]:cut[1]]).view(np.uint8).copy())
    races = sharded.sharded_check(local, info["n_words"], HostOps(256))
    q.put((rank, sorted((int(k), int(w), int(e)) for k, w, e in zip(races["kernel"], races["word"],
                                                                    races["epoch"]))))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_equal_one(oracle_mod):
    from paper_2401_04701_gb300 import tracegen as tg
    tr, info = tg.gen_global_mix(tg.seed_for(2, 30), inject=True, n_blocks=16, tile_words=8192, epochs=2, slots=4)
    want = sorted(oracle_mod.race_keys(oracle_mod.bruteforce(tr, 256)))
    assert len(want) > 0
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29600 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert got[0][1] == got[1][1] == want


def test_host_partition_and_merge_keep_races(oracle_mod):
    """The stand-ins themselves: for 1..5 ranks and random multi-kernel
    programs, partition + merge + per-rank brute force == brute force."""
    from paper_2401_04701_gb300 import sharded, tracegen as tg
    from tests import _cases as C
    rng = np.random.default_rng(33)
    for world in (1, 2, 3, 5):
        kernels = C.random_program(rng, n_threads=300, block_dim=64, n_words=200, n_acc=4000, n_st=3, n_sw=2,
                                   n_kernels=3)
        tr = tg.build_trace(kernels)
        want = oracle_mod.race_keys(oracle_mod.bruteforce(tr, 64))
        bounds = sharded.word_bounds(200, world, align=8)
        parts = np.array_split(np.arange(len(tr)), world)          # each source holds a contiguous part
        per_src = [host_partition(tr[p[0]:p[-1] + 1] if len(p) else tr[:0], bounds)[0] for p in parts]
        got = set()
        for d in range(world):
            merged = host_merge([per_src[s][d] for s in range(world)])
            bf = oracle_mod.bruteforce_parallel(merged, 64, max(1, bounds[d + 1] - bounds[d]), threads=1)
            got |= {(int(k), int(w) + bounds[d], int(e)) for k, w, e in zip(bf["kernel"], bf["word"], bf["epoch"])}
        assert got == want, world
