"""Word-range sharded check of one trace over several ranks (torch.distributed).

Each rank owns a contiguous range of the region's words and that range's
shadow.  An access only touches its own word's shadow value (Algorithm 1), so
a rank can check the accesses to its words on its own, provided it sees them
in wave order.  One check of a trace spread over the ranks (each rank holding
any part of the trace, e.g. the records its own GPU logged):

1. partition: each rank splits its records by owner rank (a stable partition,
   so every block stays wave-sorted) and rebases each word to the owner's
   range (``hr_shard_partition``);
2. exchange: one all-to-all of the per-destination blocks (the only
   collective on the data path);
3. merge: each rank merges the blocks it received into one wave-sorted trace
   (``hr_shard_merge``): inside a wave every pair is unordered (Sec. II-B), so
   any interleaving of the sources' records of one wave is a valid order;
4. check: ``hr_check_trace`` on the rank's region; the race records, words
   shifted back to the region's numbering, are all-gathered.

The partition, merge and local check are the C-ABI calls by default; the
orchestration takes them as arguments so that its collectives can be driven
on the host too.
"""
from __future__ import annotations

import numpy as np

from . import hirace

RECORD_BYTES = 16
MAX_RUNS_PER_BLOCK = 1 << 16  # waves a received block may hold (the checker's wave table size)


def word_bounds(n_words: int, world: int, align: int = 1 << 14) -> list:
    """Contiguous word ranges, rank r owning [bounds[r], bounds[r + 1]); inner
    bounds are multiples of `align` (whole shadow segments of the binned
    checker), the last is n_words."""
    per = -(-n_words // world)
    per = -(-per // align) * align
    return [min(n_words, r * per) for r in range(world)] + [n_words]


class DeviceOps:
    """Partition, merge and local check through the C-ABI on one GPU."""

    def __init__(self, device, n_words: int, block_dim: int, warp_size: int = 32, world: int = 1,
                 report_capacity: int = 1 << 22, variant: int | None = None):
        import ctypes
        import torch
        self.device = device
        self.lib = hirace.load_library()
        L, P, u32, u64 = self.lib, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
        L.hr_shard_partition_scratch_bytes.argtypes = [u64, u32]
        L.hr_shard_partition_scratch_bytes.restype = u64
        L.hr_shard_partition.argtypes = [P, u64, P, u32, P, P, P, u64, P]
        L.hr_shard_partition.restype = ctypes.c_int
        L.hr_shard_merge_scratch_bytes.argtypes = [u64]
        L.hr_shard_merge_scratch_bytes.restype = u64
        L.hr_shard_merge.argtypes = [P, P, u32, u64, P, P, u64, u64, P, P]
        L.hr_shard_merge.restype = ctypes.c_int
        self.torch = torch
        self.block_dim, self.warp_size = block_dim, warp_size
        self.report_capacity = report_capacity
        self.variant = variant
        self.status = torch.zeros(1, dtype=torch.int32, device=device)

    def _stream(self):
        return self.torch.cuda.current_stream(self.device).cuda_stream

    def partition(self, trace, bounds):
        """(blocks of the routed records, uint8 on the device; records per destination)."""
        torch = self.torch
        world = len(bounds) - 1
        n = trace.numel() // RECORD_BYTES
        d_bounds = torch.tensor(bounds, dtype=torch.int64, device=self.device)
        out = torch.empty(max(n, 1) * RECORD_BYTES, dtype=torch.uint8, device=self.device)
        counts = torch.zeros(world, dtype=torch.int64, device=self.device)
        sb = int(self.lib.hr_shard_partition_scratch_bytes(n, world))
        scratch = torch.empty(max(sb, 8), dtype=torch.uint8, device=self.device)
        rc = self.lib.hr_shard_partition(trace.data_ptr() if n else None, n, d_bounds.data_ptr(), world,
                                         out.data_ptr(), counts.data_ptr(), scratch.data_ptr(), sb, self._stream())
        if rc:
            raise hirace.HiRaceError(rc, "hr_shard_partition")
        c = [int(x) for x in counts.cpu()]
        return out[: sum(c) * RECORD_BYTES], c

    def merge(self, blocks, counts):
        """One wave-sorted trace from the received blocks (uint8 on the device)."""
        torch = self.torch
        n = sum(counts)
        starts = torch.tensor(np.concatenate([[0], np.cumsum(counts)]), dtype=torch.int64, device=self.device)
        out = torch.empty(max(n, 1) * RECORD_BYTES, dtype=torch.uint8, device=self.device)
        max_runs = max(1, min(n, MAX_RUNS_PER_BLOCK * len(counts)))
        sb = int(self.lib.hr_shard_merge_scratch_bytes(max_runs))
        scratch = torch.empty(sb, dtype=torch.uint8, device=self.device)
        rc = self.lib.hr_shard_merge(blocks.data_ptr() if n else None, starts.data_ptr(), len(counts), n,
                                     out.data_ptr(), scratch.data_ptr(), sb, max_runs, self.status.data_ptr(),
                                     self._stream())
        if rc:
            raise hirace.HiRaceError(rc, "hr_shard_merge")
        st = int(self.status.item())
        if st:
            raise hirace.HiRaceError(st, "hr_shard_merge")
        return out[: n * RECORD_BYTES]

    def check(self, trace, n_local_words):
        """Race records of the local trace on a region of the rank's words."""
        with hirace.Checker([dict(n_words=max(1, n_local_words), block_dim=self.block_dim,
                                  warp_size=self.warp_size)], report_capacity=self.report_capacity) as ck:
            if self.variant is not None:
                ck.set_variant(self.variant)
            if trace.numel():
                ck.check_trace(0, trace)
            races, status, n_total, _ = ck.report(0)
        if status != hirace.HR_OK:
            raise hirace.HiRaceError(status, "hr_check_trace (shard)")
        return races


def sharded_check(local_trace, n_words: int, ops, group=None):
    """Check one trace whose records are spread over the ranks of `group`
    (this rank holds `local_trace`, wave-sorted; a uint8 tensor of 16-byte
    records on the device the collectives use).  Returns every rank's race
    records (words in the region's numbering), the same on every rank."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    bounds = word_bounds(n_words, world)
    blocks, counts = ops.partition(local_trace, bounds)
    dev = blocks.device
    send_n = torch.tensor(counts, dtype=torch.int64, device=dev)
    recv_n = torch.empty(world, dtype=torch.int64, device=dev)
    dist.all_to_all_single(recv_n, send_n, group=group)
    rcounts = [int(x) for x in recv_n.cpu()]
    recv = torch.empty(max(1, sum(rcounts)) * RECORD_BYTES, dtype=torch.uint8, device=dev)
    dist.all_to_all_single(recv[: sum(rcounts) * RECORD_BYTES], blocks,
                           [c * RECORD_BYTES for c in rcounts], [c * RECORD_BYTES for c in counts], group=group)
    merged = ops.merge(recv[: sum(rcounts) * RECORD_BYTES], rcounts)
    races = ops.check(merged, bounds[rank + 1] - bounds[rank]).copy()
    races["word"] += np.uint32(bounds[rank])
    # all-gather the variable-size race arrays as bytes
    raw = torch.from_numpy(races.view(np.uint8).copy()).to(dev)
    sizes = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(sizes, torch.tensor([raw.numel()], dtype=torch.int64, device=dev), group=group)
    sizes = [int(s.item()) for s in sizes]
    cap = max(1, max(sizes))
    padded = torch.zeros(cap, dtype=torch.uint8, device=dev)
    padded[: raw.numel()] = raw
    parts = [torch.empty(cap, dtype=torch.uint8, device=dev) for _ in range(world)]
    dist.all_gather(parts, padded, group=group)
    out = np.concatenate([p[:s].cpu().numpy() for p, s in zip(parts, sizes)]) if world else np.zeros(0, np.uint8)
    return out.view(hirace.RACE_DTYPE)
