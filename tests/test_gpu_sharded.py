"""Device partition and merge of the word-sharded check (one GPU).

hr_shard_partition must equal the stable host partition byte for byte, and
hr_shard_merge the stable merge by wave key; then ranks emulated one after
another on this GPU (each source's part of the trace partitioned, the blocks
of each destination merged and checked on a region of that destination's
words) give together exactly the oracle's races of the whole trace.  Only
the all-to-all is left out: on one GPU a rank's received blocks are the
sources' blocks for it, concatenated in rank order.
"""
import numpy as np
import pytest

from paper_2401_04701_gb300 import tracegen as tg
from tests import _cases as C
from tests.test_sharded import host_merge, host_partition

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2401_04701_gb300 import hirace, sharded
    return hirace, sharded


def to_dev(trace):
    import torch
    return torch.from_numpy(np.ascontiguousarray(trace).view(np.uint8)).cuda()


def cases():
    rng = np.random.default_rng(41)
    out = []
    tr, info = tg.gen_global_mix(tg.seed_for(2, 31), inject=True, n_blocks=16)
    out.append((tr, info["n_words"], 256))
    tr, info = tg.gen_powerlaw_push(tg.seed_for(3, 31), log2_vertices=14, sweeps=3)
    out.append((tr, info["n_words"], 256))
    kernels = C.random_program(rng, n_threads=500, block_dim=64, n_words=40000, n_acc=20000, n_st=3, n_sw=2,
                               n_kernels=4)
    out.append((tg.build_trace(kernels), 40000, 64))
    return out


@pytest.mark.parametrize("world", [1, 2, 3, 7])
def test_partition_merge_and_emulated_ranks(oracle_mod, env, world):
    hirace, sharded = env
    for ci, (tr, n_words, bd) in enumerate(cases()):
        ops = sharded.DeviceOps("cuda", n_words, bd)
        bounds = sharded.word_bounds(n_words, world, align=1024)
        parts = np.array_split(np.arange(len(tr)), world)
        srcs = [tr[p[0]:p[-1] + 1] if len(p) else tr[:0] for p in parts]
        dev_blocks = []
        for src in srcs:
            blocks, counts = ops.partition(to_dev(src), bounds)
            want_blocks, want_counts = host_partition(src, bounds)
            assert counts == want_counts, (ci, world)
            got = blocks.cpu().numpy().view(tg.RECORD)
            assert (got.view(np.uint8) == np.concatenate(want_blocks).view(np.uint8)).all(), (ci, world)
            starts = np.concatenate([[0], np.cumsum(counts)])
            dev_blocks.append([blocks[a * 16:b * 16] for a, b in zip(starts[:-1], starts[1:])])
        races = set()
        for d in range(world):
            import torch
            recv = torch.cat([dev_blocks[s][d] for s in range(world)])
            rcounts = [dev_blocks[s][d].numel() // 16 for s in range(world)]
            merged = ops.merge(recv, rcounts)
            want_merged = host_merge([host_partition(srcs[s], bounds)[0][d] for s in range(world)])
            assert (merged.cpu().numpy() == want_merged.view(np.uint8)).all(), (ci, world, d)
            r = ops.check(merged, bounds[d + 1] - bounds[d])
            races |= {(int(k), int(w) + bounds[d], int(e)) for k, w, e in zip(r["kernel"], r["word"], r["epoch"])}
        assert races == oracle_mod.race_keys(oracle_mod.bruteforce(tr, bd)), (ci, world)


def test_merge_reports_unsorted_blocks(env):
    hirace, sharded = env
    tr = tg.build_trace([{t: [("W", t % 3), ("ST",), ("R", t % 3)] for t in range(64)}])
    acc = tr[tr["op"] <= tg.OP_A]
    bad = acc[::-1].copy()                                   # a block that is not wave-sorted
    ops = sharded.DeviceOps("cuda", 3, 64)
    with pytest.raises(hirace.HiRaceError):
        ops.merge(to_dev(np.concatenate([acc, bad])), [len(acc), len(bad)])
