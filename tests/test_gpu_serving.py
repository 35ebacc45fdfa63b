"""Serving loop: every request's result is the same alone and in the mix.

A mix of trace checks (prefixes of pooled traces of three kinds, split into
chunks so that several jobs share every batched launch) and instrumented-kernel
runs arrives over ~50 ms; the same requests are then served one at a time.
Race keys and statuses must be identical, and trace results must equal the
oracle on the same prefix.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2401_04701_gb300 import serving
    pool = serving.TracePool(torch.device("cuda", 0), scale="small")
    return serving, pool


def test_alone_equals_mix(oracle_mod, env):
    import torch
    serving, pool = env
    dev = torch.device("cuda", 0)
    reqs = serving.make_requests(77, rate=1200.0, duration=0.05, min_len=5_000, max_len=3_000_000,
                                 kernel_frac=0.3, min_grid=64, max_grid=512)
    assert len(reqs) >= 30
    mix_server = serving.Server(pool, dev, n_slots=8, slot_words=1 << 22, chunk_records=1 << 18)
    mix = mix_server.run(reqs)
    assert mix_server.iterations > 1
    assert len(mix) == len(reqs)
    alone_server = serving.Server(pool, dev, n_slots=2, slot_words=1 << 22, chunk_records=1 << 18)
    for r in reqs:
        solo = serving.Request(r.rid, 0.0, r.kind, r.source, r.length, r.seed)
        alone_server.results = {}
        got = alone_server.run([solo], warm=False)[r.rid]
        m = mix[r.rid]
        assert got.status == m.status == 0, r
        assert got.keys() == m.keys() and got.n_races == m.n_races, r
        if r.kind == "trace" and r.length <= 400_000:
            e = pool.entries[r.source]
            prefix = e["host"][: min(r.length, e["n"])]
            want = oracle_mod.race_keys(oracle_mod.bruteforce(prefix, e["block_dim"]))
            assert m.keys() == want, r


def test_kernel_jobs_overlap_trace_batches(oracle_mod, env):
    """Instrumented-kernel jobs run on streams of their own: in a mix where
    kernel jobs and trace chunks arrive together, launches of one kind are
    queued while the other kind is in flight, and every result is still the
    one the request gets alone (kernels) or the oracle's (traces)."""
    import torch
    serving, pool = env
    dev = torch.device("cuda", 0)
    R = serving.Request
    reqs = []
    for i in range(24):
        if i % 2:
            reqs.append(R(i, 0.0005 * i, "kernel", serving.KERNELS[i % 3], 256 * (64 + 32 * i), 1000 + i))
        else:
            reqs.append(R(i, 0.0005 * i, "trace", ("tree", "global", "graph")[i % 3], 150_000 + 9_000 * i, i))
    srv = serving.Server(pool, dev, n_slots=12, slot_words=1 << 22, chunk_records=1 << 15,
                         iteration_records=1 << 16)
    mix = srv.run(reqs)
    assert srv.overlapped > 0
    alone = serving.Server(pool, dev, n_slots=2, slot_words=1 << 22, chunk_records=1 << 15)
    for r in reqs:
        alone.results = {}
        got = alone.run([R(r.rid, 0.0, r.kind, r.source, r.length, r.seed)], warm=False)[r.rid]
        assert got.status == mix[r.rid].status == 0, r
        assert got.keys() == mix[r.rid].keys() and got.n_races == mix[r.rid].n_races, r
        if r.kind == "trace":
            e = pool.entries[r.source]
            want = oracle_mod.race_keys(oracle_mod.bruteforce(e["host"][: min(r.length, e["n"])], e["block_dim"]))
            assert mix[r.rid].keys() == want, r


def test_failures_stay_with_their_request(oracle_mod, env):
    """Host-side fault injection in a served mix: malformed traces end with their
    own error status, a request too large for any slot is refused at once, a
    request that overruns its timeout is cancelled and its slot reused, and every
    other request still gets the oracle's races."""
    import torch
    from paper_2401_04701_gb300 import hirace, tracegen as tg
    serving, pool = env
    dev = torch.device("cuda", 0)
    tr, info = tg.gen_global_mix(tg.seed_for(5, 9), inject=True, n_blocks=8)
    unsorted = tr.copy()
    unsorted[[100, len(tr) - 100]] = unsorted[[len(tr) - 100, 100]]   # two records out of wave order
    pool._add("unsorted", unsorted, info, dev)
    pool._add("out_of_range", tr, dict(info, n_words=1 << 16), dev)  # words beyond the region
    pool._add("huge", tr, dict(info, n_words=1 << 30), dev)          # no slot holds 2^30 words
    long_tr, long_info = tg.gen_powerlaw_push(tg.seed_for(5, 10), log2_vertices=18, sweeps=4)
    pool._add("long", long_tr, long_info, dev)
    R = serving.Request
    reqs = [R(0, 0.000, "trace", "global", 400_000, 1), R(1, 0.001, "trace", "unsorted", len(tr), 2),
            R(2, 0.002, "trace", "tree", 300_000, 3), R(3, 0.003, "trace", "out_of_range", len(tr), 4),
            R(4, 0.004, "trace", "huge", 1000, 5), R(5, 0.005, "trace", "long", len(long_tr), 6, timeout=1e-4),
            R(6, 0.006, "kernel", "stencil", 1 << 16, 7), R(7, 0.007, "trace", "graph", 200_000, 8)]
    srv = serving.Server(pool, dev, n_slots=3, slot_words=1 << 22, chunk_records=1 << 16,
                         iteration_records=1 << 17)
    res = srv.run(reqs)
    name = lambda rid: hirace.STATUS.get(res[rid].status, res[rid].status)
    assert name(1) == "HR_ERR_ORDER" and name(3) == "HR_ERR_RANGE" and name(4) == "HR_ERR_OOM"
    assert res[5].status == serving.CANCELLED
    for rid in (0, 2, 7):
        r = reqs[rid]
        e = pool.entries[r.source]
        want = oracle_mod.race_keys(oracle_mod.bruteforce(e["host"][: min(r.length, e["n"])], e["block_dim"]))
        assert res[rid].status == hirace.HR_OK and res[rid].keys() == want, r
    assert res[6].status == hirace.HR_OK
    assert sorted(srv.free) == [0, 1, 2] and srv.used == 0   # every slot came back
