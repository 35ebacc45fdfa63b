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
