"""Batched multi-threshold queries and the continuous-batching server.

Every request's result must be exactly the same alone (pj_query) and in the
mix (pj_query_multi batches, server batches); integer results, tolerance 0.
"""
import threading
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1111_7171_gb300 import passjoin as pj
from paper_1111_7171_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def resident():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()
    S = synth.generate("short", 4, n=30000) + [b"", b"a", b"ab", b"abc", b"abcd"]
    idx = pj.pj_build_index(S, 4)
    yield S, idx
    idx.free()


def requests(S, n_req, seed):
    reqs = synth.query_stream(S, n_req, seed=seed, tau_max=4, max_batch=300)
    reqs.append(([b"", b"b", b"ab"], 2))  # short queries, short indexed strings
    return reqs


def test_query_multi_equals_oracle_and_single(resident):
    S, idx = resident
    sb, so = synth.pack(S)
    reqs = requests(S, 12, seed=3)
    batch = [q for qs, _ in reqs for q in qs]
    taus = [t for qs, t in reqs for _ in qs]
    got = pj.pj_query_multi(idx, batch, taus).pairs
    base = 0
    for qs, t in reqs:
        sel = got[(got["a"] >= base) & (got["a"] < base + len(qs))].copy()
        sel["a"] -= base
        alone = pj.pj_query(idx, qs, t).pairs
        assert np.array_equal(sel, alone)
        qb, qo = synth.pack(qs)
        assert np.array_equal(alone, oracle.join(qb, qo, sb, so, t))
        base += len(qs)


def test_server_results_equal_alone_in_the_mix(resident):
    S, idx = resident
    reqs = requests(S, 60, seed=5)
    want = [pj.pj_query(idx, qs, t).pairs for qs, t in reqs]
    srv = pj.Server(idx, slots=3)
    try:
        tickets = [srv.submit(qs, t) for qs, t in reqs]
        for tk, w in zip(tickets, want):
            res, times = srv.wait(tk, timeout_ms=60000)
            assert np.array_equal(res.pairs, w)
            assert times["batch_requests"] >= 1
        st = srv.stats()
        assert st["requests"] == len(reqs)
        assert st["batches"] < len(reqs)           # requests were batched together
        assert st["max_batch_requests"] > 1
    finally:
        srv.stop()


def test_server_concurrent_submitters_and_overlap(resident):
    S, idx = resident
    reqs = requests(S, 40, seed=9)
    want = [pj.pj_query(idx, qs, t).pairs for qs, t in reqs]
    srv = pj.Server(idx, slots=3, max_batch_queries=400)
    errors = []
    try:
        def worker(k0):
            for k in range(k0, len(reqs), 4):
                tk = srv.submit(*reqs[k])
                res, _ = srv.wait(tk)
                if not np.array_equal(res.pairs, want[k]):
                    errors.append(k)
        th = [threading.Thread(target=worker, args=(k,)) for k in range(4)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        assert not errors
        assert srv.stats()["requests"] == len(reqs)
    finally:
        srv.stop()


def test_server_timeout_and_cancel(resident):
    S, idx = resident
    srv = pj.Server(idx, slots=1)
    try:
        big = synth.generate("short", 4, n=4000, seed=77)
        tk = srv.submit(big, 4)
        try:
            res, _ = srv.wait(tk, timeout_ms=0)   # almost surely still queued or running
        except pj.PJError as e:
            assert e.code == pj.PJ_ETIMEDOUT
            res, _ = srv.wait(tk)
        assert np.array_equal(res.pairs, pj.pj_query(idx, big, 4).pairs)
        # cancel: block the single slot with a big request, then cancel a queued one
        t1 = srv.submit(big, 4)
        t2 = srv.submit(big[:100], 3)
        srv.cancel(t2)
        with pytest.raises(pj.PJError) as e:
            srv.wait(t2)
        assert e.value.code == pj.PJ_ECANCELED
        srv.wait(t1)
        with pytest.raises(pj.PJError):
            srv.wait(t1)  # a ticket is collected once
    finally:
        srv.stop()
