"""Query plans: the multi-threshold query pipeline replayed as a CUDA graph.

A plan's result for a batch must equal pj_query_multi's (and so pj_query's
per query, and the oracle's) exactly, whatever its capacities: integer
results, tolerance 0.  Covered: graph reuse across different batches, empty
and single-query batches, a batch at the plan's limits, capacity growth from
one-entry buffers (re-recorded graph), indexed strings too short to
partition (fallback kernel), a lazy index, launch accounting, argument
errors, and the server running its batches through plans.
"""
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


def mixed_batch(S, n_req, seed, max_batch=300):
    reqs = synth.query_stream(S, n_req, seed=seed, tau_max=4, max_batch=max_batch)
    reqs.append(([b"", b"b", b"ab"], 2))
    reqs.append(([b"abcd", b"xbcd"], 0))
    batch = [q for qs, _ in reqs for q in qs]
    taus = np.array([t for qs, t in reqs for _ in qs], dtype=np.uint8)
    return batch, taus


def test_plan_equals_query_multi_and_oracle(resident):
    S, idx = resident
    sb, so = synth.pack(S)
    plan = pj.Plan(idx, max_queries=4096, max_bytes=1 << 20)
    try:
        for seed in (1, 2, 3):  # one graph, several different batches
            batch, taus = mixed_batch(S, 10, seed)
            got = plan.query(batch, taus)
            want = pj.pj_query_multi(idx, batch, taus)
            assert np.array_equal(got.pairs, want.pairs)
            for key in ("lookups", "candidates", "accepted", "hits", "dp_cells", "fallback_pairs"):
                assert got.stats[key] == want.stats[key], key
        # the oracle on one batch, per threshold
        batch, taus = mixed_batch(S, 6, 11)
        got = plan.query(batch, taus).pairs
        for t in np.unique(taus).tolist():
            sel = np.flatnonzero(taus == t)
            qb, qo = synth.pack([batch[k] for k in sel.tolist()])
            w = oracle.join(qb, qo, sb, so, int(t))
            g = got[np.isin(got["a"], sel)].copy()
            g["a"] = np.searchsorted(sel, g["a"])
            assert np.array_equal(g, w), t
        info = plan.info()
        assert info["runs"] >= 4 and info["graph_kernels"] > 10
    finally:
        plan.free()


def test_plan_empty_single_and_full_batches(resident):
    S, idx = resident
    plan = pj.Plan(idx, max_queries=64, max_bytes=64 * 80)
    try:
        assert len(plan.query([], [])) == 0
        one = [S[123]]
        assert np.array_equal(plan.query(one, [3]).pairs, pj.pj_query(idx, one, 3).pairs)
        full = [S[k][:80] for k in range(0, 6400, 100)]  # exactly 64 queries, at most 64 * 80 bytes
        taus = np.arange(64, dtype=np.uint8) % 5
        assert np.array_equal(plan.query(full, taus).pairs, pj.pj_query_multi(idx, full, taus).pairs)
        assert len(plan.query([], [])) == 0  # empty again after a full one
    finally:
        plan.free()


def test_plan_grows_from_tiny_capacities(resident):
    S, idx = resident
    plan = pj.Plan(idx, max_queries=2048, max_bytes=1 << 20, hits_capacity=1, accepted_capacity=1, pairs_capacity=1)
    try:
        batch, taus = mixed_batch(S, 8, 21)
        want = pj.pj_query_multi(idx, batch, taus).pairs
        assert len(want) > 1
        got = plan.query(batch, taus).pairs
        assert np.array_equal(got, want)
        info = plan.info()
        assert info["recaptures"] >= 3  # hits, accepted matches and pairs each grew
        assert info["hits_capacity"] > 1 and info["accepted_capacity"] > 1 and info["pairs_capacity"] > 1
        # grown buffers stay; the next batch needs no new recording
        batch2, taus2 = mixed_batch(S, 8, 22)
        before = plan.info()["recaptures"]
        assert np.array_equal(plan.query(batch2, taus2).pairs, pj.pj_query_multi(idx, batch2, taus2).pairs)
        assert plan.info()["recaptures"] >= before
    finally:
        plan.free()


def test_plan_short_indexed_strings_use_the_fallback():
    # indexed strings of length <= tau have no even partition
    S = [b"", b"a", b"b", b"ab", b"ba", b"abc", b"abd", b"abcd", b"abcde", b"zzzzzz", b"abcdef"]
    sb, so = synth.pack(S)
    idx = pj.pj_build_index(S, 3)
    plan = pj.Plan(idx, max_queries=16, max_bytes=256)
    try:
        Q = [b"", b"a", b"abc", b"abcd", b"zz", b"abcdefg", b"q"]
        for t in range(4):
            got = plan.query(Q, np.full(len(Q), t, dtype=np.uint8)).pairs
            qb, qo = synth.pack(Q)
            assert np.array_equal(got, oracle.join(qb, qo, sb, so, t)), t
        taus = np.array([0, 1, 2, 3, 1, 2, 3], dtype=np.uint8)
        assert np.array_equal(plan.query(Q, taus).pairs, pj.pj_query_multi(idx, Q, taus).pairs)
    finally:
        plan.free()
        idx.free()


def test_plan_builds_every_threshold_of_a_lazy_index():
    S = synth.generate("short", 3, n=4000)
    idx = pj.pj_build_index(S, 3, lazy_partitions=True)
    try:
        plan = pj.Plan(idx, max_queries=512)
        Q = [S[k] for k in range(0, 4000, 9)]
        taus = np.arange(len(Q), dtype=np.uint8) % 4
        got = plan.query(Q, taus).pairs
        plan.free()
        assert np.array_equal(got, pj.pj_query_multi(idx, Q, taus).pairs)
    finally:
        idx.free()


def test_plan_launch_accounting(resident):
    S, idx = resident
    plan = pj.Plan(idx, max_queries=1024)
    try:
        batch, taus = mixed_batch(S, 4, 31, max_batch=100)
        plan.query(batch, taus)  # sizes settle
        k = plan.info()["graph_kernels"]
        r0 = plan.info()["recaptures"]
        before = pj.pj_kernel_launches()
        plan.query(batch, taus)
        assert plan.info()["recaptures"] == r0
        assert pj.pj_kernel_launches() - before == k
    finally:
        plan.free()


def test_plan_argument_errors(resident):
    S, idx = resident
    plan = pj.Plan(idx, max_queries=4, max_bytes=32)
    try:
        with pytest.raises(pj.PJError) as e:
            plan.query([b"a"] * 5, 1)
        assert e.value.code == pj.PJ_EINVAL
        with pytest.raises(pj.PJError) as e:
            plan.query([b"x" * 33], 1)
        assert e.value.code == pj.PJ_EINVAL
        with pytest.raises(pj.PJError) as e:
            plan.query([b"abc"], 5)  # above tau_max
        assert e.value.code == pj.PJ_EINVAL
        dev = (torch.tensor([97, 98], dtype=torch.uint8, device="cuda"),
               torch.tensor([0, 2], dtype=torch.int64, device="cuda"))
        with pytest.raises(pj.PJError) as e:
            plan.query(dev, 1)
        assert e.value.code == pj.PJ_EINVAL
        # the plan still works after rejected calls
        assert np.array_equal(plan.query([S[7]], 2).pairs, pj.pj_query(idx, [S[7]], 2).pairs)
    finally:
        plan.free()
    with pytest.raises(pj.PJError) as e:
        pj.Plan(idx, max_queries=0)
    assert e.value.code == pj.PJ_EINVAL


def test_server_with_plans_equals_alone(resident):
    S, idx = resident
    reqs = synth.query_stream(S, 50, seed=41, tau_max=4, max_batch=300)
    reqs.append(([b"", b"b", b"ab"], 2))
    want = [pj.pj_query(idx, qs, t).pairs for qs, t in reqs]
    srv = pj.Server(idx, slots=2, max_batch_queries=1024, max_batch_bytes=1 << 20, use_plans=True)
    try:
        tickets = [srv.submit(qs, t) for qs, t in reqs]
        for tk, w in zip(tickets, want):
            res, _ = srv.wait(tk, timeout_ms=60000)
            assert np.array_equal(res.pairs, w)
        # a single request above the plans' query limit runs on the eager path
        big = [S[k] for k in range(0, 2 * 1024 * 10, 10)]
        tk = srv.submit(big, 1)
        res, _ = srv.wait(tk, timeout_ms=60000)
        assert np.array_equal(res.pairs, pj.pj_query(idx, big, 1).pairs)
    finally:
        srv.stop()
