"""Full-size parity: every workload at every one of its thresholds, and the
serving workload on its 1M-string resident index.

At the workloads' full sizes (1M short, 500k medium, 100k long strings) the
brute-force oracle cannot run every whole join, so the GPU self join (the
launch configuration bench.py times: resident device input, lazy threshold
index, autotuned verification, results in device memory) is checked on
outputs the oracle computes one by one:
  * every reported pair is well formed (a < b, sorted, unique, ed <= tau);
  * sampled reported pairs have exactly the oracle's ED (full DP);
  * for PROBES sampled strings -- half uniform over the set, half taken from
    reported pairs -- the set of partners with ED <= tau and their ED equals
    the oracle's one-against-all result over the whole set (banded DP,
    pinned to the plain DP by the CPU tests).
Where the whole join fits the host cores in seconds (long strings at
tau = 8) the complete pair set is compared with the oracle's.

The serving check builds the 1M-string index for tau_max = 4, runs a stream
of requests with mixed thresholds through the continuous-batching server with
graph-captured plans, and compares each sampled query's pairs with the
oracle's.  Integer work: the tolerance is zero (Def. 1, Sec. 2; Theorem 6).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1111_7171_gb300 import passjoin as pj
from paper_1111_7171_gb300 import synth

pytestmark = pytest.mark.gpu

PROBES = 600
ED_SAMPLES = 2000

FULL_SIZE = [("short", t) for t in (1, 2, 3, 4)] + [("medium", t) for t in (2, 4, 6, 8)] + \
            [("long", t) for t in (8, 16, 32)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    yield


def bench_launch_self_join(buf, off, tau):
    """The self join as bench.py runs it (device input, lazy index, autotune,
    device results), copied back to the host."""
    db = torch.from_numpy(buf).cuda()
    do = torch.from_numpy(off.astype(np.int64)).cuda()
    idx = pj.pj_build_index((db, do), tau, lazy_partitions=True, results_on_device=True, autotune=True)
    try:
        r = pj.pj_self_join(idx, tau)
        pairs, stats = r.to_host(), r.stats
        r.free()
    finally:
        idx.free()
    return pairs, stats


def partner_sets(a, b, ed, probes):
    """{probe: {(partner, ed)}} for the probes, from pairs (a < b)."""
    out = {x: set() for x in probes}
    m = np.isin(a, probes)
    for x, y, e in zip(a[m].tolist(), b[m].tolist(), ed[m].tolist()):
        out[x].add((y, e))
    m = np.isin(b, probes)
    for x, y, e in zip(b[m].tolist(), a[m].tolist(), ed[m].tolist()):
        out[x].add((y, e))
    return out


@pytest.mark.parametrize("name,tau", FULL_SIZE)
def test_full_size_sampled(name, tau):
    strings = synth.generate(name, tau)
    buf, off = synth.pack(strings)
    pairs, stats = bench_launch_self_join(buf, off, tau)
    a = pairs["a"].astype(np.int64)
    b = pairs["b"].astype(np.int64)
    ed = pairs["ed"].astype(np.int64)
    n = len(strings)
    assert len(pairs) > 0
    assert (a < b).all() and (b < n).all() and (ed <= tau).all()
    key = a * n + b
    assert (np.diff(key) > 0).all(), "pairs must be sorted and unique"

    rng = np.random.default_rng(1000 + tau)
    # reported pairs have the oracle's exact ED (full Wagner-Fischer)
    for k in rng.choice(len(pairs), size=min(ED_SAMPLES, len(pairs)), replace=False).tolist():
        assert oracle.ed(strings[a[k]], strings[b[k]]) == ed[k], (name, tau, a[k], b[k])

    # partner sets of sampled probe strings: half uniform, half from pairs
    probes = set(rng.choice(n, size=PROBES // 2, replace=False).tolist())
    from_pairs = rng.choice(len(pairs), size=min(len(pairs), PROBES), replace=False)
    for k in from_pairs.tolist():
        if len(probes) >= PROBES:
            break
        probes.add(int(a[k]) if k % 2 else int(b[k]))
    probes = np.array(sorted(probes), dtype=np.int64)
    qb, qo = synth.pack([strings[x] for x in probes.tolist()])
    want = oracle.similar_to(qb, qo, buf, off, tau, banded=True, exclude=probes)
    got = partner_sets(a, b, ed, probes)
    wa = want["a"].astype(np.int64)
    for qi, x in enumerate(probes.tolist()):
        w = want[wa == qi]
        want_set = {(int(y), int(e)) for y, e in zip(w["b"], w["ed"])}
        assert got[x] == want_set, (name, tau, x, len(got[x]), len(want_set))
    assert sum(len(s) for s in got.values()) > 0, "the sample must contain similar pairs"


def test_full_size_complete_long_tau8():
    """Long strings at tau = 8: the whole pair set against the oracle's whole
    self join (banded DP, all host cores)."""
    strings = synth.generate("long", 8)
    buf, off = synth.pack(strings)
    pairs, _ = bench_launch_self_join(buf, off, 8)
    want = oracle.self_join(buf, off, 8, banded=True)
    assert len(want) > 0
    assert np.array_equal(pairs, want)


@pytest.mark.parametrize("name,tau", [("medium", 4), ("long", 32), ("medium", 8)])
def test_full_size_graph_replay_and_forms_agree(name, tau, monkeypatch):
    """At full size, the tuned self join replayed from its recorded CUDA graph
    (graph_joins; the fused kernel where the tuner picks it), the chunked
    pipeline (PJ_FUSED=0) and the fused kernel on every probe (PJ_FUSED=1)
    return the same pair set; that set is checked against the oracle by
    test_full_size_sampled."""
    strings = synth.generate(name, tau)
    buf, off = synth.pack(strings)
    db = torch.from_numpy(buf).cuda()
    do = torch.from_numpy(off.astype(np.int64)).cuda()

    def join(graph, fused):
        if fused is None:
            monkeypatch.delenv("PJ_FUSED", raising=False)
        else:
            monkeypatch.setenv("PJ_FUSED", fused)
        idx = pj.pj_build_index((db, do), tau, results_on_device=True, autotune=True, graph_joins=graph)
        try:
            out = []
            for _ in range(2 if graph else 1):
                r = pj.pj_self_join(idx, tau)
                out.append((r.to_host(), r.stats["graph_replay"]))
                r.free()
            return out[-1]
        finally:
            idx.free()

    replayed, was_replay = join(True, None)
    assert was_replay == 1
    chunked, _ = join(False, "0")
    fused, _ = join(False, "1")
    assert len(chunked) > 0
    assert np.array_equal(replayed, chunked), (name, tau, "graph replay")
    assert np.array_equal(fused, chunked), (name, tau, "fused kernel")


def test_serving_full_size_mixed_tau():
    """The serving workload: 1M short strings resident (tau_max = 4), a stream
    of requests of 1..4096 queries with tau uniform in 1..4, run through the
    continuous-batching server with graph-captured plans (several requests
    per batch, batches overlapping).  Sampled queries of every request have
    exactly the oracle's partner set."""
    strings = synth.generate("short", 4)
    buf, off = synth.pack(strings)
    reqs = synth.query_stream(strings, 160, seed=4000, tau_max=4, max_batch=4096)
    idx = pj.pj_build_index(strings, 4)
    srv = pj.Server(idx, slots=3, use_plans=True)
    try:
        tickets = [srv.submit(qs, t) for qs, t in reqs]
        results = [srv.wait(tk)[0].pairs for tk in tickets]
        st = srv.stats()
    finally:
        srv.stop()
        idx.free()
    assert st["requests"] == len(reqs) and st["max_batch_requests"] > 1

    rng = np.random.default_rng(44)
    by_tau = {t: [] for t in range(1, 5)}  # tau -> [(request, position)]
    for r, (qs, t) in enumerate(reqs):
        k = min(len(qs), 8)
        for p in rng.choice(len(qs), size=k, replace=False).tolist():
            by_tau[t].append((r, p))
    checked = found = 0
    for t, picks in by_tau.items():
        if not picks:
            continue
        qb, qo = synth.pack([reqs[r][0][p] for r, p in picks])
        want = oracle.similar_to(qb, qo, buf, off, t, banded=True)
        wa = want["a"].astype(np.int64)
        for qi, (r, p) in enumerate(picks):
            w = want[wa == qi]
            want_set = {(int(y), int(e)) for y, e in zip(w["b"], w["ed"])}
            res = results[r]
            m = res["a"] == p
            got_set = {(int(y), int(e)) for y, e in zip(res["b"][m], res["ed"][m])}
            assert got_set == want_set, (t, r, p, len(got_set), len(want_set))
            checked += 1
            found += len(want_set)
    assert checked >= 500 and found > 0
