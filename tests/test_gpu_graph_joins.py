"""Self-join graphs: a repeated self join of an unchanged index replayed as
one recorded CUDA graph (pj_options.graph_joins).

A replayed join must equal the eager join and the oracle exactly (integer
results, tolerance 0), and report the same counts.  Covered: extension
verification with indexed strings too short to partition (the fallback
kernel), distinct-pair verification with a thread and with a warp per pair,
host and device results, several thresholds of one index, an eager join
taken in several probe chunks, replays whose counts overflow the recorded
capacities (falling back to the eager join), joins that are not recorded
(too many probe groups, a warp-per-candidate range), an index without
graph joins, and launch accounting.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1111_7171_gb300 import passjoin as pj
from paper_1111_7171_gb300 import synth

pytestmark = pytest.mark.gpu

COUNTS = ("lookups", "candidates", "accepted", "hits", "dp_cells", "fallback_pairs", "filtered", "distinct_pairs")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    yield


def cpu_self(strings, tau, banded=False):
    b, o = synth.pack(strings)
    return oracle.self_join(b, o, tau, banded=banded)


def joins(strings, tau, runs=3, tau_max=None, **kw):
    idx = pj.pj_build_index(strings, tau if tau_max is None else tau_max, graph_joins=True, **kw)
    try:
        return [pj.pj_self_join(idx, tau) for _ in range(runs)]
    finally:
        idx.free()


def check_replays(rs, want, what, counts=COUNTS):
    assert rs[0].stats["graph_replay"] == 0, what  # the eager join that gets recorded
    for k, r in enumerate(rs):
        assert np.array_equal(np.asarray(r.pairs), want), f"{what} run {k}"
        for key in counts:
            assert r.stats[key] == rs[0].stats[key], f"{what} run {k} {key}"
    for r in rs[1:]:
        assert r.stats["graph_replay"] == 1, what
        assert r.stats["graph_ms"] > 0.0, what
        for key in COUNTS:  # replays repeat exactly
            assert r.stats[key] == rs[1].stats[key], f"{what} replay {key}"


def test_graph_replay_extension_verification(monkeypatch):
    monkeypatch.setenv("PJ_VERIFY_PAIRS", "0")
    for name, tau, n, banded in [("short", 4, 4000, False), ("short2k", 2, 2000, False), ("medium", 6, 2500, True)]:
        strings = synth.generate(name, tau, n=n) + [b"", b"a", b"ab", b"abc", b"abcd"]
        check_replays(joins(strings, tau), cpu_self(strings, tau, banded=banded), f"{name} tau={tau}")


@pytest.mark.parametrize("mode", ["1", "2"])
def test_graph_replay_distinct_pairs(monkeypatch, mode):
    monkeypatch.setenv("PJ_VERIFY_PAIRS", mode)
    for name, tau, n, banded in [("short", 3, 3000, False), ("medium", 8, 2500, True), ("long", 32, 600, True)]:
        strings = synth.generate(name, tau, n=n) + [b"", b"xy"]
        rs = joins(strings, tau)
        check_replays(rs, cpu_self(strings, tau, banded=banded), f"{name} tau={tau} pairs={mode}")
        assert rs[1].stats["verify_mode"] == 2  # distinct pairs
        assert 0 < rs[1].stats["distinct_pairs"] <= rs[1].stats["candidates"]


def test_graph_replay_default_modes_and_thresholds():
    """Default verification choice; each threshold of one index keeps its own
    graph, interleaved with the others."""
    strings = synth.generate("short", 4, n=5000)
    idx = pj.pj_build_index(strings, 4, graph_joins=True)
    try:
        first = {}
        for rep in range(3):
            for tau in (4, 1, 2, 0):
                r = pj.pj_self_join(idx, tau)
                assert np.array_equal(r.pairs, cpu_self(strings, tau)) if rep == 0 else \
                    np.array_equal(r.pairs, first[tau].pairs), (tau, rep)
                assert r.stats["graph_replay"] == (0 if rep == 0 else 1), (tau, rep)
                first.setdefault(tau, r)
    finally:
        idx.free()
    strings = synth.generate("long", 16, n=700)
    check_replays(joins(strings, 16), cpu_self(strings, 16, banded=True), "long default")


def test_graph_replay_results_on_device():
    strings = synth.generate("short", 3, n=3000) + [b"", b"q"]
    idx = pj.pj_build_index(strings, 3, graph_joins=True, results_on_device=True)
    try:
        want = cpu_self(strings, 3)
        for k in range(3):
            r = pj.pj_self_join(idx, 3)
            assert isinstance(r, pj.DeviceResult)
            assert r.stats["graph_replay"] == (1 if k else 0)
            host = r.to_host()
            r.free()
            assert np.array_equal(host, want), k
    finally:
        idx.free()


def test_joins_that_are_not_recorded(monkeypatch):
    monkeypatch.setenv("PJ_VERIFY_PAIRS", "0")
    strings = synth.generate("short", 3, n=3000)
    want = cpu_self(strings, 3)
    monkeypatch.setenv("PJ_GRAPH_MAX_GROUPS", "1000")  # more probe groups than a graph may hold
    rs = joins(strings, 3)
    assert all(r.stats["graph_replay"] == 0 for r in rs)
    assert all(np.array_equal(r.pairs, want) for r in rs)
    monkeypatch.delenv("PJ_GRAPH_MAX_GROUPS")
    monkeypatch.setenv("PJ_WARP_MIN_LEN", "20")  # a warp-per-candidate range
    rs = joins(strings, 3)
    assert all(r.stats["graph_replay"] == 0 for r in rs)
    assert all(np.array_equal(r.pairs, want) for r in rs)
    monkeypatch.delenv("PJ_WARP_MIN_LEN")
    idx = pj.pj_build_index(strings, 3)  # graph joins off
    try:
        assert all(pj.pj_self_join(idx, 3).stats["graph_replay"] == 0 for _ in range(2))
    finally:
        idx.free()


def test_graph_replay_after_chunked_eager_join(monkeypatch):
    """The eager join probes in several chunks, the recorded graph in one
    pass: same pairs and probe counts.  In mode L a pair found from probes of
    two chunks is made distinct, and verified, once per chunk, so the
    verification counts may differ there."""
    monkeypatch.setenv("PJ_GROUP_BUDGET", "2000")
    probe_counts = ("lookups", "candidates", "hits", "fallback_pairs")
    for mode in ("0", "1"):
        monkeypatch.setenv("PJ_VERIFY_PAIRS", mode)
        strings = synth.generate("short", 3, n=3000)
        check_replays(joins(strings, 3), cpu_self(strings, 3), f"chunked eager pairs={mode}",
                      COUNTS if mode == "0" else probe_counts)


@pytest.mark.parametrize("mode", ["0", "1"])
def test_replays_that_overflow_fall_back(monkeypatch, mode):
    """Graphs recorded with half the eager run's counts as capacities (hits,
    candidates, accepted matches, pairs): every replay overflows, is
    discarded, and the join runs eagerly -- same pairs, graph_replay 0."""
    monkeypatch.setenv("PJ_GRAPH_TIGHT", "1")
    monkeypatch.setenv("PJ_VERIFY_PAIRS", mode)
    strings = synth.generate("short", 3, n=3000) + [b"", b"ab"]
    want = cpu_self(strings, 3)
    rs = joins(strings, 3, runs=4)
    assert all(r.stats["graph_replay"] == 0 for r in rs)
    assert all(np.array_equal(r.pairs, want) for r in rs)
    for key in COUNTS:
        assert all(r.stats[key] == rs[0].stats[key] for r in rs), key


def test_graph_replay_empty_and_tiny():
    for strings in ([b"abc"], [b"", b""], [b"abcdef", b"abcdeg"], [b"a", b"b", b"c"]):
        for tau in (0, 1, 2):
            rs = joins(strings, tau)
            want = cpu_self(strings, tau)
            assert all(np.array_equal(np.asarray(r.pairs), want) for r in rs), (strings, tau)


def test_graph_replay_launch_accounting():
    strings = synth.generate("short", 2, n=3000)
    idx = pj.pj_build_index(strings, 2, graph_joins=True)
    try:
        pj.pj_self_join(idx, 2)
        pj.pj_self_join(idx, 2)
        before = pj.pj_kernel_launches()
        r = pj.pj_self_join(idx, 2)
        k = pj.pj_kernel_launches() - before
        assert r.stats["graph_replay"] == 1
        assert 8 <= k <= 64  # the recorded pipeline's kernels, counted once per replay
        before = pj.pj_kernel_launches()
        assert pj.pj_self_join(idx, 2).stats["graph_replay"] == 1
        assert pj.pj_kernel_launches() - before == k
    finally:
        idx.free()


@pytest.mark.parametrize("mode", ["1", "2"])
def test_graph_replay_fused(monkeypatch, mode):
    """The fused self join recorded into the graph: k_fused_self over the
    probes from PJ_FUSED_FROM, the chunked mode-L pipeline over the shorter
    ones, the overflow and long-run lists gathered and verified on the device.
    Replays equal the oracle; the probe counts repeat (which pairs leave the
    kernel through the overflow lists depends on timing, so the verification
    counts may differ); replays whose lists or buffers outgrow the recorded
    capacities are discarded."""
    monkeypatch.setenv("PJ_FUSED", mode)
    probe_counts = ("lookups", "candidates", "hits", "fallback_pairs")
    cases = [("medium", 8, 2500, True, "0"), ("medium", 8, 2500, True, "80"), ("long", 32, 600, True, "0"),
             ("short", 4, 3000, False, "16")]
    for name, tau, n, banded, frm in cases:
        monkeypatch.setenv("PJ_FUSED_FROM", frm)
        strings = synth.generate(name, tau, n=n) + [b"", b"xy"]
        rs = joins(strings, tau)
        check_replays(rs, cpu_self(strings, tau, banded=banded), f"{name} tau={tau} fused={mode} from {frm}",
                      probe_counts)
        assert all(r.stats["fused"] == 1 for r in rs)
    monkeypatch.setenv("PJ_FUSED_FROM", "0")
    base = synth.generate("medium", 8, n=1500)
    strings = base + [base[7]] * 300 + [base[11]] * 40  # long runs and full lists
    check_replays(joins(strings, 8), cpu_self(strings, 8, banded=True), f"copies fused={mode}", probe_counts)
    monkeypatch.setenv("PJ_GRAPH_TIGHT", "1")
    rs = joins(strings, 8, runs=3)
    assert all(r.stats["graph_replay"] == 0 for r in rs)
    want = cpu_self(strings, 8, banded=True)
    assert all(np.array_equal(np.asarray(r.pairs), want) for r in rs)
