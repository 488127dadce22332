"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Integer work, so the bar is bit-exact: the sorted (a, b, ed) arrays must be
equal.  Sizes here span many tiles, warps and posting runs and include ragged
tails; full-size workloads are checked on sampled outputs that the oracle
computes one by one (tests/test_gpu_fullsize.py).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import method as M
from paper_1111_7171_gb300 import passjoin as pj
from paper_1111_7171_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    yield


def gpu_self(strings, tau, tau_max=None):
    idx = pj.pj_build_index(strings, tau if tau_max is None else tau_max)
    try:
        return pj.pj_self_join(idx, tau)
    finally:
        idx.free()


def cpu_self(strings, tau, banded=False):
    b, o = synth.pack(strings)
    return oracle.self_join(b, o, tau, banded=banded)


def assert_same(got, want, what=""):
    got = np.asarray(got)
    if len(got) != len(want) or not np.array_equal(got, want):
        gs = set(map(tuple, got.tolist()))
        ws = set(map(tuple, want.tolist()))
        raise AssertionError(f"{what}: {len(got)} vs {len(want)} pairs; "
                             f"extra {sorted(gs - ws)[:5]} missing {sorted(ws - gs)[:5]}")


# --------------------------------------------------------------- workloads --

@pytest.mark.parametrize("tau", [0, 1, 2, 3])
def test_short2k_full(tau):
    strings = synth.generate("short2k", 2)
    assert_same(gpu_self(strings, tau).pairs, cpu_self(strings, tau), f"short2k tau={tau}")


@pytest.mark.parametrize("tau", [1, 2, 3, 4])
def test_short_subsample(tau):
    strings = synth.generate("short", tau, n=6000)
    assert_same(gpu_self(strings, tau).pairs, cpu_self(strings, tau), f"short n=6000 tau={tau}")


@pytest.mark.parametrize("tau", [2, 4, 6, 8])
def test_medium_subsample(tau):
    strings = synth.generate("medium", tau, n=5000)
    assert_same(gpu_self(strings, tau).pairs, cpu_self(strings, tau, banded=True), f"medium tau={tau}")


@pytest.mark.parametrize("tau", [8, 16, 32])
def test_long_subsample(tau):
    strings = synth.generate("long", tau, n=1200)
    assert_same(gpu_self(strings, tau).pairs, cpu_self(strings, tau, banded=True), f"long tau={tau}")


def test_index_reuse_across_tau():
    """One index built for tau_max answers every smaller tau exactly."""
    strings = synth.generate("short", 4, n=3000)
    idx = pj.pj_build_index(strings, 4)
    try:
        for tau in range(0, 5):
            assert_same(pj.pj_self_join(idx, tau).pairs, cpu_self(strings, tau), f"tau={tau}")
    finally:
        idx.free()


def test_candidate_and_accept_counts_match_algorithm():
    """The kernels examine exactly the (s, r, i, p) matches of Alg. 1 with
    multi-match selection (visiting by length, then by the first eight
    bytes, then id: the store's order) and accept exactly the ones extension
    verification accepts."""
    strings = synth.generate("short", 3, n=700)
    strings += [strings[5][:6] + b"zz" + strings[5][8:], strings[5][:9] + b"q"]  # shared first 8 bytes
    st = {}
    M.pass_join_self(strings, 3, order="prefix8", stats=st)
    res = gpu_self(strings, 3)
    assert res.stats["candidates"] == st["tuples"]
    assert res.stats["accepted"] == st["accepted"]


# --------------------------------------------------------- R x S and query --

def _rs_sets(seed, tau):
    S = synth.generate("short", tau, n=2500, seed=seed)
    S += [b"", b"a", b"ab", b"abc"[:tau], b"zz"]
    R = synth.generate("short", tau, n=800, seed=seed + 1)
    rng = np.random.default_rng(seed)
    for k in rng.integers(0, len(S), size=300).tolist():
        s = bytearray(S[k])
        for _ in range(int(rng.integers(0, tau + 1))):
            if s and rng.random() < 0.4:
                del s[int(rng.integers(0, len(s)))]
            else:
                s.insert(int(rng.integers(0, len(s) + 1)), ord("a") + int(rng.integers(0, 26)))
        R.append(bytes(s))
    R += [b"", b"b", b"abcd"]
    return R, S


@pytest.mark.parametrize("tau", [1, 2, 4])
def test_join_rs(tau):
    R, S = _rs_sets(40 + tau, tau)
    rb, ro = synth.pack(R)
    sb, so = synth.pack(S)
    assert_same(pj.pj_join(R, S, tau).pairs, oracle.join(rb, ro, sb, so, tau), f"join tau={tau}")


def test_query_against_resident_index():
    R, S = _rs_sets(77, 4)
    sb, so = synth.pack(S)
    idx = pj.pj_build_index(S, 4)
    try:
        for tau in (1, 2, 3, 4):
            batch = R[tau * 100:(tau + 1) * 150]
            qb, qo = synth.pack(batch)
            assert_same(pj.pj_query(idx, batch, tau).pairs, oracle.join(qb, qo, sb, so, tau), f"query tau={tau}")
    finally:
        idx.free()


def test_device_inputs_match_host_inputs():
    strings = synth.generate("medium", 4, n=2000)
    b, o = synth.pack(strings)
    db = torch.from_numpy(b).cuda()
    do = torch.from_numpy(o.astype(np.int64)).cuda()
    idx = pj.pj_build_index((db, do), 4)
    try:
        assert_same(pj.pj_self_join(idx, 4).pairs, cpu_self(strings, 4, banded=True), "device input")
    finally:
        idx.free()


def test_results_on_device():
    strings = synth.generate("short", 2, n=3000)
    idx = pj.pj_build_index(strings, 2, results_on_device=True)
    try:
        r = pj.pj_self_join(idx, 2)
        assert isinstance(r, pj.DeviceResult)
        host = r.to_host()
        r.free()
        assert_same(host, cpu_self(strings, 2), "device results")
    finally:
        idx.free()


# ------------------------------------------------------------- edge cases --

def test_empty_and_single():
    for strings in ([], [b""], [b"abc"], [b"", b""], [b"a", b""]):
        for tau in (0, 1, 3):
            assert_same(gpu_self(strings, tau).pairs, cpu_self(strings, tau), f"{strings} tau={tau}")


def test_all_identical_one_posting_run():
    strings = [b"abcdefgh"] * 700 + [b"abcdefgX", b"Xbcdefgh"]
    for tau in (0, 1, 2):
        assert_same(gpu_self(strings, tau).pairs, cpu_self(strings, tau), f"identical tau={tau}")


def test_one_symbol_alphabet():
    rng = np.random.default_rng(3)
    strings = [b"a" * int(k) for k in rng.integers(0, 30, size=400)]
    for tau in (1, 3, 5):
        assert_same(gpu_self(strings, tau).pairs, cpu_self(strings, tau), f"unary tau={tau}")


def test_lengths_around_tau_plus_one():
    rng = np.random.default_rng(5)
    strings = []
    for _ in range(900):
        L = int(rng.integers(0, 9))
        strings.append(bytes(rng.choice(list(b"abc"), size=L).tolist()))
    for tau in (2, 3, 4, 6):
        assert_same(gpu_self(strings, tau).pairs, cpu_self(strings, tau), f"short lengths tau={tau}")


def test_long_strings_beyond_staging():
    rng = np.random.default_rng(9)
    base = bytes(rng.integers(97, 101, size=5000).tolist())
    strings = [base]
    for k in range(6):
        s = bytearray(base)
        for _ in range(k):
            s[int(rng.integers(0, len(s)))] = ord("z")
        strings.append(bytes(s))
    strings += [bytes(rng.integers(97, 101, size=int(L)).tolist()) for L in rng.integers(4990, 5010, size=20)]
    for tau in (3, 8):
        assert_same(gpu_self(strings, tau).pairs, cpu_self(strings, tau, banded=True), f"5000-byte tau={tau}")


def test_invalid_arguments():
    idx = pj.pj_build_index([b"abc", b"abd"], 2)
    try:
        with pytest.raises(pj.PJError) as e:
            pj.pj_self_join(idx, 3)
        assert e.value.code == pj.PJ_EINVAL
        with pytest.raises(pj.PJError):
            pj.pj_self_join(idx, -1)
    finally:
        idx.free()
    with pytest.raises(pj.PJError) as e:
        pj.pj_build_index([b"abc"], pj.PJ_TAU_LIMIT + 1)
    assert e.value.code == pj.PJ_EINVAL
    with pytest.raises(pj.PJError) as e:
        pj.pj_build_index((np.frombuffer(b"abcdef", np.uint8), np.array([0, 4, 2, 6], np.uint64)), 1)
    assert e.value.code == pj.PJ_EINVAL
    with pytest.raises(pj.PJError) as e:
        pj.pj_join([b"a"], [b"b"], pj.PJ_TAU_LIMIT + 1)
    assert e.value.code == pj.PJ_EINVAL


def test_index_audit(monkeypatch):
    """PJ_CHECK_INDEX=1 audits every partition on the host after it is built:
    runs tile the postings, fingerprints and presence bitmap match the stored
    keys, at least half the slots are empty.  Includes a partition with no
    partitioned strings (every string shorter than tau + 1)."""
    monkeypatch.setenv("PJ_CHECK_INDEX", "1")
    for strings, tau in [(synth.generate("short", 4, n=3000), 4), (synth.generate("long", 16, n=300), 16),
                         ([b"", b"a", b"ab"], 3)]:
        idx = pj.pj_build_index(strings, tau)
        try:
            for t in sorted({0, tau // 2, tau}):
                assert_same(pj.pj_self_join(idx, t).pairs, cpu_self(strings, t, banded=len(strings) == 300),
                            f"audited tau={t}")
        finally:
            idx.free()


def test_lazy_partitions_match_eager():
    strings = synth.generate("short", 3, n=3000)
    want = cpu_self(strings, 3)
    idx = pj.pj_build_index(strings, 4, lazy_partitions=True)
    try:
        r = pj.pj_self_join(idx, 3)
        assert r.stats["partition_ms"] > 0
        assert_same(r.pairs, want, "lazy tau=3")
        r2 = pj.pj_self_join(idx, 3)  # built once
        assert r2.stats["partition_ms"] == 0
        assert_same(r2.pairs, want, "lazy again")
    finally:
        idx.free()


def test_stats_timings_and_launch_counter():
    strings = synth.generate("medium", 4, n=2000)
    before = pj.pj_kernel_launches()
    idx = pj.pj_build_index(strings, 4)
    r = pj.pj_self_join(idx, 4)
    idx.free()
    assert pj.pj_kernel_launches() - before >= 10
    assert r.stats["verify_ms"] > 0 and r.stats["probe_ms"] > 0 and r.stats["dedupe_ms"] > 0
    assert r.stats["hits"] > 0 and r.stats["candidates"] >= r.stats["hits"]


def test_chunked_probe_multi_launch_and_buffer_growth(monkeypatch):
    """Small probe chunks, small verification launches and a tiny initial
    accepted-match buffer (with and without the room reserved before the
    first launch: launches that overflow it run again into a grown buffer)
    must give the same exact result."""
    strings = synth.generate("short", 3, n=5000)
    want = cpu_self(strings, 3)
    monkeypatch.setenv("PJ_GROUP_BUDGET", "3000")
    monkeypatch.setenv("PJ_LAUNCH_CANDS", "5000")
    monkeypatch.setenv("PJ_ACCEPT_INITIAL", "7")
    r = gpu_self(strings, 3)
    assert_same(r.pairs, want, "chunked")
    monkeypatch.setenv("PJ_ACCEPT_RESERVE", "0")
    assert_same(gpu_self(strings, 3).pairs, want, "chunked, buffer grown on overflow")
    monkeypatch.delenv("PJ_GROUP_BUDGET")
    monkeypatch.delenv("PJ_LAUNCH_CANDS")
    assert_same(gpu_self(strings, 3).pairs, want, "one launch, buffer grown on overflow")
    monkeypatch.delenv("PJ_ACCEPT_RESERVE")
    R, S = _rs_sets(5, 2)
    rb, ro = synth.pack(R)
    sb, so = synth.pack(S)
    assert_same(pj.pj_join(R, S, 2).pairs, oracle.join(rb, ro, sb, so, 2), "chunked join")


@pytest.mark.parametrize("cut", ["0", "60"])
def test_warp_per_pair_verification(monkeypatch, cut):
    """Candidates of probes at least PJ_WARP_MIN_LEN long are verified one
    warp per candidate (shuffle-scan band, ballot early exit): same exact
    result as the thread-per-candidate path, alone (0) and mixed (60)."""
    monkeypatch.setenv("PJ_WARP_MIN_LEN", cut)
    cases = [("short2k", 2, 2000, False), ("short", 4, 3000, False), ("medium", 8, 2500, True),
             ("long", 32, 600, True), ("long", 8, 600, True)]
    for name, tau, n, banded in cases:
        strings = synth.generate(name, tau, n=n)
        assert_same(gpu_self(strings, tau).pairs, cpu_self(strings, tau, banded=banded), f"{name} tau={tau} cut={cut}")


@pytest.mark.parametrize("mode", ["0", "1"])
def test_probe_interleaving_both_ways(monkeypatch, mode):
    """Probe groups taken probe by probe (0) or interleaved across 32-probe
    blocks (1), with and without the warp cut-over inside a block and with
    chunks that end mid-block: same exact result."""
    monkeypatch.setenv("PJ_PROBE_INTERLEAVE", mode)
    cases = [("short", 4, 3001, False, None), ("short2k", 2, 2000, False, "12"), ("medium", 6, 1999, True, "90"),
             ("long", 16, 333, True, "0")]
    for name, tau, n, banded, cut in cases:
        if cut is None:
            monkeypatch.delenv("PJ_WARP_MIN_LEN", raising=False)
        else:
            monkeypatch.setenv("PJ_WARP_MIN_LEN", cut)
        strings = synth.generate(name, tau, n=n)
        want = cpu_self(strings, tau, banded=banded)
        assert_same(gpu_self(strings, tau).pairs, want, f"{name} tau={tau} interleave={mode}")
    monkeypatch.setenv("PJ_GROUP_BUDGET", str(25 * 45))  # 45 probes per chunk at tau = 4
    strings = synth.generate("short", 4, n=2000)
    assert_same(gpu_self(strings, 4).pairs, cpu_self(strings, 4), f"chunked interleave={mode}")
    R, S = _rs_sets(5, 2)
    rb, ro = synth.pack(R)
    sb, so = synth.pack(S)
    assert_same(pj.pj_join(R, S, 2).pairs, oracle.join(rb, ro, sb, so, 2), f"join interleave={mode}")


@pytest.mark.parametrize("mode", ["1", "2"])
def test_distinct_pair_verification(monkeypatch, mode):
    """Mode L: candidate pairs made distinct by a sort and verified once over
    the whole strings (thread per pair 1, warp per pair 2): same exact
    result, for self joins (with chunks and a growing accepted buffer) and
    R x S joins."""
    monkeypatch.setenv("PJ_VERIFY_PAIRS", mode)
    cases = [("short2k", 2, 2000, False), ("short", 4, 3000, False), ("medium", 8, 2500, True),
             ("long", 32, 600, True), ("long", 8, 600, True)]
    for name, tau, n, banded in cases:
        strings = synth.generate(name, tau, n=n)
        r = gpu_self(strings, tau)
        assert_same(r.pairs, cpu_self(strings, tau, banded=banded), f"{name} tau={tau} pairs={mode}")
    monkeypatch.setenv("PJ_GROUP_BUDGET", "3000")
    monkeypatch.setenv("PJ_ACCEPT_INITIAL", "5")
    strings = synth.generate("short", 3, n=3000)
    assert_same(gpu_self(strings, 3).pairs, cpu_self(strings, 3), f"chunked pairs={mode}")
    R, S = _rs_sets(7, 3)
    rb, ro = synth.pack(R)
    sb, so = synth.pack(S)
    assert_same(pj.pj_join(R, S, 3).pairs, oracle.join(rb, ro, sb, so, 3), f"join pairs={mode}")


@pytest.mark.parametrize("queued", ["0", "1"])
def test_direct_and_queued_verification(monkeypatch, queued):
    """Thread-per-candidate verification straight (0) or behind the screen
    and per-warp queues (1): same exact result, with launch chunks that end
    inside a warp's candidates."""
    monkeypatch.setenv("PJ_VERIFY_QUEUE", queued)
    monkeypatch.setenv("PJ_VERIFY_PAIRS", "0")
    for name, tau, n, banded in [("short", 4, 4000, False), ("short2k", 2, 2000, False), ("medium", 4, 3000, True)]:
        strings = synth.generate(name, tau, n=n)
        assert_same(gpu_self(strings, tau).pairs, cpu_self(strings, tau, banded=banded), f"{name} queued={queued}")
    monkeypatch.setenv("PJ_LAUNCH_CANDS", "777")
    strings = synth.generate("short", 3, n=2500)
    r = gpu_self(strings, 3)
    assert_same(r.pairs, cpu_self(strings, 3), f"short launches queued={queued}")
    assert r.stats["filtered"] > 0
    R, S = _rs_sets(9, 2)
    rb, ro = synth.pack(R)
    sb, so = synth.pack(S)
    assert_same(pj.pj_join(R, S, 2).pairs, oracle.join(rb, ro, sb, so, 2), f"join queued={queued}")


def test_autotuned_self_join(monkeypatch, tmp_path):
    """The autotuner picks the cut-over and block size per workload signature
    (cached for the process and in PJ_AUTOTUNE_CACHE); results stay exact."""
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("PJ_AUTOTUNE_CACHE", str(cache))
    for name, tau, n, banded in [("long", 16, 700, True), ("medium", 4, 3000, True)]:
        strings = synth.generate(name, tau, n=n)
        want = cpu_self(strings, tau, banded=banded)
        idx = pj.pj_build_index(strings, tau, autotune=True)
        try:
            r1 = pj.pj_self_join(idx, tau)
            r2 = pj.pj_self_join(idx, tau)
        finally:
            idx.free()
        assert_same(r1.pairs, want, f"autotuned {name}")
        assert_same(r2.pairs, want, f"autotuned again {name}")
        assert r1.stats["verify_block"] in (128, 256, 512)
        assert r2.stats["tune_ms"] == 0.0  # decision cached
        assert (r1.stats["warp_min_len"], r1.stats["verify_block"]) == (r2.stats["warp_min_len"], r2.stats["verify_block"])
    lines = cache.read_text().strip().splitlines()
    assert len(lines) == 2 and all(line.count("|") == 4 for line in lines)


@pytest.mark.parametrize("queued", ["0", "1"])
def test_thread_extension_verification_wide_bands(monkeypatch, queued):
    """Extension verification with one thread per candidate at thresholds
    above 8 (Sec. 5.2, Alg. 3): the sides run the band of 17 (tau <= 16) or
    33 (tau <= 32) diagonals held in one thread's registers.  The library
    sends long strings to whole-pair or warp verification by default, so
    both are switched off here; straight (0) and behind the screen queue (1)."""
    monkeypatch.setenv("PJ_VERIFY_PAIRS", "0")
    monkeypatch.setenv("PJ_WARP_MIN_LEN", "65536")
    monkeypatch.setenv("PJ_VERIFY_QUEUE", queued)
    for name, tau, n in [("medium", 8, 3000), ("long", 16, 800), ("long", 32, 600), ("medium", 12, 2000)]:
        strings = synth.generate(name, tau, n=n)
        r = gpu_self(strings, tau)
        assert r.stats["verify_mode"] == 1, "extension verification expected"
        assert r.stats["warp_min_len"] == 65536, "thread per candidate expected"
        assert r.stats["accepted"] > 0
        assert_same(r.pairs, cpu_self(strings, tau, banded=True), f"{name} tau={tau} thread extension")


@pytest.mark.parametrize("name,tau,n", [("short2k", 2, 2000), ("short", 1, 3000), ("short", 4, 3000),
                                        ("medium", 6, 1500), ("long", 16, 300)])
def test_selection_counts_match_algorithm(name, tau, n):
    """The selection ablation of Sec. 4 (Fig. 12's four methods) counted on
    the device equals the counts of the oracle's own windows over Alg. 1's
    visiting order, and the multi-match-aware count is exactly what the self
    join looks up."""
    strings = synth.generate(name, tau, n=n)
    want = M.selection_counts(strings, tau)
    idx = pj.pj_build_index(strings, tau, lazy_partitions=True)
    try:
        got = pj.pj_count_selection(idx, tau)
        r = pj.pj_self_join(idx, tau)
    finally:
        idx.free()
    assert got == {"length_based": want["length"], "shift_based": want["shift"],
                   "position_aware": want["position"], "multi_match": want["multi"], "groups": want["groups"]}
    assert got["length_based"] > got["shift_based"] >= got["position_aware"] >= got["multi_match"] > 0
    assert r.stats["lookups"] == got["multi_match"]


def _with_short_strings(strings, tau):
    # strings too short to partition (length <= tau) exercise the fallback
    return strings + [b"", b"a", b"ab", b"abc"[:tau], b"zz"]


@pytest.mark.parametrize("name,tau,n,banded", [("short", 3, 5000, False), ("medium", 6, 2000, True),
                                               ("long", 16, 500, True)])
def test_shards_partition_the_self_join(name, tau, n, banded):
    """pj_self_join_shard: the probe ranges of k shards give disjoint pair
    sets whose union is exactly the self join (each pair is found by the
    later of its strings, Alg. 1), for k = 1, 3 and 7."""
    strings = _with_short_strings(synth.generate(name, tau, n=n), tau)
    want = cpu_self(strings, tau, banded=banded)
    idx = pj.pj_build_index(strings, tau)
    try:
        for k in (1, 3, 7):
            parts = [pj.pj_self_join_shard(idx, tau, s, k).pairs for s in range(k)]
            assert all((np.diff(p["a"].astype(np.int64) * (1 << 32) + p["b"]) > 0).all() for p in parts if len(p) > 1)
            got = np.concatenate(parts)
            got = got[np.lexsort((got["b"], got["a"]))]
            assert_same(got, want, f"{name} tau={tau} shards={k}")
    finally:
        idx.free()


def test_stream_self_join_under_a_small_budget():
    """pj_self_join_stream: windows of consecutive probing strings (by length)
    joined one at a time under a device budget far below the whole join's
    needs; the result equals the oracle's and pj_self_join's, the windows are
    several, and the device memory held never passed the budget."""
    tau = 3
    strings = _with_short_strings(synth.generate("short", tau, n=12000), tau)
    budget = 24 << 20
    r = pj.pj_self_join_stream(strings, tau, device_budget=budget)
    assert r.stats["windows"] >= 3
    assert 0 < r.stats["device_peak"] <= budget
    assert_same(r.pairs, cpu_self(strings, tau, banded=True), "stream")
    assert_same(r.pairs, gpu_self(strings, tau).pairs, "stream vs pj_self_join")
    # no budget: one window of the whole set
    r1 = pj.pj_self_join_stream(strings, tau)
    assert r1.stats["windows"] == 1
    assert_same(r1.pairs, r.pairs, "stream, one window")


def test_device_budget_refuses_instead_of_allocating():
    """pj_options.device_budget: an index whose join would need more device
    memory than the budget fails with PJ_ENOMEM (nothing beyond the budget is
    allocated), and a generous budget gives the exact result and reports its
    peak."""
    strings = synth.generate("short", 4, n=20000)
    small = pj.pj_build_index(strings, 4, device_budget=16 << 20, lazy_partitions=True)  # the store fits
    try:
        with pytest.raises(pj.PJError) as e:
            pj.pj_self_join(small, 4)
        assert e.value.code == pj.PJ_ENOMEM and "budget" in str(e.value)
    finally:
        small.free()
    big = pj.pj_build_index(strings, 4, device_budget=2 << 30)
    try:
        r = pj.pj_self_join(big, 4)
    finally:
        big.free()
    assert 0 < r.stats["device_peak"] <= 2 << 30
    assert_same(r.pairs, cpu_self(strings, 4), "budgeted self join")


def _prefix_families(strings, n_fam, size, seed):
    """Families of same-length strings that share long prefixes: a string of
    the set and copies of it with one substitution in their last quarter."""
    rng = np.random.default_rng(seed)
    out = []
    for k in rng.choice(len(strings), size=n_fam, replace=False).tolist():
        base = bytearray(strings[k])
        for _ in range(size):
            s = bytearray(base)
            pos = len(s) - 1 - int(rng.integers(0, max(1, len(s) // 4)))
            s[pos] = ord("a") + int(rng.integers(0, 26))
            out.append(bytes(s))
    return strings + out


@pytest.mark.parametrize("mode", ["1", "2"])
def test_shared_prefix_verification(monkeypatch, mode):
    """Sec. 5.3 on the GPU: distinct pairs verified with the DP rows of
    common prefixes shared between consecutive pairs of a probe (thread per
    run of pairs 1, warp per run 2).  Same exact result as without sharing
    and as the oracle, and fewer DP cells."""
    monkeypatch.setenv("PJ_VERIFY_PAIRS", mode)
    for name, tau, n in [("medium", 8, 2500), ("long", 16, 500), ("short", 4, 3000)]:
        strings = _prefix_families(synth.generate(name, tau, n=n), 40, 6, seed=tau)
        want = cpu_self(strings, tau, banded=True)
        monkeypatch.setenv("PJ_SHARE_PREFIX", "1")
        r1 = gpu_self(strings, tau)
        monkeypatch.setenv("PJ_SHARE_PREFIX", "0")
        r0 = gpu_self(strings, tau)
        assert_same(r1.pairs, want, f"{name} tau={tau} shared")
        assert_same(r0.pairs, want, f"{name} tau={tau} not shared")
        assert r1.stats["verify_mode"] == 2
        assert r1.stats["dp_cells"] < r0.stats["dp_cells"], (name, r1.stats["dp_cells"], r0.stats["dp_cells"])


@pytest.mark.parametrize("name,tau,n,banded", [("short", 4, 4000, False), ("short", 2, 3000, False),
                                               ("medium", 8, 2500, True), ("long", 16, 500, True)])
def test_center_partition(name, tau, n, banded):
    """The centred partition scheme (the longer segments in the middle):
    self joins, R x S joins and queries equal the oracle, and the kernels
    examine exactly the Alg. 1 matches the oracle enumerates with that
    scheme."""
    strings = _with_short_strings(synth.generate(name, tau, n=n), tau)
    want = cpu_self(strings, tau, banded=banded)
    idx = pj.pj_build_index(strings, tau, partition="center")
    try:
        assert_same(pj.pj_self_join(idx, tau).pairs, want, f"{name} tau={tau} center")
        R = synth.generate(name, tau, n=200, seed=99) + strings[:100]
        rb, ro = synth.pack(R)
        sb, so = synth.pack(strings)
        want_rs = oracle.join(rb, ro, sb, so, tau, banded=True)
        assert_same(pj.pj_query(idx, R, tau).pairs, want_rs, f"{name} tau={tau} center query")
    finally:
        idx.free()
    assert_same(pj.pj_join(R, strings, tau, partition="center").pairs, want_rs, f"{name} tau={tau} center join")


def test_center_partition_candidates_match_algorithm():
    """With the centred scheme the kernels examine exactly the (s, r, i, p)
    matches of Alg. 1 under that scheme (store order), and accept exactly
    those extension verification accepts; fewer than under the even
    partition on short strings."""
    strings = synth.generate("short", 4, n=900)
    counts = {}
    for scheme in ("even", "center"):
        st = {}
        M.pass_join_self(strings, 4, order="prefix8", stats=st, scheme=scheme)
        idx = pj.pj_build_index(strings, 4, partition=scheme)
        try:
            r = pj.pj_self_join(idx, 4)
            sel = pj.pj_count_selection(idx, 4)
        finally:
            idx.free()
        assert r.stats["candidates"] == st["tuples"], scheme
        assert r.stats["accepted"] == st["accepted"], scheme
        assert sel["multi_match"] == M.selection_counts(strings, 4, scheme=scheme)["multi"]
        counts[scheme] = st["tuples"]
    assert counts["center"] < counts["even"]


def _copies(strings, n_fam, size, seed):
    """`size` exact copies of `n_fam` strings of the set, appended."""
    rng = np.random.default_rng(seed)
    picks = rng.choice(len(strings), size=n_fam, replace=False).tolist()
    return strings + [strings[k] for k in picks for _ in range(size)]


@pytest.mark.parametrize("mode", ["1", "2"])
def test_fused_self_join(monkeypatch, mode):
    """Mode L by the fused persistent kernel (selection, lookups, distinct
    pairs and verification of a work item in shared memory; thread per pair
    1, warp per pair 2): the same exact result as the oracle, with items
    whose distinct pairs overflow the warp's list and posting runs long
    enough to leave the kernel (copies of a string), with the short probes
    in the chunked pipeline (PJ_FUSED_FROM), and with an accepted-match
    buffer that has to grow."""
    monkeypatch.setenv("PJ_FUSED", mode)
    cases = [("short2k", 2, 2000, False), ("short", 4, 3000, False), ("medium", 8, 2500, True),
             ("long", 32, 600, True), ("long", 8, 600, True)]
    for name, tau, n, banded in cases:
        strings = synth.generate(name, tau, n=n)
        r = gpu_self(strings, tau)
        assert_same(r.pairs, cpu_self(strings, tau, banded=banded), f"{name} tau={tau} fused={mode}")
        assert r.stats["fused"] == 1 and r.stats["verify_mode"] == 2
        assert r.stats["distinct_pairs"] > 0 and r.stats["candidates"] >= r.stats["distinct_pairs"]
    for size in (50, 700):
        strings = _copies(synth.generate("medium", 8, n=1500), 2, size, seed=size)
        r = gpu_self(strings, 8)
        assert_same(r.pairs, cpu_self(strings, 8, banded=True), f"copies {size} fused={mode}")
    # probes shorter than PJ_FUSED_FROM in the chunked mode-L pipeline, the rest fused
    for name, tau, n, banded, cut in [("medium", 8, 2500, True, "80"), ("short", 4, 3000, False, "16"),
                                      ("long", 16, 600, True, "1000")]:
        monkeypatch.setenv("PJ_FUSED_FROM", cut)
        strings = synth.generate(name, tau, n=n)
        assert_same(gpu_self(strings, tau).pairs, cpu_self(strings, tau, banded=banded),
                    f"{name} tau={tau} fused={mode} from {cut}")
    monkeypatch.delenv("PJ_FUSED_FROM")
    monkeypatch.setenv("PJ_ACCEPT_INITIAL", "5")  # the fused launch re-runs into a grown buffer
    strings = synth.generate("short", 3, n=3000)
    assert_same(gpu_self(strings, 3).pairs, cpu_self(strings, 3), f"grown buffer fused={mode}")
