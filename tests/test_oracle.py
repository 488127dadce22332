"""Pins for the CPU oracle (CPU only).

The oracle is checked against things other than itself: values the paper
prints in its worked examples (tests/golden/paper_examples.json), a
breadth-first search over single-character edit operations (the definition
of ED in Sec. 2, independent of the DP recurrence), algebraic properties of a
metric, and brute force on tiny inputs.
"""
import functools
import itertools
import json
import os
import random

import numpy as np
import pytest

import oracle
from oracle import method as M

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")))


# --------------------------------------------------- independent ED checks --

def bfs_distances(src: str, alphabet: str, max_len: int) -> dict:
    """Shortest number of single-character insert/delete/substitute steps from
    src to every string over the alphabet of length <= max_len (Sec. 2's
    definition of ED, evaluated as a graph search)."""
    dist = {src: 0}
    frontier = [src]
    while frontier:
        nxt = []
        for u in frontier:
            d = dist[u]
            cand = set()
            for p in range(len(u) + 1):
                if len(u) < max_len:
                    for c in alphabet:
                        cand.add(u[:p] + c + u[p:])
                if p < len(u):
                    cand.add(u[:p] + u[p + 1:])
                    for c in alphabet:
                        cand.add(u[:p] + c + u[p + 1:])
            for v in cand:
                if v not in dist:
                    dist[v] = d + 1
                    nxt.append(v)
        frontier = nxt
    return dist


def all_strings(alphabet: str, max_len: int):
    for L in range(max_len + 1):
        for t in itertools.product(alphabet, repeat=L):
            yield "".join(t)


@functools.lru_cache(maxsize=None)
def ed_alignments(a: str, b: str) -> int:
    """ED as the minimum cost of an alignment, recursing on the LAST column
    of the alignment (a different decomposition from the oracle's row scan)."""
    if not a:
        return len(b)
    if not b:
        return len(a)
    return min(ed_alignments(a[:-1], b) + 1, ed_alignments(a, b[:-1]) + 1,
               ed_alignments(a[:-1], b[:-1]) + (a[-1] != b[-1]))


@pytest.mark.parametrize("alphabet,max_len", [("ab", 5), ("abc", 4)])
def test_ed_equals_edit_graph_search(alphabet, max_len):
    words = list(all_strings(alphabet, max_len))
    for src in words:
        dist = bfs_distances(src, alphabet, max_len)
        for dst in words:
            assert oracle.ed(src.encode(), dst.encode()) == dist[dst], (src, dst)


def test_ed_paper_values():
    for e in GOLDEN["ed"]:
        assert oracle.ed(e["r"].encode(), e["s"].encode()) == e["ed"], e["cite"]
    for e in GOLDEN["similar"]:
        d = oracle.ed(e["r"].encode(), e["s"].encode())
        assert (d <= e["tau"]) == e["similar"], e["cite"]


def test_ed_metric_properties():
    rng = random.Random(7)
    words = ["".join(rng.choice("abcd") for _ in range(rng.randint(0, 14))) for _ in range(60)]
    for a in words:
        assert oracle.ed(a.encode(), a.encode()) == 0
        for b in words:
            d = oracle.ed(a.encode(), b.encode())
            assert d == oracle.ed(b.encode(), a.encode())
            assert abs(len(a) - len(b)) <= d <= max(len(a), len(b))
            assert d == ed_alignments(a, b)
    for a, b, c in zip(words, words[1:], words[2:]):
        assert oracle.ed(a.encode(), c.encode()) <= oracle.ed(a.encode(), b.encode()) + oracle.ed(b.encode(), c.encode())


def test_banded_equals_capped_full():
    rng = random.Random(11)
    for _ in range(3000):
        a = "".join(rng.choice("abc") for _ in range(rng.randint(0, 25)))
        b = "".join(rng.choice("abc") for _ in range(rng.randint(0, 25)))
        tau = rng.randint(0, 8)
        full = oracle.ed(a.encode(), b.encode())
        assert oracle.ed_banded(a.encode(), b.encode(), tau) == min(tau + 1, full), (a, b, tau)


# ------------------------------------------------------------- join sets --

def brute_pairs(strings, tau):
    out = []
    for x in range(len(strings)):
        for y in range(x + 1, len(strings)):
            d = ed_alignments(strings[x].decode(), strings[y].decode())
            if d <= tau:
                out.append((x, y, d))
    return out


def as_tuples(arr):
    return [(int(r["a"]), int(r["b"]), int(r["ed"])) for r in arr]


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("tau", [0, 1, 2, 3])
def test_self_join_matches_brute_force(seed, tau):
    rng = random.Random(100 * seed + tau)
    base = ["".join(rng.choice("abc") for _ in range(rng.randint(0, 9))) for _ in range(25)]
    strings = [s.encode() for s in base]
    for s in list(strings[:10]):  # near duplicates
        t = bytearray(s)
        if t:
            t[rng.randrange(len(t))] = ord(rng.choice("abc"))
        strings.append(bytes(t))
    strings.append(strings[0])  # exact duplicate -> ed 0
    b, o = oracle.pack(strings)
    for banded in (False, True):
        got = as_tuples(oracle.self_join(b, o, tau, banded=banded))
        assert got == brute_pairs(strings, tau)


def test_join_and_similar_to_match_brute_force():
    rng = random.Random(5)
    R = ["".join(rng.choice("ab") for _ in range(rng.randint(0, 8))).encode() for _ in range(15)]
    S = ["".join(rng.choice("ab") for _ in range(rng.randint(0, 8))).encode() for _ in range(20)]
    tau = 2
    want = [(a, b, ed_alignments(R[a].decode(), S[b].decode())) for a in range(len(R)) for b in range(len(S))
            if ed_alignments(R[a].decode(), S[b].decode()) <= tau]
    rb, ro = oracle.pack(R)
    sb, so = oracle.pack(S)
    assert as_tuples(oracle.join(rb, ro, sb, so, tau)) == want
    assert as_tuples(oracle.join(rb, ro, sb, so, tau, banded=True)) == want
    assert as_tuples(oracle.similar_to(rb, ro, sb, so, tau)) == want
    # self-join through similar_to with the diagonal excluded
    sj = as_tuples(oracle.self_join(sb, so, tau))
    st = as_tuples(oracle.similar_to(sb, so, sb, so, tau, exclude=np.arange(len(S))))
    assert sorted((min(a, b), max(a, b), d) for a, b, d in st if a < b) == sj


def test_table1_answer_set():
    T = [s.encode() for s in GOLDEN["table1"]["strings"]]
    b, o = oracle.pack(T)
    got = as_tuples(oracle.self_join(b, o, 3))
    # Sec. 2: <kaushik chakrab (s4), caushik chakrabar (s2)> is similar at tau = 3;
    # the other pairs the paper discusses are not (Sec. 2, 3.2, 5.1).
    assert (1, 3) in [(a, bb) for a, bb, _ in got]
    assert got == brute_pairs(T, 3)


def test_lemma1_every_result_shares_a_segment():
    """Lemma 1: if ED(r, s) <= tau, s contains a substring equal to one of the
    tau + 1 segments of r (checked on every oracle result pair)."""
    strings = []
    rng = random.Random(3)
    for _ in range(60):
        s = "".join(rng.choice("abcd") for _ in range(rng.randint(3, 14)))
        strings.append(s.encode())
        t = bytearray(s.encode())
        for _ in range(rng.randint(0, 3)):
            t[rng.randrange(len(t))] = ord(rng.choice("abcd"))
        strings.append(bytes(t))
    b, o = oracle.pack(strings)
    for tau in (1, 2, 3):
        for a, bb, _ in as_tuples(oracle.self_join(b, o, tau)):
            for r, s in ((strings[a], strings[bb]), (strings[bb], strings[a])):
                if len(r) >= tau + 1:
                    assert any(seg in s for seg in M.segments(r, tau))


# ------------------------------------------------------- the method steps --

def test_even_partition_paper_example():
    for e in GOLDEN["partition"]:
        assert [x.decode() for x in M.segments(e["s"].encode(), e["tau"])] == e["segments"], e["cite"]
        L, t = len(e["s"]), e["tau"]
        assert L - (L // (t + 1)) * (t + 1) == e["k"]


def test_even_partition_shape():
    for L in range(1, 80):
        for tau in range(0, L):
            segs = M.even_partition(L, tau)
            lens = [n for _, n in segs]
            assert len(segs) == tau + 1 and sum(lens) == L
            assert max(lens) - min(lens) <= 1 and lens == sorted(lens)  # longer ones last
            assert all(segs[k][0] + segs[k][1] == segs[k + 1][0] for k in range(tau))


def test_selection_paper_example():
    g = GOLDEN["selection"]
    s, l, tau = g["s"].encode(), g["l"], g["tau"]
    pos = [[w.decode() for w in ws] for ws in M.selected_substrings(s, l, tau, "position")]
    mul = [[w.decode() for w in ws] for ws in M.selected_substrings(s, l, tau, "multi")]
    assert pos == g["position"] and sum(map(len, pos)) == g["position_count"]
    assert mul == g["multi"] and sum(map(len, mul)) == g["multi_count"]
    sh = M.select_windows(len(s), l, tau, "shift", clip=False)
    assert sum(hi - lo + 1 for _, lo, hi, _ in sh) == g["shift_unclipped_count"]
    # left-side-only windows printed in Sec. 4.2 (1-based, not yet clipped by the right side)
    segs = M.even_partition(l, tau)
    left = [[P - (i - 1) + 1, P + (i - 1) + 1] for i, (P, _) in enumerate(segs, start=1)]
    assert left == g["multi_left_windows_1based"]
    D = len(s) - l
    right = [[P + D - (tau + 1 - i) + 1, P + D + (tau + 1 - i) + 1] for i, (P, _) in enumerate(segs, start=1)]
    assert right[2:] == g["multi_right_windows_1based_seg3_seg4"]


def test_selection_count_formulas():
    for tau in range(0, 9):
        for l in range(tau + 1, 70):
            for D in range(0, tau + 1):
                ls = l + D
                w = lambda m, clip=True: sum(max(0, hi - lo + 1) for _, lo, hi, _ in M.select_windows(ls, l, tau, m, clip))
                assert w("length") == (tau + 1) * (ls + 1) - l            # Sec. 4
                assert w("shift", False) == (tau + 1) * (2 * tau + 1)      # Sec. 4
                # Sec. 4.1 states (tau+1)^2; the two floors give exactly that when
                # tau - D is even and one position fewer per segment otherwise.
                per_seg = (tau - D) // 2 + (tau + D) // 2 + 1
                assert w("position", False) == (tau + 1) * per_seg <= (tau + 1) ** 2
                if (tau - D) % 2 == 0:
                    assert w("position", False) == (tau + 1) ** 2
                assert w("multi") == M.lemma2_count(tau, D)                 # Lemma 2
                assert w("multi", False) == M.lemma2_count(tau, D)          # never clipped for D >= 0


def test_selection_counts_two_strings_of_length_15():
    """Sec. 6.1's worked count for |s| = l = 15, tau = 1: the length-based
    method selects (tau+1)(|s|+1) - l = 17 substrings and the multi-match
    method floor((tau^2 - D^2)/2) + tau + 1 = 2.  The shift-based window
    [P_i - 1, P_i + 1] holds 2 tau + 1 = 3 positions per segment (6 in the
    paper's count), of which 2 per segment exist in s (p >= 0 and p <= |s| -
    l_i: segment 1 starts at 0, segment 2 ends at |s|); the position-aware
    window of Sec. 4.1 has floor((tau - D)/2) + floor((tau + D)/2) + 1 = 1
    position per segment at D = 0 (the paper's (tau+1)^2 = 4 holds for even
    tau - D).  Only the second string probes (the first has nothing visited
    before it)."""
    a, b = b"abcdefghijklmno", b"bcdefghijklmnop"
    got = M.selection_counts([a, b], 1)
    assert got == {"length": 17, "shift": 4, "position": 2, "multi": 2, "groups": 2}
    # a length not visited before the probe selects nothing
    assert M.selection_counts([a, b"xyz"], 1)["groups"] == 0


def test_lemma3_subset_chain():
    for tau in range(0, 7):
        for l in range(tau + 1, 40):
            for D in range(0, tau + 1):
                ls = l + D
                sets = {}
                for m in ("length", "shift", "position", "multi"):
                    sets[m] = {(i, p) for i, lo, hi, _ in M.select_windows(ls, l, tau, m) for p in range(lo, hi + 1)}
                assert sets["multi"] <= sets["position"] <= sets["shift"] <= sets["length"]


def _tiny_pairs(alphabet, max_len, min_len):
    words = [w.encode() for w in all_strings(alphabet, max_len) if len(w) >= min_len]
    return words


@pytest.mark.parametrize("tau", [1, 2, 3])
def test_multi_match_completeness_exhaustive(tau):
    """Theorem 2 (and the signed-length reading for R != S): for every pair
    with ED <= tau and an indexed string r of length >= tau + 1, some segment
    i of r equals s[p : p + l_i] for a p in the multi-match window -- for the
    even partition (Sec. 3.1) and for the centred scheme, whose segments also
    depend on the length alone."""
    words = _tiny_pairs("ab", 7, 0)
    for scheme in ("even", "center"):
        _completeness(words, tau, scheme)


def _completeness(words, tau, scheme):
    for r in words:
        if len(r) < tau + 1:
            continue
        segs = M.partition(len(r), tau, scheme)
        for s in words:
            if abs(len(s) - len(r)) > tau or ed_alignments(r.decode(), s.decode()) > tau:
                continue
            wins = M.select_windows(len(s), len(r), tau, "multi", scheme=scheme)
            assert any(s[p:p + li] == r[P:P + li]
                       for (i, lo, hi, li), (P, _) in zip(wins, segs) for p in range(lo, hi + 1)), (r, s)


def test_verification_paper_examples():
    for e in GOLDEN["verification"]:
        fn = M.verify_string_pair if e["method"] == "length_aware" else M.verify_naive
        d, rows = fn(e["s"].encode(), e["r"].encode(), e["tau"], return_rows=True)
        assert (d, rows) == (e["result"], e["stop_row"]), e["cite"]


def test_verify_string_pair_is_capped_ed():
    """Length-aware band + Lemma 4 return exactly min(tau' + 1, ED)."""
    words = _tiny_pairs("abc", 4, 0)
    for a in words:
        for b in words:
            d = ed_alignments(a.decode(), b.decode())
            for t in range(0, 5):
                assert M.verify_string_pair(a, b, t) == min(t + 1, d), (a, b, t)
                assert M.verify_naive(a, b, t) == min(t + 1, d)
    rng = random.Random(9)
    for _ in range(1500):
        a = "".join(rng.choice("abc") for _ in range(rng.randint(0, 22))).encode()
        b = "".join(rng.choice("abc") for _ in range(rng.randint(0, 22))).encode()
        t = rng.randint(0, 7)
        assert M.verify_string_pair(a, b, t) == min(t + 1, ed_alignments(a.decode(), b.decode()))


def test_extension_paper_example():
    for e in GOLDEN["extension"]:
        r, s = e["r"].encode(), e["s"].encode()
        segs = M.segments(r, e["tau"])
        assert segs[e["i"] - 1].decode() == e["segment"]
        assert s[e["p"]:e["p"] + len(e["segment"])].decode() == e["segment"]
        ok, _ = M.extension_verify(r, s, e["i"], e["p"], e["tau"])
        assert ok == e["accepted"], e["cite"]


def test_extension_min_over_matches_is_ed():
    """Theorem 5 plus the exact-ed reading: over the multi-match tuples of a
    pair, some tuple is accepted iff ED <= tau, and the least accepted
    d_l + d_r equals ED.  Checked for D >= 0 and D < 0 (R != S probing)."""
    rng = random.Random(21)
    for trial in range(4000):
        tau = rng.randint(1, 4)
        r = "".join(rng.choice("abc") for _ in range(rng.randint(tau + 1, 16))).encode()
        s = bytearray(r)
        for _ in range(rng.randint(0, tau + 1)):
            k = rng.randint(0, 2)
            if k == 0:
                s.insert(rng.randint(0, len(s)), ord(rng.choice("abc")))
            elif k == 1 and s:
                del s[rng.randrange(len(s))]
            elif s:
                s[rng.randrange(len(s))] = ord(rng.choice("abc"))
        s = bytes(s)
        d = ed_alignments(r.decode(), s.decode())
        best = None
        for i, lo, hi, li in M.select_windows(len(s), len(r), tau, "multi"):
            for p in range(lo, hi + 1):
                ok, dd = M.extension_verify(r, s, i, p, tau)
                if ok:
                    assert dd >= d
                    best = dd if best is None else min(best, dd)
        if d <= tau:
            assert best == d, (r, s, tau)
        else:
            assert best is None


@pytest.mark.parametrize("order,scheme", [("alphabetical", "even"), ("id", "even"), ("prefix8", "center")])
@pytest.mark.parametrize("tau", [0, 1, 2, 3])
def test_pass_join_equals_definition(order, scheme, tau):
    """Theorem 6: Alg. 1 with multi-match selection and extension verification
    returns exactly the pairs of Def. 1, with exact ED (short and empty
    strings included)."""
    rng = random.Random(31 + tau)
    strings = [b"", b"", b"a", b"ab"]
    for _ in range(45):
        s = "".join(rng.choice("abc") for _ in range(rng.randint(1, 11))).encode()
        strings.append(s)
        t = bytearray(s)
        for _ in range(rng.randint(0, tau + 1)):
            if t and rng.random() < 0.5:
                t[rng.randrange(len(t))] = ord(rng.choice("abc"))
            else:
                t.insert(rng.randint(0, len(t)), ord(rng.choice("abc")))
        strings.append(bytes(t))
    got = M.pass_join_self(strings, tau, order=order, scheme=scheme)
    want = {(a, b): d for a, b, d in brute_pairs(strings, tau)}
    assert got == want


def test_center_partition_shape():
    """The centred scheme keeps the even partition's segment lengths (floor
    or ceil of |s| / (tau + 1), Sec. 3.1) and puts the longer ones in one
    run around the middle; with |s| a multiple of tau + 1 both schemes are
    the same."""
    assert M.center_partition(13, 3) == [(0, 3), (3, 4), (7, 3), (10, 3)]   # k = 1, even parts: the left middle
    assert M.center_partition(14, 3) == [(0, 3), (3, 4), (7, 4), (11, 3)]   # k = 2: both middles
    assert M.center_partition(16, 4) == [(0, 3), (3, 3), (6, 4), (10, 3), (13, 3)]  # k = 1, odd parts: the middle
    assert M.center_partition(18, 4) == [(0, 3), (3, 4), (7, 4), (11, 4), (15, 3)]  # k = 3
    assert M.center_partition(19, 4) == [(0, 4), (4, 4), (8, 4), (12, 4), (16, 3)]  # k = 4: ties to the left
    for L in range(1, 90):
        for tau in range(0, min(L, 33)):
            even, cen = M.even_partition(L, tau), M.center_partition(L, tau)
            assert sorted(n for _, n in even) == sorted(n for _, n in cen)
            assert all(cen[k][0] + cen[k][1] == cen[k + 1][0] for k in range(tau))
            longer = [i for i, (_, n) in enumerate(cen) if n > L // (tau + 1)]
            assert longer == list(range(longer[0], longer[0] + len(longer))) if longer else True
            if longer:  # centred: equally many on each side, one more on the left at most
                left, right = longer[0], tau - longer[-1]
                assert 0 <= right - left <= 1 or 0 <= left - right <= 1
            if L % (tau + 1) == 0:
                assert even == cen


def test_pass_join_table1():
    T = [s.encode() for s in GOLDEN["table1"]["strings"]]
    assert M.pass_join_self(T, 3) == {(1, 3): 3}


@pytest.mark.parametrize("tau", [1, 2, 3])
def test_pass_join_rs_equals_definition(tau):
    rng = random.Random(77 + tau)
    S = [b"", b"a"] + ["".join(rng.choice("ab") for _ in range(rng.randint(1, 10))).encode() for _ in range(40)]
    R = [b"", b"b"]
    for s in S[:30]:
        t = bytearray(s)
        for _ in range(rng.randint(0, tau)):
            k = rng.randint(0, 2)
            if k == 0:
                t.insert(rng.randint(0, len(t)), ord(rng.choice("ab")))
            elif k == 1 and t:
                del t[rng.randrange(len(t))]
            elif t:
                t[rng.randrange(len(t))] = ord(rng.choice("ab"))
        R.append(bytes(t))
    got = M.pass_join_rs(R, S, tau)
    want = {}
    for a in range(len(R)):
        for b in range(len(S)):
            d = ed_alignments(R[a].decode(), S[b].decode())
            if d <= tau:
                want[(a, b)] = d
    assert got == want
