"""Pass-Join's own steps, written out plainly for small inputs.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): nothing in the CUDA
path imports this module.

Every function follows one passage of the paper, in the paper's order and
notation.  Positions are 0-based here: the paper's start position p (1-based)
is ``p - 1`` in this module, and its segment start p_i is ``P[i-1]``.

* ``even_partition``       -- Sec. 3.1 (even-partition scheme);
  ``center_partition``     -- a second scheme (Sec. 3.1 leaves other schemes
                              to future work): the same lengths, the longer
                              segments in the middle.
* ``select_windows``       -- Sec. 4 (length- and shift-based), Sec. 4.1
                              (position-aware, W_p), Sec. 4.2 (multi-match-aware,
                              W_m) and Alg. 2.
* ``verify_string_pair``   -- Sec. 5.1 (length-aware band, expected edit
                              distance E(i, j), Lemma 4) = VERIFYSTRINGPAIR of
                              Alg. 3; ``verify_naive`` is the 2*tau+1 band with
                              prefix pruning that Sec. 5.1 and Sec. 6.2 compare
                              against.
* ``extension_verify``     -- Sec. 5.2 and Alg. 3 (tau_l = i - 1,
                              tau_r = tau + 1 - i).
* ``pass_join_self`` / ``pass_join_rs`` -- Alg. 1 and the R != S variant of
                              Sec. 3.2.

Readings taken where the paper is silent:
strings shorter than tau + 1 have no even partition (footnote to Sec. 3.1), so
pairs whose indexed string is that short are verified directly; the exact
``ed`` of a reported pair is the minimum d_l + d_r over the accepted
(segment, position) matches of that pair; for R != S the windows of Sec. 4.2
are used with a signed length difference.
"""
from __future__ import annotations

from collections import defaultdict

INF = float("inf")


# ------------------------------------------------------------ Sec. 3.1 ----

def even_partition(length: int, tau: int) -> list[tuple[int, int]]:
    """Even partition of a string of the given length into tau + 1 segments.

    Each segment has floor(|s|/(tau+1)) or ceil(|s|/(tau+1)) characters; with
    k = |s| - floor(|s|/(tau+1)) * (tau+1), the LAST k segments are the longer
    ones.  Returns [(start, length)] for i = 1..tau+1 (0-based starts).
    Requires |s| >= tau + 1 (footnote to Sec. 3.1).
    """
    if length < tau + 1:
        raise ValueError("even partition needs |s| >= tau + 1")
    base = length // (tau + 1)
    k = length - base * (tau + 1)
    segs = []
    start = 0
    for i in range(1, tau + 2):
        li = base + 1 if i > tau + 1 - k else base
        segs.append((start, li))
        start += li
    assert start == length
    return segs


def center_partition(length: int, tau: int) -> list[tuple[int, int]]:
    """A second partition scheme (the paper leaves other schemes to future
    work, Sec. 3.1, and notes that its techniques extend to them): the same
    segment lengths as the even partition -- floor(|s|/(tau+1)), and k of
    them one longer -- but the k longer segments are the k closest to the
    middle (segments ordered by |2i - (tau + 2)|, ties to the left), where
    the multi-match windows of Sec. 4.2 are widest, so that the more
    selective segments are looked up at the most positions.  Returns
    [(start, length)] for i = 1..tau+1 (0-based starts)."""
    if length < tau + 1:
        raise ValueError("a partition needs |s| >= tau + 1")
    m = tau + 1
    base = length // m
    k = length - base * m
    by_centrality = sorted(range(1, m + 1), key=lambda i: (abs(2 * i - (m + 1)), i))
    longer = set(by_centrality[:k])
    segs, start = [], 0
    for i in range(1, m + 1):
        li = base + 1 if i in longer else base
        segs.append((start, li))
        start += li
    assert start == length
    return segs


PARTITIONS = {"even": even_partition, "center": center_partition}


def partition(length: int, tau: int, scheme: str = "even") -> list[tuple[int, int]]:
    """The segments of a length-|s| string under a partition scheme."""
    return PARTITIONS[scheme](length, tau)


def segments(s: bytes, tau: int, scheme: str = "even") -> list[bytes]:
    return [s[p:p + n] for p, n in partition(len(s), tau, scheme)]


# ---------------------------------------------------------- Sec. 4 / 4.x ---

def select_windows(s_len: int, l: int, tau: int, method: str = "multi",
                   clip: bool = True, scheme: str = "even") -> list[tuple[int, int, int, int]]:
    """Start-position windows of the selected substrings of s for L_l^i.

    Returns [(i, lo, hi, l_i)] for i = 1..tau+1; positions p in [lo, hi]
    (0-based, inclusive) give the substrings s[p : p + l_i].  ``clip`` keeps
    only positions where the substring exists (0 <= p <= |s| - l_i); the
    paper's closed-form counts for the shift- and position-aware rules are the
    unclipped window sizes.

    method:
      "length"   -- every substring of length l_i            (Sec. 4)
      "shift"    -- p in [p_i - tau, p_i + tau]               (Sec. 4)
      "position" -- p in [p_i - floor((tau - D)/2),
                          p_i + floor((tau + D)/2)]            (Sec. 4.1)
      "multi"    -- p in [max(bot_l, bot_r), min(top_l, top_r)] with
                    bot_l/top_l = p_i -/+ (i - 1) and
                    bot_r/top_r = p_i + D -/+ (tau + 1 - i)   (Sec. 4.2)
    where D = |s| - l (may be negative for R != S joins).
    """
    D = s_len - l
    out = []
    for i, (P, li) in enumerate(partition(l, tau, scheme), start=1):
        last = s_len - li  # last start position at which s[p:p+l_i] exists
        if method == "length":
            lo, hi = 0, last
        elif method == "shift":
            lo, hi = P - tau, P + tau
        elif method == "position":
            lo, hi = P - (tau - D) // 2, P + (tau + D) // 2
        elif method == "multi":
            lo = max(P - (i - 1), P + D - (tau + 1 - i))
            hi = min(P + (i - 1), P + D + (tau + 1 - i))
        else:
            raise ValueError(method)
        if clip:
            lo, hi = max(lo, 0), min(hi, last)
        out.append((i, lo, hi, li))
    return out


def selected_substrings(s: bytes, l: int, tau: int, method: str = "multi"):
    """W(s, L_l^i) for every i (Alg. 2): list over i of the substrings s[p, l_i]."""
    res = []
    for i, lo, hi, li in select_windows(len(s), l, tau, method, clip=True):
        res.append([s[p:p + li] for p in range(lo, hi + 1)])
    return res


def lemma2_count(tau: int, delta: int) -> int:
    """|W_m(s, l)| = floor((tau^2 - D^2)/2) + tau + 1 (Lemma 2)."""
    return (tau * tau - delta * delta) // 2 + tau + 1


# -------------------------------------------------------------- Sec. 5.1 ---

def verify_string_pair(s: bytes, r: bytes, tau: int, return_rows: bool = False):
    """VERIFYSTRINGPAIR(s, r, tau') of Alg. 3: min(tau' + 1, ED(s, r)).

    Length-aware verification (Sec. 5.1): with |s| >= |r| (swap otherwise) and
    D = |s| - |r| <= tau, row i of M only holds the cells
    j in [i - floor((tau - D)/2), i + floor((tau + D)/2)]; cells outside are
    treated as larger than tau.  After each row the expected edit distances
    E(i, j) = M(i, j) + |(|s| - j) - (|r| - i)| are checked: if all exceed tau
    the pair is dissimilar (Lemma 4) and tau + 1 is returned.

    With return_rows, also returns the last row computed (the row after which
    the scan stopped, or |r| when it ran to the end).
    """
    if len(s) < len(r):
        s, r = r, s
    D = len(s) - len(r)
    if D > tau:
        return (tau + 1, 0) if return_rows else tau + 1
    lo_off = (tau - D) // 2
    hi_off = (tau + D) // 2
    ns, nr = len(s), len(r)

    def band(i):
        return max(0, i - lo_off), min(ns, i + hi_off)

    prev = {}
    a, b = band(0)
    for j in range(a, b + 1):
        prev[j] = j  # M(0, j) = j
    rows = 0
    for i in range(1, nr + 1):
        cur = {}
        a, b = band(i)
        for j in range(a, b + 1):
            if j == 0:
                cur[j] = i  # M(i, 0) = i
                continue
            delta = 0 if r[i - 1] == s[j - 1] else 1
            cur[j] = min(prev.get(j, INF) + 1, cur.get(j - 1, INF) + 1,
                         prev.get(j - 1, INF) + delta)
        rows = i
        expected = [cur[j] + abs((ns - j) - (nr - i)) for j in cur]
        if all(e > tau for e in expected):
            return (tau + 1, rows) if return_rows else tau + 1
        prev = cur
    d = prev.get(ns, INF)
    d = tau + 1 if d > tau else int(d)
    return (d, rows) if return_rows else d


def verify_naive(s: bytes, r: bytes, tau: int, return_rows: bool = False):
    """The baseline verification of Sec. 5.1 / Sec. 6.2 ("2tau+1"): cells with
    |i - j| <= tau, stop when every value of a row exceeds tau (prefix
    pruning).  Returns min(tau + 1, ED)."""
    if abs(len(s) - len(r)) > tau:
        return (tau + 1, 0) if return_rows else tau + 1
    ns, nr = len(s), len(r)
    prev = {j: j for j in range(0, min(ns, tau) + 1)}
    rows = 0
    for i in range(1, nr + 1):
        cur = {}
        for j in range(max(0, i - tau), min(ns, i + tau) + 1):
            if j == 0:
                cur[j] = i
                continue
            delta = 0 if r[i - 1] == s[j - 1] else 1
            cur[j] = min(prev.get(j, INF) + 1, cur.get(j - 1, INF) + 1,
                         prev.get(j - 1, INF) + delta)
        rows = i
        if all(v > tau for v in cur.values()):
            return (tau + 1, rows) if return_rows else tau + 1
        prev = cur
    d = prev.get(ns, INF)
    d = tau + 1 if d > tau else int(d)
    return (d, rows) if return_rows else d


# -------------------------------------------------------------- Sec. 5.2 ---

def extension_verify(r: bytes, s: bytes, i: int, p: int, tau: int, scheme: str = "even"):
    """Extension-based verification of one match (Sec. 5.2, Alg. 3).

    r is the indexed string (its i-th even segment w = r[P_i : P_i + l_i]);
    s contains w at position p.  Split both around w, then
      d_l = VERIFYSTRINGPAIR(s_l, r_l, tau_l = i - 1);
      if d_l <= tau_l: d_r = VERIFYSTRINGPAIR(s_r, r_r, tau_r = tau + 1 - i);
      accept iff d_r <= tau_r.
    Returns (accepted, d_l + d_r).  A segment that does not equal s[p : p+l_i]
    is not a match and is rejected.
    """
    P, li = partition(len(r), tau, scheme)[i - 1]
    if s[p:p + li] != r[P:P + li] or p < 0:
        return False, None
    tau_l, tau_r = i - 1, tau + 1 - i
    d_l = verify_string_pair(s[:p], r[:P], tau_l)
    if d_l > tau_l:
        return False, None
    d_r = verify_string_pair(s[p + li:], r[P + li:], tau_r)
    if d_r > tau_r:
        return False, None
    return True, d_l + d_r


# ------------------------------------------------------------- Alg. 1 -----

def _direct_ed(a: bytes, b: bytes) -> int:
    """Plain Wagner-Fischer (Sec. 5.1 recurrence), used by the fallback for
    strings too short to partition."""
    prev = list(range(len(b) + 1))
    for i in range(1, len(a) + 1):
        cur = [i] + [0] * len(b)
        for j in range(1, len(b) + 1):
            cur[j] = min(prev[j] + 1, cur[j - 1] + 1,
                         prev[j - 1] + (0 if a[i - 1] == b[j - 1] else 1))
        prev = cur
    return prev[len(b)]


def pass_join_self(strings: list[bytes], tau: int, order: str = "alphabetical",
                   method: str = "multi", stats: dict | None = None, scheme: str = "even"):
    """Alg. 1 PASS-JOIN(S, tau) with multi-match selection and extension
    verification.  Returns {(a, b): ed} over input ids with a < b.

    order: "alphabetical" visits by (length, string), the order Alg. 1 sorts into;
    "id" visits by (length, input id); "prefix8" by (length, first eight
    bytes, input id).  The result set is the same; the visiting order only
    decides which string of a pair probes the other.
    stats (optional dict) receives "tuples" (candidate (s, r, i, p) matches
    after the visited-before rule), "lookups" and "accepted".
    """
    n = len(strings)
    if order == "alphabetical":
        visit = sorted(range(n), key=lambda k: (len(strings[k]), strings[k], k))
    elif order == "prefix8":
        visit = sorted(range(n), key=lambda k: (len(strings[k]), strings[k][:8], k))
    else:
        visit = sorted(range(n), key=lambda k: (len(strings[k]), k))
    index = defaultdict(lambda: defaultdict(list))  # (l, i) -> segment -> ids
    best: dict[tuple[int, int], int] = {}
    tuples = lookups = accepted = 0
    visited: list[int] = []
    for sid in visit:
        s = strings[sid]
        ls = len(s)
        # Alg. 1, probing step: L_l^i for |s| - tau <= l <= |s|
        for l in range(max(tau + 1, ls - tau), ls + 1):
            for i, lo, hi, li in select_windows(ls, l, tau, method, clip=True, scheme=scheme):
                lists = index.get((l, i))
                for p in range(lo, hi + 1):
                    lookups += 1
                    if lists is None:
                        continue
                    for rid in lists.get(s[p:p + li], ()):
                        tuples += 1
                        ok, d = extension_verify(strings[rid], s, i, p, tau, scheme)
                        if ok:
                            accepted += 1
                            key = (min(rid, sid), max(rid, sid))
                            best[key] = min(best.get(key, d), d)
        # strings too short to partition: verify directly against visited ones
        for rid in visited:
            r = strings[rid]
            if len(r) <= tau and ls - len(r) <= tau:
                d = _direct_ed(r, s)
                if d <= tau:
                    key = (min(rid, sid), max(rid, sid))
                    best[key] = d
        visited.append(sid)
        # Alg. 1, indexing step: insert s's segments into L_{|s|}^i
        if ls >= tau + 1:
            for i, seg in enumerate(segments(s, tau, scheme), start=1):
                index[(ls, i)][seg].append(sid)
    if stats is not None:
        stats.update(tuples=tuples, lookups=lookups, accepted=accepted)
    return best


def selection_counts(strings: list[bytes], tau: int, scheme: str = "even") -> dict:
    """Substrings each selection method of Sec. 4 selects over Alg. 1's self
    join (visiting by length; the order within a length does not change the
    counts, since only the first string of a length has no string of its own
    length before it): for every probing string s,
    every l in [max(tau + 1, |s| - tau), |s|] whose inverted lists are
    non-empty when s probes them (some string of length l visited before s),
    and every segment i, the number of existing substrings s[p, l_i] in the
    method's window (``select_windows`` with clipping).  Returns the totals per
    method ("length", "shift", "position", "multi") and "groups", the number
    of (s, l, i) combinations counted."""
    visit = sorted(range(len(strings)), key=lambda k: (len(strings[k]), k))
    counts = {"length": 0, "shift": 0, "position": 0, "multi": 0, "groups": 0}
    indexed_lengths: set[int] = set()
    for sid in visit:
        ls = len(strings[sid])
        for l in range(max(tau + 1, ls - tau), ls + 1):
            if l not in indexed_lengths:
                continue
            counts["groups"] += tau + 1
            for m in ("length", "shift", "position", "multi"):
                counts[m] += sum(max(0, hi - lo + 1)
                                 for _, lo, hi, _ in select_windows(ls, l, tau, m, clip=True, scheme=scheme))
        if ls >= tau + 1:
            indexed_lengths.add(ls)
    return counts


def pass_join_rs(R: list[bytes], S: list[bytes], tau: int, stats: dict | None = None, scheme: str = "even"):
    """R != S join (Sec. 3.2): index S, probe each r in R against the lengths
    [|r| - tau, |r| + tau] with the Sec. 4.2 windows at signed D = |r| - l.
    Returns {(a in R, b in S): ed}."""
    index = defaultdict(lambda: defaultdict(list))
    short = []
    for sid, s in enumerate(S):
        if len(s) >= tau + 1:
            for i, seg in enumerate(segments(s, tau, scheme), start=1):
                index[(len(s), i)][seg].append(sid)
        else:
            short.append(sid)
    best: dict[tuple[int, int], int] = {}
    tuples = 0
    for qid, q in enumerate(R):
        lq = len(q)
        for l in range(max(tau + 1, lq - tau), lq + tau + 1):
            for i, lo, hi, li in select_windows(lq, l, tau, "multi", clip=True, scheme=scheme):
                lists = index.get((l, i))
                if lists is None:
                    continue
                for p in range(lo, hi + 1):
                    for sid in lists.get(q[p:p + li], ()):
                        tuples += 1
                        ok, d = extension_verify(S[sid], q, i, p, tau, scheme)
                        if ok:
                            key = (qid, sid)
                            best[key] = min(best.get(key, d), d)
        for sid in short:
            if abs(len(S[sid]) - lq) <= tau:
                d = _direct_ed(q, S[sid])
                if d <= tau:
                    best[(qid, sid)] = d
    if stats is not None:
        stats.update(tuples=tuples)
    return best
