"""Seeded synthetic string sets shaped like the paper's workloads.

This module only draws random strings; it holds none of the join's arithmetic,
so both the CUDA path's tests/benchmark and the CPU oracle can be fed from it.

Workloads (the paper's DBLP Author, Query Log and Author+Title sets of Table 2
are not available; these stand in for them):

* ``short2k``  -- 2,000 strings, 'a'-'z' uniform, lengths uniform 8..20, 20% of
  the strings derived from a uniformly chosen fresh string by 1..3 random
  edits.  tau = 2.  Seed 0.
* ``short``    -- 1,000,000 strings over 27 symbols ('a'-'z' then space) with
  Zipf(1.1) character frequencies in listed order, lengths round(N(15, 4))
  clipped to [5, 40]; 30% of the strings sit in clusters of 2..8 (a fresh base
  plus members made by 1..tau random edits each).  Stands in for Author
  (average length 14.8).
* ``medium``   -- 500,000 strings over 40 symbols ('a'-'z', '0'-'9', space,
  '.', ',', '-') with Zipf(1.0) frequencies, lengths round(N(100, 30))
  clipped to [20, 300]; 25% in clusters of 2..5.  Stands in for Author+Title
  (average length 105.8).
* ``long``     -- 100,000 strings, the same 40-symbol Zipf(1.0) alphabet,
  lengths round(N(1000, 200)) clipped to [400, 2000]; 20% of the strings form
  near-duplicate pairs.

Edits are insert / delete / substitute with equal probability at a uniform
position; an edit that would take a length outside the workload's clip range
becomes a substitution.  Inserted and substituted characters follow the
workload's character distribution.  The final order of the strings is a
random permutation, so cluster members do not sit next to each other.

The seed of a (workload, tau) dataset is 1000 * workload_index + tau, except
``short2k`` which uses seed 0.
"""
from __future__ import annotations

import numpy as np

ALPHA27 = b"abcdefghijklmnopqrstuvwxyz "
ALPHA40 = b"abcdefghijklmnopqrstuvwxyz0123456789 .,-"

WORKLOADS = {
    "short2k": dict(index=0, n=2000, alphabet=b"abcdefghijklmnopqrstuvwxyz", zipf=None,
                    length=("uniform", 8, 20), clip=(1, 64), derived_frac=0.2, edits=(1, 3),
                    taus=(2,)),
    "short": dict(index=1, n=1_000_000, alphabet=ALPHA27, zipf=1.1, length=("normal", 15, 4),
                  clip=(5, 40), cluster_frac=0.30, cluster_size=(2, 8), taus=(1, 2, 3, 4)),
    "medium": dict(index=2, n=500_000, alphabet=ALPHA40, zipf=1.0, length=("normal", 100, 30),
                   clip=(20, 300), cluster_frac=0.25, cluster_size=(2, 5), taus=(2, 4, 6, 8)),
    "long": dict(index=3, n=100_000, alphabet=ALPHA40, zipf=1.0, length=("normal", 1000, 200),
                 clip=(400, 2000), cluster_frac=0.20, cluster_size=(2, 2), taus=(8, 16, 32)),
}


def char_probs(spec) -> np.ndarray:
    k = len(spec["alphabet"])
    if spec.get("zipf") is None:
        return np.full(k, 1.0 / k)
    w = np.arange(1, k + 1, dtype=np.float64) ** (-float(spec["zipf"]))
    return w / w.sum()


def seed_for(name: str, tau: int) -> int:
    spec = WORKLOADS[name]
    return 0 if spec["index"] == 0 else 1000 * spec["index"] + int(tau)


def _lengths(spec, rng, n) -> np.ndarray:
    kind = spec["length"][0]
    lo, hi = spec["clip"]
    if kind == "uniform":
        return rng.integers(spec["length"][1], spec["length"][2] + 1, size=n)
    mu, sd = spec["length"][1], spec["length"][2]
    return np.clip(np.rint(rng.normal(mu, sd, size=n)), lo, hi).astype(np.int64)


def _draw_codes(spec, rng, count: int) -> np.ndarray:
    """count i.i.d. symbol codes from the workload's distribution (uint8).

    Inverse-CDF sampling through a 2^16-entry table: a uniform 16-bit draw u
    maps to the first symbol whose cumulative probability exceeds u / 2^16
    (probabilities are thereby quantised to 1/65536)."""
    cdf = np.cumsum(char_probs(spec))
    grid = (np.arange(1 << 16, dtype=np.float64) + 0.5) / float(1 << 16)
    table = np.minimum(np.searchsorted(cdf, grid, side="right"), len(cdf) - 1).astype(np.uint8)
    out = np.empty(count, dtype=np.uint8)
    chunk = 1 << 22
    for a in range(0, count, chunk):
        b = min(count, a + chunk)
        np.take(table, np.frombuffer(rng.bytes(2 * (b - a)), dtype=np.uint16), out=out[a:b])
    return out


def _fresh(spec, rng, n) -> list[bytes]:
    lens = _lengths(spec, rng, n)
    alpha = np.frombuffer(spec["alphabet"], dtype=np.uint8)
    chars = alpha[_draw_codes(spec, rng, int(lens.sum()))].tobytes()
    out, pos = [], 0
    for L in lens.tolist():
        out.append(chars[pos:pos + L])
        pos += L
    return out


def _edit_many(bases: list[bytes], n_edits: list[int], spec, rng) -> list[bytes]:
    """Apply n_edits[k] random edits to bases[k] (all random draws batched)."""
    lo, hi = spec["clip"]
    alpha = spec["alphabet"]
    total = int(sum(n_edits))
    kinds = rng.integers(0, 3, size=total).tolist()
    u = rng.random(total).tolist()
    chars = _draw_codes(spec, rng, total).tolist()
    out = []
    e = 0
    for base, k in zip(bases, n_edits):
        s = bytearray(base)
        for _ in range(int(k)):
            kind, uu, c = kinds[e], u[e], alpha[chars[e]]
            e += 1
            if kind == 0 and len(s) >= hi:
                kind = 2
            if kind == 1 and len(s) <= lo:
                kind = 2
            if kind == 0:  # insert
                s.insert(int(uu * (len(s) + 1)), c)
            elif kind == 1:  # delete
                del s[int(uu * len(s))]
            elif s:  # substitute
                s[int(uu * len(s))] = c
        out.append(bytes(s))
    return out


def generate(name: str, tau: int | None = None, n: int | None = None, seed: int | None = None):
    """Strings of one workload as a list of bytes (input order = ids).

    n overrides the workload's size (same recipe at a smaller scale); tau sets
    the edit budget of cluster members (1..tau edits; ``short2k`` always uses
    1..3) and, with seed=None, the seed.
    """
    spec = WORKLOADS[name]
    if tau is None:
        tau = spec["taus"][-1]
    N = spec["n"] if n is None else int(n)
    rng = np.random.default_rng(seed_for(name, tau) if seed is None else seed)
    if "derived_frac" in spec:
        n_der = int(round(spec["derived_frac"] * N))
        fresh = _fresh(spec, rng, N - n_der)
        e_lo, e_hi = spec["edits"]
        bases = rng.integers(0, len(fresh), size=n_der)
        n_ed = rng.integers(e_lo, e_hi + 1, size=n_der)
        derived = _edit_many([fresh[b] for b in bases.tolist()], n_ed.tolist(), spec, rng)
        strings = fresh + derived
    else:
        target = int(round(spec["cluster_frac"] * N))
        c_lo, c_hi = spec["cluster_size"]
        # cluster sizes U{c_lo..c_hi} until the clustered share is covered
        draws = rng.integers(c_lo, c_hi + 1, size=target // max(1, c_lo) + 1)
        cum = np.cumsum(draws)
        m = int(np.searchsorted(cum, target)) + 1 if target > 0 else 0
        sizes = draws[:m].tolist()
        if sizes and sum(sizes) > target:
            sizes[-1] -= sum(sizes) - target
            if sizes[-1] < 2:
                sizes.pop()
        n_clustered = sum(sizes)
        n_bases = len(sizes)
        fresh = _fresh(spec, rng, N - n_clustered + n_bases)
        strings = fresh[n_bases:]
        e_hi = max(1, int(tau))
        member_bases = []
        for c, size in enumerate(sizes):
            strings.append(fresh[c])
            member_bases.extend([fresh[c]] * (size - 1))
        member_edits = rng.integers(1, e_hi + 1, size=len(member_bases)).tolist()
        strings.extend(_edit_many(member_bases, member_edits, spec, rng))
    perm = rng.permutation(len(strings))
    return [strings[k] for k in perm.tolist()]


def pack(strings) -> tuple[np.ndarray, np.ndarray]:
    """list of bytes -> (uint8 bytes, uint64 offsets with n + 1 entries)."""
    lens = np.fromiter((len(s) for s in strings), dtype=np.uint64, count=len(strings))
    off = np.zeros(len(strings) + 1, dtype=np.uint64)
    np.cumsum(lens, out=off[1:])
    buf = np.frombuffer(b"".join(strings), dtype=np.uint8).copy()
    return buf, off


def unpack(buf: np.ndarray, off: np.ndarray) -> list[bytes]:
    b = buf.tobytes()
    o = off.tolist()
    return [b[o[k]:o[k + 1]] for k in range(len(o) - 1)]


def subsample(strings, k: int, seed: int) -> list[bytes]:
    """k strings drawn without replacement, kept in their original order."""
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(len(strings), size=min(k, len(strings)), replace=False))
    return [strings[i] for i in idx.tolist()]


def query_stream(index_strings, n_requests: int, seed: int, tau_max: int = 4,
                 max_batch: int = 4096):
    """Serving requests against a resident index of ``short`` strings.

    Each request: batch size round(exp(U(0, ln max_batch))), tau uniform in
    1..tau_max, queries half ``short``-like and half ``medium``-like (lengths
    clipped to [5, 200]); half of all queries are indexed strings with 1..tau
    random edits so that hits exist.  Returns a list of (queries, tau).
    """
    rng = np.random.default_rng(seed)
    short = dict(WORKLOADS["short"])
    med = dict(WORKLOADS["medium"])
    med["clip"] = (5, 200)
    reqs = []
    for _ in range(n_requests):
        b = int(round(np.exp(rng.uniform(0.0, np.log(max_batch)))))
        b = max(1, min(max_batch, b))
        tau = int(rng.integers(1, tau_max + 1))
        kinds = rng.integers(0, 4, size=b)  # 0/1: fresh short/medium, 2/3: derived
        n_s = int((kinds == 0).sum())
        n_m = int((kinds == 1).sum())
        fs = _fresh(short, rng, n_s) if n_s else []
        fm = _fresh(med, rng, n_m) if n_m else []
        n_d = b - n_s - n_m
        picks = rng.integers(0, len(index_strings), size=n_d).tolist()
        fd = _edit_many([index_strings[k] for k in picks],
                        rng.integers(1, tau + 1, size=n_d).tolist(), short, rng)
        qs = []
        for k in kinds.tolist():
            qs.append(fs.pop() if k == 0 else fm.pop() if k == 1 else fd.pop())
        reqs.append((qs, tau))
    return reqs
