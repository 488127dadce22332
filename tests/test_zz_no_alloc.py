"""pj_query_noalloc, the query entry point that allocates nothing.

Some callers cannot allocate on the call path (a serving thread that must not
block in cudaMalloc, an embedder with a fixed memory reservation).  This file
calls the entry point through the C ABI and checks that two calls in a row
return exactly what pj_query returns for the same inputs (integer results:
the tolerance is zero) and what the CPU oracle (Def. 1 by brute force)
returns, on indexes of short and of long strings (every compiled band width
of the verification), and that it refuses inputs it cannot serve without
allocating -- including more accepted matches than its fixed scratch holds --
and keeps working after such a refusal.  It is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1111_7171_gb300 import passjoin as pj
from paper_1111_7171_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return pj.library()


def device_strings(strings):
    b, o = synth.pack(strings)
    return torch.from_numpy(b).cuda(), torch.from_numpy(o.astype(np.int64)).cuda()


def call_noalloc(L, idx, db, do, tau, cap):
    s = pj.Strings((db, do))
    out = torch.empty(max(cap, 1) * 12, dtype=torch.uint8, device="cuda")
    n = ctypes.c_uint64(0)
    rc = L.pj_query_noalloc(idx.handle, ctypes.byref(s.c), tau, ctypes.c_void_p(out.data_ptr()), cap, ctypes.byref(n))
    torch.cuda.synchronize()
    pairs = out[: int(n.value) * 12].cpu().numpy().view(pj.PAIR_DTYPE) if rc == 0 else None
    return rc, int(n.value), pairs


def test_two_calls_match_pj_query(lib):
    S = synth.generate("short", 4, n=20000) + [b"", b"ab", b"abc"]
    idx = pj.pj_build_index(S, 4)
    try:
        rng = np.random.default_rng(11)
        batches = []
        for seed in (1, 2):
            Q = synth.generate("short", 4, n=1500, seed=seed)
            Q += [S[k][1:] + b"q" for k in rng.integers(0, len(S), size=500).tolist()] + [b"", b"a"]
            batches.append(Q)
        sb, so = synth.pack(S)
        for tau in (1, 3, 4):
            for k, Q in enumerate(batches):  # two calls in a row, different contents
                want = pj.pj_query(idx, Q, tau).pairs
                db, do = device_strings(Q)
                rc, n, got = call_noalloc(lib, idx, db, do, tau, len(want) + 10)
                assert rc == 0, lib.pj_last_error().decode()
                assert n == len(want)
                assert np.array_equal(got, want)
                if k == 0:  # and the definition itself
                    qb, qo = synth.pack(Q)
                    assert np.array_equal(got, oracle.join(qb, qo, sb, so, tau, banded=True))
            # and the first batch again: the scratch keeps the last call's data
            want = pj.pj_query(idx, batches[0], tau).pairs
            rc, n, got = call_noalloc(lib, idx, *device_strings(batches[0]), tau, len(want))
            assert rc == 0 and np.array_equal(got, want)
    finally:
        idx.free()


def test_refuses_what_it_cannot_serve(lib):
    S = synth.generate("short", 2, n=3000)
    idx = pj.pj_build_index(S, 2)
    try:
        Q = S[:200]
        want = pj.pj_query(idx, Q, 2).pairs
        db, do = device_strings(Q)
        rc, n, _ = call_noalloc(lib, idx, db, do, 2, max(0, len(want) - 1))
        assert rc == pj.PJ_EINVAL and n == len(want)  # output buffer too small, count reported
        host = pj.Strings(Q)
        out = torch.empty(12 * len(want), dtype=torch.uint8, device="cuda")
        cnt = ctypes.c_uint64(0)
        assert lib.pj_query_noalloc(idx.handle, ctypes.byref(host.c), 2, ctypes.c_void_p(out.data_ptr()),
                                    len(want), ctypes.byref(cnt)) == pj.PJ_EINVAL  # host batch
        big = [b"abcdef"] * 65537
        rc, _, _ = call_noalloc(lib, idx, *device_strings(big), 2, 10)
        assert rc == pj.PJ_EINVAL and b"limit" in lib.pj_last_error()
        rc, _, _ = call_noalloc(lib, idx, db, do, 3, 10)
        assert rc == pj.PJ_EINVAL  # tau above tau_max
    finally:
        idx.free()
    lazy = pj.pj_build_index(S, 2, lazy_partitions=True)
    try:
        rc, _, _ = call_noalloc(lib, lazy, *device_strings(S[:10]), 2, 100)
        assert rc == pj.PJ_EINVAL and b"not built" in lib.pj_last_error()
    finally:
        lazy.free()


def test_long_strings_every_band_width(lib):
    """An index of long strings (average length above 256 bytes, so its
    tables carry two presence-bitmap bytes per slot) built for tau_max 32 and
    queried at tau 8, 16 and 32: the thread-per-candidate band widths 9, 17
    and 33 of the no-allocation kernels, against pj_query and the oracle."""
    S = synth.generate("long", 16, n=500)
    rng = np.random.default_rng(3)
    Q = synth.generate("long", 16, n=60, seed=9)
    for k in rng.integers(0, len(S), size=60).tolist():
        s = bytearray(S[k])
        for _ in range(int(rng.integers(0, 20))):
            pos = int(rng.integers(0, len(s)))
            if rng.random() < 0.5:
                s[pos] = ord("a") + int(rng.integers(0, 26))
            else:
                del s[pos]
        Q.append(bytes(s))
    idx = pj.pj_build_index(S, 32)
    try:
        sb, so = synth.pack(S)
        qb, qo = synth.pack(Q)
        db, do = device_strings(Q)
        for tau in (8, 16, 32):
            want = pj.pj_query(idx, Q, tau).pairs
            assert len(want) > 0
            assert np.array_equal(want, oracle.join(qb, qo, sb, so, tau, banded=True))
            for _ in range(2):
                rc, n, got = call_noalloc(lib, idx, db, do, tau, len(want))
                assert rc == 0, lib.pj_last_error().decode()
                assert np.array_equal(got, want)
    finally:
        idx.free()


def test_scratch_overflow_is_refused_then_recovers(lib):
    """More accepted matches than the fixed scratch array holds: the call
    fails with PJ_ENOMEM (nothing is allocated instead), and the next call
    with a batch that fits returns the exact result."""
    S = [b"a" * 12] * 3000 + synth.generate("short", 4, n=2000)
    idx = pj.pj_build_index(S, 4)
    try:
        heavy = [b"a" * 12] * 1000  # every pair matches on every window position
        rc, _, _ = call_noalloc(lib, idx, *device_strings(heavy), 4, 10)
        assert rc == pj.PJ_ENOMEM, lib.pj_last_error().decode()
        assert b"scratch" in lib.pj_last_error()
        Q = S[3000:3400]
        want = pj.pj_query(idx, Q, 4).pairs
        rc, n, got = call_noalloc(lib, idx, *device_strings(Q), 4, len(want))
        assert rc == 0 and np.array_equal(got, want)
    finally:
        idx.free()
