"""pj_query_noalloc, the query entry point that allocates nothing.

Some callers cannot allocate on the call path (a serving thread that must not
block in cudaMalloc, an embedder with a fixed memory reservation).  This file
calls the entry point through the C ABI and checks that two calls in a row
return exactly what pj_query returns for the same inputs (integer results:
the tolerance is zero), and that it refuses inputs it cannot serve without
allocating.  It is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

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
        for tau in (1, 3, 4):
            for Q in batches:  # two calls in a row, different contents
                want = pj.pj_query(idx, Q, tau).pairs
                db, do = device_strings(Q)
                rc, n, got = call_noalloc(lib, idx, db, do, tau, len(want) + 10)
                assert rc == 0, lib.pj_last_error().decode()
                assert n == len(want)
                assert np.array_equal(got, want)
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
