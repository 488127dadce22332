"""The probe/verify kernels' per-thread logic, run on the CPU.

tests/host_logic/probe_emu.cu includes the same __host__ __device__ functions
the kernels call (group windows, lookups, extension verification) and runs
them through the kernels' two phases on the host.  Its pair sets must equal
the oracle's, and its candidate / accepted counts must equal those of the
paper's algorithm (oracle.method, visiting by length then id).  CPU only.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from oracle import method as M
from paper_1111_7171_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "host_logic", "probe_emu.cu")
CSRC = os.path.join(ROOT, "paper_1111_7171_gb300", "csrc")


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path_factory.mktemp("emu") / "probe_emu"
    subprocess.run([nvcc, "-std=c++17", "-O2", "-I", CSRC, "-I", os.path.join(ROOT, "include"), "-o", str(exe), SRC],
                   check=True)
    return str(exe)


def run_emu(exe, tmp, strings, tau, queries=None):
    b, o = synth.pack(strings)
    (tmp / "b").write_bytes(b.tobytes())
    (tmp / "o").write_bytes(o.tobytes())
    args = [exe, str(tmp / "b"), str(tmp / "o"), str(tau)]
    if queries is not None:
        qb, qo = synth.pack(queries)
        (tmp / "qb").write_bytes(qb.tobytes())
        (tmp / "qo").write_bytes(qo.tobytes())
        args += [str(tmp / "qb"), str(tmp / "qo")]
    out = subprocess.run(args, capture_output=True, text=True, check=True).stdout.split("\n")
    st = list(map(int, out[0].split()[1:]))
    pairs = np.array([tuple(map(int, line.split())) for line in out[1:] if line.strip()],
                     dtype=np.int64).reshape(-1, 3)
    return st, pairs


def oracle_self(strings, tau):
    b, o = synth.pack(strings)
    r = oracle.self_join(b, o, tau)
    return np.stack([r["a"], r["b"], r["ed"]], axis=1).astype(np.int64) if len(r) else np.zeros((0, 3), np.int64)


@pytest.mark.parametrize("name,tau,n", [("short2k", 2, 2000), ("short", 1, 3000), ("short", 2, 3000),
                                        ("short", 4, 2000), ("medium", 4, 800), ("medium", 8, 600),
                                        ("long", 16, 150)])
def test_self_join_logic(emu, tmp_path, name, tau, n):
    strings = synth.generate(name, tau, n=n)
    st, pairs = run_emu(emu, tmp_path, strings, tau)
    assert st[4] == 0
    want = oracle_self(strings, tau) if name != "long" else None
    if want is None:
        b, o = synth.pack(strings)
        r = oracle.self_join(b, o, tau, banded=True)
        want = np.stack([r["a"], r["b"], r["ed"]], axis=1).astype(np.int64) if len(r) else np.zeros((0, 3), np.int64)
    assert np.array_equal(pairs, want)


def test_self_join_logic_without_fingerprints(emu, tmp_path, monkeypatch):
    monkeypatch.setenv("PJ_EMU_NO_FP", "1")  # plain linear probing over the slots
    strings = synth.generate("short", 3, n=2000)
    st, pairs = run_emu(emu, tmp_path, strings, 3)
    assert np.array_equal(pairs, oracle_self(strings, 3))


def test_fingerprint_buckets_match_linear_probing(tmp_path):
    """table_find reads eight fingerprint bytes per load; its answers must be
    those of plain linear probing, for present and absent keys, clustered
    runs and runs that wrap past the last slot."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "table_check"
    subprocess.run([nvcc, "-std=c++17", "-O2", "-I", CSRC, "-I", os.path.join(ROOT, "include"), "-o", str(exe),
                    os.path.join(ROOT, "tests", "host_logic", "table_check.cu")], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    assert out[0] == "cases" and int(out[1]) > 100000 and out[2:] == ["bad", "0"]


def test_counts_equal_the_algorithm(emu, tmp_path):
    strings = synth.generate("short", 3, n=500)
    st, _ = run_emu(emu, tmp_path, strings, 3)
    ref = {}
    M.pass_join_self(strings, 3, order="id", stats=ref)
    assert st[1] == ref["tuples"] and st[2] == ref["accepted"]


def test_short_and_empty_strings(emu, tmp_path):
    rng = np.random.default_rng(2)
    strings = [bytes(rng.choice(list(b"ab"), size=int(L)).tolist()) for L in rng.integers(0, 7, size=300)]
    for tau in (0, 1, 2, 3):
        st, pairs = run_emu(emu, tmp_path, strings, tau)
        assert np.array_equal(pairs, oracle_self(strings, tau)), tau


def test_rs_join_logic(emu, tmp_path):
    S = synth.generate("short", 3, n=1500) + [b"", b"ab", b"abc"]
    R = synth.generate("short", 3, n=400, seed=5) + [s[1:] for s in S[:200]] + [s + b"x" for s in S[200:300]] + [b""]
    st, pairs = run_emu(emu, tmp_path, S, 3, queries=R)
    rb, ro = synth.pack(R)
    sb, so = synth.pack(S)
    r = oracle.join(rb, ro, sb, so, 3)
    want = np.stack([r["a"], r["b"], r["ed"]], axis=1).astype(np.int64)
    assert np.array_equal(pairs, want)


def test_vsp_widths_match_plain_dp(tmp_path):
    """VERIFYSTRINGPAIR (Sec. 5.1, Alg. 3) at every compiled band width, 2 to
    33 diagonals, equals min(t + 1, ED) of the plain DP; so does its
    shared-prefix form (Sec. 5.3) over runs of strings with common prefixes,
    resuming from kept rows as the mode-L kernel does."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "vsp_check"
    subprocess.run([nvcc, "-std=c++17", "-O2", "-I", CSRC, "-o", str(exe),
                    os.path.join(ROOT, "tests", "host_logic", "vsp_check.cu")], check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines()
    shared = [ln.split() for ln in lines if ln.startswith("shared")]
    assert len(shared) == 3
    for toks in shared:  # the shared-prefix form (Sec. 5.3): exact, and it does share rows
        vals = dict(tok.split("=") for tok in toks[1:])
        assert vals["bad"] == "0", toks
        assert int(vals["resumed"]) > 1000 and int(vals["rows_saved"]) > 10000 and int(vals["skipped"]) > 100
    out = " ".join(ln for ln in lines if not ln.startswith("shared")).split()
    widths = [tok.split("=")[1] for tok in out if tok.startswith("W=")]
    assert widths == ["2", "3", "5", "9", "17", "33"]
    assert all(tok == "bad=0" for tok in out if tok.startswith("bad="))
    # the long edited pairs put many distances next to the threshold, where a
    # wrong band edge or early exit would show
    assert all(int(tok.split("=")[1]) > 5000 for tok in out if tok.startswith("near="))


def test_even_partition_by_reciprocal_matches_division(tmp_path):
    """The kernels' division-free even partition equals the rule of Sec. 3.1
    (plain integer division) for every length < 2^16 and 1..33 segments."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "segment_check"
    subprocess.run([nvcc, "-std=c++17", "-O2", "-I", CSRC, "-I", os.path.join(ROOT, "include"), "-o", str(exe),
                    os.path.join(ROOT, "tests", "host_logic", "segment_check.cu")], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    assert out.strip().endswith("bad=0"), out


def test_character_set_bound_never_exceeds_edit_distance(tmp_path):
    """The bound that rejects candidates before verification is a lower bound
    of the edit distance of Def. 1 (plain DP), for every alphabet size."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "bound_check"
    subprocess.run([nvcc, "-std=c++17", "-O2", "-I", CSRC, "-I", os.path.join(ROOT, "include"), "-o", str(exe),
                    os.path.join(ROOT, "tests", "host_logic", "bound_check.cu")], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    vals = dict(tok.split("=") for tok in out)
    assert vals["bad"] == "0", out
    assert int(vals["tight"]) > 1000  # the bound is often exact, so it has teeth
    assert int(vals["side_tight"]) > 1000


def test_partition_schemes_match_the_oracle(tmp_path):
    """The kernels' closed form of both partition schemes (the paper's even
    partition, Sec. 3.1, and the centred scheme) gives exactly the segments
    of the oracle's definitions (oracle/method.py) for every length up to 160
    and 1..33 segments."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "scheme_dump"
    subprocess.run([nvcc, "-std=c++17", "-O2", "-I", CSRC, "-I", os.path.join(ROOT, "include"), "-o", str(exe),
                    os.path.join(ROOT, "tests", "host_logic", "scheme_dump.cu")], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines()
    schemes = {0: M.even_partition, 1: M.center_partition}
    n = 0
    for line in out:
        f = [int(x) for x in line.split()]
        scheme, parts, length = f[:3]
        got = [(f[3 + 2 * k], f[4 + 2 * k]) for k in range(parts)]
        assert got == schemes[scheme](length, parts - 1), (scheme, parts, length)
        n += 1
    assert n == 2 * sum(161 - p for p in range(1, 34))


def test_fused_work_items_cover_every_probe_once(tmp_path):
    """The fused self join's work items (fused_item: items from the two ends
    of the length order in turn) cover every probe of the range exactly once,
    for probe ranges of 1..300 probes at several starts and 1..40 probes per
    item."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "fused_items"
    subprocess.run([nvcc, "-std=c++17", "-O2", "-I", CSRC, "-I", os.path.join(ROOT, "include"), "-o", str(exe),
                    os.path.join(ROOT, "tests", "host_logic", "fused_items.cu")], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True).stdout.strip()
    assert out == f"ok {4 * 300 * 40}", out

