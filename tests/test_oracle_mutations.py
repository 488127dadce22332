"""Planted mistakes: the oracle's pins must catch plausible bugs.

Each case copies an oracle source into a temporary directory, plants one
mistake (a dropped term, a wrong sign or index, a transposed operand), builds
or loads the copy, and checks that the pins of test_oracle.py reject it.  The
committed oracle is never modified.
"""
import ctypes
import importlib.util
import json
import os
import random
import subprocess

import numpy as np
import pytest

from test_oracle import GOLDEN, all_strings, bfs_distances, ed_alignments

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
C_SRC = os.path.join(ROOT, "oracle", "passjoin_oracle.c")
PY_SRC = os.path.join(ROOT, "oracle", "method.py")

C_MUTANTS = {
    "delta_inverted": ("(r[i - 1] == s[j - 1] ? 0 : 1);\n      int32_t m", "(r[i - 1] == s[j - 1] ? 1 : 0);\n      int32_t m"),
    "first_row_zero": ("row_prev[j] = (int32_t)j; /* M(0, j) = j */", "row_prev[j] = 0;"),
    "first_col_zero": ("row_cur[0] = (int32_t)i; /* M(i, 0) = i */", "row_cur[0] = 0;"),
    "no_insert_cost": ("int32_t ins = row_cur[j - 1] + 1;\n      int32_t sub = row_prev[j - 1] + (r[i - 1] == s[j - 1] ? 0 : 1);\n      int32_t m",
                       "int32_t ins = row_cur[j - 1];\n      int32_t sub = row_prev[j - 1] + (r[i - 1] == s[j - 1] ? 0 : 1);\n      int32_t m"),
    "diag_index": ("int32_t sub = row_prev[j - 1] + (r[i - 1] == s[j - 1] ? 0 : 1);\n      int32_t m",
                   "int32_t sub = row_prev[j] + (r[i - 1] == s[j - 1] ? 0 : 1);\n      int32_t m"),
    "char_index": ("(r[i - 1] == s[j - 1] ? 0 : 1);\n      int32_t m", "(r[i - 1] == s[j] ? 0 : 1);\n      int32_t m"),
    "length_filter_off_by_one": ("if (dl > tau) continue; /* length filter */", "if (dl >= tau) continue;"),
    "self_pairs_included": ("for (int64_t y = self ? x + 1 : 0; y < nb; ++y)", "for (int64_t y = self ? x : 0; y < nb; ++y)"),
}


def _build_mutant(tmp_path, name, old, new):
    src = open(C_SRC).read()
    assert src.count(old) >= 1, name
    src = src.replace(old, new, 1)
    c = tmp_path / f"{name}.c"
    c.write_text(src)
    so = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O1", "-fopenmp", "-shared", "-fPIC", "-o", str(so), str(c)], check=True)
    L = ctypes.CDLL(str(so))
    u8p = ctypes.POINTER(ctypes.c_uint8)
    L.oracle_ed.argtypes = [u8p, ctypes.c_int64, u8p, ctypes.c_int64]
    L.oracle_ed.restype = ctypes.c_int32
    return L


def _ed(L, a: bytes, b: bytes) -> int:
    aa = np.frombuffer(a + b"\0", np.uint8).copy()
    bb = np.frombuffer(b + b"\0", np.uint8).copy()
    p = ctypes.POINTER(ctypes.c_uint8)
    return int(L.oracle_ed(aa.ctypes.data_as(p), len(a), bb.ctypes.data_as(p), len(b)))


def _c_pins_pass(L, tmp_path, name) -> bool:
    words = list(all_strings("ab", 4))
    for src in words:
        dist = bfs_distances(src, "ab", 4)
        for dst in words:
            if _ed(L, src.encode(), dst.encode()) != dist[dst]:
                return False
    for e in GOLDEN["ed"]:
        if _ed(L, e["r"].encode(), e["s"].encode()) != e["ed"]:
            return False
    return True


@pytest.mark.parametrize("name", [k for k in C_MUTANTS if k not in ("length_filter_off_by_one", "self_pairs_included")])
def test_c_ed_mutants_are_caught(tmp_path, name):
    old, new = C_MUTANTS[name]
    L = _build_mutant(tmp_path, name, old, new)
    assert not _c_pins_pass(L, tmp_path, name)


@pytest.mark.parametrize("name", ["length_filter_off_by_one", "self_pairs_included"])
def test_c_join_mutants_are_caught(tmp_path, name):
    """Join-level mistakes are caught by the brute-force join comparison."""
    old, new = C_MUTANTS[name]
    src = open(C_SRC).read().replace(old, new, 1)
    c = tmp_path / f"{name}.c"
    c.write_text(src)
    so = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O1", "-fopenmp", "-shared", "-fPIC", "-o", str(so), str(c)], check=True)
    import oracle as O
    saved = O._lib
    try:
        O._lib = None
        orig = O.build
        O.build = lambda: str(so)
        rng = random.Random(4)
        strings = [("".join(rng.choice("ab") for _ in range(rng.randint(0, 6)))).encode() for _ in range(30)]
        b, o = O.pack(strings)
        got = [(int(r["a"]), int(r["b"]), int(r["ed"])) for r in O.self_join(b, o, 2)]
        want = [(x, y, ed_alignments(strings[x].decode(), strings[y].decode()))
                for x in range(len(strings)) for y in range(x + 1, len(strings))
                if ed_alignments(strings[x].decode(), strings[y].decode()) <= 2]
        assert got != want
    finally:
        O.build = orig
        O._lib = saved


PY_MUTANTS = {
    "partition_longer_first": ("li = base + 1 if i > tau + 1 - k else base", "li = base + 1 if i <= k else base"),
    "multi_left_dropped": ("lo = max(P - (i - 1), P + D - (tau + 1 - i))", "lo = P + D - (tau + 1 - i)"),
    "multi_right_sign": ("hi = min(P + (i - 1), P + D + (tau + 1 - i))", "hi = min(P + (i - 1), P - D + (tau + 1 - i))"),
    "multi_right_index": ("lo = max(P - (i - 1), P + D - (tau + 1 - i))", "lo = max(P - (i - 1), P + D - (tau - i))"),
    "position_floor_swapped": ("lo, hi = P - (tau - D) // 2, P + (tau + D) // 2", "lo, hi = P - (tau + D) // 2, P + (tau - D) // 2"),
    "tau_l_off_by_one": ("tau_l, tau_r = i - 1, tau + 1 - i", "tau_l, tau_r = i - 2, tau + 1 - i"),
    "tau_r_off_by_one": ("tau_l, tau_r = i - 1, tau + 1 - i", "tau_l, tau_r = i - 1, tau - i"),
    "expected_ed_dropped": ("expected = [cur[j] + abs((ns - j) - (nr - i)) for j in cur]", "expected = [cur[j] for j in cur]"),
    "expected_ed_transposed": ("expected = [cur[j] + abs((ns - j) - (nr - i)) for j in cur]", "expected = [cur[j] + abs((ns - i) - (nr - j)) for j in cur]"),
    "band_offsets_swapped": ("lo_off = (tau - D) // 2\n    hi_off = (tau + D) // 2", "lo_off = (tau + D) // 2\n    hi_off = (tau - D) // 2"),
    "segment_not_compared": ("if s[p:p + li] != r[P:P + li] or p < 0:", "if p < 0:"),
    # centred partition scheme: longer segments off the middle, ties the other way, or swapped lengths
    "center_off_by_one": ("key=lambda i: (abs(2 * i - (m + 1)), i))", "key=lambda i: (abs(2 * i - m), i))"),
    "center_ties_right": ("key=lambda i: (abs(2 * i - (m + 1)), i))", "key=lambda i: (abs(2 * i - (m + 1)), -i))"),
    "center_short_middle": ("li = base + 1 if i in longer else base\n", "li = base if i in longer else base + 1\n"),
}


def _load_method_mutant(tmp_path, name):
    old, new = PY_MUTANTS[name]
    src = open(PY_SRC).read()
    assert src.count(old) == 1, name
    path = tmp_path / f"method_{name}.py"
    path.write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location(f"method_{name}", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _method_pins_pass(Mm) -> bool:
    import test_oracle as T
    checks = [T.test_even_partition_paper_example, T.test_even_partition_shape,
              T.test_selection_paper_example, T.test_selection_count_formulas,
              T.test_lemma3_subset_chain, T.test_verification_paper_examples,
              T.test_verify_string_pair_is_capped_ed, T.test_extension_paper_example,
              T.test_extension_min_over_matches_is_ed, T.test_pass_join_table1,
              lambda: T.test_multi_match_completeness_exhaustive(2),
              lambda: T.test_pass_join_equals_definition("id", "even", 2),
              lambda: T.test_pass_join_equals_definition("prefix8", "center", 2),
              T.test_center_partition_shape]
    saved = T.M
    T.M = Mm
    try:
        for chk in checks:
            try:
                chk()
            except (AssertionError, ValueError, IndexError, KeyError, TypeError):
                return False
        return True
    finally:
        T.M = saved


@pytest.mark.parametrize("name", sorted(PY_MUTANTS))
def test_method_mutants_are_caught(tmp_path, name):
    assert not _method_pins_pass(_load_method_mutant(tmp_path, name))


def test_unmutated_sources_pass(tmp_path):
    from oracle import method as Mm
    assert _method_pins_pass(Mm)
