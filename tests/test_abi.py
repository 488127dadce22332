"""C ABI checks that need no GPU: the library builds, loads and exports every
function include/passjoin.h declares; the binding rejects bad input before
any device call."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "passjoin.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1111_7171_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(pj_[a-z_0-9]+)\s*\(", text)
    return sorted(set(n for n in names if not n.endswith("_fn")))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pj_build_index", "pj_self_join", "pj_join", "pj_query", "pj_result_free",
                     "pj_index_free", "pj_strerror"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in passjoin.h but not exported"


def test_strerror_and_options_init_without_gpu(lib):
    lib.pj_strerror.restype = ctypes.c_char_p
    assert lib.pj_strerror(0) == b"PJ_OK"
    assert b"EINVAL" in lib.pj_strerror(-1)
    from paper_1111_7171_gb300 import passjoin as pj
    opt = pj.pj_options()
    opt.verify_mode = 7
    pj.library().pj_options_init(ctypes.byref(opt))
    assert opt.verify_mode == 0 and opt.results_on_device == 0 and not opt.stream


def test_null_arguments_rejected_without_device_work(lib):
    from paper_1111_7171_gb300 import passjoin as pj
    L = pj.library()
    h = ctypes.c_void_p()
    assert L.pj_build_index(None, 2, None, ctypes.byref(h)) == pj.PJ_EINVAL
    assert L.pj_self_join(None, 1, ctypes.byref(pj.pj_result())) == pj.PJ_EINVAL
    assert L.pj_query(None, None, 1, ctypes.byref(pj.pj_result())) == pj.PJ_EINVAL
    s = pj.Strings([b"ab"])
    assert L.pj_build_index(ctypes.byref(s.c), 33, None, ctypes.byref(h)) == pj.PJ_EINVAL
    assert L.pj_join(ctypes.byref(s.c), ctypes.byref(s.c), -1, None, ctypes.byref(pj.pj_result())) == pj.PJ_EINVAL
    assert L.pj_count_selection(None, 1, ctypes.byref(pj.pj_selection())) == pj.PJ_EINVAL
    assert L.pj_calibrate(None) == pj.PJ_EINVAL
    assert L.pj_self_join_shard(None, 1, 0, 1, ctypes.byref(pj.pj_result())) == pj.PJ_EINVAL
    assert L.pj_self_join_stream(None, 1, None, ctypes.byref(pj.pj_result())) == pj.PJ_EINVAL
    assert L.pj_self_join_stream(ctypes.byref(s.c), 33, None, ctypes.byref(pj.pj_result())) == pj.PJ_EINVAL
    L.pj_result_free(None)
    L.pj_index_free(None)


def test_struct_layouts_match_header(tmp_path):
    """ctypes mirrors of the ABI structs have the C compiler's sizes and offsets."""
    import subprocess
    from paper_1111_7171_gb300 import passjoin as pj
    src = tmp_path / "layout.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "passjoin.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(pj_strings), sizeof(pj_pair), sizeof(pj_stats),
         sizeof(pj_result), sizeof(pj_options), offsetof(pj_result, stats));
  printf("%zu %zu %zu\\n", offsetof(pj_options, verify_mode), offsetof(pj_options, results_on_device),
         offsetof(pj_result, priv));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    sizes = [int(x) for x in out]
    assert sizes[0] == ctypes.sizeof(pj.pj_strings)
    assert sizes[1] == pj.PAIR_DTYPE.itemsize
    assert sizes[2] == ctypes.sizeof(pj.pj_stats)
    assert sizes[3] == ctypes.sizeof(pj.pj_result)
    assert sizes[4] == ctypes.sizeof(pj.pj_options)
    assert sizes[5] == pj.pj_result.stats.offset
    assert sizes[6] == pj.pj_options.verify_mode.offset
    assert sizes[7] == pj.pj_options.results_on_device.offset
    assert sizes[8] == pj.pj_result.priv.offset


def test_every_struct_field_matches_header(tmp_path):
    """Every field offset and size of every ctypes mirror equals the C compiler's."""
    import subprocess
    from paper_1111_7171_gb300 import passjoin as pj
    structs = [pj.pj_strings, pj.pj_stats, pj.pj_result, pj.pj_options, pj.pj_server_options,
               pj.pj_request_times, pj.pj_server_counters, pj.pj_plan_options, pj.pj_plan_info,
               pj.pj_selection, pj.pj_calibration]
    lines = []
    for st in structs:
        name = st.__name__
        lines.append(f'  printf("{name} sizeof %zu\\n", sizeof({name}));')
        for f, _ in st._fields_:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    src = tmp_path / "fields.c"
    src.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"passjoin.h\"\nint main(void) {\n" +
                   "\n".join(lines) + "\n  return 0;\n}\n")
    exe = tmp_path / "fields"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines()
    want = {}
    for line in out:
        name, field, value = line.split()
        want[(name, field)] = int(value)
    for st in structs:
        assert want[(st.__name__, "sizeof")] == ctypes.sizeof(st), st.__name__
        for f, _ in st._fields_:
            assert want[(st.__name__, f)] == getattr(st, f).offset, (st.__name__, f)


def test_plan_entry_points_reject_null_without_device_work(lib):
    from paper_1111_7171_gb300 import passjoin as pj
    L = pj.library()
    o = pj.pj_plan_options()
    L.pj_plan_options_init(ctypes.byref(o))
    assert o.max_queries == 4096 and o.max_bytes == 1 << 20 and o.hits_capacity == 0
    h = ctypes.c_void_p()
    assert L.pj_plan_create(None, ctypes.byref(o), ctypes.byref(h)) == pj.PJ_EINVAL
    assert not h.value
    assert L.pj_plan_query(None, None, None, ctypes.byref(pj.pj_result())) == pj.PJ_EINVAL
    assert L.pj_plan_get_info(None, ctypes.byref(pj.pj_plan_info())) == pj.PJ_EINVAL
    L.pj_plan_free(None)
    so = pj.pj_server_options()
    so.use_plans = 5
    L.pj_server_options_init(ctypes.byref(so))
    assert so.use_plans == 0 and so.slots == 3


def test_binding_marshals_string_sets():
    from paper_1111_7171_gb300 import passjoin as pj
    s = pj.Strings([b"abc", b"", b"de"])
    assert s.n == 3 and s.c.on_device == 0
    buf = np.frombuffer(b"xxabcde", np.uint8)
    s2 = pj.Strings((buf, np.array([2, 5, 7], np.uint64)))
    assert s2.n == 2


def test_synth_is_deterministic():
    from paper_1111_7171_gb300 import synth
    a = synth.generate("short", 3, n=2000)
    b = synth.generate("short", 3, n=2000)
    assert a == b and len(a) == 2000
    assert synth.generate("short2k", 2)[:5] == synth.generate("short2k", 2)[:5]
    lens = np.array([len(s) for s in synth.generate("medium", 4, n=3000)])
    assert lens.min() >= 20 and lens.max() <= 300 and 90 < lens.mean() < 110
