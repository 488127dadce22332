"""CPU oracle for the Pass-Join similarity join.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA path (``paper_1111_7171_gb300``) and
never imports it.

Two layers:

* ``passjoin_oracle.c`` (loaded here through ctypes): the plain definition of
  the result -- Def. 1 (Sec. 2) evaluated by brute force: length filter, then
  the Wagner-Fischer recurrence of Sec. 5.1 on every surviving pair.
* ``oracle.method``: the paper's own steps in the paper's order (even
  partition, Sec. 3.1; the four substring-selection rules, Sec. 4; length-aware
  verification with expected-edit-distance early termination, Sec. 5.1 and
  Lemma 4; extension-based verification, Sec. 5.2 and Alg. 3; the Pass-Join
  loop, Alg. 1), pure Python for small inputs.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "passjoin_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_lock = threading.Lock()
_lib = None


class OraclePair(ctypes.Structure):
    _fields_ = [("a", ctypes.c_uint32), ("b", ctypes.c_uint32), ("ed", ctypes.c_uint32)]


PAIR_DTYPE = np.dtype([("a", np.uint32), ("b", np.uint32), ("ed", np.uint32)])


def _lib_path() -> str:
    with open(_SRC, "rb") as f:
        tag = hashlib.sha1(f.read()).hexdigest()[:12]
    return os.path.join(_BUILD_DIR, f"liboracle_{tag}.so")


def build() -> str:
    """Compile the C oracle with gcc (OpenMP) into oracle/_build/.  Idempotent."""
    path = _lib_path()
    if os.path.exists(path):
        return path
    os.makedirs(_BUILD_DIR, exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-std=c11", "-Wall", "-shared", "-fPIC", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            u8p = ctypes.POINTER(ctypes.c_uint8)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            i64p = ctypes.POINTER(ctypes.c_int64)
            pp = ctypes.POINTER(OraclePair)
            L.oracle_ed.argtypes = [u8p, ctypes.c_int64, u8p, ctypes.c_int64]
            L.oracle_ed.restype = ctypes.c_int32
            L.oracle_ed_banded.argtypes = [u8p, ctypes.c_int64, u8p, ctypes.c_int64, ctypes.c_int32]
            L.oracle_ed_banded.restype = ctypes.c_int32
            L.oracle_self_join.argtypes = [u8p, u64p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int,
                                           pp, ctypes.c_int64, ctypes.c_int]
            L.oracle_self_join.restype = ctypes.c_int64
            L.oracle_join.argtypes = [u8p, u64p, ctypes.c_int64, u8p, u64p, ctypes.c_int64,
                                      ctypes.c_int32, ctypes.c_int, pp, ctypes.c_int64, ctypes.c_int]
            L.oracle_join.restype = ctypes.c_int64
            L.oracle_similar_to.argtypes = [u8p, u64p, ctypes.c_int64, u8p, u64p, ctypes.c_int64,
                                            ctypes.c_int32, ctypes.c_int, i64p, pp, ctypes.c_int64,
                                            ctypes.c_int]
            L.oracle_similar_to.restype = ctypes.c_int64
            L.oracle_num_threads.argtypes = []
            L.oracle_num_threads.restype = ctypes.c_int
            _lib = L
    return _lib


# ----------------------------------------------------------------- helpers --

def pack(strings) -> tuple[np.ndarray, np.ndarray]:
    """list of bytes -> (uint8 bytes, uint64 offsets[n+1])."""
    lens = np.fromiter((len(s) for s in strings), dtype=np.uint64, count=len(strings))
    off = np.zeros(len(strings) + 1, dtype=np.uint64)
    np.cumsum(lens, out=off[1:])
    buf = np.frombuffer(b"".join(strings), dtype=np.uint8).copy() if len(strings) else np.zeros(0, np.uint8)
    if buf.size == 0:
        buf = np.zeros(1, np.uint8)  # keep a valid pointer for empty inputs
    return buf, off


def _u8(a: np.ndarray):
    a = np.ascontiguousarray(a, dtype=np.uint8)
    if a.size == 0:
        a = np.zeros(1, np.uint8)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _u64(a: np.ndarray):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def ed(r: bytes, s: bytes) -> int:
    """ED(r, s) by the full Wagner-Fischer DP (Sec. 5.1)."""
    ra, rp = _u8(np.frombuffer(r, np.uint8))
    sa, sp = _u8(np.frombuffer(s, np.uint8))
    return int(lib().oracle_ed(rp, len(r), sp, len(s)))


def ed_banded(r: bytes, s: bytes, tau: int) -> int:
    """min(tau + 1, ED(r, s)) by the 2*tau+1 band with row-minimum cutoff."""
    ra, rp = _u8(np.frombuffer(r, np.uint8))
    sa, sp = _u8(np.frombuffer(s, np.uint8))
    return int(lib().oracle_ed_banded(rp, len(r), sp, len(s), tau))


def _run_with_retry(fn, cap=1 << 16):
    while True:
        out = np.zeros(max(cap, 1), dtype=PAIR_DTYPE)
        total = fn(out.ctypes.data_as(ctypes.POINTER(OraclePair)), cap)
        if total < 0:
            raise RuntimeError("oracle failed (allocation or invalid tau)")
        if total <= cap:
            return out[:total].copy()
        cap = int(total)


def self_join(bytes_: np.ndarray, offsets: np.ndarray, tau: int, banded: bool = False,
              nthreads: int = 0) -> np.ndarray:
    """All pairs a < b of one set with ED <= tau, sorted; structured (a, b, ed)."""
    b, bp = _u8(bytes_)
    o, op = _u64(offsets)
    n = len(o) - 1
    return _run_with_retry(lambda out, cap: lib().oracle_self_join(
        bp, op, n, tau, int(banded), out, cap, nthreads))


def join(rbytes, roff, sbytes, soff, tau: int, banded: bool = False, nthreads: int = 0) -> np.ndarray:
    """All (a in R, b in S) with ED <= tau, sorted; structured (a, b, ed)."""
    rb, rbp = _u8(rbytes)
    ro, rop = _u64(roff)
    sb, sbp = _u8(sbytes)
    so, sop = _u64(soff)
    return _run_with_retry(lambda out, cap: lib().oracle_join(
        rbp, rop, len(ro) - 1, sbp, sop, len(so) - 1, tau, int(banded), out, cap, nthreads))


def similar_to(qbytes, qoff, sbytes, soff, tau: int, banded: bool = True, exclude=None,
               nthreads: int = 0) -> np.ndarray:
    """For each query q, all y in S with ED(q, y) <= tau; (a=q, b=y, ed)."""
    qb, qbp = _u8(qbytes)
    qo, qop = _u64(qoff)
    sb, sbp = _u8(sbytes)
    so, sop = _u64(soff)
    if exclude is not None:
        ex = np.ascontiguousarray(exclude, dtype=np.int64)
        exp = ex.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    else:
        ex, exp = None, None
    return _run_with_retry(lambda out, cap: lib().oracle_similar_to(
        qbp, qop, len(qo) - 1, sbp, sop, len(so) - 1, tau, int(banded), exp, out, cap, nthreads))


def num_threads() -> int:
    return int(lib().oracle_num_threads())
