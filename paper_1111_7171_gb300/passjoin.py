"""Thin Python binding of libpassjoin (the C ABI in include/passjoin.h).

Argument marshalling only: every step of the join runs in the library's CUDA
kernels.  PyTorch supplies device memory (the library's allocator callbacks
draw from torch's caching allocator) and the stream (torch's current stream
unless one is given).  There is no CPU fallback: if the library or a GPU is
missing, every call raises.

Strings can be given as
  * a list of ``bytes``;
  * ``(bytes_u8, offsets_u64)`` numpy arrays (host), or
  * ``(bytes_u8, offsets)`` torch CUDA tensors (uint8 and int64/uint64), which
    the library reads in place.

Results are numpy structured arrays with fields (a, b, ed) sorted by (a, b);
``DeviceResult`` keeps them in device memory.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libpassjoin.so")

PJ_OK, PJ_EINVAL, PJ_ENOMEM, PJ_ECUDA, PJ_ETIMEDOUT, PJ_ECANCELED = 0, -1, -2, -3, -4, -5
PJ_TAU_LIMIT = 32
PAIR_DTYPE = np.dtype([("a", np.uint32), ("b", np.uint32), ("ed", np.uint32)])
PARTITIONS = {"even": 0, "center": 1}  # pj_options.partition (PJ_PARTITION_EVEN / PJ_PARTITION_CENTER)


class PJError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str):
        super().__init__(f"{where}: {detail} (code {code})")
        self.code = code


class pj_strings(ctypes.Structure):
    _fields_ = [("bytes", ctypes.c_void_p), ("offsets", ctypes.c_void_p), ("n", ctypes.c_uint32),
                ("on_device", ctypes.c_int)]


class pj_stats(ctypes.Structure):
    _fields_ = [("lookups", ctypes.c_uint64), ("candidates", ctypes.c_uint64), ("accepted", ctypes.c_uint64),
                ("dp_cells", ctypes.c_uint64), ("fallback_pairs", ctypes.c_uint64), ("hits", ctypes.c_uint64),
                ("probe_ms", ctypes.c_float), ("verify_ms", ctypes.c_float), ("fallback_ms", ctypes.c_float),
                ("dedupe_ms", ctypes.c_float), ("partition_ms", ctypes.c_float), ("verify_block", ctypes.c_int32),
                ("warp_min_len", ctypes.c_int32), ("tune_ms", ctypes.c_float), ("verify_mode", ctypes.c_int32),
                ("pair_warp", ctypes.c_int32), ("filtered", ctypes.c_uint64),
                ("distinct_pairs", ctypes.c_uint64), ("graph_replay", ctypes.c_int32), ("graph_ms", ctypes.c_float),
                ("device_peak", ctypes.c_uint64), ("windows", ctypes.c_uint32),
                ("fused", ctypes.c_int32)]


class pj_result(ctypes.Structure):
    _fields_ = [("pairs", ctypes.c_void_p), ("count", ctypes.c_uint64), ("on_device", ctypes.c_int),
                ("stats", pj_stats), ("priv", ctypes.c_void_p)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class pj_options(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", ctypes.c_void_p),
                ("verify_mode", ctypes.c_int), ("results_on_device", ctypes.c_int), ("lazy_partitions", ctypes.c_int),
                ("autotune", ctypes.c_int), ("graph_joins", ctypes.c_int), ("device_budget", ctypes.c_uint64),
                ("autotune_cache", ctypes.c_char_p), ("partition", ctypes.c_int)]


class pj_server_options(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int), ("max_batch_queries", ctypes.c_uint32), ("max_batch_bytes", ctypes.c_uint64),
                ("bytes_per_query", ctypes.c_uint64), ("device_reserve", ctypes.c_uint64), ("use_plans", ctypes.c_int)]


class pj_plan_options(ctypes.Structure):
    _fields_ = [("max_queries", ctypes.c_uint32), ("max_bytes", ctypes.c_uint64), ("hits_capacity", ctypes.c_uint64),
                ("accepted_capacity", ctypes.c_uint64), ("pairs_capacity", ctypes.c_uint64)]


class pj_plan_info(ctypes.Structure):
    _fields_ = [("runs", ctypes.c_uint64), ("recaptures", ctypes.c_uint64), ("graph_nodes", ctypes.c_uint32),
                ("graph_kernels", ctypes.c_uint32), ("hits_capacity", ctypes.c_uint64),
                ("accepted_capacity", ctypes.c_uint64), ("pairs_capacity", ctypes.c_uint64),
                ("device_bytes", ctypes.c_uint64), ("host_bytes", ctypes.c_uint64)]


class pj_selection(ctypes.Structure):
    _fields_ = [("length_based", ctypes.c_uint64), ("shift_based", ctypes.c_uint64),
                ("position_aware", ctypes.c_uint64), ("multi_match", ctypes.c_uint64), ("groups", ctypes.c_uint64)]


class pj_calibration(ctypes.Structure):
    _fields_ = [("dp_cells_per_s", ctypes.c_double), ("int32_ops_per_s", ctypes.c_double),
                ("l2_read_bytes_per_s", ctypes.c_double),
                ("sm_mhz", ctypes.c_double), ("sm_count", ctypes.c_int32)]


class pj_request_times(ctypes.Structure):
    _fields_ = [("queue_ms", ctypes.c_float), ("service_ms", ctypes.c_float), ("batch_requests", ctypes.c_uint32)]


class pj_server_counters(ctypes.Structure):
    _fields_ = [("requests", ctypes.c_uint64), ("batches", ctypes.c_uint64), ("queries", ctypes.c_uint64),
                ("max_batch_requests", ctypes.c_uint64), ("max_in_flight", ctypes.c_uint32),
                ("pending", ctypes.c_uint64)]


_lib = None
_lib_lock = threading.Lock()


def library():
    """Load libpassjoin.so (raises if it has not been built)."""
    global _lib
    with _lib_lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libpassjoin.so is not built ({LIB_PATH}); run "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = ctypes.CDLL(LIB_PATH)
            P = ctypes.POINTER
            L.pj_options_init.argtypes = [P(pj_options)]
            L.pj_options_init.restype = None
            L.pj_build_index.argtypes = [P(pj_strings), ctypes.c_int, P(pj_options), P(ctypes.c_void_p)]
            L.pj_build_index.restype = ctypes.c_int
            L.pj_self_join.argtypes = [ctypes.c_void_p, ctypes.c_int, P(pj_result)]
            L.pj_self_join.restype = ctypes.c_int
            L.pj_join.argtypes = [P(pj_strings), P(pj_strings), ctypes.c_int, P(pj_options), P(pj_result)]
            L.pj_join.restype = ctypes.c_int
            L.pj_query.argtypes = [ctypes.c_void_p, P(pj_strings), ctypes.c_int, P(pj_result)]
            L.pj_query.restype = ctypes.c_int
            L.pj_result_free.argtypes = [P(pj_result)]
            L.pj_result_free.restype = None
            L.pj_index_free.argtypes = [ctypes.c_void_p]
            L.pj_index_free.restype = None
            L.pj_index_size.argtypes = [ctypes.c_void_p]
            L.pj_index_size.restype = ctypes.c_uint32
            L.pj_index_tau_max.argtypes = [ctypes.c_void_p]
            L.pj_index_tau_max.restype = ctypes.c_int
            L.pj_index_device_bytes.argtypes = [ctypes.c_void_p]
            L.pj_index_device_bytes.restype = ctypes.c_uint64
            L.pj_query_multi.argtypes = [ctypes.c_void_p, P(pj_strings), ctypes.c_void_p, P(pj_result)]
            L.pj_query_multi.restype = ctypes.c_int
            L.pj_server_options_init.argtypes = [P(pj_server_options)]
            L.pj_server_options_init.restype = None
            L.pj_server_start.argtypes = [ctypes.c_void_p, P(pj_server_options), P(ctypes.c_void_p)]
            L.pj_server_start.restype = ctypes.c_int
            L.pj_server_submit.argtypes = [ctypes.c_void_p, P(pj_strings), ctypes.c_int, P(ctypes.c_uint64)]
            L.pj_server_submit.restype = ctypes.c_int
            L.pj_server_wait.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, P(pj_result),
                                         P(pj_request_times)]
            L.pj_server_wait.restype = ctypes.c_int
            L.pj_server_cancel.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
            L.pj_server_cancel.restype = ctypes.c_int
            L.pj_server_stats.argtypes = [ctypes.c_void_p, P(pj_server_counters)]
            L.pj_server_stats.restype = ctypes.c_int
            L.pj_server_stop.argtypes = [ctypes.c_void_p]
            L.pj_server_stop.restype = None
            L.pj_query_noalloc.argtypes = [ctypes.c_void_p, P(pj_strings), ctypes.c_int, ctypes.c_void_p,
                                           ctypes.c_uint64, P(ctypes.c_uint64)]
            L.pj_query_noalloc.restype = ctypes.c_int
            L.pj_plan_options_init.argtypes = [P(pj_plan_options)]
            L.pj_plan_options_init.restype = None
            L.pj_plan_create.argtypes = [ctypes.c_void_p, P(pj_plan_options), P(ctypes.c_void_p)]
            L.pj_plan_create.restype = ctypes.c_int
            L.pj_plan_query.argtypes = [ctypes.c_void_p, P(pj_strings), ctypes.c_void_p, P(pj_result)]
            L.pj_plan_query.restype = ctypes.c_int
            L.pj_plan_get_info.argtypes = [ctypes.c_void_p, P(pj_plan_info)]
            L.pj_plan_get_info.restype = ctypes.c_int
            L.pj_plan_free.argtypes = [ctypes.c_void_p]
            L.pj_plan_free.restype = None
            L.pj_self_join_shard.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32,
                                             P(pj_result)]
            L.pj_self_join_shard.restype = ctypes.c_int
            L.pj_self_join_stream.argtypes = [P(pj_strings), ctypes.c_int, P(pj_options), P(pj_result)]
            L.pj_self_join_stream.restype = ctypes.c_int
            L.pj_calibrate.argtypes = [P(pj_calibration)]
            L.pj_calibrate.restype = ctypes.c_int
            L.pj_count_selection.argtypes = [ctypes.c_void_p, ctypes.c_int, P(pj_selection)]
            L.pj_count_selection.restype = ctypes.c_int
            L.pj_index_build_ms.argtypes = [ctypes.c_void_p]
            L.pj_index_build_ms.restype = ctypes.c_float
            L.pj_kernel_launches.argtypes = []
            L.pj_kernel_launches.restype = ctypes.c_uint64
            L.pj_strerror.argtypes = [ctypes.c_int]
            L.pj_strerror.restype = ctypes.c_char_p
            L.pj_last_error.argtypes = []
            L.pj_last_error.restype = ctypes.c_char_p
            _lib = L
    return _lib


def _check(code: int, where: str):
    if code != PJ_OK:
        L = library()
        raise PJError(code, where, f"{L.pj_strerror(code).decode()}: {L.pj_last_error().decode()}")


# ------------------------------------------------------------- allocator --

def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libpassjoin needs a CUDA GPU; torch.cuda.is_available() is False")
    return torch


_LOG_ALLOC = bool(os.environ.get("PJ_LOG_ALLOC"))


@ALLOC_FN
def _torch_alloc(ctx, nbytes, stream):
    try:
        import torch
        ptr = torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), stream or 0)
        if _LOG_ALLOC:
            print(f"[alloc] {ptr:#x} {int(nbytes)} stream={stream}", flush=True)
        return ptr
    except Exception:  # reported to the caller as PJ_ENOMEM
        return None


@FREE_FN
def _torch_free(ctx, ptr, stream):
    import torch
    if _LOG_ALLOC:
        print(f"[free]  {ptr:#x}", flush=True)
    torch.cuda.caching_allocator_delete(ptr)


def make_options(stream=None, results_on_device: bool = False, torch_allocator: bool = True,
                 lazy_partitions: bool = False, autotune: bool = False, graph_joins: bool = False,
                 device_budget: int = 0, autotune_cache: str | None = None,
                 partition: str = "even") -> pj_options:
    torch = _torch()
    opt = pj_options()
    library().pj_options_init(ctypes.byref(opt))
    if stream is None:
        stream = torch.cuda.current_stream()
    opt.stream = ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream) or 0))
    if torch_allocator:
        opt.alloc = _torch_alloc
        opt.free = _torch_free
    opt.results_on_device = 1 if results_on_device else 0
    opt.lazy_partitions = 1 if lazy_partitions else 0
    opt.autotune = 1 if autotune else 0
    opt.graph_joins = 1 if graph_joins else 0
    opt.device_budget = int(device_budget)
    # the library copies the path at pj_build_index; the bytes object lives
    # as long as the options
    opt.autotune_cache = os.fsencode(autotune_cache) if autotune_cache else None
    opt.partition = PARTITIONS[partition]
    return opt


# --------------------------------------------------------------- strings --

class Strings:
    """Marshalled pj_strings plus the buffers that back it."""

    def __init__(self, data):
        self._keep = []
        s = pj_strings()
        if isinstance(data, (list, tuple)) and (len(data) == 0 or isinstance(data[0], (bytes, bytearray))) \
                and not (isinstance(data, tuple) and len(data) == 2 and hasattr(data[0], "dtype")):
            lens = np.fromiter((len(x) for x in data), dtype=np.uint64, count=len(data))
            off = np.zeros(len(data) + 1, dtype=np.uint64)
            np.cumsum(lens, out=off[1:])
            buf = np.frombuffer(b"".join(data), dtype=np.uint8) if len(data) else np.zeros(0, np.uint8)
            self._host(s, buf, off)
        elif isinstance(data, tuple) and len(data) == 2:
            b, o = data
            if hasattr(b, "is_cuda") and b.is_cuda:
                if o.numel() != 0 and not o.is_cuda:
                    raise ValueError("device bytes need device offsets")
                b = b.contiguous()
                o = o.contiguous()
                self._keep += [b, o]
                s.bytes = ctypes.c_void_p(b.data_ptr() if b.numel() else 0)
                s.offsets = ctypes.c_void_p(o.data_ptr())
                s.n = o.numel() - 1
                s.on_device = 1
            else:
                self._host(s, np.asarray(b, dtype=np.uint8), np.asarray(o, dtype=np.uint64))
        else:
            raise TypeError("strings must be a list of bytes or a (bytes, offsets) pair")
        self.c = s
        self.n = int(s.n)

    def _host(self, s, buf, off):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        if buf.size == 0:
            buf = np.zeros(1, np.uint8)
        off = np.ascontiguousarray(off, dtype=np.uint64)
        self._keep += [buf, off]
        s.bytes = ctypes.c_void_p(buf.ctypes.data)
        s.offsets = ctypes.c_void_p(off.ctypes.data)
        s.n = len(off) - 1
        s.on_device = 0


# ---------------------------------------------------------------- results --

class JoinResult:
    """Host result: ``pairs`` (structured a, b, ed) and ``stats`` (dict)."""

    def __init__(self, pairs: np.ndarray, stats: dict):
        self.pairs = pairs
        self.stats = stats

    def __len__(self):
        return len(self.pairs)


class _DeviceBytes:
    """__cuda_array_interface__ view of a raw device byte range."""

    def __init__(self, ptr: int, nbytes: int):
        self.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (ptr, False),
                                         "version": 3, "strides": None}


class DeviceResult:
    """Result left in device memory; ``count``, ``stats``, ``to_host()``, ``free()``."""

    def __init__(self, res: pj_result):
        self._res = res
        self.count = int(res.count)
        self.stats = _stats(res.stats)
        self.ptr = int(res.pairs or 0)

    def tensor(self):
        """The pairs as a uint8 torch CUDA tensor view (count * 12 bytes)."""
        torch = _torch()
        return torch.as_tensor(_DeviceBytes(self.ptr, self.count * PAIR_DTYPE.itemsize), device="cuda")

    def to_host(self) -> np.ndarray:
        if self.count == 0:
            return np.zeros(0, dtype=PAIR_DTYPE)
        return self.tensor().cpu().numpy().view(PAIR_DTYPE).copy()

    def free(self):
        if self._res is not None:
            library().pj_result_free(ctypes.byref(self._res))
            self._res = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _stats(st: pj_stats) -> dict:
    return dict(lookups=int(st.lookups), candidates=int(st.candidates), accepted=int(st.accepted),
                dp_cells=int(st.dp_cells), fallback_pairs=int(st.fallback_pairs), hits=int(st.hits),
                probe_ms=float(st.probe_ms), verify_ms=float(st.verify_ms), fallback_ms=float(st.fallback_ms),
                dedupe_ms=float(st.dedupe_ms), partition_ms=float(st.partition_ms),
                verify_block=int(st.verify_block), warp_min_len=int(st.warp_min_len), tune_ms=float(st.tune_ms),
                verify_mode=int(st.verify_mode), pair_warp=int(st.pair_warp), filtered=int(st.filtered),
                distinct_pairs=int(st.distinct_pairs), graph_replay=int(st.graph_replay),
                graph_ms=float(st.graph_ms), device_peak=int(st.device_peak), windows=int(st.windows),
                fused=int(st.fused))


class _HostPairs:
    """Owner of a host pj_result whose pairs a numpy array views without a
    copy; pj_result_free runs when the last view is gone."""

    def __init__(self, res: pj_result):
        self.res = res

    def __del__(self):
        try:
            library().pj_result_free(ctypes.byref(self.res))
        except Exception:
            pass


def _take(res: pj_result):
    if res.on_device:
        return DeviceResult(res)
    n = int(res.count)
    stats = _stats(res.stats)
    if n:
        raw = (ctypes.c_uint8 * (n * PAIR_DTYPE.itemsize)).from_address(res.pairs)
        raw._owner = _HostPairs(res)  # the library's buffer lives as long as the array
        pairs = np.frombuffer(raw, dtype=PAIR_DTYPE)
    else:
        pairs = np.zeros(0, dtype=PAIR_DTYPE)
        library().pj_result_free(ctypes.byref(res))
    return JoinResult(pairs, stats)


# ----------------------------------------------------------------- index --

class Index:
    """A resident segment index (pj_index*)."""

    def __init__(self, handle, options, strings_keepalive):
        self._h = handle
        self._opt = options
        self._keep = strings_keepalive

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("index already freed")
        return self._h

    @property
    def n(self) -> int:
        return int(library().pj_index_size(self.handle))

    @property
    def tau_max(self) -> int:
        return int(library().pj_index_tau_max(self.handle))

    @property
    def device_bytes(self) -> int:
        return int(library().pj_index_device_bytes(self.handle))

    @property
    def build_ms(self) -> float:
        return float(library().pj_index_build_ms(self.handle))

    def free(self):
        if self._h:
            library().pj_index_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# ------------------------------------------------------------ entry points --

def pj_kernel_launches() -> int:
    """pj_kernel_launches: kernels launched by the library since it was loaded."""
    return int(library().pj_kernel_launches())


def pj_build_index(strings, tau_max: int, stream=None, results_on_device: bool = False,
                   lazy_partitions: bool = False, autotune: bool = False, graph_joins: bool = False,
                   device_budget: int = 0, autotune_cache: str | None = None, partition: str = "even") -> Index:
    """pj_build_index: resident segment index for thresholds 0..tau_max.

    results_on_device: results stay in device memory (DeviceResult).
    lazy_partitions: a threshold's segment index is built on its first use.
    autotune: each threshold's self join picks its verification form by timing.
    graph_joins: after a threshold's first self join, later self joins of it
    replay that join recorded as one CUDA graph (pj_options.graph_joins).
    device_budget: most device bytes the index and its calls may hold at once
    (0 = no limit; beyond it a call fails with PJ_ENOMEM).
    autotune_cache: file keeping autotuning decisions across processes.
    partition: "even" (the paper's even partition) or "center" (the longer
    segments in the middle; same results)."""
    opt = make_options(stream, results_on_device, lazy_partitions=lazy_partitions, autotune=autotune,
                       graph_joins=graph_joins, device_budget=device_budget, autotune_cache=autotune_cache,
                       partition=partition)
    S = Strings(strings)
    h = ctypes.c_void_p()
    _check(library().pj_build_index(ctypes.byref(S.c), int(tau_max), ctypes.byref(opt), ctypes.byref(h)),
           "pj_build_index")
    return Index(h, opt, None)


def pj_self_join(index: Index, tau: int):
    """pj_self_join: all pairs a < b of the indexed set with ED <= tau."""
    res = pj_result()
    _check(library().pj_self_join(index.handle, int(tau), ctypes.byref(res)), "pj_self_join")
    return _take(res)


def pj_calibrate() -> dict:
    """pj_calibrate: measured DP-cell rate, int32 throughput, L2 read
    bandwidth and SM clock of the current device (the rooflines' ceilings)."""
    _torch()
    out = pj_calibration()
    _check(library().pj_calibrate(ctypes.byref(out)), "pj_calibrate")
    return {f: (int(getattr(out, f)) if f == "sm_count" else float(getattr(out, f))) for f, _ in pj_calibration._fields_}


def pj_count_selection(index: Index, tau: int) -> dict:
    """pj_count_selection: substrings each selection method of Sec. 4 would
    look up over the self join at threshold tau (length-based, shift-based,
    position-aware, multi-match-aware) and the groups counted."""
    out = pj_selection()
    _check(library().pj_count_selection(index.handle, int(tau), ctypes.byref(out)), "pj_count_selection")
    return {f: int(getattr(out, f)) for f, _ in pj_selection._fields_}


def pj_self_join_shard(index: Index, tau: int, shard: int, n_shards: int):
    """pj_self_join_shard: the part of pj_self_join whose later string (in
    Alg. 1's visiting order) is among shard `shard` of `n_shards` equal probe
    ranges; the shards are disjoint and together give the whole join."""
    res = pj_result()
    _check(library().pj_self_join_shard(index.handle, int(tau), int(shard), int(n_shards), ctypes.byref(res)),
           "pj_self_join_shard")
    return _take(res)


def pj_self_join_stream(strings, tau: int, device_budget: int = 0, stream=None, autotune: bool = False,
                        partition: str = "even"):
    """pj_self_join_stream: the self join of host strings, window by window of
    lengths, holding at most `device_budget` device bytes at once (0 = three
    quarters of the free device memory).  Host result."""
    opt = make_options(stream, autotune=autotune, device_budget=device_budget, partition=partition)
    S = Strings(strings)
    res = pj_result()
    _check(library().pj_self_join_stream(ctypes.byref(S.c), int(tau), ctypes.byref(opt), ctypes.byref(res)),
           "pj_self_join_stream")
    return _take(res)


def pj_join(R, S, tau: int, stream=None, results_on_device: bool = False, device_budget: int = 0,
            partition: str = "even"):
    """pj_join: all (a in R, b in S) with ED <= tau."""
    opt = make_options(stream, results_on_device, device_budget=device_budget, partition=partition)
    r, s = Strings(R), Strings(S)
    res = pj_result()
    _check(library().pj_join(ctypes.byref(r.c), ctypes.byref(s.c), int(tau), ctypes.byref(opt), ctypes.byref(res)),
           "pj_join")
    return _take(res)


def pj_query(index: Index, batch, tau: int):
    """pj_query: (query position, indexed id) pairs with ED <= tau."""
    b = Strings(batch)
    res = pj_result()
    _check(library().pj_query(index.handle, ctypes.byref(b.c), int(tau), ctypes.byref(res)), "pj_query")
    return _take(res)


def pj_query_noalloc(index: Index, batch, tau: int, out_pairs, out_cap: int) -> int:
    """pj_query_noalloc: probe a device-resident batch into a caller-owned
    device buffer (``out_pairs``: a CUDA tensor or a device address holding
    ``out_cap`` pj_pair entries) without allocating.  Returns the pair count."""
    b = Strings(batch)
    ptr = out_pairs.data_ptr() if hasattr(out_pairs, "data_ptr") else int(out_pairs)
    n = ctypes.c_uint64(0)
    _check(library().pj_query_noalloc(index.handle, ctypes.byref(b.c), int(tau), ctypes.c_void_p(ptr),
                                      int(out_cap), ctypes.byref(n)), "pj_query_noalloc")
    return int(n.value)


def pj_query_multi(index: Index, batch, taus):
    """pj_query_multi: one batched probe where query q uses threshold taus[q]."""
    b = Strings(batch)
    t = np.ascontiguousarray(np.asarray(taus, dtype=np.uint8))
    if len(t) != b.n:
        raise ValueError("one threshold per query")
    res = pj_result()
    _check(library().pj_query_multi(index.handle, ctypes.byref(b.c), ctypes.c_void_p(t.ctypes.data if len(t) else 0),
                                    ctypes.byref(res)), "pj_query_multi")
    return _take(res)


class Plan:
    """pj_plan_*: the multi-threshold query pipeline recorded into a CUDA
    graph, replayed once per batch of host strings."""

    def __init__(self, index: Index, max_queries: int = 4096, max_bytes: int = 1 << 20, hits_capacity: int = 0,
                 accepted_capacity: int = 0, pairs_capacity: int = 0):
        _torch()
        L = library()
        o = pj_plan_options()
        L.pj_plan_options_init(ctypes.byref(o))
        o.max_queries, o.max_bytes = max_queries, max_bytes
        o.hits_capacity, o.accepted_capacity, o.pairs_capacity = hits_capacity, accepted_capacity, pairs_capacity
        h = ctypes.c_void_p()
        _check(L.pj_plan_create(index.handle, ctypes.byref(o), ctypes.byref(h)), "pj_plan_create")
        self._h = h
        self._index = index

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("plan already freed")
        return self._h

    def query(self, batch, taus):
        """pj_plan_query: host batch, query q at threshold taus[q] (an int
        applies to every query)."""
        b = Strings(batch)
        if np.isscalar(taus):
            taus = np.full(b.n, int(taus), dtype=np.uint8)
        t = np.ascontiguousarray(np.asarray(taus, dtype=np.uint8))
        if len(t) != b.n:
            raise ValueError("one threshold per query")
        res = pj_result()
        _check(library().pj_plan_query(self.handle, ctypes.byref(b.c), ctypes.c_void_p(t.ctypes.data if len(t) else 0),
                                       ctypes.byref(res)), "pj_plan_query")
        return _take(res)

    def info(self) -> dict:
        i = pj_plan_info()
        _check(library().pj_plan_get_info(self.handle, ctypes.byref(i)), "pj_plan_get_info")
        return {f: int(getattr(i, f)) for f, _ in pj_plan_info._fields_}

    def free(self):
        if self._h:
            library().pj_plan_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Server:
    """pj_server_*: continuous-batching query server over a resident index."""

    def __init__(self, index: Index, slots: int = 3, max_batch_queries: int = 1 << 16,
                 max_batch_bytes: int = 16 << 20, bytes_per_query: int = 64 << 10, device_reserve: int = 2 << 30,
                 use_plans: bool = False):
        _torch()
        L = library()
        o = pj_server_options()
        L.pj_server_options_init(ctypes.byref(o))
        o.slots, o.max_batch_queries, o.max_batch_bytes = slots, max_batch_queries, max_batch_bytes
        o.bytes_per_query, o.device_reserve = bytes_per_query, device_reserve
        o.use_plans = 1 if use_plans else 0
        h = ctypes.c_void_p()
        _check(L.pj_server_start(index.handle, ctypes.byref(o), ctypes.byref(h)), "pj_server_start")
        self._h = h
        self._index = index

    def submit(self, strings, tau: int) -> int:
        s = Strings(strings)
        t = ctypes.c_uint64(0)
        _check(library().pj_server_submit(self._h, ctypes.byref(s.c), int(tau), ctypes.byref(t)), "pj_server_submit")
        return int(t.value)

    def wait(self, ticket: int, timeout_ms: int = -1):
        """Returns (JoinResult, times dict); raises PJError (code PJ_ETIMEDOUT,
        PJ_ECANCELED, ...) otherwise."""
        res = pj_result()
        tm = pj_request_times()
        _check(library().pj_server_wait(self._h, int(ticket), int(timeout_ms), ctypes.byref(res), ctypes.byref(tm)),
               "pj_server_wait")
        times = dict(queue_ms=float(tm.queue_ms), service_ms=float(tm.service_ms),
                     batch_requests=int(tm.batch_requests))
        return _take(res), times

    def cancel(self, ticket: int):
        _check(library().pj_server_cancel(self._h, int(ticket)), "pj_server_cancel")

    def stats(self) -> dict:
        c = pj_server_counters()
        _check(library().pj_server_stats(self._h, ctypes.byref(c)), "pj_server_stats")
        return {f: int(getattr(c, f)) for f, _ in pj_server_counters._fields_}

    def stop(self):
        if self._h:
            library().pj_server_stop(self._h)
            self._h = None

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass
