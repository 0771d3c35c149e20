"""Python binding of libkc.so (include/kclique.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
graph work of its own: the path runs in the library's CUDA kernels.  PyTorch
is used only for device memory and streams (tensors on the GPU are passed as
raw device pointers).  If libkc.so cannot be built or loaded, ``load()``
raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from functools import lru_cache

import numpy as np

from . import build as _build

KC_OK = 0
KC_E_INVALID_ARG = 1
KC_E_INVALID_GRAPH = 2
KC_E_OOM = 3
KC_E_CAPACITY = 4
KC_E_DEVICE_TIMEOUT = 5
KC_E_CUDA = 6
KC_E_BUSY = 7
KC_E_UNSUPPORTED = 8
KC_E_NOT_FOUND = 9

KC_HOST_PTRS = 0x1
KC_DEVICE_PTRS = 0x2
KC_CANONICALIZE = 0x4

KC_MAX_K = 64
KC_MAX_OUTDEG = 1024

# Every entry point include/kclique.h declares (checked by the CPU tests).
EXPORTS = (
    "kc_create", "kc_destroy", "kc_upload", "kc_free_graph", "kc_graph_info_get", "kc_export_dag",
    "kc_count", "kc_list", "kc_list_range", "kc_last_stats", "kc_last_upload_stats", "kc_strerror",
    "kc_last_error", "kc_count_dag_noalloc", "kc_count_batched", "kc_serve_start", "kc_serve_submit",
    "kc_serve_submit_csr", "kc_serve_poll", "kc_serve_wait", "kc_serve_stats_get", "kc_serve_stop",
    "kc_tune",
)

KC_SERVE_COUNT = 0
KC_SERVE_LIST = 1

KC_NODE_PARALLEL = 0
KC_EDGE_PARALLEL = 1


class KcError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        name = kc_strerror(status) if status else "KC_OK"
        super().__init__(f"{what}: {name}" if what else name)


class kc_opts(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("no_memo", ctypes.c_uint32),
        ("no_prune", ctypes.c_uint32),
        ("split_threshold", ctypes.c_uint32),
        ("memo_bytes", ctypes.c_uint64),
        ("spin_limit", ctypes.c_uint64),
        ("decomposition", ctypes.c_uint32),
        ("autotune", ctypes.c_uint32),
        ("tune_cache", ctypes.c_char_p),
        ("no_plex", ctypes.c_uint32),
        ("memo_min_k", ctypes.c_uint32),
    ]


class kc_tune_result(ctypes.Structure):
    _fields_ = [
        ("split_threshold", ctypes.c_uint32),
        ("warps_small", ctypes.c_uint32),
        ("warps_large", ctypes.c_uint32),
        ("probes", ctypes.c_uint32),
        ("memo_bytes", ctypes.c_uint64),
        ("ms_default", ctypes.c_float),
        ("ms_tuned", ctypes.c_float),
        ("cached", ctypes.c_uint32),
        ("key", ctypes.c_char * 116),
    ]


class kc_graph_info(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_uint32),
        ("degeneracy", ctypes.c_uint32),
        ("m", ctypes.c_uint64),
        ("max_out_degree", ctypes.c_uint32),
        ("peel_rounds", ctypes.c_uint32),
    ]


class kc_stats(ctypes.Structure):
    _fields_ = [
        ("ms_bin", ctypes.c_float),
        ("ms_enum", ctypes.c_float),
        ("ms_total", ctypes.c_float),
        ("enum_launches", ctypes.c_uint32),
        ("total_launches", ctypes.c_uint32),
        ("roots_total", ctypes.c_uint64),
        ("roots_pruned", ctypes.c_uint64),
        ("roots_heavy", ctypes.c_uint64),
        ("build_words", ctypes.c_uint64),
        ("memo_hits", ctypes.c_uint64),
        ("memo_inserts", ctypes.c_uint64),
        ("memo_full", ctypes.c_uint64),
        ("memo_frames", ctypes.c_uint64),
        ("ms_tier", ctypes.c_float * 6),
        ("roots_tier", ctypes.c_uint32 * 6),
        ("word_ops", ctypes.c_uint64),
        ("warp_ns_build", ctypes.c_uint64),
        ("warp_ns_busy", ctypes.c_uint64),
        ("memo_peak", ctypes.c_uint64),
        ("plex_frames", ctypes.c_uint64),
    ]


class kc_upload_stats(ctypes.Structure):
    _fields_ = [
        ("ms_copy", ctypes.c_float),
        ("ms_canon", ctypes.c_float),
        ("ms_peel", ctypes.c_float),
        ("ms_orient", ctypes.c_float),
        ("ms_total", ctypes.c_float),
        ("launches", ctypes.c_uint32),
    ]


class kc_serve_opts(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("lanes", ctypes.c_uint32),
        ("max_batch", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32),
        ("mem_cap_bytes", ctypes.c_uint64),
    ]


class kc_serve_result(ctypes.Structure):
    _fields_ = [
        ("count", ctypes.c_uint64),
        ("status", ctypes.c_int32),
        ("batch_size", ctypes.c_uint32),
        ("t_submit_ns", ctypes.c_uint64),
        ("t_start_ns", ctypes.c_uint64),
        ("t_done_ns", ctypes.c_uint64),
        ("checksum", ctypes.c_uint64),
        ("mode", ctypes.c_uint32),
        ("enumerated", ctypes.c_uint32),
    ]


class kc_serve_stats(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_uint64),
        ("completed", ctypes.c_uint64),
        ("failed", ctypes.c_uint64),
        ("batches", ctypes.c_uint64),
        ("p50_ms", ctypes.c_double),
        ("p99_ms", ctypes.c_double),
        ("mean_batch", ctypes.c_double),
        ("req_per_s", ctypes.c_double),
        ("cliques_per_s", ctypes.c_double),
        ("peak_reserved_bytes", ctypes.c_uint64),
        ("p50_enum_ms", ctypes.c_double),
        ("p99_enum_ms", ctypes.c_double),
        ("lane_scratch_bytes", ctypes.c_uint64),
    ]


def _struct_dict(s) -> dict:
    out = {}
    for name, _ in s._fields_:
        v = getattr(s, name)
        out[name] = list(v) if isinstance(v, ctypes.Array) else v
    return out


@lru_cache(maxsize=1)
def load(path: str | None = None) -> ctypes.CDLL:
    """Load libkc.so (building it first if the sources changed; KC_LIBRARY names another build)."""
    path = path or os.environ.get("KC_LIBRARY") or _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libkc.so missing at {path}")
    lib = ctypes.CDLL(path)
    P, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    pu64 = ctypes.POINTER(u64)
    sig = {
        "kc_create": (i32, [ctypes.POINTER(P), i32, ctypes.POINTER(kc_opts)]),
        "kc_destroy": (i32, [P]),
        "kc_upload": (i32, [P, u32, P, P, u32, ctypes.POINTER(u32), P]),
        "kc_free_graph": (i32, [P, u32]),
        "kc_graph_info_get": (i32, [P, u32, ctypes.POINTER(kc_graph_info)]),
        "kc_export_dag": (i32, [P, u32, P, P, P, P]),
        "kc_count": (i32, [P, u32, u32, pu64, P]),
        "kc_list": (i32, [P, u32, u32, P, u64, pu64, pu64, pu64, P]),
        "kc_list_range": (i32, [P, u32, u32, u32, u32, P, u64, pu64, pu64, pu64, P]),
        "kc_last_stats": (i32, [P, ctypes.POINTER(kc_stats)]),
        "kc_last_upload_stats": (i32, [P, ctypes.POINTER(kc_upload_stats)]),
        "kc_strerror": (ctypes.c_char_p, [i32]),
        "kc_last_error": (ctypes.c_char_p, [P]),
        "kc_count_dag_noalloc": (i32, [u32, P, P, u32, pu64, P]),
        "kc_count_batched": (i32, [P, P, P, u32, P, P]),
        "kc_serve_start": (i32, [P, ctypes.POINTER(kc_serve_opts)]),
        "kc_serve_submit": (i32, [P, u32, u32, u32, pu64]),
        "kc_serve_submit_csr": (i32, [P, u32, P, P, u32, u32, u32, pu64]),
        "kc_serve_poll": (i32, [P, u64, ctypes.POINTER(kc_serve_result)]),
        "kc_serve_wait": (i32, [P, u64, ctypes.c_int64, ctypes.POINTER(kc_serve_result)]),
        "kc_serve_stats_get": (i32, [P, ctypes.POINTER(kc_serve_stats)]),
        "kc_serve_stop": (i32, [P]),
        "kc_tune": (i32, [P, P, P, u32, ctypes.POINTER(kc_tune_result)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


def _check(st: int, what: str):
    if st != KC_OK:
        raise KcError(st, what)


def _ptr(x):
    """Raw pointer of a numpy array (host) or a torch tensor (host or device)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(x.data_ptr())


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


# ------------------------------------------------------- C-ABI mirror
def kc_strerror(status: int) -> str:
    return load().kc_strerror(int(status)).decode()


def kc_create(device: int = 0, no_memo: bool = False, no_prune: bool = False, memo_bytes: int = 0,
              spin_limit: int = 0, split_threshold: int = 0, decomposition: int = 0, autotune: bool = False,
              tune_cache: str | None = None, no_plex: bool = False, memo_min_k: int = 0) -> int:
    o = kc_opts(ctypes.sizeof(kc_opts), int(no_memo), int(no_prune), int(split_threshold), int(memo_bytes),
                int(spin_limit), int(decomposition), int(autotune), tune_cache.encode() if tune_cache else None,
                int(no_plex), int(memo_min_k))
    h = ctypes.c_void_p()
    _check(load().kc_create(ctypes.byref(h), int(device), ctypes.byref(o)), "kc_create")
    return h.value


def kc_destroy(ctx: int) -> None:
    _check(load().kc_destroy(ctypes.c_void_p(ctx)), "kc_destroy")


def kc_upload(ctx: int, n: int, rowptr, col, flags: int, stream=None) -> int:
    g = ctypes.c_uint32(0)
    st = load().kc_upload(ctypes.c_void_p(ctx), int(n), _ptr(rowptr), _ptr(col), int(flags), ctypes.byref(g),
                          _stream(stream))
    _check(st, "kc_upload")
    return int(g.value)


def kc_free_graph(ctx: int, g: int) -> None:
    _check(load().kc_free_graph(ctypes.c_void_p(ctx), int(g)), "kc_free_graph")


def kc_graph_info_get(ctx: int, g: int) -> dict:
    info = kc_graph_info()
    _check(load().kc_graph_info_get(ctypes.c_void_p(ctx), int(g), ctypes.byref(info)), "kc_graph_info_get")
    return _struct_dict(info)


def kc_export_dag(ctx: int, g: int):
    info = kc_graph_info_get(ctx, g)
    n, m = info["n"], info["m"]
    core = np.zeros(max(n, 1), dtype=np.uint32)
    rank = np.zeros(max(n, 1), dtype=np.uint32)
    orow = np.zeros(n + 1, dtype=np.uint64)
    ocol = np.zeros(max(m, 1), dtype=np.uint32)
    _check(load().kc_export_dag(ctypes.c_void_p(ctx), int(g), _ptr(core), _ptr(rank), _ptr(orow), _ptr(ocol)),
           "kc_export_dag")
    return core[:n], rank[:n], orow, ocol[:m]


def kc_count(ctx: int, g: int, k: int, stream=None) -> int:
    c = ctypes.c_uint64(0)
    _check(load().kc_count(ctypes.c_void_p(ctx), int(g), int(k), ctypes.byref(c), _stream(stream)), "kc_count")
    return int(c.value)


def kc_list(ctx: int, g: int, k: int, d_buf=None, cap: int = 0, stream=None, allow_capacity: bool = False):
    """Returns (written, total, checksum); d_buf is a device tensor of >= cap*k 32-bit ints."""
    w, t, s = ctypes.c_uint64(0), ctypes.c_uint64(0), ctypes.c_uint64(0)
    st = load().kc_list(ctypes.c_void_p(ctx), int(g), int(k), _ptr(d_buf), int(cap), ctypes.byref(w), ctypes.byref(t),
                        ctypes.byref(s), _stream(stream))
    if not (allow_capacity and st == KC_E_CAPACITY):
        _check(st, "kc_list")
    return int(w.value), int(t.value), int(s.value)


def kc_list_range(ctx: int, g: int, k: int, root_lo: int, root_hi: int, d_buf=None, cap: int = 0, stream=None,
                  allow_capacity: bool = False):
    w, t, s = ctypes.c_uint64(0), ctypes.c_uint64(0), ctypes.c_uint64(0)
    st = load().kc_list_range(ctypes.c_void_p(ctx), int(g), int(k), int(root_lo), int(root_hi), _ptr(d_buf), int(cap),
                              ctypes.byref(w), ctypes.byref(t), ctypes.byref(s), _stream(stream))
    if not (allow_capacity and st == KC_E_CAPACITY):
        _check(st, "kc_list_range")
    return int(w.value), int(t.value), int(s.value)


def kc_last_stats(ctx: int) -> dict:
    s = kc_stats()
    _check(load().kc_last_stats(ctypes.c_void_p(ctx), ctypes.byref(s)), "kc_last_stats")
    return _struct_dict(s)


def kc_last_upload_stats(ctx: int) -> dict:
    s = kc_upload_stats()
    _check(load().kc_last_upload_stats(ctypes.c_void_p(ctx), ctypes.byref(s)), "kc_last_upload_stats")
    return _struct_dict(s)


def kc_count_batched(ctx: int, graphs, ks, stream=None) -> list[int]:
    """Counts of (graphs[i], ks[i]) for every i, in one batched enumeration."""
    g = np.ascontiguousarray(graphs, dtype=np.uint32)
    k = np.ascontiguousarray(ks, dtype=np.uint32)
    if g.shape != k.shape:
        raise ValueError("graphs and ks differ in length")
    out = np.zeros(max(g.size, 1), dtype=np.uint64)
    _check(load().kc_count_batched(ctypes.c_void_p(ctx), _ptr(g), _ptr(k), int(g.size), _ptr(out), _stream(stream)),
           "kc_count_batched")
    return [int(x) for x in out[: g.size]]


def kc_tune(ctx: int, graphs, ks) -> dict:
    """Times the batched count of (graphs[i], ks[i]) under candidate launch
    settings and applies the fastest to the context; returns the choice."""
    g = np.ascontiguousarray(graphs, dtype=np.uint32)
    k = np.ascontiguousarray(ks, dtype=np.uint32)
    if g.shape != k.shape:
        raise ValueError("graphs and ks differ in length")
    r = kc_tune_result()
    _check(load().kc_tune(ctypes.c_void_p(ctx), _ptr(g), _ptr(k), int(g.size), ctypes.byref(r)), "kc_tune")
    d = _struct_dict(r)
    d["key"] = r.key.decode()
    return d


def kc_serve_start(ctx: int, lanes: int = 0, max_batch: int = 0, mem_cap_bytes: int = 0) -> None:
    o = kc_serve_opts(ctypes.sizeof(kc_serve_opts), int(lanes), int(max_batch), 0, int(mem_cap_bytes))
    _check(load().kc_serve_start(ctypes.c_void_p(ctx), ctypes.byref(o)), "kc_serve_start")


def kc_serve_submit(ctx: int, g: int, k: int, mode: int = KC_SERVE_COUNT) -> int:
    t = ctypes.c_uint64(0)
    _check(load().kc_serve_submit(ctypes.c_void_p(ctx), int(g), int(k), int(mode), ctypes.byref(t)),
           "kc_serve_submit")
    return int(t.value)


def kc_serve_submit_csr(ctx: int, n: int, rowptr, col, k: int, canonicalize: bool = False,
                        mode: int = KC_SERVE_COUNT) -> int:
    rowptr = np.ascontiguousarray(rowptr, dtype=np.uint64)
    col = np.ascontiguousarray(col, dtype=np.uint32)
    t = ctypes.c_uint64(0)
    flags = KC_HOST_PTRS | (KC_CANONICALIZE if canonicalize else 0)
    _check(load().kc_serve_submit_csr(ctypes.c_void_p(ctx), int(n), _ptr(rowptr), _ptr(col) if col.size else None,
                                      flags, int(k), int(mode), ctypes.byref(t)), "kc_serve_submit_csr")
    return int(t.value)


def kc_serve_poll(ctx: int, ticket: int):
    """The request's result dict once complete, else None (queued or running)."""
    r = kc_serve_result()
    st = load().kc_serve_poll(ctypes.c_void_p(ctx), int(ticket), ctypes.byref(r))
    if st == KC_E_BUSY:
        return None
    _check(st, "kc_serve_poll")
    return _struct_dict(r)


def kc_serve_wait(ctx: int, ticket: int, timeout_ms: int = -1):
    r = kc_serve_result()
    st = load().kc_serve_wait(ctypes.c_void_p(ctx), int(ticket), int(timeout_ms), ctypes.byref(r))
    if st == KC_E_BUSY:
        return None
    _check(st, "kc_serve_wait")
    return _struct_dict(r)


def kc_serve_stats_get(ctx: int) -> dict:
    s = kc_serve_stats()
    _check(load().kc_serve_stats_get(ctypes.c_void_p(ctx), ctypes.byref(s)), "kc_serve_stats_get")
    return _struct_dict(s)


def kc_serve_stop(ctx: int) -> None:
    _check(load().kc_serve_stop(ctypes.c_void_p(ctx)), "kc_serve_stop")


def kc_count_dag_noalloc(n: int, d_orow, d_ocol, k: int, stream=None) -> int:
    """Count k-cliques of a device-resident rank-space DAG without any allocation
    inside the library (for callers that must not allocate); see kclique.h."""
    c = ctypes.c_uint64(0)
    _check(load().kc_count_dag_noalloc(int(n), _ptr(d_orow), _ptr(d_ocol), int(k), ctypes.byref(c), _stream(stream)),
           "kc_count_dag_noalloc")
    return int(c.value)


def kc_last_error(ctx: int) -> str:
    return load().kc_last_error(ctypes.c_void_p(ctx)).decode()


# ------------------------------------------------------- convenience
class Context:
    """Owns a kc_ctx; methods forward to the C entry points."""

    def __init__(self, device: int = 0, **opts):
        self.h = kc_create(device, **opts)

    def close(self):
        if self.h:
            kc_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def upload_host(self, n: int, rowptr: np.ndarray, col: np.ndarray, canonicalize: bool = False, stream=None) -> int:
        rowptr = np.ascontiguousarray(rowptr, dtype=np.uint64)
        col = np.ascontiguousarray(col, dtype=np.uint32)
        if col.size == 0:
            col = np.zeros(1, dtype=np.uint32)
        flags = KC_HOST_PTRS | (KC_CANONICALIZE if canonicalize else 0)
        return kc_upload(self.h, n, rowptr, col, flags, stream)

    def upload_device(self, n: int, rowptr, col, canonicalize: bool = False, stream=None) -> int:
        flags = KC_DEVICE_PTRS | (KC_CANONICALIZE if canonicalize else 0)
        return kc_upload(self.h, n, rowptr, col, flags, stream)

    def free(self, g: int):
        kc_free_graph(self.h, g)

    def info(self, g: int) -> dict:
        return kc_graph_info_get(self.h, g)

    def count(self, g: int, k: int, stream=None) -> int:
        return kc_count(self.h, g, k, stream)

    def list(self, g: int, k: int, d_buf=None, cap: int = 0, stream=None, allow_capacity: bool = False):
        return kc_list(self.h, g, k, d_buf, cap, stream, allow_capacity)

    def list_range(self, g: int, k: int, lo: int, hi: int, d_buf=None, cap: int = 0, stream=None,
                   allow_capacity: bool = False):
        return kc_list_range(self.h, g, k, lo, hi, d_buf, cap, stream, allow_capacity)

    def tune(self, graphs, ks) -> dict:
        return kc_tune(self.h, graphs, ks)

    def count_batched(self, graphs, ks, stream=None) -> list[int]:
        return kc_count_batched(self.h, graphs, ks, stream)

    def stats(self) -> dict:
        return kc_last_stats(self.h)

    def upload_stats(self) -> dict:
        return kc_last_upload_stats(self.h)

    def export_dag(self, g: int):
        return kc_export_dag(self.h, g)
