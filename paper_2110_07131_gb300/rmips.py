"""Thin Python binding of librmips (argument marshalling only).

Every step of the reverse k-MIPS path runs in the CUDA library; this module
only converts numpy arrays / torch tensors to pointers and sizes and calls the
C ABI declared in ``include/rmips.h``.  Importing it does not touch the GPU;
the library is built (if needed) and loaded on first use, and any failure to
build or load raises -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

__all__ = [
    "RmipsError", "Index", "load_library", "rmips_build_index", "rmips_query",
    "rmips_query_batch", "rmips_query_batch_async", "rmips_index_get_info", "rmips_last_query_stats",
    "rmips_index_save", "rmips_index_load", "rmips_index_rebuild", "rmips_topk_join",
    "rmips_index_export", "rmips_free_index", "rmips_status_string", "rmips_exact_sign_host",
    "rmips_profile_enable", "rmips_profile_read", "rmips_query_noalloc", "rmips_query_async", "rmips_index_tune", "EXPORTED_SYMBOLS",
    "FP32", "BF16", "FP16", "Server",
]

FP32, BF16, FP16 = 0, 1, 2
_PREC = {"fp32": FP32, "bf16": BF16, "fp16": FP16, FP32: FP32, BF16: BF16, FP16: FP16}

STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_K_RANGE", 3: "ERR_NONFINITE", 4: "ERR_OOM",
          5: "ERR_CAPACITY", 6: "ERR_TIMEOUT", 7: "ERR_CUDA", 8: "ERR_INTERNAL", 9: "ERR_BUSY"}

EXPORTED_SYMBOLS = [
    "rmips_build_index", "rmips_query", "rmips_query_batch", "rmips_query_batch_async", "rmips_index_get_info",
    "rmips_last_query_stats", "rmips_index_export", "rmips_free_index", "rmips_status_string",
    "rmips_last_error", "rmips_exact_sign_host", "rmips_profile_enable", "rmips_profile_read",
    "rmips_query_noalloc", "rmips_debug_tc_tile", "rmips_server_create", "rmips_server_submit",
    "rmips_server_submit_many", "rmips_server_wait", "rmips_server_wait_many", "rmips_server_get_stats",
    "rmips_server_destroy", "rmips_index_save", "rmips_index_load", "rmips_index_rebuild", "rmips_topk_join",
    "rmips_query_async", "rmips_index_tune", "rmips_server_add_segment",
]


class RmipsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class BuildOpts(C.Structure):
    _fields_ = [("k_max", C.c_int32), ("block_size", C.c_int32), ("p_prime", C.c_int64),
                ("precision", C.c_int32), ("flags", C.c_int32), ("tune_cache", C.c_char_p)]


class Segment(C.Structure):
    _fields_ = [("kind", C.c_int32), ("reserved", C.c_int32), ("begin", C.c_int64), ("end", C.c_int64),
                ("ids", C.POINTER(C.c_int64)), ("n_ids", C.c_int64)]


class IndexInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("m", C.c_int64), ("d", C.c_int32), ("k_max", C.c_int32),
                ("block_size", C.c_int32), ("precision", C.c_int32), ("n_blocks", C.c_int64),
                ("p_prime", C.c_int64), ("incomplete", C.c_int64), ("device_bytes", C.c_int64),
                ("build_ms", C.c_double), ("tuned", C.c_int32), ("batch_stages", C.c_int32),
                ("single_stages", C.c_int32), ("build_kind", C.c_int32), ("tune_ms", C.c_double)]


class Profile(C.Structure):
    _fields_ = [("filter_launches", C.c_int64), ("filter_ms", C.c_double), ("filter_alg_bytes", C.c_double),
                ("users_tested", C.c_int64), ("blocks_pruned", C.c_int64), ("blocks_total", C.c_int64),
                ("mfilter_launches", C.c_int64), ("mfilter_ms", C.c_double), ("mfilter_pairs", C.c_int64),
                ("mfilter_alg_flops", C.c_double), ("mfilter_tiles", C.c_int64),
                ("mfilter_wait", C.c_double * 11), ("mfilter_cycles", C.c_double * 4),
                ("mfilter_active_tiles", C.c_int64)]


class ServerOpts(C.Structure):
    _fields_ = [("max_batch", C.c_int32), ("max_wait_us", C.c_int32), ("streams", C.c_int32),
                ("single_max", C.c_int32), ("max_pending", C.c_int64), ("max_device_bytes", C.c_int64),
                ("result_ids_per_request", C.c_int64), ("spin_us", C.c_int32), ("reserved", C.c_int32)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("rejected", C.c_int64),
                ("pending", C.c_int64), ("batches", C.c_int64), ("mean_batch", C.c_double),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("max_ms", C.c_double),
                ("reserved_ids", C.c_int64), ("reservable_ids", C.c_int64), ("batches_one_by_one", C.c_int64)]


class QueryStats(C.Structure):
    _fields_ = [("blocks_total", C.c_int64), ("blocks_pruned", C.c_int64), ("users_tested", C.c_int64),
                ("yes_fast", C.c_int64), ("todo", C.c_int64), ("exact_calls", C.c_int64),
                ("result", C.c_int64)]


_lib = None
_lock = threading.Lock()
LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "librmips.so")


def load_library(build_if_missing: bool = True):
    """Load librmips.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            from . import build_lib
            build_lib.build()
        if not os.path.exists(LIB_PATH):
            raise RmipsError(7, f"CUDA library not found at {LIB_PATH}")
        lib = C.CDLL(LIB_PATH)
        P, I64, I32, VP = C.c_void_p, C.c_int64, C.c_int32, C.c_void_p
        lib.rmips_build_index.argtypes = [P, I64, P, I64, I32, C.POINTER(BuildOpts), VP, C.POINTER(VP)]
        lib.rmips_query.argtypes = [VP, P, I32, C.POINTER(Segment), P, I64, C.POINTER(I64), VP]
        lib.rmips_query_batch.argtypes = [VP, P, I64, P, C.POINTER(Segment), P, I64, P, VP]
        lib.rmips_query_batch_async.argtypes = [VP, P, I64, P, P, I64, P, P, VP]
        lib.rmips_query_async.argtypes = [VP, P, I32, P, I64, P, VP]
        lib.rmips_index_tune.argtypes = [VP, C.c_char_p, VP]
        lib.rmips_index_save.argtypes = [VP, C.c_char_p]
        lib.rmips_index_load.argtypes = [C.c_char_p, VP, C.POINTER(VP)]
        lib.rmips_index_rebuild.argtypes = [VP, I32, VP, C.POINTER(VP)]
        lib.rmips_topk_join.argtypes = [VP, I32, P, VP]
        lib.rmips_index_get_info.argtypes = [VP, C.POINTER(IndexInfo)]
        lib.rmips_last_query_stats.argtypes = [VP, C.POINTER(QueryStats)]
        lib.rmips_index_export.argtypes = [VP, I32, P, I64]
        lib.rmips_free_index.argtypes = [VP]
        lib.rmips_free_index.restype = None
        lib.rmips_status_string.argtypes = [I32]
        lib.rmips_status_string.restype = C.c_char_p
        lib.rmips_last_error.argtypes = []
        lib.rmips_last_error.restype = C.c_char_p
        lib.rmips_exact_sign_host.argtypes = [P, P, P, I32]
        lib.rmips_exact_sign_host.restype = I32
        lib.rmips_profile_enable.argtypes = [VP, I32]
        lib.rmips_profile_read.argtypes = [VP, C.POINTER(Profile)]
        lib.rmips_query_noalloc.argtypes = [VP, P, I32, P, I64, C.POINTER(I64), VP]
        lib.rmips_debug_tc_tile.argtypes = [P, P, P, I32, VP]
        lib.rmips_server_create.argtypes = [VP, C.POINTER(ServerOpts), C.POINTER(VP)]
        lib.rmips_server_submit.argtypes = [VP, P, I32, C.POINTER(Segment), C.POINTER(I64)]
        lib.rmips_server_submit_many.argtypes = [VP, P, I64, P, C.POINTER(Segment), P]
        lib.rmips_server_wait.argtypes = [VP, I64, P, I64, C.POINTER(I64), C.POINTER(C.c_double), I32]
        lib.rmips_server_get_stats.argtypes = [VP, C.POINTER(ServerStats)]
        lib.rmips_server_wait_many.argtypes = [VP, P, I64, P, I64, P, P, I32]
        lib.rmips_server_destroy.argtypes = [VP]
        lib.rmips_server_add_segment.argtypes = [VP, P, I64, C.POINTER(C.c_int32)]
        lib.rmips_server_destroy.restype = None
        for name in ("rmips_build_index", "rmips_query", "rmips_query_batch", "rmips_query_batch_async",
                     "rmips_index_save", "rmips_index_load", "rmips_index_rebuild", "rmips_topk_join",
                     "rmips_index_get_info",
                     "rmips_last_query_stats", "rmips_index_export", "rmips_profile_enable",
                     "rmips_profile_read", "rmips_query_noalloc", "rmips_debug_tc_tile",
                     "rmips_server_create", "rmips_server_submit", "rmips_server_submit_many",
                     "rmips_server_wait", "rmips_server_wait_many", "rmips_server_get_stats",
                     "rmips_query_async", "rmips_index_tune", "rmips_server_add_segment"):
            getattr(lib, name).restype = I32
        _lib = lib
        return lib


def _check(st: int):
    if st != 0:
        msg = _lib.rmips_last_error().decode(errors="replace")
        raise RmipsError(st, msg)


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr_f32(x, shape_last=None):
    """Pointer to a C-contiguous float32 buffer (numpy or torch), plus a keep-alive."""
    if _is_torch(x):
        import torch
        if x.dtype != torch.float32 or not x.is_contiguous():
            x = x.to(torch.float32).contiguous()
        return x.data_ptr(), x
    a = np.ascontiguousarray(x, dtype=np.float32)
    return a.ctypes.data, a


def _ptr_i32(x):
    if _is_torch(x):
        import torch
        if x.dtype != torch.int32 or not x.is_contiguous():
            x = x.to(torch.int32).contiguous()
        return x.data_ptr(), x
    a = np.ascontiguousarray(x, dtype=np.int32)
    return a.ctypes.data, a


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return getattr(stream, "cuda_stream", None)


def _segment(seg, keep):
    """Build a Segment from None, (begin, end) or an id array."""
    if seg is None:
        return None
    s = Segment()
    if isinstance(seg, tuple) and len(seg) == 2 and seg[0] == "registered":
        s.kind, s.begin = 3, int(seg[1])
    elif isinstance(seg, tuple) and len(seg) == 2:
        s.kind, s.begin, s.end = 1, int(seg[0]), int(seg[1])
    else:
        ids = np.ascontiguousarray(seg, dtype=np.int64)
        keep.append(ids)
        s.kind = 2
        s.ids = ids.ctypes.data_as(C.POINTER(C.c_int64))
        s.n_ids = ids.shape[0]
    return s


class Index:
    """Owning handle of a device-resident index (freed on ``close`` / GC)."""

    def __init__(self, handle: int, n: int, m: int, d: int, k_max: int):
        self.handle = C.c_void_p(handle)
        self.n, self.m, self.d, self.k_max = n, m, d, k_max

    def close(self):
        if self.handle and self.handle.value:
            _lib.rmips_free_index(self.handle)
            self.handle = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        return rmips_index_get_info(self)

    def query(self, q, k, **kw):
        return rmips_query(self, q, k, **kw)

    def query_batch(self, qs, ks, **kw):
        return rmips_query_batch(self, qs, ks, **kw)


def rmips_build_index(Q, P, k_max: int, block_size: int = 32, p_prime: int = 0,
                      precision="fp32", batch_tensor_cores: bool = True, build_tensor_cores: bool = True,
                      block_filter: bool = True, autotune: bool = False, tune_cache: str | None = None,
                      stream=None) -> Index:
    """Build the index of Algorithm 1 from users Q [n, d] and items P [m, d].

    ``batch_tensor_cores=False`` keeps the batched filter on CUDA cores;
    ``build_tensor_cores=False`` selects candidates on CUDA cores;
    ``block_filter=False`` switches Lemma 3 off (the no-blocks ablation);
    ``autotune=True`` (or a ``tune_cache`` file) ends the build with the
    autotuner (``rmips_index_tune``)."""
    load_library()
    qp, qk = _ptr_f32(Q)
    pp, pk = _ptr_f32(P)
    n, d = int(qk.shape[0]), int(qk.shape[1])
    m = int(pk.shape[0])
    if int(pk.shape[1]) != d:
        raise RmipsError(1, "Q and P differ in dimension")
    opts = BuildOpts(int(k_max), int(block_size), int(p_prime), _PREC[precision],
                     (0 if batch_tensor_cores else 1) | (0 if build_tensor_cores else 2) |
                     (0 if block_filter else 4) | (8 if autotune else 0),
                     tune_cache.encode() if tune_cache else None)
    out = C.c_void_p()
    _check(_lib.rmips_build_index(qp, n, pp, m, d, C.byref(opts), _stream(stream), C.byref(out)))
    return Index(out.value, n, m, d, int(k_max))


def rmips_index_save(index: Index, path: str):
    """Write the index to a file (see rmips_index_load)."""
    _check(_lib.rmips_index_save(index.handle, os.fsencode(path)))


def rmips_index_load(path: str, stream=None) -> Index:
    """Read an index written by rmips_index_save onto the current device."""
    load_library()
    out = C.c_void_p()
    _check(_lib.rmips_index_load(os.fsencode(path), _stream(stream), C.byref(out)))
    h = Index(out.value, 0, 0, 0, 0)
    info = rmips_index_get_info(h)
    h.n, h.m, h.d, h.k_max = info["n"], info["m"], info["d"], info["k_max"]
    return h


def rmips_index_rebuild(index: Index, k_max: int, stream=None) -> Index:
    """A new index over the same users and items with another k_max (Algorithm 1 again)."""
    out = C.c_void_p()
    _check(_lib.rmips_index_rebuild(index.handle, int(k_max), _stream(stream), C.byref(out)))
    return Index(out.value, index.n, index.m, index.d, int(k_max))


def rmips_topk_join(index: Index, k: int, out=None, stream=None):
    """k-MIPS of every user (Definition 1): [n, k] item ids, descending inner product."""
    if out is None:
        out = np.empty((index.n, int(k)), dtype=np.int64)
        _check(_lib.rmips_topk_join(index.handle, int(k), out.ctypes.data, _stream(stream)))
        return out
    ptr = out.data_ptr() if _is_torch(out) else out.ctypes.data
    _check(_lib.rmips_topk_join(index.handle, int(k), ptr, _stream(stream)))
    return out


def rmips_query(index: Index, q, k: int, segment=None, capacity=None, out=None, stream=None) -> np.ndarray:
    """Reverse k-MIPS of one query; ascending user ids (numpy int64, or ``out`` if given)."""
    keep = []
    qp, qk = _ptr_f32(q)
    seg = _segment(segment, keep)
    cnt = C.c_int64(0)
    if out is None:
        cap = index.n if capacity is None else int(capacity)
        buf = np.empty(max(cap, 1), dtype=np.int64)
        optr = buf.ctypes.data
    else:
        buf = out
        cap = int(out.numel() if _is_torch(out) else out.shape[0])
        optr = out.data_ptr() if _is_torch(out) else out.ctypes.data
    _check(_lib.rmips_query(index.handle, qp, int(k), C.byref(seg) if seg is not None else None,
                            optr, cap, C.byref(cnt), _stream(stream)))
    return buf[:cnt.value]


def rmips_query_noalloc(index: Index, q, k: int, out, stream=None) -> int:
    """Allocation-free single query (see ``include/rmips.h``).

    ``out`` must be a device tensor of int64; returns the result size (the
    first that many entries of ``out`` hold the ascending ids).
    """
    qp, qk = _ptr_f32(q)
    cnt = C.c_int64(0)
    cap = int(out.numel())
    _check(_lib.rmips_query_noalloc(index.handle, qp, int(k), out.data_ptr(), cap, C.byref(cnt),
                                    _stream(stream)))
    return cnt.value


def rmips_debug_tc_tile(A, B, D, kind="tf32", stream=None):
    """One 128x64x64 tensor-core tile (device tensors): D = A @ B.T in TF32, BF16 or FP16."""
    load_library()
    kid = {"tf32": 0, "bf16": 1, "fp16": 2}[kind]
    _check(_lib.rmips_debug_tc_tile(A.data_ptr(), B.data_ptr(), D.data_ptr(), kid, _stream(stream)))


def rmips_query_batch(index: Index, qs, ks, segments=None, capacity=None, out=None, stream=None):
    """Reverse k-MIPS of many queries: returns ``(ids, offsets)`` in CSR form."""
    keep = []
    qp, qk = _ptr_f32(qs)
    nq = int(qk.shape[0])
    if np.isscalar(ks):
        ks = np.full(nq, int(ks), dtype=np.int32)
    kp, kk = _ptr_i32(ks)
    segs = None
    if segments is not None:
        arr = (Segment * nq)()
        for j, sg in enumerate(segments):
            s = _segment(sg, keep)
            arr[j] = s if s is not None else Segment()
        segs = arr
    offs = np.zeros(nq + 1, dtype=np.int64)
    if out is not None:
        cap = int(out.numel() if _is_torch(out) else out.shape[0])
        optr = out.data_ptr() if _is_torch(out) else out.ctypes.data
        _check(_lib.rmips_query_batch(index.handle, qp, nq, kp, segs, optr, cap, offs.ctypes.data,
                                      _stream(stream)))
        return out[:offs[-1]], offs
    cap = int(capacity) if capacity is not None else max(1024, nq * 64)
    while True:
        buf = np.empty(max(cap, 1), dtype=np.int64)
        st = _lib.rmips_query_batch(index.handle, qp, nq, kp, segs, buf.ctypes.data, cap,
                                    offs.ctypes.data, _stream(stream))
        if st == 5 and capacity is None:
            cap = int(offs[-1])
            continue
        _check(st)
        return buf[:offs[-1]], offs


def rmips_query_batch_async(index: Index, qs, ks, out, offsets, done, stream=None):
    """Queue a batch on ``stream`` without waiting (torch CUDA tensors only).

    qs float32 [nq, d], ks int32 [nq], out int64 [capacity], offsets int64
    [nq + 1], done int64 [2]: when the stream has passed the call, offsets is
    the CSR index of out and done = (status, number of ids)."""
    for t in (qs, ks, out, offsets, done):
        if not _is_torch(t) or not t.is_cuda or not t.is_contiguous():
            raise RmipsError(1, "rmips_query_batch_async takes contiguous CUDA tensors")
    nq = int(qs.shape[0])
    if ks.dtype.itemsize != 4 or out.dtype.itemsize != 8 or offsets.numel() < nq + 1 or done.numel() < 2:
        raise RmipsError(1, "ks int32, out / offsets / done int64, offsets nq + 1, done 2")
    _check(_lib.rmips_query_batch_async(index.handle, qs.data_ptr(), nq, ks.data_ptr(), out.data_ptr(),
                                        int(out.numel()), offsets.data_ptr(), done.data_ptr(), _stream(stream)))


def rmips_query_async(index: Index, q, k: int, out, done, stream=None):
    """Queue one query on ``stream`` without waiting (torch CUDA tensors only).

    q float32 [d], out int64 [capacity], done int64 [2]: when the stream has
    passed the call, out[:done[1]] holds the ascending ids and done[0] the
    status."""
    for t in (q, out, done):
        if not _is_torch(t) or not t.is_cuda or not t.is_contiguous():
            raise RmipsError(1, "rmips_query_async takes contiguous CUDA tensors")
    if q.dtype.itemsize != 4 or out.dtype.itemsize != 8 or done.numel() < 2 or done.dtype.itemsize != 8:
        raise RmipsError(1, "q float32, out / done int64, done 2")
    _check(_lib.rmips_query_async(index.handle, q.data_ptr(), int(k), out.data_ptr(), int(out.numel()),
                                  done.data_ptr(), _stream(stream)))


def rmips_index_tune(index: Index, tune_cache: str | None = None, stream=None) -> dict:
    """Run the autotuner on an index; returns the index info with the choices."""
    _check(_lib.rmips_index_tune(index.handle, tune_cache.encode() if tune_cache else None, _stream(stream)))
    return rmips_index_get_info(index)


def rmips_index_get_info(index: Index) -> dict:
    info = IndexInfo()
    _check(_lib.rmips_index_get_info(index.handle, C.byref(info)))
    return {f: getattr(info, f) for f, _ in IndexInfo._fields_}


def rmips_last_query_stats(index: Index) -> dict:
    st = QueryStats()
    _check(_lib.rmips_last_query_stats(index.handle, C.byref(st)))
    return {f: getattr(st, f) for f, _ in QueryStats._fields_}


_FIELDS = {"permQ": (0, np.int32), "permP": (1, np.int32), "lo": (2, np.float32), "hi": (3, np.float32),
           "LB": (4, np.float32), "hdr": (5, np.float32), "unorm": (6, np.float32),
           "pnorm": (7, np.float32), "incomplete": (8, np.uint8)}


def rmips_index_export(index: Index, field: str) -> np.ndarray:
    info = rmips_index_get_info(index)
    n, m, k_max, nb = info["n"], info["m"], info["k_max"], info["n_blocks"]
    shapes = {"permQ": (n,), "permP": (m,), "lo": (k_max, n), "hi": (k_max, n), "LB": (k_max, nb),
              "hdr": (nb,), "unorm": (n,), "pnorm": (m,),
              "incomplete": (n,) if info["p_prime"] == m else (0,)}
    fid, dt = _FIELDS[field]
    arr = np.empty(shapes[field], dtype=dt)
    _check(_lib.rmips_index_export(index.handle, fid, arr.ctypes.data if arr.size else
                                   np.empty(1, dt).ctypes.data, arr.nbytes))
    return arr


def rmips_profile_enable(index: Index, enable=True):
    """enable: False/0 off, True/1 kernel timing, 2 timing plus pipeline counters."""
    level = 2 if enable == 2 else (1 if enable else 0)
    _check(_lib.rmips_profile_enable(index.handle, level))


def rmips_profile_read(index: Index) -> dict:
    pr = Profile()
    _check(_lib.rmips_profile_read(index.handle, C.byref(pr)))
    out = {}
    for f, _ in Profile._fields_:
        v = getattr(pr, f)
        out[f] = list(v) if hasattr(v, "__len__") else v
    return out


def rmips_free_index(index: Index):
    index.close()


def rmips_status_string(status: int) -> str:
    load_library()
    return _lib.rmips_status_string(int(status)).decode()


def rmips_exact_sign_host(u, a, b) -> int:
    """Sign of u.a - u.b in exact arithmetic (host-side integer accumulator)."""
    load_library()
    u = np.ascontiguousarray(u, np.float32)
    a = np.ascontiguousarray(a, np.float32)
    b = np.ascontiguousarray(b, np.float32)
    return int(_lib.rmips_exact_sign_host(u.ctypes.data, a.ctypes.data, b.ctypes.data, u.shape[0]))


class Server:
    """Continuous-batching request loop over an index (see ``include/rmips.h``)."""

    def __init__(self, index: Index, max_batch: int = 4096, max_wait_us: int = 200, streams: int = 2,
                 max_pending: int = 1 << 20, max_device_bytes: int = 0, result_ids_per_request: int = 0,
                 single_max: int = 0, spin_us: int = 0):
        load_library()
        self.index = index                       # keeps the index alive
        opts = ServerOpts(int(max_batch), int(max_wait_us), int(streams), int(single_max), int(max_pending),
                          int(max_device_bytes), int(result_ids_per_request), int(spin_us), 0)
        h = C.c_void_p()
        _check(_lib.rmips_server_create(index.handle, C.byref(opts), C.byref(h)))
        self.handle = h

    def add_segment(self, ids) -> int:
        """Registers a user segment; use it as the segment ``("registered", handle)``."""
        a = np.ascontiguousarray(ids, np.int64)
        h = C.c_int32(0)
        _check(_lib.rmips_server_add_segment(self.handle, a.ctypes.data, a.shape[0], C.byref(h)))
        return h.value

    def submit(self, q, k: int, segment=None) -> int:
        keep = []
        qa = np.ascontiguousarray(q, np.float32)
        seg = _segment(segment, keep)
        t = C.c_int64(0)
        _check(_lib.rmips_server_submit(self.handle, qa.ctypes.data, int(k),
                                        C.byref(seg) if seg is not None else None, C.byref(t)))
        return t.value

    def submit_many(self, qs, ks, segments=None) -> np.ndarray:
        keep = []
        qa = np.ascontiguousarray(qs, np.float32)
        nq = qa.shape[0]
        ka = np.ascontiguousarray(np.broadcast_to(np.asarray(ks), (nq,)), np.int32)
        segs = None
        if segments is not None:
            segs = (Segment * nq)()
            for j, sg in enumerate(segments):
                s = _segment(sg, keep)
                segs[j] = s if s is not None else Segment()
        tickets = np.empty(nq, np.int64)
        _check(_lib.rmips_server_submit_many(self.handle, qa.ctypes.data, nq, ka.ctypes.data, segs,
                                             tickets.ctypes.data))
        return tickets

    def wait(self, ticket: int, timeout_ms: int = -1, capacity: int | None = None):
        """Returns ``(ids, latency_ms)``."""
        cap = self.index.n if capacity is None else int(capacity)
        buf = np.empty(max(cap, 1), np.int64)
        cnt = C.c_int64(0)
        lat = C.c_double(0.0)
        _check(_lib.rmips_server_wait(self.handle, int(ticket), buf.ctypes.data, cap, C.byref(cnt),
                                      C.byref(lat), int(timeout_ms)))
        return buf[:cnt.value], lat.value

    def wait_many(self, tickets, timeout_ms: int = -1, capacity: int | None = None):
        """Results of many requests: ``(ids, offsets, latencies_ms)`` in CSR form."""
        t = np.ascontiguousarray(tickets, np.int64)
        nt = t.shape[0]
        cap = max(1024, nt * 64) if capacity is None else int(capacity)
        offs = np.zeros(nt + 1, np.int64)
        lat = np.zeros(max(nt, 1), np.float64)
        while True:
            buf = np.empty(max(cap, 1), np.int64)
            st = _lib.rmips_server_wait_many(self.handle, t.ctypes.data, nt, buf.ctypes.data, cap,
                                             offs.ctypes.data, lat.ctypes.data, int(timeout_ms))
            if st == 5 and capacity is None:
                cap = int(offs[-1])
                continue
            _check(st)
            return buf[:offs[-1]], offs, lat[:nt]

    def stats(self) -> dict:
        st = ServerStats()
        _check(_lib.rmips_server_get_stats(self.handle, C.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if self.handle and self.handle.value:
            _lib.rmips_server_destroy(self.handle)
            self.handle = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
