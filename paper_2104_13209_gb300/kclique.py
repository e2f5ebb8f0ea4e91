"""Thin Python binding of libkclique (include/kclique.h).

Argument marshalling only: every step of the counting path runs inside the
CUDA library.  Host arrays are numpy arrays; device arrays may be given as
torch CUDA tensors (their data pointers are passed straight through).  The
library must have been built (``paper_2104_13209_gb300.build.build()``);
importing this module on a machine without it raises at first use -- there
is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

KC_OK = 0
KC_E_INVALID_ARG = 1
KC_E_INVALID_GRAPH = 2
KC_E_NO_MEMORY = 3
KC_E_OVERFLOW = 4
KC_E_TIMEOUT = 5
KC_E_CUDA = 6
KC_E_INTERNAL = 7
KC_E_UNSUPPORTED = 8
KC_E_REFUSED = 9

KC_ORIENT_DEGREE = 0
KC_ORIENT_DEGENERACY = 1
KC_SCHEME_AUTO = 0
KC_SCHEME_VC = 1
KC_SCHEME_EC = 2
KC_SCHEME_VC_LIST = 3
KC_SCHEME_EC_LIST = 4

KC_FLAG_TOTAL_OVERFLOW = 1
KC_FLAG_VERTEX_OVERFLOW = 2
KC_FLAG_TIMEOUT = 4
KC_FLAG_INTERNAL = 8
KC_FLAG_TOTAL_OVERFLOW128 = 16

_ORIENT = {"degree": KC_ORIENT_DEGREE, "degeneracy": KC_ORIENT_DEGENERACY}
_SCHEME = {"auto": KC_SCHEME_AUTO, "vc": KC_SCHEME_VC, "ec": KC_SCHEME_EC, "vc-list": KC_SCHEME_VC_LIST,
           "ec-list": KC_SCHEME_EC_LIST}

# Every exported symbol of include/kclique.h.
EXPORTED = [
    "kc_last_error", "kc_status_name", "kc_version", "kc_graph_create", "kc_graph_destroy", "kc_graph_info_get",
    "kc_graph_export", "kc_count", "kc_count128", "kc_count_async", "kc_count_noalloc", "kc_graph_reserve", "kc_count_all",
    "kc_count_all128",
    "kc_graph_set_time_limit", "kc_launch_count", "kc_graph_last_work", "kc_graph_last_sm_work", "kc_list_cliques",
    "kc_batch_create", "kc_batch_destroy", "kc_batch_graph_info", "kc_batch_set_time_limit", "kc_batch_count",
    "kc_batch_tune", "kc_batch_capture", "kc_batch_exec_launch", "kc_batch_exec_destroy",
    "kc_server_create", "kc_server_add_graph", "kc_server_set_time_limit", "kc_server_submit", "kc_server_poll",
    "kc_server_stats", "kc_server_shape", "kc_server_destroy",
]

KC_SERVER_SERIAL = 1
SHAPE_UNKNOWN, SHAPE_FITS, SHAPE_EXPENSIVE = 0, 1, 2
KC_SERVER_AUTO_TRAVERSAL = 2
KC_SERVER_REFUSE_EXPENSIVE = 4


class kc_graph_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("d_max", ctypes.c_uint32), ("num_edges", ctypes.c_uint64),
                ("degeneracy", ctypes.c_uint32), ("orient", ctypes.c_int32), ("device_bytes", ctypes.c_uint64),
                ("orient_ms", ctypes.c_float)]


class kc_result(ctypes.Structure):
    _fields_ = [("total", ctypes.c_uint64), ("total_hi", ctypes.c_uint64), ("flags", ctypes.c_uint32),
                ("status", ctypes.c_uint32), ("words", ctypes.c_uint64)]


class kc_server_result(ctypes.Structure):
    _fields_ = [("total", ctypes.c_uint64), ("total_hi", ctypes.c_uint64), ("flags", ctypes.c_uint32),
                ("status", ctypes.c_int32), ("graph_id", ctypes.c_uint32), ("k", ctypes.c_uint32),
                ("pivot", ctypes.c_int32), ("launch", ctypes.c_uint32), ("t_submit_ms", ctypes.c_double),
                ("t_admit_ms", ctypes.c_double), ("t_done_ms", ctypes.c_double)]


KC_TUNE_MAX = 256


class kc_tune_entry(ctypes.Structure):
    _fields_ = [("dclass", ctypes.c_uint32), ("k", ctypes.c_uint32), ("scheme", ctypes.c_int32),
                ("subwarp", ctypes.c_uint32), ("chunk", ctypes.c_uint32), ("ms", ctypes.c_float)]


class kc_tune(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("e", kc_tune_entry * KC_TUNE_MAX)]


RESULT_BYTES = ctypes.sizeof(kc_result)


class KCError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{status_name(status)}: {message}")
        self.status = status
        self.message = message


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libkclique.so (raising if it is absent and build_if_missing is False)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise ImportError(f"libkclique.so is not built ({path}); run paper_2104_13209_gb300.build.build()")
        _build.build()
    lib = ctypes.CDLL(path)
    vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    lib.kc_last_error.restype = ctypes.c_char_p
    lib.kc_last_error.argtypes = []
    lib.kc_status_name.restype = ctypes.c_char_p
    lib.kc_status_name.argtypes = [i32]
    lib.kc_version.restype = i32
    lib.kc_launch_count.restype = u64
    lib.kc_launch_count.argtypes = []
    lib.kc_graph_create.argtypes = [vp, vp, u32, u64, i32, i32, i32, vp, ctypes.POINTER(vp)]
    lib.kc_graph_destroy.argtypes = [vp]
    lib.kc_graph_info_get.argtypes = [vp, ctypes.POINTER(kc_graph_info)]
    lib.kc_graph_export.argtypes = [vp, vp, vp, vp, vp]
    lib.kc_count.argtypes = [vp, u32, i32, i32, u32, ctypes.POINTER(u64), vp, ctypes.POINTER(u32), vp]
    lib.kc_count128.argtypes = [vp, u32, i32, i32, u32, ctypes.POINTER(u64), ctypes.POINTER(u64),
                                ctypes.POINTER(u32), vp]
    lib.kc_count_async.argtypes = [vp, u32, i32, i32, u32, vp, vp, vp]
    lib.kc_count_noalloc.argtypes = [vp, u32, i32, u32, vp, vp]
    lib.kc_graph_reserve.argtypes = [vp, u32, i32, i32, vp]
    lib.kc_count_all.argtypes = [vp, vp, vp, u32, ctypes.POINTER(u32), u32, vp, vp]
    lib.kc_count_all128.argtypes = [vp, vp, vp, vp, u32, ctypes.POINTER(u32), u32, vp, vp]
    lib.kc_graph_set_time_limit.argtypes = [vp, ctypes.c_double]
    lib.kc_graph_last_work.argtypes = [vp, ctypes.POINTER(u64)]
    lib.kc_graph_last_work.restype = i32
    lib.kc_graph_last_sm_work.argtypes = [vp, vp, u32, ctypes.POINTER(u32)]
    lib.kc_graph_last_sm_work.restype = i32
    lib.kc_list_cliques.argtypes = [vp, u32, vp, u64, ctypes.POINTER(u64), vp]
    lib.kc_list_cliques.restype = i32
    lib.kc_batch_create.argtypes = [vp, vp, u32, u64, vp, u32, i32, i32, i32, vp, ctypes.POINTER(vp)]
    lib.kc_batch_destroy.argtypes = [vp]
    lib.kc_batch_graph_info.argtypes = [vp, u32, ctypes.POINTER(u32), ctypes.POINTER(u64), ctypes.POINTER(u32)]
    lib.kc_batch_set_time_limit.argtypes = [vp, ctypes.c_double]
    lib.kc_batch_count.argtypes = [vp, vp, vp, u32, vp, vp, vp]
    lib.kc_batch_tune.argtypes = [vp, vp, vp, u32, u32, ctypes.POINTER(kc_tune), vp]
    lib.kc_batch_capture.argtypes = [vp, vp, vp, u32, vp, vp, ctypes.POINTER(vp)]
    lib.kc_batch_exec_launch.argtypes = [vp, vp]
    lib.kc_batch_exec_destroy.argtypes = [vp]
    lib.kc_server_create.argtypes = [ctypes.c_size_t, u32, u32, i32, ctypes.POINTER(vp)]
    lib.kc_server_add_graph.argtypes = [vp, vp, vp, u32, u64, i32, i32, i32, ctypes.POINTER(u32)]
    lib.kc_server_set_time_limit.argtypes = [vp, ctypes.c_double]
    lib.kc_server_submit.argtypes = [vp, u32, u32, i32, ctypes.POINTER(u64)]
    lib.kc_server_poll.argtypes = [vp, u64, ctypes.POINTER(kc_server_result), i32]
    lib.kc_server_stats.argtypes = [vp, ctypes.POINTER(u64), ctypes.POINTER(u64), ctypes.POINTER(u64)]
    lib.kc_server_shape.argtypes = [vp, u32, u32, i32, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_double)]
    lib.kc_server_destroy.argtypes = [vp]
    for f in ("kc_server_create", "kc_server_add_graph", "kc_server_set_time_limit", "kc_server_submit",
              "kc_server_poll", "kc_server_stats", "kc_server_shape", "kc_server_destroy"):
        getattr(lib, f).restype = i32
    for f in ("kc_batch_create", "kc_batch_destroy", "kc_batch_graph_info", "kc_batch_set_time_limit",
              "kc_batch_count", "kc_batch_tune", "kc_batch_capture", "kc_batch_exec_launch", "kc_batch_exec_destroy"):
        getattr(lib, f).restype = i32
    for f in ("kc_graph_create", "kc_graph_destroy", "kc_graph_info_get", "kc_graph_export", "kc_count",
              "kc_count128", "kc_count_async", "kc_count_noalloc", "kc_graph_reserve", "kc_count_all", "kc_count_all128",
              "kc_graph_set_time_limit"):
        getattr(lib, f).restype = i32
    _lib = lib
    return lib


def status_name(s: int) -> str:
    try:
        return load().kc_status_name(s).decode()
    except Exception:  # library not loadable: plain number
        return f"status {s}"


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load().kc_launch_count())


def last_error() -> str:
    return load().kc_last_error().decode()


def _check(st: int, allow=(KC_OK,)) -> int:
    if st not in allow:
        raise KCError(st, last_error())
    return st


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr_of(x):
    """(pointer, keepalive, on_device) of a numpy array or torch tensor."""
    if x is None:
        return None, None, False
    if _is_torch(x):
        if not x.is_contiguous():
            x = x.contiguous()
        return x.data_ptr(), x, x.is_cuda
    a = np.ascontiguousarray(x)
    return a.ctypes.data, a, False


@dataclass
class CountResult:
    total: int            # exact count (both words)
    flags: int
    overflow: bool        # exceeded 2^64 - 1
    words: int = 0        # bitmap words intersected by the traversal
    status: int = KC_OK   # per-query status of a batched count

    @property
    def total_u64(self) -> int:
        return self.total & ((1 << 64) - 1)


class Graph:
    """A resident, oriented graph (kc_graph_create)."""

    def __init__(self, row_ptr, col_idx, n: int | None = None, orient: str = "degeneracy", validate: bool = True,
                 stream=None):
        lib = load()
        rp, rp_keep, rp_dev = _ptr_of(row_ptr if _is_torch(row_ptr) else np.asarray(row_ptr, dtype=np.uint32))
        ci, ci_keep, ci_dev = _ptr_of(col_idx if _is_torch(col_idx) else np.asarray(col_idx, dtype=np.uint32))
        if rp_dev != ci_dev:
            raise ValueError("row_ptr and col_idx must both be on the host or both on the device")
        if n is None:
            n = (rp_keep.numel() if _is_torch(rp_keep) else rp_keep.size) - 1
        nnz = ci_keep.numel() if _is_torch(ci_keep) else ci_keep.size
        h = ctypes.c_void_p()
        _check(lib.kc_graph_create(rp, ci if nnz else None, n, nnz, int(rp_dev), _ORIENT[orient], int(validate),
                                   _stream_ptr(stream), ctypes.byref(h)))
        self._h = h
        self.n = n
        self.orient = orient

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            load().kc_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        i = kc_graph_info()
        _check(load().kc_graph_info_get(self._h, ctypes.byref(i)))
        return {f: getattr(i, f) for f, _ in kc_graph_info._fields_}

    def last_work(self) -> int:
        """Work units of the last synchronous count (see kc_graph_last_work)."""
        u = ctypes.c_uint64()
        _check(load().kc_graph_last_work(self._h, ctypes.byref(u)))
        return u.value

    def set_time_limit(self, seconds: float):
        _check(load().kc_graph_set_time_limit(self._h, float(seconds)))

    def list_cliques(self, k: int, cap: int | None = None, stream=None):
        """(number of k-cliques, uint32 array [min(count, cap), k] of input vertex ids) via kc_list_cliques;
        cap defaults to the count (one counting call by the bitmap traversal first)."""
        import torch

        lib = load()
        if cap is None:
            cap = self.count(k, stream=stream).total
        buf = torch.empty(max(cap * k, 1), dtype=torch.int32, device="cuda")
        cnt = ctypes.c_uint64()
        _check(lib.kc_list_cliques(self._h, k, buf.data_ptr() if cap else None, cap, ctypes.byref(cnt),
                                   _stream_ptr(stream)))
        rows = min(cnt.value, cap)
        out = buf[: rows * k].cpu().numpy().view(np.uint32).reshape(rows, k)
        return cnt.value, out

    def last_sm_work(self) -> np.ndarray:
        """Work units per SM of the last orientation-mode count (kc_graph_last_sm_work)."""
        lib = load()
        slots = ctypes.c_uint32()
        _check(lib.kc_graph_last_sm_work(self._h, None, 0, ctypes.byref(slots)))
        out = np.zeros(max(slots.value, 1), dtype=np.uint64)
        _check(lib.kc_graph_last_sm_work(self._h, out.ctypes.data, slots.value, ctypes.byref(slots)))
        return out[: slots.value]

    def export(self, core: bool = False):
        """(dag_row_ptr, dag_col, new_of_old, core or None) as numpy arrays."""
        inf = self.info()
        n, m = inf["n"], inf["num_edges"]
        rp = np.zeros(n + 1, dtype=np.uint32)
        col = np.zeros(max(m, 1), dtype=np.uint32)
        nof = np.zeros(max(n, 1), dtype=np.uint32)
        cr = np.zeros(max(n, 1), dtype=np.uint32) if core else None
        _check(load().kc_graph_export(self._h, rp.ctypes.data, col.ctypes.data, nof.ctypes.data,
                                      cr.ctypes.data if core else None))
        return rp, col[:m], nof[:n], (cr[:n] if core else None)

    def count(self, k: int, pivot: bool = False, scheme: str = "auto", subwarp: int = 0, stream=None) -> CountResult:
        lo, hi, fl = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint32()
        _check(load().kc_count128(self._h, k, int(pivot), _SCHEME[scheme], subwarp, ctypes.byref(lo), ctypes.byref(hi),
                                  ctypes.byref(fl), _stream_ptr(stream)), allow=(KC_OK, KC_E_OVERFLOW))
        total = (hi.value << 64) | lo.value
        return CountResult(total, fl.value, total >= (1 << 64) or bool(fl.value & KC_FLAG_TOTAL_OVERFLOW))

    def count_per_vertex(self, k: int, pivot: bool = True, scheme: str = "auto", stream=None):
        """(total mod 2^64, per-vertex counts mod 2^64 as uint64[n], flags) via kc_count."""
        tot, fl = ctypes.c_uint64(), ctypes.c_uint32()
        pv = np.zeros(max(self.n, 1), dtype=np.uint64)
        _check(load().kc_count(self._h, k, int(pivot), _SCHEME[scheme], 0, ctypes.byref(tot), pv.ctypes.data,
                               ctypes.byref(fl), _stream_ptr(stream)), allow=(KC_OK, KC_E_OVERFLOW))
        return tot.value, pv[: self.n], fl.value

    def count_all(self, cap: int | None = None, per_vertex_k: int = 0, stream=None):
        """Every clique size by pivoting: (counts uint64[cap], overflow uint8[cap], omega, per-vertex or None)."""
        if cap is None:
            cap = self.info()["d_max"] + 3
        counts = np.zeros(cap, dtype=np.uint64)
        ovf = np.zeros(cap, dtype=np.uint8)
        om = ctypes.c_uint32()
        pv = np.zeros(max(self.n, 1), dtype=np.uint64) if per_vertex_k else None
        _check(load().kc_count_all(self._h, counts.ctypes.data, ovf.ctypes.data, cap, ctypes.byref(om), per_vertex_k,
                                   pv.ctypes.data if pv is not None else None, _stream_ptr(stream)),
               allow=(KC_OK, KC_E_OVERFLOW))
        return counts, ovf, om.value, (pv[: self.n] if pv is not None else None)

    def count_all128(self, cap: int | None = None, per_vertex_k: int = 0, stream=None):
        """Every clique size by pivoting, exact below 2^128: (counts as Python ints, overflow uint8[cap]
        (beyond 2^128 - 1), omega, per-vertex uint64[n] or None)."""
        if cap is None:
            cap = self.info()["d_max"] + 3
        lo = np.zeros(cap, dtype=np.uint64)
        hi = np.zeros(cap, dtype=np.uint64)
        ovf = np.zeros(cap, dtype=np.uint8)
        om = ctypes.c_uint32()
        pv = np.zeros(max(self.n, 1), dtype=np.uint64) if per_vertex_k else None
        _check(load().kc_count_all128(self._h, lo.ctypes.data, hi.ctypes.data, ovf.ctypes.data, cap, ctypes.byref(om),
                                      per_vertex_k, pv.ctypes.data if pv is not None else None, _stream_ptr(stream)),
               allow=(KC_OK, KC_E_OVERFLOW))
        counts = [(int(h) << 64) | int(x) for x, h in zip(lo, hi)]
        return counts, ovf, om.value, (pv[: self.n] if pv is not None else None)

    def count_async(self, k: int, result_dev, pivot: bool = False, scheme: str = "auto", subwarp: int = 0,
                    stream=None):
        """Enqueue a count writing a kc_result into result_dev (a CUDA tensor of >= 24 bytes)."""
        p, _, dev = _ptr_of(result_dev)
        if not dev:
            raise ValueError("result_dev must be device memory")
        _check(load().kc_count_async(self._h, k, int(pivot), _SCHEME[scheme], subwarp, p, None, _stream_ptr(stream)))

    def count_noalloc(self, k: int, result_dev, scheme: str = "auto", subwarp: int = 0, stream=None):
        """Enqueue an orientation-mode count that allocates no device memory
        (working memory is a fixed array inside the library)."""
        p, _, dev = _ptr_of(result_dev)
        if not dev:
            raise ValueError("result_dev must be device memory")
        _check(load().kc_count_noalloc(self._h, k, _SCHEME[scheme], subwarp, p, _stream_ptr(stream)))

    def reserve(self, k_max: int, pivot: bool = False, per_vertex: bool = False, stream=None):
        _check(load().kc_graph_reserve(self._h, k_max, int(pivot), int(per_vertex), _stream_ptr(stream)))


class Batch:
    """Many small graphs oriented as one block-diagonal union
    (kc_batch_create); queries (graph, k) counted in persistent launches."""

    def __init__(self, graphs=None, row_ptr=None, col_idx=None, offsets=None, orient: str = "degeneracy",
                 validate: bool = True, stream=None):
        from . import synth

        lib = load()
        if graphs is not None:
            u, offsets = synth.block_union(graphs)
            row_ptr, col_idx = u.row_ptr, u.col_idx
        rp, rp_keep, rp_dev = _ptr_of(row_ptr if _is_torch(row_ptr) else np.asarray(row_ptr, dtype=np.uint32))
        ci, ci_keep, ci_dev = _ptr_of(col_idx if _is_torch(col_idx) else np.asarray(col_idx, dtype=np.uint32))
        if rp_dev != ci_dev:
            raise ValueError("row_ptr and col_idx must both be on the host or both on the device")
        off = np.ascontiguousarray(offsets, dtype=np.uint32)
        n = int(off[-1])
        nnz = ci_keep.numel() if _is_torch(ci_keep) else ci_keep.size
        h = ctypes.c_void_p()
        _check(lib.kc_batch_create(rp, ci if nnz else None, n, nnz, off.ctypes.data, off.size - 1, int(rp_dev),
                                   _ORIENT[orient], int(validate), _stream_ptr(stream), ctypes.byref(h)))
        self._h = h
        self.num_graphs = off.size - 1

    def close(self):
        if getattr(self, "_h", None):
            load().kc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def graph_info(self, g: int):
        n, m, d = ctypes.c_uint32(), ctypes.c_uint64(), ctypes.c_uint32()
        _check(load().kc_batch_graph_info(self._h, g, ctypes.byref(n), ctypes.byref(m), ctypes.byref(d)))
        return {"n": n.value, "m": m.value, "d_max": d.value}

    def set_time_limit(self, seconds: float):
        _check(load().kc_batch_set_time_limit(self._h, float(seconds)))

    @staticmethod
    def _queries(graph_ids, ks):
        gid = np.ascontiguousarray(graph_ids, dtype=np.uint32)
        kk = np.ascontiguousarray(ks, dtype=np.uint32)
        if gid.shape != kk.shape:
            raise ValueError("graph_ids and ks differ in length")
        return gid, kk

    def count_async(self, graph_ids, ks, results_dev, tune=None, stream=None):
        """Enqueue the queries; results_dev: CUDA uint8 tensor of len * RESULT_BYTES."""
        gid, kk = self._queries(graph_ids, ks)
        p, _, dev = _ptr_of(results_dev)
        if not dev:
            raise ValueError("results_dev must be device memory")
        _check(load().kc_batch_count(self._h, gid.ctypes.data, kk.ctypes.data, gid.size, p,
                                     ctypes.byref(tune) if tune is not None else None, _stream_ptr(stream)))

    def count(self, graph_ids, ks, tune=None, stream=None) -> list[CountResult]:
        """Synchronous counts of the queries, in query order."""
        import torch

        gid, kk = self._queries(graph_ids, ks)
        res = torch.zeros(max(1, gid.size) * RESULT_BYTES, dtype=torch.uint8, device="cuda")
        self.count_async(gid, kk, res, tune=tune, stream=stream)
        if stream is not None:
            stream.synchronize()
        torch.cuda.synchronize()
        return parse_results(bytes(res.cpu().numpy()), gid.size)

    def tune(self, graph_ids, ks, sample: int = 0, stream=None) -> kc_tune:
        gid, kk = self._queries(graph_ids, ks)
        t = kc_tune()
        _check(load().kc_batch_tune(self._h, gid.ctypes.data, kk.ctypes.data, gid.size, sample, ctypes.byref(t),
                                    _stream_ptr(stream)))
        return t

    def capture(self, graph_ids, ks, results_dev, tune=None) -> "BatchExec":
        gid, kk = self._queries(graph_ids, ks)
        p, keep, dev = _ptr_of(results_dev)
        if not dev:
            raise ValueError("results_dev must be device memory")
        h = ctypes.c_void_p()
        _check(load().kc_batch_capture(self._h, gid.ctypes.data, kk.ctypes.data, gid.size, p,
                                       ctypes.byref(tune) if tune is not None else None, ctypes.byref(h)))
        return BatchExec(h, keep)


class BatchExec:
    """A captured CUDA graph of one batch of queries (kc_batch_capture)."""

    def __init__(self, h, keep):
        self._h = h
        self._keep = keep

    def launch(self, stream=None):
        _check(load().kc_batch_exec_launch(self._h, _stream_ptr(stream)))

    def close(self):
        if getattr(self, "_h", None):
            load().kc_batch_exec_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """A serving loop over resident graphs (kc_server_*): submit queries
    (graph, k, pivot) from any thread, poll their results."""

    def __init__(self, hbm_budget: int = 64 << 30, max_batch: int = 256, slots: int = 4, serial: bool = False,
                 auto_traversal: bool = False, refuse_expensive: bool = False):
        h = ctypes.c_void_p()
        flags = ((KC_SERVER_SERIAL if serial else 0) | (KC_SERVER_AUTO_TRAVERSAL if auto_traversal else 0)
                 | (KC_SERVER_REFUSE_EXPENSIVE if refuse_expensive else 0))
        _check(load().kc_server_create(hbm_budget, max_batch, slots, flags, ctypes.byref(h)))
        self._h = h

    def add_graph(self, g=None, row_ptr=None, col_idx=None, n=None, orient: str = "degeneracy",
                  validate: bool = True) -> int:
        if g is not None:
            row_ptr, col_idx, n = g.row_ptr, g.col_idx, g.n
        rp = np.ascontiguousarray(row_ptr, dtype=np.uint32)
        ci = np.ascontiguousarray(col_idx, dtype=np.uint32)
        if n is None:
            n = rp.size - 1
        gid = ctypes.c_uint32()
        _check(load().kc_server_add_graph(self._h, rp.ctypes.data, ci.ctypes.data if ci.size else None, n, ci.size,
                                          0, _ORIENT[orient], int(validate), ctypes.byref(gid)))
        return gid.value

    def set_time_limit(self, seconds: float):
        _check(load().kc_server_set_time_limit(self._h, float(seconds)))

    def submit(self, graph_id: int, k: int, pivot: bool = False) -> int:
        t = ctypes.c_uint64()
        _check(load().kc_server_submit(self._h, graph_id, k, int(pivot), ctypes.byref(t)))
        return t.value

    def poll(self, ticket: int, timeout_ms: int = -1) -> dict | None:
        """The query's result (a dict), or None if it is not done within timeout_ms."""
        r = kc_server_result()
        st = load().kc_server_poll(self._h, ticket, ctypes.byref(r), timeout_ms)
        if st == KC_E_TIMEOUT:
            return None
        _check(st)
        return {"total": (r.total_hi << 64) | r.total, "flags": r.flags, "status": r.status, "graph": r.graph_id,
                "k": r.k, "pivot": r.pivot, "launch": r.launch, "t_submit_ms": r.t_submit_ms,
                "t_admit_ms": r.t_admit_ms, "t_done_ms": r.t_done_ms}

    def stats(self) -> dict:
        a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(load().kc_server_stats(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return {"launches": a.value, "served": b.value, "resident_bytes": c.value}

    def shape(self, graph_id: int, k: int, pivot: bool) -> tuple[int, float]:
        """(state, ms) of a shape: SHAPE_UNKNOWN, SHAPE_FITS (ms: its profiled
        wall time) or SHAPE_EXPENSIVE (see kc_server_shape)."""
        st, ms = ctypes.c_int32(), ctypes.c_double()
        _check(load().kc_server_shape(self._h, graph_id, k, int(pivot), ctypes.byref(st), ctypes.byref(ms)))
        return st.value, ms.value

    def close(self):
        if getattr(self, "_h", None):
            load().kc_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tune_to_list(t: kc_tune) -> list[dict]:
    return [{"dclass": t.e[i].dclass, "k": t.e[i].k, "scheme": t.e[i].scheme, "subwarp": t.e[i].subwarp,
             "chunk": t.e[i].chunk, "ms": t.e[i].ms} for i in range(t.n)]


def tune_from_list(entries: list[dict]) -> kc_tune:
    t = kc_tune()
    for i, e in enumerate(entries[:KC_TUNE_MAX]):
        t.e[i] = kc_tune_entry(e["dclass"], e["k"], e["scheme"], e["subwarp"], e["chunk"], e.get("ms", 0.0))
    t.n = min(len(entries), KC_TUNE_MAX)
    return t


def parse_results(raw: bytes, n: int) -> list[CountResult]:
    """n consecutive kc_result records (a device result array read back)."""
    out = []
    for i in range(n):
        r = kc_result.from_buffer_copy(raw[i * RESULT_BYTES:(i + 1) * RESULT_BYTES])
        total = (r.total_hi << 64) | r.total
        out.append(CountResult(total, r.flags, total >= (1 << 64), r.words, r.status))
    return out


def parse_result(raw: bytes) -> CountResult:
    r = kc_result.from_buffer_copy(raw[:RESULT_BYTES])
    if r.status != KC_OK:
        raise KCError(r.status, "device-side failure")
    total = (r.total_hi << 64) | r.total
    return CountResult(total, r.flags, total >= (1 << 64), r.words)
