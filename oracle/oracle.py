"""Python face of the CPU oracle (``kclique_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the library.  It shares no
code with the CUDA path.  Counts come back as exact Python ints (the C side
accumulates in saturating 128-bit integers; a saturated value is reported as
``None``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kclique_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11 + OpenMP) into oracle/_build."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    vp = ctypes.c_void_p
    lib.or_canonicalize.argtypes = [ctypes.c_uint32, ctypes.c_uint64, _u32p, _u32p, _u32p, _u32p,
                                    ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]
    lib.or_canonicalize.restype = ctypes.c_int
    lib.or_degree_rank.argtypes = [ctypes.c_uint32, _u32p, _u32p]
    lib.or_degree_rank.restype = None
    lib.or_degeneracy_order.argtypes = [ctypes.c_uint32, _u32p, _u32p, _u32p, _u32p, _u32p]
    lib.or_degeneracy_order.restype = ctypes.c_uint32
    lib.or_orient.argtypes = [ctypes.c_uint32, _u32p, _u32p, _u32p, _u32p, _u32p]
    lib.or_orient.restype = ctypes.c_uint32
    lib.or_count_orient.argtypes = [ctypes.c_uint32, _u32p, _u32p, ctypes.c_uint32, vp, ctypes.c_uint32,
                                    ctypes.c_int, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                    vp, vp, vp]
    lib.or_count_orient.restype = ctypes.c_int
    lib.or_count_pivot.argtypes = [ctypes.c_uint32, _u32p, _u32p, _u32p, _u32p, ctypes.c_uint32, ctypes.c_uint32,
                                   vp, ctypes.c_uint32, ctypes.c_int, _u64p, _u64p, _u8p, ctypes.c_uint32, vp, vp,
                                   ctypes.POINTER(ctypes.c_uint32)]
    lib.or_count_pivot.restype = ctypes.c_int
    lib.or_count_vertex.argtypes = [ctypes.c_uint32, _u32p, _u32p, ctypes.c_uint32, ctypes.c_uint32,
                                    ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]
    lib.or_count_vertex.restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint32)


def _join(lo, hi) -> int:
    return (int(hi) << 64) | int(lo)


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count() or 1)


# ----------------------------------------------------------------------------

def canonicalize(n: int, src, dst) -> tuple[np.ndarray, np.ndarray]:
    """Symmetrise, drop self-loops and duplicates, sort rows (Section 3.1 input)."""
    lib = _load()
    src, dst = _u32(src), _u32(dst)
    rp = np.zeros(n + 1, dtype=np.uint32)
    cap = 2 * src.size + 1
    col = np.zeros(cap, dtype=np.uint32)
    nnz = ctypes.c_uint64()
    rc = lib.or_canonicalize(n, src.size, src, dst, rp, col, cap, ctypes.byref(nnz))
    if rc != 0:
        raise ValueError(f"or_canonicalize failed ({rc})")
    return rp, col[: nnz.value].copy()


def degree_rank(row_ptr) -> np.ndarray:
    """rank[v] in the (degree, id) order (Section 3.1, degree orientation)."""
    rp = _u32(row_ptr)
    n = rp.size - 1
    rank = np.zeros(max(n, 1), dtype=np.uint32)[:n].copy() if n else np.zeros(0, dtype=np.uint32)
    _load().or_degree_rank(n, rp, rank if n else np.zeros(1, dtype=np.uint32))
    return rank


@dataclass
class Degeneracy:
    rank: np.ndarray
    core: np.ndarray
    order: np.ndarray
    degeneracy: int


def degeneracy_order(row_ptr, col_idx) -> Degeneracy:
    """k-core removal order and core numbers (Section 3.1, degeneracy orientation)."""
    rp, ci = _u32(row_ptr), _u32(col_idx)
    n = rp.size - 1
    m = max(n, 1)
    rank = np.zeros(m, dtype=np.uint32)
    core = np.zeros(m, dtype=np.uint32)
    order = np.zeros(m, dtype=np.uint32)
    d = _load().or_degeneracy_order(n, rp, ci if ci.size else np.zeros(1, np.uint32), rank, core, order)
    return Degeneracy(rank[:n], core[:n], order[:n], int(d))


def orient(row_ptr, col_idx, rank) -> tuple[np.ndarray, np.ndarray, int]:
    """DAG keeping u->w iff rank[u] < rank[w]; returns (dag_row_ptr, dag_col, d_max)."""
    rp, ci, rk = _u32(row_ptr), _u32(col_idx), _u32(rank)
    n = rp.size - 1
    drp = np.zeros(n + 1, dtype=np.uint32)
    dci = np.zeros(max(ci.size // 2, 1), dtype=np.uint32)
    dmax = _load().or_orient(n, rp, ci if ci.size else np.zeros(1, np.uint32), rk if n else np.zeros(1, np.uint32),
                             drp, dci)
    return drp, dci[: int(drp[-1])].copy(), int(dmax)


@dataclass
class OrientResult:
    total: int | None          # None = exceeded 2^128 - 1
    per_root: np.ndarray | None  # low 64 bits per root
    per_vertex: list | None      # exact ints


def count_orient(dag_row_ptr, dag_col, k: int, roots=None, threads: int | None = None,
                 per_root: bool = False, per_vertex: bool = False) -> OrientResult:
    """c_k by the orientation traversal (Fig. 2) over a DAG."""
    lib = _load()
    rp, ci = _u32(dag_row_ptr), _u32(dag_col)
    if ci.size == 0:
        ci = np.zeros(1, dtype=np.uint32)
    n = rp.size - 1
    r = None if roots is None else _u32(roots)
    nr = n if r is None else r.size
    pr = np.zeros(max(nr, 1), dtype=np.uint64) if per_root else None
    pvl = np.zeros(max(n, 1), dtype=np.uint64) if per_vertex else None
    pvh = np.zeros(max(n, 1), dtype=np.uint64) if per_vertex else None
    lo, hi = ctypes.c_uint64(), ctypes.c_uint64()
    sat = lib.or_count_orient(n, rp, ci, k, _ptr(r), nr, threads or default_threads(), ctypes.byref(lo),
                              ctypes.byref(hi), _ptr(pr), _ptr(pvl), _ptr(pvh))
    pv = None
    if per_vertex:
        pv = [_join(a, b) for a, b in zip(pvl[:n], pvh[:n])]
    return OrientResult(None if sat else _join(lo.value, hi.value), pr[:nr] if per_root else None, pv)


@dataclass
class PivotResult:
    counts: list               # counts[j] exact int, or None if saturated (j < cap)
    max_clique: int
    per_vertex: list | None


def count_pivot(row_ptr, col_idx, dag_row_ptr, dag_col, cap: int | None = None, kfix: int = 0,
                roots=None, threads: int | None = None, per_vertex_k: int = 0) -> PivotResult:
    """All-k (kfix = 0) or fixed-k counts by the pivoting traversal (Fig. 3)."""
    lib = _load()
    rp, ci = _u32(row_ptr), _u32(col_idx)
    drp, dci = _u32(dag_row_ptr), _u32(dag_col)
    if ci.size == 0:
        ci = np.zeros(1, dtype=np.uint32)
    if dci.size == 0:
        dci = np.zeros(1, dtype=np.uint32)
    n = rp.size - 1
    dmax = int(np.diff(drp.astype(np.int64)).max()) if n else 0
    if cap is None:
        cap = dmax + 2
    cap = max(cap, 2)
    lo = np.zeros(cap, dtype=np.uint64)
    hi = np.zeros(cap, dtype=np.uint64)
    sat = np.zeros(cap, dtype=np.uint8)
    r = None if roots is None else _u32(roots)
    nr = n if r is None else r.size
    want_pv = per_vertex_k > 0
    pvl = np.zeros(max(n, 1), dtype=np.uint64) if want_pv else None
    pvh = np.zeros(max(n, 1), dtype=np.uint64) if want_pv else None
    omega = ctypes.c_uint32()
    lib.or_count_pivot(n, rp, ci, drp, dci, cap, kfix, _ptr(r), nr, threads or default_threads(), lo, hi, sat,
                       per_vertex_k, _ptr(pvl), _ptr(pvh), ctypes.byref(omega))
    counts = [None if sat[j] else _join(lo[j], hi[j]) for j in range(cap)]
    pv = [_join(a, b) for a, b in zip(pvl[:n], pvh[:n])] if want_pv else None
    return PivotResult(counts, int(omega.value), pv)


def count_vertex(row_ptr, col_idx, v: int, k: int) -> int | None:
    """c_k(v): the (k-1)-cliques of the sub-graph induced by N(v)."""
    rp, ci = _u32(row_ptr), _u32(col_idx)
    if ci.size == 0:
        ci = np.zeros(1, dtype=np.uint32)
    lo, hi = ctypes.c_uint64(), ctypes.c_uint64()
    sat = _load().or_count_vertex(rp.size - 1, rp, ci, v, k, ctypes.byref(lo), ctypes.byref(hi))
    return None if sat else _join(lo.value, hi.value)


# ----------------------------------------------------------------------------
# Convenience: whole-graph counts from an undirected CSR.
# ----------------------------------------------------------------------------

def dag_for(row_ptr, col_idx, order: str = "degree"):
    """(dag_row_ptr, dag_col, d_max, rank) for 'degree', 'degeneracy' or an explicit rank array."""
    if isinstance(order, str):
        if order == "degree":
            rank = degree_rank(row_ptr)
        elif order == "degeneracy":
            rank = degeneracy_order(row_ptr, col_idx).rank
        else:
            raise ValueError(order)
    else:
        rank = _u32(order)
    drp, dci, dmax = orient(row_ptr, col_idx, rank)
    return drp, dci, dmax, rank


def count(row_ptr, col_idx, k: int, order: str = "degree", threads: int | None = None) -> int | None:
    """c_k(G) by Fig. 2 after orienting by ``order``."""
    drp, dci, _, _ = dag_for(row_ptr, col_idx, order)
    return count_orient(drp, dci, k, threads=threads).total


def count_all(row_ptr, col_idx, order: str = "degeneracy", threads: int | None = None) -> PivotResult:
    """Every c_k(G) by Fig. 3 after orienting by ``order``."""
    drp, dci, _, _ = dag_for(row_ptr, col_idx, order)
    return count_pivot(row_ptr, col_idx, drp, dci, threads=threads)
