"""Shared helpers of the GPU tests (the CUDA path through the C ABI)."""
import math

import numpy as np

from paper_2104_13209_gb300 import build, kclique, synth

_built = False


def lib():
    global _built
    if not _built:
        build.build()
        _built = True
    return kclique.load()


def graph(g, orient="degeneracy", validate=True):
    lib()
    return kclique.Graph(g.row_ptr, g.col_idx, n=g.n, orient=orient, validate=validate)


def elementary_symmetric(parts, k):
    poly = [1]
    for a in parts:
        nxt = poly + [0]
        for i in range(len(poly)):
            nxt[i + 1] += poly[i] * a
        poly = nxt
    return poly[k] if k < len(poly) else 0


def complete_counts(n, k):
    return math.comb(n, k)


def csr_from_pairs(n, pairs):
    """Raw CSR with rows sorted as given (no canonicalisation) for invalid-graph tests."""
    rows = [[] for _ in range(n)]
    for a, b in pairs:
        rows[a].append(b)
    rp = np.zeros(n + 1, dtype=np.uint32)
    for i, r in enumerate(rows):
        rp[i + 1] = rp[i] + len(r)
    ci = np.array([x for r in rows for x in r], dtype=np.uint32)
    return rp, ci


__all__ = ["lib", "graph", "elementary_symmetric", "complete_counts", "csr_from_pairs", "synth", "kclique"]
