"""Parity at the widths the full-size workloads reach.

The R-MAT and Chung-Lu configurations have roots with 519 to 612 candidates
(17 to 20 bitmap words per row).  These graphs put the GPU's traversals at
that width and beyond, on inputs whose exact counts are known:

- K_{260,260,260} joined with K_18 (a complete multipartite graph with 18
  singleton parts): every candidate set of the first roots has 538 members
  (17 words).  Pivoting walks a chain of 18 universal pivots before it
  branches, so each warp holds more than 16 wide stack levels and spills
  the deeper ones to global memory.  Counts are the elementary symmetric
  polynomials of the part sizes; per-vertex counts those of the other parts.
- A sparse random graph C on 1,400 vertices joined with 1,500 independent
  vertices: every independent vertex is a root whose candidate set is all
  of C (1,400 members, 44 words per row), too large for shared memory, so
  the orientation traversal keeps its bitmaps and stacks in global memory,
  and pivoting keeps its adjacency there.  The join identity gives
  c_k = c_k(C) + 1500 c_{k-1}(C), with c_j(C) from the oracle.
- K_{300,300}: 300 candidates per root and no triangle.

Counts are integers: the bar is exact equality.
"""
import functools

import numpy as np
import pytest

from oracle import oracle as O
from tests.gpu_common import elementary_symmetric, graph, synth

pytestmark = pytest.mark.gpu

PARTS = [260, 260, 260] + [1] * 18
B_INDEP = 1500


@functools.lru_cache(maxsize=None)
def multipartite():
    return synth.complete_multipartite(PARTS)


@functools.lru_cache(maxsize=None)
def sparse_core():
    return synth.erdos_renyi(1400, 0.1, seed=7)


@functools.lru_cache(maxsize=None)
def join_indep():
    return synth.join(sparse_core(), synth.complete_multipartite([B_INDEP]))


@functools.lru_cache(maxsize=None)
def core_counts(kmax):
    c = sparse_core()
    drp, dci, _, _ = O.dag_for(c.row_ptr, c.col_idx, "degeneracy")
    return [1] + [O.count_orient(drp, dci, k).total for k in range(1, kmax + 1)]


def join_count(k):
    cc = core_counts(12)
    return cc[k] + B_INDEP * cc[k - 1]


def test_widths_reached():
    G = graph(multipartite())
    assert G.info()["d_max"] == 538
    G = graph(join_indep(), "degree")
    assert G.info()["d_max"] == 1400
    G = graph(join_indep(), "degeneracy")
    assert G.info()["d_max"] == 1400


@pytest.mark.parametrize("orient", ["degeneracy", "degree"])
def test_multipartite_wide_all_k_pivot(orient):
    G = graph(multipartite(), orient)
    r = len(PARTS)
    counts, ovf, om, _ = G.count_all(cap=r + 2)
    assert om == r
    for j in range(1, r + 2):
        assert ovf[j] == 0 and int(counts[j]) == elementary_symmetric(PARTS, j), j


@pytest.mark.parametrize("k", [3, 4, 6, 9, 14, 21])
def test_multipartite_wide_fixed_k_pivot(k):
    G = graph(multipartite())
    assert G.count(k, pivot=True).total == elementary_symmetric(PARTS, k)


@pytest.mark.parametrize("k", [3, 4, 5])
def test_multipartite_wide_orientation(k):
    for orient in ("degeneracy", "degree"):
        G = graph(multipartite(), orient)
        for scheme in ("vc", "ec"):
            for sw in ((4, 8, 32) if k <= 4 else (0,)):
                got = G.count(k, scheme=scheme, subwarp=sw).total
                assert got == elementary_symmetric(PARTS, k), (orient, k, scheme, sw)


@pytest.mark.parametrize("k", [3, 5, 8])
def test_multipartite_wide_per_vertex(k):
    # both traversals: pivoting, and orientation mode with either split
    G = graph(multipartite())
    label = np.repeat(np.arange(len(PARTS)), PARTS)
    for pivot, scheme in ((True, "auto"), (False, "vc"), (False, "ec")):
        tot, pv, fl = G.count_per_vertex(k, pivot=pivot, scheme=scheme)
        assert tot == elementary_symmetric(PARTS, k)
        for part in range(len(PARTS)):
            others = PARTS[:part] + PARTS[part + 1:]
            want = elementary_symmetric(others, k - 1)
            assert np.all(pv[label == part] == want), (k, part, pivot, scheme)


@pytest.mark.parametrize("orient", ["degeneracy", "degree"])
def test_global_scratch_orientation_deep(orient):
    # bitmaps of 1,400 x 44 words do not fit in shared memory: every level
    # the DFS pushes lives in global memory (k >= 5 pushes at least one)
    G = graph(join_indep(), orient)
    for k in (3, 4, 5, 6, 7):
        want = join_count(k)
        for scheme in ("vc", "ec"):
            # group widths matter to the k <= 4 traversal only
            for sw in ((1, 8, 32) if k <= 4 else (0,)):
                got = G.count(k, scheme=scheme, subwarp=sw).total
                assert got == want, (orient, k, scheme, sw)


def test_global_scratch_per_vertex_orientation():
    # per-vertex counts with 1,400-wide candidate sets (bitmaps, transposes
    # and stacks in global memory).  The join identity per vertex: a vertex v
    # of C is in c_k^C(v) + 1500 c_{k-1}^C(v) k-cliques, an independent vertex
    # in c_{k-1}(C); c^C(v) from the oracle's per-vertex counts on C.
    c = sparse_core()
    cdrp, cdci, _, _ = O.dag_for(c.row_ptr, c.col_idx, "degeneracy")
    G = graph(join_indep())
    for k in (3, 4, 5, 6):
        pk = O.count_orient(cdrp, cdci, k, per_vertex=True).per_vertex
        pk1 = O.count_orient(cdrp, cdci, k - 1, per_vertex=True).per_vertex
        want = [a + B_INDEP * b for a, b in zip(pk, pk1)] + [core_counts(12)[k - 1]] * B_INDEP
        for scheme in ("vc", "ec"):
            tot, pv, fl = G.count_per_vertex(k, pivot=False, scheme=scheme)
            assert tot == join_count(k), (k, scheme)
            assert [int(x) for x in pv] == want, (k, scheme)


def test_global_scratch_pivot():
    G = graph(join_indep())
    cc = core_counts(12)
    om_c = max(j for j in range(len(cc)) if cc[j] > 0)
    counts, ovf, om, _ = G.count_all(cap=om_c + 3)
    assert om == om_c + 1
    for j in range(1, om_c + 3):
        assert ovf[j] == 0 and int(counts[j]) == join_count(j), j
    for k in (3, 5):
        assert G.count(k, pivot=True).total == join_count(k)


def test_bipartite_wide_no_triangles():
    g = synth.complete_multipartite([300, 300])
    G = graph(g)
    assert G.info()["d_max"] == 300
    for k in (3, 4):
        assert G.count(k, scheme="vc").total == 0
        assert G.count(k, scheme="ec").total == 0
        assert G.count(k, pivot=True).total == 0
    counts, ovf, om, _ = G.count_all(cap=5)
    assert om == 2 and int(counts[2]) == 90000 and int(counts[3]) == 0
