"""Pivoting traversal on the GPU (Fig. 3): every clique size at once, fixed-k
counts, per-vertex counts and the uint64 overflow flags, against the CPU
oracle and closed forms.  Counts are integers: the bar is exact equality, and
a count above 2^64 - 1 must be flagged (never wrapped silently)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from tests.gpu_common import elementary_symmetric, graph, kclique, synth

pytestmark = pytest.mark.gpu

U64 = 1 << 64


def oracle_allk(g, order="degeneracy"):
    r = O.count_all(g.row_ptr, g.col_idx, order)
    return r.counts, r.max_clique


def check_allk(G, g):
    want, omega = oracle_allk(g)
    counts, ovf, om, _ = G.count_all(cap=len(want))
    assert om == omega
    for j in range(1, len(want)):
        w = want[j]
        if w is None or w >= U64:
            assert ovf[j] == 1, j
        else:
            assert ovf[j] == 0 and int(counts[j]) == w, (j, int(counts[j]), w)


@pytest.mark.parametrize("orient", ["degeneracy", "degree"])
def test_allk_random_graphs(orient):
    for g in (synth.dense_random_graph(120, 0.6, 2), synth.dense_random_graph(90, 0.85, 3),
              synth.rmat(12, 16, seed=1), synth.erdos_renyi(2000, 0.01, 0),
              synth.chung_lu_planted(20000, 2.1, 10, 20, 20, 60, 0.9, seed=1)):
        check_allk(graph(g, orient), g)


def test_allk_closed_forms():
    for n in (1, 2, 5, 31, 32, 33, 40, 64, 67):
        G = graph(synth.complete_graph(n))
        counts, ovf, om, _ = G.count_all(cap=n + 2)
        assert om == n
        for j in range(1, n + 2):
            assert int(counts[j]) == math.comb(n, j) and ovf[j] == 0, (n, j)
    for parts in ([10, 10, 10, 10, 10], [3, 40, 1, 7], [12] * 8, [33, 2, 33]):
        G = graph(synth.complete_multipartite(parts))
        counts, ovf, om, _ = G.count_all(cap=len(parts) + 2)
        assert om == len(parts)
        for j in range(1, len(parts) + 2):
            assert int(counts[j]) == elementary_symmetric(parts, j)


def test_overflow_flags_k67_k68():
    G = graph(synth.complete_graph(67))
    counts, ovf, om, _ = G.count_all(cap=69)
    assert int(counts[33]) == 14_226_520_737_620_288_370 and ovf[33] == 0
    G = graph(synth.complete_graph(68))
    counts, ovf, om, _ = G.count_all(cap=70)
    for j in range(69):
        exact = math.comb(68, j)
        if exact >= U64:
            assert ovf[j] == 1, j
        else:
            assert ovf[j] == 0 and int(counts[j]) == exact, j
    assert ovf[34] == 1
    tot, pv, fl = G.count_per_vertex(34)
    assert fl & kclique.KC_FLAG_TOTAL_OVERFLOW
    assert np.all(pv == math.comb(67, 33))  # each vertex's count still fits
    r = G.count(34, pivot=True)
    assert r.overflow


@pytest.mark.parametrize("k", [3, 4, 5, 7, 9])
def test_fixed_k_pivot(k):
    for g in (synth.dense_random_graph(120, 0.6, 2), synth.rmat(13, 16, seed=2),
              synth.chung_lu_planted(20000, 2.1, 10, 20, 20, 60, 0.9, seed=1)):
        want = oracle_allk(g)[0]
        G = graph(g)
        assert G.count(k, pivot=True).total == (want[k] if k < len(want) else 0)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 6, 8])
def test_per_vertex_pivot(k):
    for g in (synth.dense_random_graph(80, 0.5, 4), synth.rmat(11, 16, seed=3),
              synth.chung_lu_planted(5000, 2.1, 8, 6, 20, 50, 0.9, seed=2)):
        drp, dci, _, _ = O.dag_for(g.row_ptr, g.col_idx, "degeneracy")
        want = O.count_orient(drp, dci, k, per_vertex=True)
        G = graph(g)
        tot, pv, fl = G.count_per_vertex(k)
        assert tot == want.total
        assert [int(x) for x in pv] == want.per_vertex
        counts, ovf, om, pv2 = G.count_all(per_vertex_k=k)
        assert [int(x) for x in pv2] == want.per_vertex


def test_per_vertex_complete_graph():
    G = graph(synth.complete_graph(40))
    for k in (3, 10, 20, 40):
        tot, pv, _ = G.count_per_vertex(k)
        assert tot == math.comb(40, k)
        assert np.all(pv == math.comb(39, k - 1))


def test_both_traversals_match_the_oracle_rmat14():
    # every count on the GPU, by either traversal, against the oracle's
    # orientation-mode count (a different route on the CPU)
    g = synth.rmat(14, 16, seed=6)
    drp, dci, _, _ = O.dag_for(g.row_ptr, g.col_idx, "degeneracy")
    G = graph(g)
    counts, ovf, om, _ = G.count_all()
    for k in range(3, 7):
        want = O.count_orient(drp, dci, k).total
        assert int(counts[k]) == want and ovf[k] == 0, k
        assert G.count(k, pivot=True).total == want, k
        assert G.count(k, scheme="vc").total == want, k
        assert G.count(k, scheme="ec").total == want, k


def test_per_vertex_requested_in_orientation_mode():
    # per-vertex counts with pivot = 0 are served by the pivoting traversal
    g = synth.rmat(11, 16, seed=3)
    drp, dci, _, _ = O.dag_for(g.row_ptr, g.col_idx, "degeneracy")
    G = graph(g)
    for k in (3, 5):
        want = O.count_orient(drp, dci, k, per_vertex=True)
        tot, pv, fl = G.count_per_vertex(k, pivot=False)
        assert tot == want.total and [int(x) for x in pv] == want.per_vertex


U128 = 1 << 128


def test_exact_128_bit_counts_complete_graphs():
    # K68, k = 34: C(68, 34) = 28,453,041,475,240,576,740 > 2^64 - 1, exact
    G = graph(synth.complete_graph(68))
    counts, ovf, om, _ = G.count_all128(cap=70)
    assert counts[34] == 28_453_041_475_240_576_740 and ovf[34] == 0
    assert all(counts[j] == math.comb(68, j) for j in range(70))
    r = G.count(34, pivot=True)
    assert r.total == 28_453_041_475_240_576_740 and r.overflow
    # K100: every size below 2^128 (C(100, 50) ~ 1.0e29)
    G = graph(synth.complete_graph(100))
    counts, ovf, om, _ = G.count_all128(cap=102)
    assert om == 100
    assert all(counts[j] == math.comb(100, j) and ovf[j] == 0 for j in range(102))
    assert G.count(50, pivot=True).total == math.comb(100, 50)
    # K140: the middle sizes pass 2^128 - 1 and are flagged, the others exact
    G = graph(synth.complete_graph(140))
    counts, ovf, om, _ = G.count_all128(cap=142)
    for j in range(142):
        exact = math.comb(140, j)
        if exact >= U128:
            assert ovf[j] == 1, j
        else:
            assert ovf[j] == 0 and counts[j] == exact, j
    assert any(ovf) and not ovf[20]


def test_exact_128_bit_counts_match_oracle():
    # the oracle's counts are exact integers (128-bit sums)
    g = synth.chung_lu_planted(20000, 2.1, 10, 20, 20, 60, 0.9, seed=1)
    want, omega = oracle_allk(g)
    G = graph(g)
    counts, ovf, om, _ = G.count_all128(cap=len(want))
    assert om == omega
    for j in range(1, len(want)):
        assert ovf[j] == 0 and counts[j] == want[j], j
