"""Pins of the CPU oracle against facts it does not compute itself.

Each test ties the oracle to mathematics or to a library routine, never to
the oracle's own formulas: closed forms (C(n, k), elementary symmetric
polynomials), union/join identities, triangle-free families, trace(A^3)/6,
brute force over every k-subset, networkx core numbers and clique
enumeration, orientation invariance and the paper's worked fragments.
"""
import itertools
import json
import math
import os

import networkx as nx
import numpy as np
import pytest

from oracle import oracle as O
from paper_2104_13209_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def all_counts_orient(g, kmax, order="degree"):
    drp, dci, _, _ = O.dag_for(g.row_ptr, g.col_idx, order)
    return [O.count_orient(drp, dci, k, threads=2).total for k in range(1, kmax + 1)]


def all_counts_pivot(g, order="degeneracy"):
    """Pivot-route counts; entries past the returned cap (> clique number) are 0."""
    r = O.count_all(g.row_ptr, g.col_idx, order, threads=2)
    r.counts = r.counts + [0] * 200
    return r


def brute_force_counts(g, kmax):
    """Every k-subset tested pair by pair (itertools, an adjacency matrix)."""
    A = np.zeros((g.n, g.n), dtype=bool)
    a, b = g.edge_pairs()
    A[a, b] = True
    A[b, a] = True
    out = []
    for k in range(1, kmax + 1):
        c = 0
        for S in itertools.combinations(range(g.n), k):
            if all(A[x, y] for x, y in itertools.combinations(S, 2)):
                c += 1
        out.append(c)
    return out


def brute_force_per_vertex(g, k):
    A = np.zeros((g.n, g.n), dtype=bool)
    a, b = g.edge_pairs()
    A[a, b] = True
    A[b, a] = True
    pv = [0] * g.n
    for S in itertools.combinations(range(g.n), k):
        if all(A[x, y] for x, y in itertools.combinations(S, 2)):
            for v in S:
                pv[v] += 1
    return pv


def elementary_symmetric(parts, k):
    """e_k(a_1..a_r) by expanding prod (1 + a_i x)."""
    poly = [1]
    for a in parts:
        nxt = poly + [0]
        for i in range(len(poly)):
            nxt[i + 1] += poly[i] * a
        poly = nxt
    return poly[k] if k < len(poly) else 0


def trace_a3_over_6(g):
    """Triangles = trace(A^3) / 6 with a float64 BLAS product (exact: entries < 2^53)."""
    A = np.zeros((g.n, g.n), dtype=np.float64)
    a, b = g.edge_pairs()
    A[a, b] = 1.0
    A[b, a] = 1.0
    t = float(np.sum((A @ A) * A))
    assert t == round(t) and int(t) % 6 == 0
    return int(t) // 6


# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 13])
def test_complete_graph_closed_form(n):
    g = synth.complete_graph(n)
    for order in ("degree", "degeneracy"):
        got = all_counts_orient(g, n + 1, order)
        assert got == [math.comb(n, k) for k in range(1, n + 2)]
    piv = all_counts_pivot(g)
    assert piv.counts[1: n + 1] == [math.comb(n, k) for k in range(1, n + 1)]
    assert piv.max_clique == n


def test_complete_graph_per_vertex():
    n = 11
    g = synth.complete_graph(n)
    drp, dci, _, _ = O.dag_for(g.row_ptr, g.col_idx, "degeneracy")
    for k in (1, 2, 3, 6, 11):
        r = O.count_orient(drp, dci, k, per_vertex=True)
        assert r.per_vertex == [math.comb(n - 1, k - 1)] * n
        p = O.count_pivot(g.row_ptr, g.col_idx, drp, dci, per_vertex_k=k)
        assert p.per_vertex == [math.comb(n - 1, k - 1)] * n
        assert O.count_vertex(g.row_ptr, g.col_idx, 3, k) == math.comb(n - 1, k - 1)


def test_overflow_pins_k67_k68():
    """K_67 at k=33 fits in u64; K_68 at k=34 does not."""
    g67 = synth.complete_graph(67)
    g68 = synth.complete_graph(68)
    c67 = all_counts_pivot(g67).counts
    c68 = all_counts_pivot(g68).counts
    assert c67[33] == 14_226_520_737_620_288_370 == math.comb(67, 33)
    assert c67[33] < 2 ** 64
    assert c68[34] == 28_453_041_475_240_576_740 == math.comb(68, 34)
    assert c68[34] >= 2 ** 64
    assert c68 [1:69] == [math.comb(68, k) for k in range(1, 69)]


@pytest.mark.parametrize("parts", [[3, 3, 3], [1, 2, 3, 4], [5, 1], [2, 2, 2, 2, 2, 2], [7, 3, 3, 1, 1]])
def test_complete_multipartite(parts):
    g = synth.complete_multipartite(parts)
    r = len(parts)
    want = [elementary_symmetric(parts, k) for k in range(1, r + 3)]
    for order in ("degree", "degeneracy"):
        assert all_counts_orient(g, r + 2, order) == want
    piv = all_counts_pivot(g)
    assert piv.counts[1: r + 2] == want[: r + 1]
    assert piv.max_clique == r


def test_turan():
    g = synth.turan_graph(17, 5)
    parts = [4, 4, 3, 3, 3]
    for k in range(1, 7):
        assert O.count(g.row_ptr, g.col_idx, k) == elementary_symmetric(parts, k)


def test_disjoint_union_adds():
    g1 = synth.dense_random_graph(14, 0.6, 1)
    g2 = synth.dense_random_graph(12, 0.7, 2)
    u = synth.disjoint_union([g1, g2])
    a = all_counts_orient(g1, 8)
    b = all_counts_orient(g2, 8)
    c = all_counts_orient(u, 8)
    assert c == [x + y for x, y in zip(a, b)]


def test_join_convolution():
    g = synth.dense_random_graph(9, 0.5, 3)
    h = synth.dense_random_graph(8, 0.6, 4)
    j = synth.join(g, h)
    cg = [1] + all_counts_orient(g, 10)
    ch = [1] + all_counts_orient(h, 10)
    cj = all_counts_orient(j, 10)
    for k in range(1, 11):
        assert cj[k - 1] == sum(cg[i] * ch[k - i] for i in range(0, k + 1))
    assert all_counts_pivot(j).counts[1:11] == cj


@pytest.mark.parametrize("which", ["tree", "cycle", "bipartite"])
def test_triangle_free(which):
    g = {"tree": synth.random_tree(300, 5), "cycle": synth.cycle_graph(40),
         "bipartite": synth.random_bipartite(30, 25, 0.4, 6)}[which]
    got = all_counts_orient(g, 5)
    assert got == [g.n, g.num_edges, 0, 0, 0]
    assert all_counts_pivot(g).counts[1:4] == [g.n, g.num_edges, 0]


def test_triangles_trace_identity():
    for g in (synth.erdos_renyi(400, 0.08, 7), synth.erdos_renyi(2000, 0.01, 0), synth.rmat(10, 8, seed=3)):
        tri = trace_a3_over_6(g)
        assert O.count(g.row_ptr, g.col_idx, 3) == tri
        assert O.count(g.row_ptr, g.col_idx, 3, "degeneracy") == tri
        assert all_counts_pivot(g).counts[3] == tri


@pytest.mark.parametrize("seed,p", [(1, 0.3), (2, 0.5), (3, 0.7), (4, 0.9)])
def test_brute_force_small(seed, p):
    g = synth.dense_random_graph(15, p, seed)
    kmax = 9
    want = brute_force_counts(g, kmax)
    assert all_counts_orient(g, kmax, "degree") == want
    assert all_counts_orient(g, kmax, "degeneracy") == want
    piv = all_counts_pivot(g)
    assert piv.counts[1: kmax + 1] == want
    for k in (3, 4):
        bf = brute_force_per_vertex(g, k)
        drp, dci, _, _ = O.dag_for(g.row_ptr, g.col_idx, "degeneracy")
        assert O.count_orient(drp, dci, k, per_vertex=True).per_vertex == bf
        assert O.count_pivot(g.row_ptr, g.col_idx, drp, dci, per_vertex_k=k).per_vertex == bf
        assert [O.count_vertex(g.row_ptr, g.col_idx, v, k) for v in range(g.n)] == bf


def test_fixed_k_pivot_matches_all_k():
    g = synth.dense_random_graph(40, 0.6, 8)
    drp, dci, _, _ = O.dag_for(g.row_ptr, g.col_idx, "degeneracy")
    allk = O.count_pivot(g.row_ptr, g.col_idx, drp, dci).counts
    for k in range(3, 10):
        fixed = O.count_pivot(g.row_ptr, g.col_idx, drp, dci, kfix=k).counts[k]
        assert fixed == allk[k]


def test_networkx_cliques_and_cores():
    for seed, (n, p) in enumerate([(60, 0.3), (45, 0.5), (30, 0.75)]):
        g = synth.dense_random_graph(n, p, 100 + seed)
        G = nx.Graph()
        G.add_nodes_from(range(g.n))
        G.add_edges_from(zip(*g.edge_pairs()))
        by_size = {}
        for c in nx.enumerate_all_cliques(G):
            by_size[len(c)] = by_size.get(len(c), 0) + 1
        omega = max(by_size)
        piv = all_counts_pivot(g)
        assert piv.max_clique == omega
        assert piv.counts[1: omega + 2] == [by_size.get(k, 0) for k in range(1, omega + 2)]
        assert all_counts_orient(g, omega + 1) == [by_size.get(k, 0) for k in range(1, omega + 2)]
        core = nx.core_number(G)
        dg = O.degeneracy_order(g.row_ptr, g.col_idx)
        assert [int(x) for x in dg.core] == [core[v] for v in range(g.n)]
        assert dg.degeneracy == max(core.values())


def test_degeneracy_bounds_out_degree_and_cores_rmat():
    g = synth.rmat(12, 16, seed=1)
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    G.add_edges_from(zip(*g.edge_pairs()))
    core = nx.core_number(G)
    dg = O.degeneracy_order(g.row_ptr, g.col_idx)
    assert [int(x) for x in dg.core] == [core[v] for v in range(g.n)]
    _, _, dmax = O.orient(g.row_ptr, g.col_idx, dg.rank)
    assert dmax == dg.degeneracy


def test_orientation_invariance():
    g = synth.rmat(11, 16, seed=2)
    base = [O.count(g.row_ptr, g.col_idx, k) for k in range(1, 7)]
    for seed in (1, 2):
        rank = synth.random_permutation(g.n, seed).astype(np.uint32)
        drp, dci, _, _ = O.dag_for(g.row_ptr, g.col_idx, rank)
        assert [O.count_orient(drp, dci, k).total for k in range(1, 7)] == base
    assert [O.count(g.row_ptr, g.col_idx, k, "degeneracy") for k in range(1, 7)] == base
    assert all_counts_pivot(g).counts[1:7] == base
    assert all_counts_pivot(g, "degree").counts[1:7] == base


def test_dag_keeps_each_edge_once():
    g = synth.rmat(10, 8, seed=4)
    for order in ("degree", "degeneracy"):
        drp, dci, _, rank = O.dag_for(g.row_ptr, g.col_idx, order)
        src = np.repeat(np.arange(g.n), np.diff(drp.astype(np.int64)))
        assert dci.size == g.num_edges
        assert np.all(rank[src] < rank[dci])
        und = set(zip(*g.edge_pairs()))
        got = {(min(a, b), max(a, b)) for a, b in zip(src.tolist(), dci.tolist())}
        assert got == {(int(a), int(b)) for a, b in und}


def test_per_vertex_sum_identity():
    g = synth.rmat(10, 16, seed=5)
    drp, dci, _, _ = O.dag_for(g.row_ptr, g.col_idx, "degeneracy")
    for k in (3, 4, 5):
        r = O.count_orient(drp, dci, k, per_vertex=True)
        assert sum(r.per_vertex) == k * r.total
        p = O.count_pivot(g.row_ptr, g.col_idx, drp, dci, per_vertex_k=k)
        assert p.per_vertex == r.per_vertex
        for v in (0, 1, 17, 100):
            assert O.count_vertex(g.row_ptr, g.col_idx, v, k) == r.per_vertex[v]


def test_canonicalize_matches_definition():
    rng_u = synth.random_u64(synth.stream_key(9, 1), np.arange(3000, dtype=np.uint64)) % np.uint64(200)
    rng_v = synth.random_u64(synth.stream_key(9, 2), np.arange(3000, dtype=np.uint64)) % np.uint64(200)
    u = rng_u.astype(np.uint32)
    v = rng_v.astype(np.uint32)
    rp, col = O.canonicalize(200, u, v)
    want = {}
    for a, b in zip(u.tolist(), v.tolist()):
        if a != b:
            want.setdefault(a, set()).add(b)
            want.setdefault(b, set()).add(a)
    for x in range(200):
        assert col[rp[x]: rp[x + 1]].tolist() == sorted(want.get(x, ()))
    g = synth.edges_to_csr(200, u, v)
    assert np.array_equal(g.row_ptr, rp) and np.array_equal(g.col_idx, col)


def test_paper_fragments():
    with open(os.path.join(GOLDEN, "paper_fragments.json")) as f:
        frags = json.load(f)["fragments"]
    for fr in frags:
        g = synth.complete_graph(fr["n"])
        assert O.count(g.row_ptr, g.col_idx, fr["k"]) == fr["count"]
        assert all_counts_pivot(g).counts[fr["k"]] == fr["count"]


def test_er_config_small_counts():
    """G(2000, 0.01), seed 0: triangles and 4-cliques pinned by trace(A^3)/6
    and by brute force over (triangle, common neighbour) pairs."""
    g = synth.erdos_renyi(2000, 0.01, 0)
    a, b = g.edge_pairs()
    tri = trace_a3_over_6(g)
    G = nx.Graph()
    G.add_edges_from(zip(a.tolist(), b.tolist()))
    four = 0
    for x, y, z in (c for c in nx.enumerate_all_cliques(G) if len(c) == 3):
        common = set(G[x]) & set(G[y]) & set(G[z])
        four += sum(1 for w in common if w > max(x, y, z))
    assert O.count(g.row_ptr, g.col_idx, 3, "degeneracy") == tri
    assert O.count(g.row_ptr, g.col_idx, 4, "degeneracy") == four


@pytest.mark.parametrize("parts", [[3, 4, 5], [1, 2, 3, 4], [6, 6, 6, 6], [2, 9]])
def test_per_vertex_complete_multipartite(parts):
    # a vertex of part i lies in e_{k-1}(the other parts) k-cliques
    g = synth.complete_multipartite(parts)
    drp, dci, _, _ = O.dag_for(g.row_ptr, g.col_idx, "degeneracy")
    start = np.cumsum([0] + parts)
    for k in range(2, len(parts) + 2):
        pv = O.count_orient(drp, dci, k, per_vertex=True).per_vertex
        piv = O.count_pivot(g.row_ptr, g.col_idx, drp, dci, per_vertex_k=k).per_vertex
        for i, a in enumerate(parts):
            want = elementary_symmetric(parts[:i] + parts[i + 1:], k - 1)
            for v in range(start[i], start[i] + a):
                assert pv[v] == want and piv[v] == want, (parts, k, i)


def test_per_vertex_join_with_a_clique():
    # G join K_m: a vertex of K_m lies in sum_j c_j(G) C(m-1, k-1-j) k-cliques
    h = synth.erdos_renyi(40, 0.2, 5)
    m = 4
    g = synth.join(h, synth.complete_graph(m))
    drp, dci, _, _ = O.dag_for(g.row_ptr, g.col_idx, "degree")
    c = [1] + [O.count(h.row_ptr, h.col_idx, j) if j > 2 else (h.n if j == 1 else h.num_edges) for j in range(1, 8)]
    for k in range(2, 7):
        pv = O.count_orient(drp, dci, k, per_vertex=True).per_vertex
        want = sum(c[j] * math.comb(m - 1, k - 1 - j) for j in range(0, k))
        assert all(pv[v] == want for v in range(h.n, h.n + m)), k


def test_degree_rank_hand_computed_with_ties():
    """Degree orientation (Section 3.1) orders vertices by (degree, id).  The
    graph has a four-way degree tie, an isolated vertex and one vertex of
    largest degree; the expected ranks and DAG rows were worked out by hand:
      degrees   0:3  1:2  2:2  3:2  4:1  5:2  6:2  7:0
      order     7 (deg 0), 4 (deg 1), 1 2 3 5 6 (deg 2, ascending id), 0 (deg 3)
    Ties broken by descending id, or sorting by descending degree, give other
    ranks and other DAGs."""
    edges = [(0, 1), (0, 2), (0, 3), (1, 2), (4, 5), (5, 6), (3, 6)]
    g = synth.edges_to_csr(8, np.array([a for a, _ in edges]), np.array([b for _, b in edges]))
    rank = O.degree_rank(g.row_ptr)
    assert [int(x) for x in rank] == [7, 2, 3, 4, 1, 5, 6, 0]
    drp, dci, dmax = O.orient(g.row_ptr, g.col_idx, rank)
    rows = [sorted(int(x) for x in dci[drp[v]:drp[v + 1]]) for v in range(g.n)]
    # u -> w iff rank[u] < rank[w]
    assert rows == [[], [0, 2], [0], [0, 6], [5], [6], [], []]
    assert dmax == 2


def test_degree_rank_is_a_permutation_sorted_by_degree_then_id():
    # on R-MAT graphs (thousands of ties): consecutive ranks never decrease in
    # degree, and within one degree they increase with the id
    for seed in (1, 2):
        g = synth.rmat(11, 8, seed=seed)
        rank = O.degree_rank(g.row_ptr).astype(np.int64)
        deg = np.diff(g.row_ptr.astype(np.int64))
        order = np.empty(g.n, dtype=np.int64)
        order[rank] = np.arange(g.n)
        assert np.array_equal(np.sort(rank), np.arange(g.n))
        d = deg[order]
        assert np.all(np.diff(d) >= 0)
        same = np.diff(d) == 0
        assert np.all(np.diff(order)[same] > 0)
