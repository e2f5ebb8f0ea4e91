"""Generators of many small graphs: Barabasi-Albert, radius-1 ego networks
and the block-diagonal union (inputs only, checked against their
definitions)."""
import math

import numpy as np
import pytest

from paper_2104_13209_gb300 import synth


def test_barabasi_albert_shape_and_determinism():
    g = synth.barabasi_albert(3000, 6, seed=2)
    h = synth.barabasi_albert(3000, 6, seed=2)
    assert np.array_equal(g.row_ptr, h.row_ptr) and np.array_equal(g.col_idx, h.col_idx)
    deg = g.degrees()
    assert deg.min() >= 1
    # at most m new edges per vertex after the seed clique, and few lost to repeats
    most = 6 * 7 // 2 + (3000 - 7) * 6
    assert 0.97 * most <= g.num_edges <= most
    # preferential attachment: the early vertices collect the high degrees
    assert deg[:50].mean() > 4 * deg[-1000:].mean()


def test_ego_network_definition():
    nx = pytest.importorskip("networkx")
    g = synth.barabasi_albert(800, 4, seed=3)
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    a, b = g.edge_pairs()
    G.add_edges_from(zip(a.tolist(), b.tolist()))
    for c in (0, 5, 100, 799):
        e = synth.ego_network(g, c)
        E = nx.ego_graph(G, c, radius=1)
        assert e.n == E.number_of_nodes() and e.num_edges == E.number_of_edges()


def test_ego_networks_sizes_and_union():
    g = synth.barabasi_albert(5000, 5, seed=1)
    egos = synth.ego_networks(g, 30, 20, 300, seed=0)
    assert len(egos) == 30 and all(20 <= e.n <= 300 for e in egos)
    u, off = synth.block_union(egos)
    assert off[0] == 0 and off[-1] == u.n == sum(e.n for e in egos)
    for i, e in enumerate(egos):
        a, b = off[i], off[i + 1]
        rows = u.row_ptr[a:b + 1]
        seg = u.col_idx[rows[0]:rows[-1]]
        assert seg.size == 2 * e.num_edges and (seg.size == 0 or (seg.min() >= a and seg.max() < b))
        assert np.array_equal(seg - a, e.col_idx)


def test_serving_recipes():
    from paper_2104_13209_gb300 import workloads

    kinds = [workloads.serve_spec(i)[0] for i in range(workloads.POOL_SIZE)]
    assert kinds.count("er") == 16 and kinds.count("rmat") == 24 and kinds.count("chunglu") == 24
    for i in range(workloads.POOL_SIZE):
        s = workloads.serve_spec(i)
        if s[0] == "er":
            assert 10_000 <= s[1] <= 100_000 and 8 <= s[2] * (s[1] - 1) <= 32
        elif s[0] == "rmat":
            assert 14 <= s[1] <= 18
        else:
            assert 100_000 <= s[1] <= 1_000_000
    t, g, k, p = workloads.query_stream(2000.0, 5.0)
    t2, g2, k2, p2 = workloads.query_stream(2000.0, 5.0)
    assert np.array_equal(t, t2) and np.array_equal(g, g2) and np.array_equal(k, k2) and np.array_equal(p, p2)
    assert abs(t.size - 10_000) < 4 * math.sqrt(10_000)  # a Poisson count within 4 sigma
    assert np.all(np.diff(t) > 0) and t[-1] < 5.0
    assert g.min() >= 0 and g.max() < 64 and k.min() == 3 and k.max() == 12
    assert 0.45 < p.mean() < 0.55
