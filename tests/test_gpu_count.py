"""Orientation-mode counts on the GPU (Fig. 2) against the CPU oracle and
closed forms, over both schemes, every group width and both orientations.
Counts are integers: the bar is exact equality."""
import json
import math
import os

import pytest

from oracle import oracle as O
from tests.gpu_common import elementary_symmetric, graph, kclique, lib, synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def oracle_counts(g, ks):
    drp, dci, _, _ = O.dag_for(g.row_ptr, g.col_idx, "degeneracy")
    return {k: O.count_orient(drp, dci, k).total for k in ks}


@pytest.mark.parametrize("orient", ["degree", "degeneracy"])
def test_complete_graphs_closed_form(orient):
    for n in (1, 2, 5, 31, 32, 33, 34, 64, 70):
        G = graph(synth.complete_graph(n), orient)
        for k in range(1, min(n, 7) + 2):
            for scheme in ("vc", "ec"):
                assert G.count(k, scheme=scheme).total == math.comb(n, k), (n, k, scheme)


def test_complete_graph_large_k():
    G = graph(synth.complete_graph(36))
    for k in (30, 34, 35, 36, 37):
        assert G.count(k, scheme="vc").total == math.comb(36, k)
        assert G.count(k, scheme="ec").total == math.comb(36, k)


@pytest.mark.parametrize("parts", [[10, 10, 10, 10, 10], [3, 40, 1, 7], [12] * 8, [33, 2, 33]])
def test_multipartite_closed_form(parts):
    G = graph(synth.complete_multipartite(parts))
    for k in range(1, len(parts) + 2):
        want = elementary_symmetric(parts, k)
        for scheme in ("vc", "ec"):
            assert G.count(k, scheme=scheme).total == want, (parts, k, scheme)


@pytest.mark.parametrize("seed,n,p", [(1, 300, 0.3), (2, 120, 0.6), (3, 90, 0.85)])
def test_dense_random_every_group_width(seed, n, p):
    g = synth.dense_random_graph(n, p, seed)
    ks = [3, 4, 5, 6, 7]
    want = oracle_counts(g, ks)
    for orient in ("degree", "degeneracy"):
        G = graph(g, orient)
        for k in ks:
            for scheme in ("vc", "ec"):
                for sw in (1, 2, 4, 8, 16, 32):
                    got = G.count(k, scheme=scheme, subwarp=sw).total
                    assert got == want[k], (orient, k, scheme, sw)


@pytest.mark.parametrize("scale,ef,seed", [(12, 16, 1), (13, 16, 2), (14, 8, 4)])
def test_rmat_parity(scale, ef, seed):
    g = synth.rmat(scale, ef, seed=seed)
    ks = [3, 4, 5, 6, 7, 8]
    want = oracle_counts(g, ks)
    for orient in ("degree", "degeneracy"):
        G = graph(g, orient)
        for k in ks:
            for scheme in ("vc", "ec"):
                assert G.count(k, scheme=scheme).total == want[k], (orient, k, scheme)


def test_er_config_small():
    g = synth.erdos_renyi(2000, 0.01, 0)
    want = oracle_counts(g, [3, 4, 5])
    G = graph(g, "degeneracy")
    for k in (3, 4, 5):
        for scheme in ("vc", "ec"):
            assert G.count(k, scheme=scheme).total == want[k]


def test_union_of_cliques_ragged():
    g = synth.disjoint_union([synth.complete_graph(s) for s in (3, 17, 32, 33, 40, 65, 2, 1)])
    G = graph(g)
    for k in range(1, 9):
        want = sum(math.comb(s, k) for s in (3, 17, 32, 33, 40, 65, 2, 1))
        assert G.count(k, scheme="vc").total == want
        assert G.count(k, scheme="ec").total == want


def test_k_beyond_clique_number_and_invalid_k():
    G = graph(synth.dense_random_graph(60, 0.3, 9))
    d = G.info()["d_max"]
    assert G.count(d + 2).total == 0
    with pytest.raises(kclique.KCError) as e:
        G.count(0)
    assert e.value.status == kclique.KC_E_INVALID_ARG
    with pytest.raises(kclique.KCError):
        G.count(4, subwarp=3)


def test_rmat20_full_size_k4():
    """R-MAT scale 20 (edge factor 16), the bench's workload: k = 3 and 4
    (and 5 where stored), both schemes, both orientations, in the bench's
    launch configuration.  The stored totals were written by
    tests/golden/make_golden.py from the oracle."""
    with open(os.path.join(GOLDEN, "counts.json")) as f:
        gold = json.load(f)
    rec = gold["rmat20_ef16_s0"]
    g = synth.rmat(20, 16, seed=0)
    assert g.num_edges == rec["num_edges"]
    for orient in ("degeneracy", "degree"):
        G = graph(g, orient)
        if orient == "degeneracy":
            assert G.info()["d_max"] == rec["degeneracy_dmax"]
        for k in sorted(int(x) for x in rec["counts"]):
            for scheme in ("vc", "ec"):
                assert G.count(k, scheme=scheme).total == rec["counts"][str(k)], (orient, k, scheme)
        G.close()


@pytest.mark.parametrize("scale", [16, 17])
def test_rmat_deep_k_golden(scale):
    """R-MAT scales 16 and 17 (edge factor 16; at most 219 and 286 candidates
    under degeneracy order, so the deep traversal's wide levels and its
    re-encoded nodes both run) at the deep sizes the R-MAT-20 configuration
    asks for (k = 5, 6 and 7): both schemes, both
    orientations, against the oracle's totals stored by
    tests/golden/make_golden.py."""
    with open(os.path.join(GOLDEN, "counts.json")) as f:
        rec = json.load(f)[f"rmat{scale}_ef16_s0"]
    g = synth.rmat(scale, 16, seed=0)
    assert g.num_edges == rec["num_edges"]
    for orient in ("degeneracy", "degree"):
        G = graph(g, orient)
        if orient == "degeneracy":
            assert G.info()["d_max"] == rec["degeneracy_dmax"]
        for k in sorted(int(x) for x in rec["counts"]):
            for scheme in ("vc", "ec"):
                assert G.count(k, scheme=scheme).total == rec["counts"][str(k)], (orient, k, scheme)
        G.close()


def test_time_limit_returns_timeout_and_keeps_the_handle():
    # billions of 9-cliques: cannot finish in 50 ms; the wait ends with a
    # status, the context and the handle stay usable
    g = synth.rmat(14, 16, seed=6)
    G = graph(g)
    G.set_time_limit(0.05)
    with pytest.raises(kclique.KCError) as e:
        G.count(10, scheme="ec")
    assert e.value.status == kclique.KC_E_TIMEOUT
    G.set_time_limit(0)
    drp, dci, _, _ = O.dag_for(g.row_ptr, g.col_idx, "degeneracy")
    assert G.count(3).total == O.count_orient(drp, dci, 3).total


@pytest.mark.parametrize("gi", range(3))
def test_per_vertex_orientation_mode(gi):
    """Per-vertex counts from the orientation traversal (pivot = 0): every
    vertex's number of k-cliques, against the oracle's per-vertex counts."""
    # sizes chosen so that the oracle's per-vertex route (one step per clique)
    # stays within seconds
    g, ks = [(synth.rmat(12, 16, seed=1), (3, 4, 5, 6, 7)), (synth.dense_random_graph(120, 0.6, 2), (3, 4, 5, 6, 7, 8)),
             (synth.chung_lu_planted(20000, 2.1, 10, 20, 20, 60, 0.9, seed=1), (3, 4, 5, 6))][gi]
    drp, dci, _, _ = O.dag_for(g.row_ptr, g.col_idx, "degeneracy")
    G = graph(g)
    for k in ks:
        want = O.count_orient(drp, dci, k, per_vertex=True)
        for scheme in ("vc", "ec"):
            tot, pv, fl = G.count_per_vertex(k, pivot=False, scheme=scheme)
            assert tot == want.total, (k, scheme)
            assert [int(x) for x in pv] == want.per_vertex, (k, scheme)
            assert int(pv.sum()) == k * want.total
