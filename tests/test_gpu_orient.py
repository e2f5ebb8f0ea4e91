"""Orientation on the GPU (Section 3.1) against the CPU oracle.

Degree orientation has a unique order (degree, id), so the GPU DAG must equal
the oracle's bit for bit.  Degeneracy orientation may break ties in any peel
order; its core numbers are unique and must match exactly, its maximum
out-degree must equal the degeneracy, and the DAG must hold every undirected
edge exactly once, pointing forward in the library numbering.
"""
import numpy as np
import pytest

from oracle import oracle as O
from tests.gpu_common import csr_from_pairs, graph, kclique, lib, synth

pytestmark = pytest.mark.gpu


def _graphs():
    return [synth.rmat(12, 16, seed=1), synth.erdos_renyi(2000, 0.01, 0), synth.dense_random_graph(150, 0.3, 2),
            synth.complete_graph(20), synth.random_tree(500, 3), synth.rmat(14, 8, seed=5)]


def _dag_edges_in_input_ids(rp, col, new_of_old):
    old_of_new = np.empty_like(new_of_old)
    old_of_new[new_of_old] = np.arange(new_of_old.size, dtype=new_of_old.dtype)
    src = np.repeat(np.arange(rp.size - 1), np.diff(rp.astype(np.int64)))
    return old_of_new[src], old_of_new[col], src, col


@pytest.mark.parametrize("gi", range(6))
def test_degree_orientation_bit_exact(gi):
    g = _graphs()[gi]
    G = graph(g, "degree")
    rp, col, nof, _ = G.export()
    want_rank = O.degree_rank(g.row_ptr)
    assert np.array_equal(nof, want_rank)
    # rows ascend and edges go forward
    src = np.repeat(np.arange(g.n), np.diff(rp.astype(np.int64)))
    assert np.all(src < col)
    for r in range(min(g.n, 3000)):
        row = col[rp[r]:rp[r + 1]]
        assert np.all(row[1:] > row[:-1])
    # same DAG as the oracle, edge for edge
    a, b, _, _ = _dag_edges_in_input_ids(rp, col, nof)
    drp, dci, dmax, _ = O.dag_for(g.row_ptr, g.col_idx, "degree")
    osrc = np.repeat(np.arange(g.n), np.diff(drp.astype(np.int64)))
    got = np.sort(a.astype(np.uint64) * g.n + b)
    want = np.sort(osrc.astype(np.uint64) * g.n + dci)
    assert np.array_equal(got, want)
    assert G.info()["d_max"] == dmax


@pytest.mark.parametrize("gi", range(6))
def test_degeneracy_orientation(gi):
    g = _graphs()[gi]
    G = graph(g, "degeneracy")
    rp, col, nof, core = G.export(core=True)
    dg = O.degeneracy_order(g.row_ptr, g.col_idx)
    assert np.array_equal(core, dg.core)
    info = G.info()
    assert info["degeneracy"] == dg.degeneracy
    assert info["d_max"] == dg.degeneracy
    assert np.array_equal(np.sort(nof), np.arange(g.n))
    a, b, src, dst = _dag_edges_in_input_ids(rp, col, nof)
    assert np.all(src < dst)
    # a peel order: every vertex has at most core(v) out-neighbours
    outdeg = np.diff(rp.astype(np.int64))
    old_of_new = np.empty_like(nof)
    old_of_new[nof] = np.arange(g.n, dtype=nof.dtype)
    assert np.all(outdeg <= core[old_of_new])
    und = np.sort(np.minimum(a, b).astype(np.uint64) * g.n + np.maximum(a, b))
    lo, hi = g.edge_pairs()
    assert np.array_equal(und, np.sort(lo.astype(np.uint64) * g.n + hi))


def test_invalid_graphs_rejected():
    lib()
    bad = {
        "asymmetric": csr_from_pairs(3, [(0, 1), (1, 0), (1, 2)]),
        "self-loop": csr_from_pairs(2, [(0, 0), (0, 1), (1, 0)]),
        "unsorted": csr_from_pairs(3, [(0, 2), (0, 1), (1, 0), (2, 0)]),
        "duplicate": csr_from_pairs(2, [(0, 1), (0, 1), (1, 0), (1, 0)]),
    }
    for name, (rp, ci) in bad.items():
        with pytest.raises(kclique.KCError) as e:
            kclique.Graph(rp, ci, orient="degeneracy")
        assert e.value.status == kclique.KC_E_INVALID_GRAPH, name
    rp = np.array([0, 1, 2], dtype=np.uint32)
    ci = np.array([1, 5], dtype=np.uint32)
    with pytest.raises(kclique.KCError) as e:
        kclique.Graph(rp, ci)
    assert e.value.status == kclique.KC_E_INVALID_GRAPH
    rp = np.array([0, 2, 1], dtype=np.uint32)  # not monotone
    ci = np.array([1, 0], dtype=np.uint32)
    with pytest.raises(kclique.KCError) as e:
        kclique.Graph(rp, ci)
    assert e.value.status == kclique.KC_E_INVALID_GRAPH


def test_empty_and_edgeless():
    lib()
    G = kclique.Graph(np.zeros(1, dtype=np.uint32), np.zeros(0, dtype=np.uint32), n=0)
    assert G.info()["n"] == 0
    assert G.count(1).total == 0
    assert G.count(3).total == 0
    G = kclique.Graph(np.zeros(6, dtype=np.uint32), np.zeros(0, dtype=np.uint32), n=5, orient="degree")
    assert [G.count(k).total for k in (1, 2, 3)] == [5, 0, 0]
