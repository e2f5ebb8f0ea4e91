"""k-clique listing (kc_list_cliques): the list traversal writes out every
clique it closes.  The listed sets are compared with the reference listing
of tests/clique_listing_ref.py (pinned on the CPU by
tests/test_listing_ref.py), their number with the oracle's count, and a
truncated listing with the full count."""
import itertools
import math

import pytest

from oracle import oracle as O
from tests.clique_listing_ref import brute_force_cliques
from tests.gpu_common import graph, kclique, synth

pytestmark = pytest.mark.gpu

pytest.importorskip("torch")


def listed_set(rows):
    return {tuple(sorted(r.tolist())) for r in rows}


@pytest.mark.parametrize("gi", range(3))
def test_listing_matches_brute_force(gi):
    g = [synth.dense_random_graph(40, 0.5, 5), synth.rmat(9, 8, seed=3), synth.erdos_renyi(300, 0.08, 2)][gi]
    for orient in ("degeneracy", "degree"):
        G = graph(g, orient)
        for k in (3, 4, 5, 6):
            want = brute_force_cliques(g, k)
            cnt, rows = G.list_cliques(k)
            assert cnt == len(want) == rows.shape[0], (orient, k)
            got = listed_set(rows)
            assert len(got) == cnt  # no clique listed twice
            assert got == want, (orient, k)
        G.close()


def test_listing_complete_graph_and_count():
    G = graph(synth.complete_graph(12))
    cnt, rows = G.list_cliques(5)
    assert cnt == math.comb(12, 5)
    assert listed_set(rows) == set(itertools.combinations(range(12), 5))
    g = synth.rmat(11, 16, seed=7)
    G = graph(g)
    drp, dci, _, _ = O.dag_for(g.row_ptr, g.col_idx, "degeneracy")
    for k in (3, 4, 5):
        cnt, rows = G.list_cliques(k)
        assert cnt == O.count_orient(drp, dci, k).total == rows.shape[0]


def test_listing_truncated_and_limits():
    g = synth.dense_random_graph(50, 0.5, 8)
    G = graph(g)
    full = brute_force_cliques(g, 4)
    cap = len(full) // 3
    cnt, rows = G.list_cliques(4, cap=cap)
    assert cnt == len(full) and rows.shape[0] == cap
    got = listed_set(rows)
    assert len(got) == cap and got <= full  # distinct cliques of the graph
    cnt0, rows0 = G.list_cliques(4, cap=0)
    assert cnt0 == len(full) and rows0.shape == (0, 4)
    for k in (2, 17):
        with pytest.raises(kclique.KCError) as e:
            G.list_cliques(k, cap=0)
        assert e.value.status == kclique.KC_E_UNSUPPORTED
    T = graph(synth.random_tree(30, seed=4))  # out-degree 1: no triangle, and no launch
    cnt, rows = T.list_cliques(3, cap=4)
    assert cnt == 0 and rows.shape == (0, 3)
