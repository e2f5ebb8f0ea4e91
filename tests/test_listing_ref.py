"""Pins of the reference listing used by the GPU listing tests, against
facts outside it: every k-subset of a complete graph, the subsets that pass
a pairwise adjacency test on tiny random graphs, the elementary symmetric
polynomials on complete multipartite graphs, and the oracle's counts."""
import itertools
import math

import pytest

from oracle import oracle as O
from paper_2104_13209_gb300 import synth
from tests.clique_listing_ref import brute_force_cliques


def test_complete_graph_lists_every_subset():
    g = synth.complete_graph(9)
    for k in range(1, 10):
        assert brute_force_cliques(g, k) == set(itertools.combinations(range(9), k))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_tiny_random_graphs_against_pairwise_test(seed):
    g = synth.dense_random_graph(14, 0.55, seed)
    adj = {(int(u), int(v)) for u in range(g.n) for v in g.col_idx[g.row_ptr[u]:g.row_ptr[u + 1]]}
    for k in range(3, 8):
        want = {S for S in itertools.combinations(range(g.n), k)
                if all((a, b) in adj for a, b in itertools.combinations(S, 2))}
        assert brute_force_cliques(g, k) == want


def test_multipartite_counts():
    parts = [3, 5, 2, 4]
    g = synth.complete_multipartite(parts)
    for k in range(1, 6):
        e = sum(math.prod(c) for c in itertools.combinations(parts, k))
        assert len(brute_force_cliques(g, k)) == e


def test_random_graphs_against_the_oracle():
    for g in (synth.rmat(9, 8, seed=3), synth.dense_random_graph(40, 0.5, 5)):
        drp, dci, _, _ = O.dag_for(g.row_ptr, g.col_idx, "degeneracy")
        for k in (3, 4, 5, 6):
            assert len(brute_force_cliques(g, k)) == O.count_orient(drp, dci, k).total
