"""The orientation traversal without the binary encoding (schemes vc-list and
ec-list: sorted vertex lists intersected by binary search, the paper's
comparison point in Sections 3.4 and 4.3), and the per-SM work counters of
the orientation-mode counts (the load balance of Fig. 7).

Counts are integers: the bar is exact equality with the oracle or the closed
form.  The per-SM counters must add up to the count's work units."""
import math

import pytest

from oracle import oracle as O
from tests.gpu_common import elementary_symmetric, graph, kclique, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

LIST_SCHEMES = ("vc-list", "ec-list")


def oracle_counts(g, ks):
    drp, dci, _, _ = O.dag_for(g.row_ptr, g.col_idx, "degeneracy")
    return {k: O.count_orient(drp, dci, k).total for k in ks}


# (graph, sizes): the list traversal does one warp-wide intersection per
# tree node, so the sizes stop where the node count reaches ~10^7
CASES = [
    (lambda: synth.rmat(12, 16, seed=1), [3, 4, 5]),
    (lambda: synth.rmat(13, 8, seed=4), [3, 4, 5]),
    (lambda: synth.dense_random_graph(120, 0.6, 2), [3, 4, 5, 6, 7]),
    (lambda: synth.erdos_renyi(2000, 0.01, 0), [3, 4, 5]),
]


@pytest.mark.parametrize("gi", range(len(CASES)))
def test_list_schemes_match_oracle(gi):
    make, ks = CASES[gi]
    g = make()
    want = oracle_counts(g, ks)
    for orient in ("degeneracy", "degree"):
        G = graph(g, orient)
        for k in ks:
            for scheme in LIST_SCHEMES:
                assert G.count(k, scheme=scheme).total == want[k], (orient, k, scheme)
        G.close()


def test_list_schemes_closed_forms():
    for n in (5, 33, 40):
        G = graph(synth.complete_graph(n))
        for k in range(1, min(n, 6) + 2):
            for scheme in LIST_SCHEMES:
                assert G.count(k, scheme=scheme).total == math.comb(n, k), (n, k, scheme)
        G.close()
    parts = [3, 40, 1, 7, 12, 12]
    G = graph(synth.complete_multipartite(parts))
    for k in range(1, len(parts) + 2):
        for scheme in LIST_SCHEMES:
            assert G.count(k, scheme=scheme).total == elementary_symmetric(parts, k), (k, scheme)


def test_list_schemes_limits():
    K = graph(synth.complete_graph(30))  # 29 candidates: k = 17 reaches the traversal
    with pytest.raises(kclique.KCError) as e:
        K.count(17, scheme="vc-list")
    assert e.value.status == kclique.KC_E_UNSUPPORTED
    assert graph(synth.complete_graph(18)).count(16, scheme="ec-list").total == math.comb(18, 16)
    g = synth.dense_random_graph(60, 0.5, 3)
    G = graph(g)
    with pytest.raises(kclique.KCError) as e:
        G.count_per_vertex(4, pivot=False, scheme="ec-list")
    assert e.value.status == kclique.KC_E_UNSUPPORTED
    d = G.info()["d_max"]
    assert G.count(d + 2, scheme="vc-list").total == 0
    # the handle stays usable
    drp, dci, _, _ = O.dag_for(g.row_ptr, g.col_idx, "degeneracy")
    assert G.count(4, scheme="ec-list").total == O.count_orient(drp, dci, 4).total


def test_list_scheme_time_limit():
    g = synth.rmat(14, 16, seed=6)
    G = graph(g)
    G.set_time_limit(0.05)
    with pytest.raises(kclique.KCError) as e:
        G.count(12, scheme="vc-list")
    assert e.value.status == kclique.KC_E_TIMEOUT
    G.set_time_limit(0)
    drp, dci, _, _ = O.dag_for(g.row_ptr, g.col_idx, "degeneracy")
    assert G.count(3, scheme="vc-list").total == O.count_orient(drp, dci, 3).total


def test_per_sm_work_adds_up():
    """Every orientation-mode kernel splits its work units by SM: the bitmap
    traversal for k <= 4 (both splits), the deep traversal (k >= 5) and the
    list traversal.  The split must add up to kc_graph_last_work, spread over
    more than one SM on a graph of thousands of roots, and cover at least the
    device's SMs."""
    g = synth.rmat(14, 16, seed=2)
    G = graph(g)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for k, scheme in ((4, "vc"), (4, "ec"), (5, "vc"), (6, "ec"), (3, "vc-list"), (4, "ec-list")):
        G.count(k, scheme=scheme)
        per_sm = G.last_sm_work()
        assert per_sm.size >= sms
        assert int(per_sm.astype(object).sum()) == G.last_work() > 0, (k, scheme)
        assert (per_sm > 0).sum() > 1, (k, scheme)
    G.count(2)  # no launch: every counter reads 0
    assert int(G.last_sm_work().sum()) == 0
