"""kc_count_noalloc: the orientation-mode count with its working memory in a
fixed array inside the library instead of graph-owned device allocations.

Its totals must equal kc_count's on the same graph, call after call: the
array keeps the previous call's contents, so a second call in a row checks
that everything that must start at zero is cleared.  This file runs last so
that the array has been through the rest of the suite's kernels first."""
import pytest

from tests.gpu_common import graph, kclique, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _noalloc(G, k, scheme):
    res = torch.zeros(kclique.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    G.count_noalloc(k, res, scheme=scheme)
    torch.cuda.synchronize()
    return kclique.parse_result(bytes(res.cpu().numpy()))


CASES = [
    (synth.rmat(13, 16, seed=2), "degeneracy", [3, 4, 5, 6]),
    (synth.dense_random_graph(120, 0.6, 2), "degree", [3, 5, 8]),
    (synth.chung_lu_planted(20000, 2.1, 10, 20, 20, 60, 0.9, seed=1), "degeneracy", [4, 7]),
    (synth.complete_graph(50), "degeneracy", [1, 2, 3, 4, 48, 50, 51]),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_noalloc_matches_count_twice_in_a_row(case):
    g, orient, ks = CASES[case]
    G = graph(g, orient)
    for k in ks:
        for scheme in ("vc", "ec"):
            want = G.count(k, scheme=scheme)
            first = _noalloc(G, k, scheme)
            second = _noalloc(G, k, scheme)
            assert first.total == want.total == second.total, (case, k, scheme)
            assert first.flags == want.flags == second.flags


def test_noalloc_rejects_what_needs_global_scratch():
    # out-degree 1499 in a complete graph: the per-block bitmaps need global memory
    G = graph(synth.complete_graph(1500), "degree")
    res = torch.zeros(kclique.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    with pytest.raises(kclique.KCError) as e:
        G.count_noalloc(4, res)
    assert e.value.status == kclique.KC_E_UNSUPPORTED
    assert G.count(3).total == 1500 * 1499 * 1498 // 6
