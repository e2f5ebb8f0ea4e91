"""kc_count_noalloc: the orientation-mode count with its working memory in a
fixed array inside the library instead of graph-owned device allocations.

Some callers cannot let a library allocate device memory: every byte of it
belongs to another allocator (a framework's caching pool, an arena carved
up at start-up), or a cudaFree would synchronise the device inside a
latency-critical loop.  This entry point serves them.

Its totals must equal the oracle's (the Fig. 2 traversal on the CPU).  The
array keeps the previous call's contents, so every case runs twice in a
row, and a call with many big roots is followed by one with few, to check
that everything that must start at zero is cleared.  The first call on a
fresh handle must leave the handle's device memory unchanged.  The file is
collected last so that a failure here stops a `-x` run only after every
other test has run."""
import functools
import math

import pytest

from oracle import oracle as O
from tests.gpu_common import graph, kclique, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _noalloc(G, k, scheme):
    res = torch.zeros(kclique.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    G.count_noalloc(k, res, scheme=scheme)
    torch.cuda.synchronize()
    return kclique.parse_result(bytes(res.cpu().numpy()))


@functools.lru_cache(maxsize=None)
def _oracle(case, k):
    g, _, _ = CASES[case]
    if case == COMPLETE:
        # C(n, k) (the oracle's pinned closed form); its plain recursion
        # does not prune by size and would walk 2^50 nodes at k = 48
        return math.comb(g.n, k)
    drp, dci, _, _ = O.dag_for(g.row_ptr, g.col_idx, "degeneracy")
    return O.count_orient(drp, dci, k).total


CASES = [
    (synth.rmat(13, 16, seed=2), "degeneracy", [3, 4, 5, 6]),
    (synth.dense_random_graph(120, 0.6, 2), "degree", [3, 5, 8]),
    (synth.chung_lu_planted(20000, 2.1, 10, 20, 20, 60, 0.9, seed=1), "degeneracy", [4, 7]),
    (synth.complete_graph(50), "degeneracy", [1, 2, 3, 4, 48, 50, 51]),
]
COMPLETE = 3


@pytest.mark.parametrize("case", range(len(CASES)))
def test_noalloc_matches_oracle_twice_in_a_row(case):
    g, orient, ks = CASES[case]
    G = graph(g, orient)
    bytes0 = G.info()["device_bytes"]
    for k in ks:
        want = _oracle(case, k)
        for scheme in ("vc", "ec"):
            first = _noalloc(G, k, scheme)
            second = _noalloc(G, k, scheme)
            assert first.total == want == second.total, (case, k, scheme)
            assert first.flags == second.flags == 0
    # no count through the handle's own buffers ran: nothing was allocated
    assert G.info()["device_bytes"] == bytes0


def test_noalloc_many_big_roots_then_few():
    # R-MAT 14 at k = 5 has thousands of roots with more than 32 candidates
    # (one task counter each in the array); the dense graph that follows has
    # a hundred.  Stale counters from the first call would cut the second.
    big, small = synth.rmat(14, 16, seed=5), synth.dense_random_graph(100, 0.7, 11)
    Gb, Gs = graph(big), graph(small)
    for g, G, k in ((big, Gb, 5), (small, Gs, 6), (big, Gb, 4), (small, Gs, 3)):
        drp, dci, _, _ = O.dag_for(g.row_ptr, g.col_idx, "degeneracy")
        want = O.count_orient(drp, dci, k).total
        for scheme in ("vc", "ec"):
            assert _noalloc(G, k, scheme).total == want, (g.name, k, scheme)


def test_noalloc_rejects_what_needs_global_scratch():
    # out-degree 1499 in a complete graph: the per-block bitmaps need global memory
    G = graph(synth.complete_graph(1500), "degree")
    res = torch.zeros(kclique.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    with pytest.raises(kclique.KCError) as e:
        G.count_noalloc(4, res)
    assert e.value.status == kclique.KC_E_UNSUPPORTED
    assert G.count(3).total == 1500 * 1499 * 1498 // 6
