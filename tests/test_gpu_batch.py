"""Batched counts (kc_batch_*): many small graphs oriented as one union and
counted, each with its own k, in persistent launches -- every result equal
to the CPU oracle's count of that graph alone, for every launch
configuration, and the same when replayed from a captured CUDA graph."""
import numpy as np
import pytest

from oracle import oracle as O
from tests.gpu_common import kclique, lib, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def mixed_graphs():
    gs = [synth.complete_graph(1), synth.complete_graph(5), synth.complete_graph(12), synth.complete_graph(40),
          synth.complete_multipartite([3, 4, 5]), synth.complete_multipartite([12] * 6),
          synth.dense_random_graph(60, 0.5, 1), synth.dense_random_graph(120, 0.6, 2), synth.rmat(9, 8, seed=1),
          synth.cycle_graph(9), synth.edges_to_csr(3, np.zeros(0), np.zeros(0), "empty3")]
    ba = synth.barabasi_albert(3000, 8, seed=4)
    gs += synth.ego_networks(ba, 40, 20, 400, seed=1)
    return gs


def oracle_counts(gs, qs):
    memo = {}
    out = []
    for g, k in qs:
        key = (g, k)
        if key not in memo:
            h = gs[g]
            memo[key] = h.n if k == 1 else (h.num_edges if k == 2 else O.count(h.row_ptr, h.col_idx, k))
        out.append(memo[key])
    return out


def queries(gs, ks):
    return [(g, k) for g in range(len(gs)) for k in ks]


def test_batch_matches_oracle():
    lib()
    gs = mixed_graphs()
    B = kclique.Batch(gs)
    qs = queries(gs, [1, 2, 3, 4, 5, 6, 8, 13])
    want = oracle_counts(gs, qs)
    got = B.count([g for g, _ in qs], [k for _, k in qs])
    assert [r.total for r in got] == want
    assert all(r.status == kclique.KC_OK and r.flags == 0 for r in got)
    for g in (0, 3, 9):
        info = B.graph_info(g)
        assert info["n"] == gs[g].n and info["m"] == gs[g].num_edges


@pytest.mark.parametrize("scheme", [kclique.KC_SCHEME_VC, kclique.KC_SCHEME_EC])
@pytest.mark.parametrize("subwarp", [1, 4, 32])
@pytest.mark.parametrize("chunk", [1, 8])
def test_batch_every_configuration(scheme, subwarp, chunk):
    lib()
    gs = mixed_graphs()
    B = kclique.Batch(gs, orient="degree")
    qs = queries(gs, [3, 4, 6, 7])
    entries = [{"dclass": c, "k": k, "scheme": scheme, "subwarp": subwarp, "chunk": chunk}
               for c in range(7) for k in (3, 4, 6, 7)]
    got = B.count([g for g, _ in qs], [k for _, k in qs], tune=kclique.tune_from_list(entries))
    assert [r.total for r in got] == oracle_counts(gs, qs)


def test_batch_uneven_queries_repeated_graphs():
    lib()
    gs = mixed_graphs()
    B = kclique.Batch(gs)
    key = synth.stream_key(1, 0xB1)
    n = 600
    gid = (synth.uniform(key, np.arange(n, dtype=np.uint64)) * len(gs)).astype(np.int64)
    ks = 3 + (synth.uniform(synth.stream_key(1, 0xB2), np.arange(n, dtype=np.uint64)) * 6).astype(np.int64)
    qs = list(zip(gid.tolist(), ks.tolist()))
    got = B.count(gid, ks)
    assert [r.total for r in got] == oracle_counts(gs, qs)


def test_batch_capture_replay_and_tune():
    lib()
    gs = mixed_graphs()
    B = kclique.Batch(gs)
    qs = queries(gs, [3, 4, 5, 7])
    gid, ks = [g for g, _ in qs], [k for _, k in qs]
    want = oracle_counts(gs, qs)
    t = B.tune(gid, ks, sample=16)
    entries = kclique.tune_to_list(t)
    assert entries and all(e["subwarp"] in (2, 4, 8, 32) for e in entries if e["k"] >= 3)
    assert [r.total for r in B.count(gid, ks, tune=t)] == want
    res = torch.zeros(len(qs) * kclique.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    ex = B.capture(gid, ks, res, tune=t)
    for _ in range(2):
        res.zero_()
        ex.launch()
        torch.cuda.synchronize()
        got = kclique.parse_results(bytes(res.cpu().numpy()), len(qs))
        assert [r.total for r in got] == want
    ex.close()


def test_batch_rejects_edges_between_graphs():
    lib()
    a, b = synth.complete_graph(4), synth.complete_graph(3)
    u, off = synth.block_union([a, b])
    # move one edge of the first graph so that it joins vertex 3 to vertex 4
    x, y = u.edge_pairs()
    x = x.copy()
    y = y.copy()
    i = int(np.nonzero((x == 2) & (y == 3))[0][0])
    x[i], y[i] = 3, 4
    bad = synth.edges_to_csr(u.n, x, y)
    with pytest.raises(kclique.KCError) as e:
        kclique.Batch(row_ptr=bad.row_ptr, col_idx=bad.col_idx, offsets=off)
    assert e.value.status == kclique.KC_E_INVALID_GRAPH


def test_batch_invalid_queries():
    lib()
    B = kclique.Batch([synth.complete_graph(4)])
    with pytest.raises(kclique.KCError):
        B.count([1], [3])
    with pytest.raises(kclique.KCError):
        B.count([0], [0])
