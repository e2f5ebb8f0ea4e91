"""The serving loop (kc_server_*): queries of different graphs, k and modes
admitted while others run, batched on the fly -- each result equal to the
CPU oracle's count, the same when the query runs alone and in the mix, and
a query that runs out of time does not disturb the others."""
import pytest

from oracle import oracle as O
from tests.gpu_common import kclique, lib, synth

pytestmark = pytest.mark.gpu


def pool():
    return [synth.erdos_renyi(2000, 0.01, 0), synth.rmat(12, 16, seed=1), synth.complete_graph(30),
            synth.complete_multipartite([10] * 6), synth.dense_random_graph(100, 0.5, 3),
            synth.chung_lu_planted(20000, 2.1, 10, 20, 20, 60, 0.9, seed=1)]


def want(gs, g, k):
    h = gs[g]
    return h.n if k == 1 else (h.num_edges if k == 2 else O.count(h.row_ptr, h.col_idx, k))


def queries(gs):
    return [(g, k, p) for g in range(len(gs)) for k in (1, 2, 3, 4, 5, 7) for p in (0, 1)]


def make_server(gs, **kw):
    lib()
    S = kclique.Server(**kw)
    ids = [S.add_graph(h) for h in gs]
    assert ids == list(range(len(gs)))
    return S


def wait(S, t):
    r = S.poll(t, 120000)
    assert r is not None, "query not served within two minutes"
    return r


def check(r, gs, g, k):
    assert r["status"] == kclique.KC_OK and r["flags"] == 0, r
    assert r["total"] == want(gs, g, k), (g, k, r)
    assert r["t_submit_ms"] <= r["t_admit_ms"] <= r["t_done_ms"]


def test_server_alone_and_mixed():
    gs = pool()
    qs = queries(gs)
    S = make_server(gs, max_batch=64, slots=3)
    alone = []
    for g, k, p in qs:
        r = wait(S, S.submit(g, k, bool(p)))
        check(r, gs, g, k)
        alone.append(r["total"])
    tickets = [S.submit(g, k, bool(p)) for g, k, p in qs * 3]
    mixed = [wait(S, t) for t in tickets]
    for (g, k, p), r in zip(qs * 3, mixed):
        check(r, gs, g, k)
    assert [r["total"] for r in mixed] == alone * 3
    st = S.stats()
    assert st["served"] == 4 * len(qs) and st["launches"] <= st["served"]
    S.close()


def test_server_serial_baseline():
    gs = pool()
    qs = queries(gs)
    S = make_server(gs, serial=True)
    tickets = [S.submit(g, k, bool(p)) for g, k, p in qs]
    for (g, k, p), t in zip(qs, tickets):
        check(wait(S, t), gs, g, k)
    assert S.stats()["launches"] == sum(1 for _ in qs)
    S.close()


def test_server_timeout_is_per_query():
    gs = [synth.rmat(14, 16, seed=6), synth.complete_graph(20), synth.erdos_renyi(2000, 0.01, 0)]
    S = make_server(gs, max_batch=64, slots=2)
    S.set_time_limit(0.3)
    heavy = S.submit(0, 10)  # billions of 9-cliques to enumerate: cannot finish in 0.3 s
    light = [S.submit(1, 5), S.submit(2, 3), S.submit(1, 20), S.submit(2, 4)]
    r = wait(S, heavy)
    assert r["status"] == kclique.KC_E_TIMEOUT
    for t, (g, k) in zip(light, [(1, 5), (2, 3), (1, 20), (2, 4)]):
        check(wait(S, t), gs, g, k)
    S.close()


def test_server_budget_and_arguments():
    lib()
    with pytest.raises(kclique.KCError):
        kclique.Server(hbm_budget=1 << 10)
    S = kclique.Server(hbm_budget=8 << 20, max_batch=16, slots=1)
    S.add_graph(synth.complete_graph(10))
    with pytest.raises(kclique.KCError) as e:
        S.add_graph(synth.rmat(17, 16, seed=1))  # its DAG alone exceeds the budget
    assert e.value.status == kclique.KC_E_NO_MEMORY
    with pytest.raises(kclique.KCError):
        S.submit(5, 3)
    with pytest.raises(kclique.KCError):
        S.submit(0, 0)
    assert wait(S, S.submit(0, 4))["total"] == 210
    S.close()


def test_server_auto_traversal_same_counts():
    # the traversal chosen by k (Section 4.5) counts exactly what the
    # requested one counts
    gs = pool()
    qs = queries(gs)
    S = make_server(gs, max_batch=64, slots=3, auto_traversal=True)
    tickets = [S.submit(g, k, bool(p)) for g, k, p in qs]
    for (g, k, p), t in zip(qs, tickets):
        r = wait(S, t)
        check(r, gs, g, k)
        assert r["pivot"] == (1 if k >= 7 else 0)
    S.close()


def test_server_refuses_a_shape_that_ran_out_of_time():
    gs = [synth.rmat(14, 16, seed=6), synth.complete_graph(20)]
    S = make_server(gs, max_batch=64, slots=2, refuse_expensive=True)
    S.set_time_limit(0.3)
    first = wait(S, S.submit(0, 10))  # cannot finish in 0.3 s
    assert first["status"] == kclique.KC_E_TIMEOUT
    again = wait(S, S.submit(0, 10))  # the same shape: refused at admission
    assert again["status"] == kclique.KC_E_REFUSED
    assert again["t_admit_ms"] == again["t_submit_ms"] == again["t_done_ms"]
    check(wait(S, S.submit(1, 5)), gs, 1, 5)  # other shapes are still served
    check(wait(S, S.submit(0, 3)), gs, 0, 3)
    S.close()


def test_server_profile_picks_the_traversal_and_refuses():
    # with a time limit, adding a graph measures its cost profile; queries
    # then take the traversal that finished there, and a shape that ran out
    # of time in both traversals is refused at admission without a launch
    import math

    gs = [synth.rmat(14, 16, seed=6), synth.complete_graph(40), synth.erdos_renyi(2000, 0.01, 0)]
    lib()
    S = kclique.Server(max_batch=64, slots=2, auto_traversal=True, refuse_expensive=True)
    S.set_time_limit(0.3)
    for h in gs:
        S.add_graph(h)
    # R-MAT 14: k = 3 finishes by graph orientation; k = 10 needs seconds in
    # either traversal (about 4.5 s and more than 0.4 s on a whole GB300)
    assert S.shape(0, 3, False)[0] == kclique.SHAPE_FITS
    assert S.shape(0, 10, False)[0] == kclique.SHAPE_EXPENSIVE
    launches = S.stats()["launches"]
    r = wait(S, S.submit(0, 10, False))
    assert r["status"] == kclique.KC_E_REFUSED and r["t_admit_ms"] == r["t_done_ms"]
    assert S.stats()["launches"] == launches
    check(wait(S, S.submit(0, 4, True)), gs, 0, 4)
    # K40: orientation enumerates C(40, k) leaves; pivoting is one path
    st_or, _ = S.shape(1, 20, False)
    st_pv, ms_pv = S.shape(1, 20, True)
    assert st_pv == kclique.SHAPE_FITS and ms_pv > 0
    r = wait(S, S.submit(1, 20, False))
    assert r["status"] == kclique.KC_OK and r["total"] == math.comb(40, 20)
    assert r["pivot"] == (1 if st_or == kclique.SHAPE_EXPENSIVE else 0)
    r = wait(S, S.submit(1, 3, True))
    assert r["status"] == kclique.KC_OK and r["total"] == math.comb(40, 3) and r["pivot"] == 0
    # ER: every profiled k finishes by orientation
    for k in (3, 4, 5):
        assert S.shape(2, k, False)[0] == kclique.SHAPE_FITS
        r = wait(S, S.submit(2, k, True))
        check(r, gs, 2, k)
        assert r["pivot"] == 0
    S.close()
