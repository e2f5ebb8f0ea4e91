"""Reference k-clique listing for the listing tests: every clique of a small
graph, found by extending cliques one vertex at a time over increasing ids,
so that each clique is reached exactly once.  Plain Python sets, for graphs
of a few hundred vertices.  Pinned by tests/test_listing_ref.py."""


def brute_force_cliques(g, k):
    """Every k-clique of the CSR graph g as a sorted tuple of vertex ids."""
    adj = [set(g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]].tolist()) for v in range(g.n)]
    out = []

    def extend(clique, cand):
        if len(clique) == k:
            out.append(tuple(clique))
            return
        for x in sorted(cand):
            extend(clique + [x], {y for y in cand if y > x} & adj[x])

    for v in range(g.n):
        extend([v], {y for y in adj[v] if y > v})
    return set(out)
