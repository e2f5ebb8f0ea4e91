"""Seeded synthetic graph generators (inputs only: no k-clique arithmetic here).

Every generator draws its randomness from SplitMix64 used as a counter-based
generator (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): output i of a stream is the SplitMix64 finaliser
applied to ``key + (i + 1) * 0x9E3779B97F4A7C15``.  A stream key is derived
from ``(seed, tag)`` the same way, so every draw is a pure function of
``(seed, tag, counter)`` and does not depend on numpy's generator versions.

The graphs stand in for the paper's SNAP workloads (Section 4.1): they are
symmetrised, stripped of self-loops and duplicate edges and returned as a u32
CSR ``(row_ptr[n+1], col_idx[nnz])`` with every row sorted ascending.

Both the CUDA path's tests/bench and the CPU oracle's tests consume these
graphs; nothing in this module counts, orients or intersects anything.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser on a uint64 array (wrapping arithmetic)."""
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def stream_key(seed: int, tag: int) -> int:
    """64-bit key of the stream named ``tag`` under ``seed``."""
    x = np.array([((seed & 0xFFFFFFFF) << 24 | (tag & 0xFFFFFF)) & _MASK64], dtype=np.uint64)
    return int(_mix(x)[0])


def random_u64(key: int, counters: np.ndarray) -> np.ndarray:
    """Outputs ``counters`` (uint64 array) of the stream with 64-bit ``key``."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(key) + (c + np.uint64(1)) * _GOLDEN
    return _mix(z)


def uniform(key: int, counters: np.ndarray) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of ``random_u64``."""
    return (random_u64(key, counters) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


# ----------------------------------------------------------------------------
# CSR assembly
# ----------------------------------------------------------------------------

@dataclass
class CSRGraph:
    """Simple undirected graph as a symmetric u32 CSR with sorted rows."""

    n: int
    row_ptr: np.ndarray  # uint32[n+1]
    col_idx: np.ndarray  # uint32[nnz], nnz = 2 * num_edges
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def num_edges(self) -> int:
        return self.nnz // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr.astype(np.int64))

    def edge_pairs(self) -> tuple[np.ndarray, np.ndarray]:
        """Each undirected edge once, as (lo, hi) with lo < hi."""
        src = np.repeat(np.arange(self.n, dtype=np.int64), self.degrees())
        dst = self.col_idx.astype(np.int64)
        keep = src < dst
        return src[keep], dst[keep]


def edges_to_csr(n: int, u: np.ndarray, v: np.ndarray, name: str = "") -> CSRGraph:
    """Symmetrise, drop self-loops and duplicates, sort rows; return the CSR."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    if u.size and (u.min() < 0 or v.min() < 0 or u.max() >= n or v.max() >= n):
        raise ValueError("edge endpoint out of range")
    keep = u != v
    lo = np.minimum(u[keep], v[keep]).astype(np.uint64)
    hi = np.maximum(u[keep], v[keep]).astype(np.uint64)
    key = lo * np.uint64(n) + hi
    key.sort()  # sorted distinct keys (the same values as np.unique, much faster at 10^8 keys)
    if key.size:
        key = key[np.concatenate(([True], key[1:] != key[:-1]))]
    lo = (key // np.uint64(n)).astype(np.int64)
    hi = (key % np.uint64(n)).astype(np.int64)
    both = np.concatenate([key, hi.astype(np.uint64) * np.uint64(n) + lo.astype(np.uint64)])
    both.sort()  # every (src, dst) once, ordered by source then destination
    src = (both // np.uint64(n)).astype(np.int64)
    dst = (both % np.uint64(n)).astype(np.int64)
    if dst.size >= (1 << 32):
        raise ValueError("nnz does not fit in u32")
    counts = np.bincount(src, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.uint32)
    np.cumsum(counts, out=row_ptr[1:])
    return CSRGraph(n=n, row_ptr=row_ptr, col_idx=dst.astype(np.uint32), name=name)


def disjoint_union(graphs: list[CSRGraph], name: str = "") -> CSRGraph:
    """Vertex-disjoint union; vertex ids of graph i are shifted by the sizes before it."""
    us, vs, off = [], [], 0
    for g in graphs:
        a, b = g.edge_pairs()
        us.append(a + off)
        vs.append(b + off)
        off += g.n
    return edges_to_csr(off, np.concatenate(us) if us else np.zeros(0), np.concatenate(vs) if vs else np.zeros(0), name)


def relabel(g: CSRGraph, perm: np.ndarray, name: str = "") -> CSRGraph:
    """The same graph with vertex v renamed perm[v]."""
    a, b = g.edge_pairs()
    perm = np.asarray(perm, dtype=np.int64)
    return edges_to_csr(g.n, perm[a], perm[b], name or g.name)


def random_permutation(n: int, seed: int, tag: int = 0x5E) -> np.ndarray:
    """A seeded permutation of range(n) (sort by random keys)."""
    keys = random_u64(stream_key(seed, tag), np.arange(n, dtype=np.uint64))
    return np.argsort(keys, kind="stable").astype(np.int64)


# ----------------------------------------------------------------------------
# Deterministic families with known clique counts (used as test inputs)
# ----------------------------------------------------------------------------

def complete_graph(n: int) -> CSRGraph:
    i, j = np.triu_indices(n, 1)
    return edges_to_csr(n, i, j, f"K{n}")


def complete_multipartite(parts: list[int]) -> CSRGraph:
    """K_{a1,...,ar}: vertices in different parts are adjacent, same part not."""
    n = int(sum(parts))
    label = np.repeat(np.arange(len(parts)), parts)
    i, j = np.triu_indices(n, 1)
    keep = label[i] != label[j]
    return edges_to_csr(n, i[keep], j[keep], "K_" + ",".join(map(str, parts)))


def turan_graph(n: int, r: int) -> CSRGraph:
    """T(n, r): complete r-partite with part sizes as equal as possible."""
    parts = [n // r + (1 if i < n % r else 0) for i in range(r)]
    g = complete_multipartite([p for p in parts if p > 0])
    g.name = f"T({n},{r})"
    return g


def join(g: CSRGraph, h: CSRGraph) -> CSRGraph:
    """G join H: disjoint union plus every edge between V(G) and V(H)."""
    a, b = g.edge_pairs()
    c, d = h.edge_pairs()
    x, y = np.meshgrid(np.arange(g.n), np.arange(h.n) + g.n, indexing="ij")
    u = np.concatenate([a, c + g.n, x.ravel()])
    v = np.concatenate([b, d + g.n, y.ravel()])
    return edges_to_csr(g.n + h.n, u, v, f"({g.name})v({h.name})")


def cycle_graph(n: int) -> CSRGraph:
    i = np.arange(n)
    return edges_to_csr(n, i, (i + 1) % n, f"C{n}")


def random_tree(n: int, seed: int) -> CSRGraph:
    """Vertex i > 0 attaches to a uniformly drawn earlier vertex."""
    if n <= 1:
        return edges_to_csr(n, np.zeros(0), np.zeros(0), f"tree{n}")
    i = np.arange(1, n, dtype=np.int64)
    par = np.floor(uniform(stream_key(seed, 0x7E), i.astype(np.uint64)) * i).astype(np.int64)
    return edges_to_csr(n, i, par, f"tree{n}")


def random_bipartite(a: int, b: int, p: float, seed: int) -> CSRGraph:
    i, j = np.meshgrid(np.arange(a), np.arange(b) + a, indexing="ij")
    i, j = i.ravel(), j.ravel()
    keep = uniform(stream_key(seed, 0xB1), np.arange(i.size, dtype=np.uint64)) < p
    return edges_to_csr(a + b, i[keep], j[keep], f"bip({a},{b},{p})")


def dense_random_graph(n: int, p: float, seed: int) -> CSRGraph:
    """G(n, p) by one Bernoulli draw per pair (for small n)."""
    i, j = np.triu_indices(n, 1)
    keep = uniform(stream_key(seed, 0xD5), np.arange(i.size, dtype=np.uint64)) < p
    return edges_to_csr(n, i[keep], j[keep], f"G({n},{p})s{seed}")


# ----------------------------------------------------------------------------
# Erdos-Renyi G(n, p) by geometric skipping (Batagelj and Brandes, 2005)
# ----------------------------------------------------------------------------

def _pair_from_linear(n: int, L: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Map a linear index over pairs i<j (row-major) to (i, j)."""
    L = L.astype(np.int64)
    b = 2 * n - 1
    i = np.floor((b - np.sqrt(np.maximum(b * b - 8.0 * L, 0.0))) / 2).astype(np.int64)
    i = np.clip(i, 0, n - 2)
    off = i * (2 * n - i - 1) // 2
    # fix rounding: make off(i) <= L < off(i+1)
    for _ in range(3):
        too_big = off > L
        i = np.where(too_big, i - 1, i)
        off = i * (2 * n - i - 1) // 2
        nxt = (i + 1) * (2 * n - i - 2) // 2
        too_small = L >= nxt
        i = np.where(too_small, i + 1, i)
        off = i * (2 * n - i - 1) // 2
    j = L - off + i + 1
    return i, j


def erdos_renyi(n: int, p: float, seed: int = 0) -> CSRGraph:
    """G(n, p): each of the n(n-1)/2 pairs is an edge independently with prob p.

    Gaps between successive edges in the row-major pair order are geometric;
    the k-th gap is drawn from counter k of the stream (seed, 0xE5).
    """
    N = n * (n - 1) // 2
    if p <= 0 or N == 0:
        return edges_to_csr(n, np.zeros(0), np.zeros(0), f"ER({n},{p})")
    if p >= 1:
        return complete_graph(n)
    key = stream_key(seed, 0xE5)
    logq = math.log1p(-p)
    pos_all = []
    last = -1
    drawn = 0
    batch = int(N * p * 1.05) + 1024
    while True:
        u = uniform(key, np.arange(drawn, drawn + batch, dtype=np.uint64))
        drawn += batch
        gaps = np.floor(np.log1p(-u) / logq).astype(np.int64)
        pos = last + np.cumsum(gaps + 1)
        inside = pos < N
        pos_all.append(pos[inside])
        if not inside.all():
            break
        last = int(pos[-1])
    L = np.concatenate(pos_all)
    i, j = _pair_from_linear(n, L)
    return edges_to_csr(n, i, j, f"ER({n},{p})s{seed}")


# ----------------------------------------------------------------------------
# R-MAT (Chakrabarti, Zhan and Faloutsos, SDM 2004)
# ----------------------------------------------------------------------------

def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 0) -> CSRGraph:
    """R-MAT with 2**scale vertices and edge_factor * 2**scale generated edges.

    Edge e descends ``scale`` levels; at level l the quadrant is chosen by
    counter ``e * scale + l`` of the stream (seed, 0xA7), most significant bit
    first.  No noise and no vertex permutation; the result is symmetrised and
    deduplicated by ``edges_to_csr``.
    """
    n = 1 << scale
    m = edge_factor * n
    key = stream_key(seed, 0xA7)
    src = np.zeros(m, dtype=np.int64)
    dst = np.zeros(m, dtype=np.int64)
    base = np.arange(m, dtype=np.uint64) * np.uint64(scale)
    ab, abc = a + b, a + b + c
    for lvl in range(scale):
        u = uniform(key, base + np.uint64(lvl))
        bit_s = (u >= ab).astype(np.int64)
        bit_d = (((u >= a) & (u < ab)) | (u >= abc)).astype(np.int64)
        src = (src << 1) | bit_s
        dst = (dst << 1) | bit_d
    return edges_to_csr(n, src, dst, f"RMAT{scale}-ef{edge_factor}s{seed}")


# ----------------------------------------------------------------------------
# Chung-Lu power-law graph with planted dense communities
# ----------------------------------------------------------------------------

def chung_lu_planted(n: int, beta: float = 2.1, mean_deg: float = 30.0, ncomm: int = 0, size_min: int = 40,
                     size_max: int = 200, p_in: float = 0.9, seed: int = 0) -> CSRGraph:
    """Power-law background plus vertex-disjoint dense communities.

    Background (the fast Chung-Lu sampler of Pinar, Seshadhri and Kolda, 2012):
    weights w_i proportional to (i + 1)^(-1/(beta - 1)), scaled to mean
    ``mean_deg`` and capped at sqrt(sum w); round(sum(w) / 2) edges whose two
    endpoints are drawn independently with probability proportional to w
    (streams (seed, 0xC1) and (seed, 0xC2)).  Communities: ``ncomm`` groups with
    sizes uniform in [size_min, size_max] (stream (seed, 0xC3)) taken as
    consecutive blocks of a seeded permutation (so they are vertex-disjoint),
    each pair inside a group an edge with probability p_in (stream
    (seed, 0xC4), one counter per pair).  Loops and duplicates are removed.
    """
    i = np.arange(n, dtype=np.float64)
    w = (i + 1.0) ** (-1.0 / (beta - 1.0))
    w *= mean_deg * n / w.sum()
    w = np.minimum(w, math.sqrt(w.sum()))
    m = int(round(w.sum() / 2))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    cnt = np.arange(m, dtype=np.uint64)
    u = np.searchsorted(cdf, uniform(stream_key(seed, 0xC1), cnt), side="right")
    v = np.searchsorted(cdf, uniform(stream_key(seed, 0xC2), cnt), side="right")
    u = np.minimum(u, n - 1)
    v = np.minimum(v, n - 1)
    us, vs = [u], [v]
    if ncomm:
        sizes = size_min + np.floor(uniform(stream_key(seed, 0xC3), np.arange(ncomm, dtype=np.uint64)) *
                                    (size_max - size_min + 1)).astype(np.int64)
        if sizes.sum() > n:
            raise ValueError("communities do not fit in the graph")
        perm = random_permutation(n, seed, 0xC5)
        key = stream_key(seed, 0xC4)
        start, pair_base = 0, 0
        for s in sizes.tolist():
            members = perm[start:start + s]
            a, b = np.triu_indices(s, 1)
            keep = uniform(key, np.arange(pair_base, pair_base + a.size, dtype=np.uint64)) < p_in
            us.append(members[a[keep]])
            vs.append(members[b[keep]])
            start += s
            pair_base += a.size
    return edges_to_csr(n, np.concatenate(us), np.concatenate(vs), f"CL{n}-b{beta}-d{mean_deg}-c{ncomm}s{seed}")


# ----------------------------------------------------------------------------
# Barabasi-Albert graphs and their ego networks (many small graphs)
# ----------------------------------------------------------------------------

def barabasi_albert(n: int, m: int, seed: int = 0) -> CSRGraph:
    """Preferential attachment (Barabasi and Albert, 1999) from a seed clique
    of m + 1 vertices: vertex t >= m + 1 draws m endpoints, each a uniformly
    chosen entry of the endpoint list of every earlier edge (so an earlier
    vertex is chosen with probability proportional to its degree).  Draw j of
    vertex t is counter (t - m - 1) * m + j of stream (seed, 0xBA).  Repeated
    picks of one vertex collapse into one edge, so a few vertices get fewer
    than m edges.  The endpoint list is never materialised: position p of it
    is resolved by following earlier draws (an odd position of a new edge is
    that edge's own draw), all draws at once.
    """
    m0 = m + 1
    if n < m0:
        raise ValueError("n must be at least m + 1")
    su, sv = np.triu_indices(m0, 1)
    seed_end = np.empty(2 * su.size, dtype=np.int64)
    seed_end[0::2] = su
    seed_end[1::2] = sv
    e_seed = su.size
    nt = n - m0
    cnt = np.arange(nt * m, dtype=np.uint64)
    edge = np.arange(nt * m, dtype=np.int64)
    src = m0 + edge // m
    # draws of edge e: a position among the 2 * (edges before its vertex)
    before = e_seed + (edge // m) * m
    pos = np.floor(uniform(stream_key(seed, 0xBA), cnt) * (2 * before)).astype(np.int64)
    pos = np.minimum(pos, 2 * before - 1)
    tgt = np.full(nt * m, -1, dtype=np.int64)
    cur = pos.copy()
    todo = np.arange(nt * m)
    for _ in range(200):
        if todo.size == 0:
            break
        p = cur[todo]
        in_seed = p < 2 * e_seed
        tgt[todo[in_seed]] = seed_end[p[in_seed]]
        q = p[~in_seed] - 2 * e_seed
        rest = todo[~in_seed]
        even = (q % 2) == 0
        tgt[rest[even]] = m0 + (q[even] // 2) // m       # the source of an earlier new edge
        cur[rest[~even]] = pos[q[~even] // 2]             # the target of an earlier new edge: its draw
        todo = rest[~even]
    if todo.size:
        raise RuntimeError("endpoint resolution did not converge")
    u = np.concatenate([su, src])
    v = np.concatenate([sv, tgt])
    return edges_to_csr(n, u, v, f"BA{n}-m{m}s{seed}")


def ego_network(g: CSRGraph, c: int) -> CSRGraph:
    """Radius-1 ego network of c: c, its neighbours and every edge among
    them, relabelled 0..size-1 in increasing id order."""
    rp, ci = g.row_ptr, g.col_idx
    nodes = np.unique(np.concatenate([[c], ci[rp[c]:rp[c + 1]]]).astype(np.int64))
    us, vs = [], []
    for i, x in enumerate(nodes.tolist()):
        nb = ci[rp[x]:rp[x + 1]].astype(np.int64)
        j = np.searchsorted(nodes, nb)
        j = np.minimum(j, nodes.size - 1)
        hit = nodes[j] == nb
        us.append(np.full(int(hit.sum()), i, dtype=np.int64))
        vs.append(j[hit])
    return edges_to_csr(int(nodes.size), np.concatenate(us), np.concatenate(vs), f"ego{c}")


def ego_networks(g: CSRGraph, count: int, size_min: int, size_max: int, seed: int = 0) -> list[CSRGraph]:
    """`count` ego networks of distinct centres drawn uniformly (a seeded
    permutation, stream (seed, 0xE6)) among the vertices whose ego network
    has size_min..size_max vertices (degree + 1)."""
    deg = np.diff(g.row_ptr.astype(np.int64))
    ok = np.nonzero((deg + 1 >= size_min) & (deg + 1 <= size_max))[0]
    if ok.size < count:
        raise ValueError(f"only {ok.size} eligible centres")
    centres = ok[random_permutation(ok.size, seed, 0xE6)[:count]]
    return [ego_network(g, int(c)) for c in centres]


def block_union(graphs: list[CSRGraph]) -> tuple[CSRGraph, np.ndarray]:
    """Block-diagonal union of the graphs and the vertex offsets (len + 1)."""
    off = np.zeros(len(graphs) + 1, dtype=np.uint32)
    np.cumsum([h.n for h in graphs], out=off[1:])
    rps, cis, base_e = [np.zeros(1, dtype=np.uint64)], [], 0
    for h, o in zip(graphs, off[:-1]):
        rps.append(h.row_ptr[1:].astype(np.uint64) + np.uint64(base_e))
        cis.append(h.col_idx.astype(np.uint64) + np.uint64(o))
        base_e += int(h.row_ptr[-1])
    if base_e >= (1 << 32):
        raise ValueError("nnz does not fit in u32")
    rp = np.concatenate(rps).astype(np.uint32)
    ci = (np.concatenate(cis) if cis else np.zeros(0, dtype=np.uint64)).astype(np.uint32)
    return CSRGraph(int(off[-1]), rp, ci, f"union{len(graphs)}"), off
