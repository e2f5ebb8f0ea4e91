"""Seeded inputs of the batched and serving workloads (inputs only: no
k-clique arithmetic here).

Batched: 4,096 radius-1 ego networks of a Barabasi-Albert graph BA(n =
500,000, m = 20) (seed 0) with 50 to 5,000 vertices each (centres seed 0),
each queried once with k uniform in 3..8 (stream (1, 0xB3)).

Serving: a pool of 64 graphs --
  - 16 Erdos-Renyi graphs, n uniform in [10^4, 10^5], mean degree uniform in
    [8, 32];
  - 24 R-MAT graphs (edge factor 16, a/b/c/d = .57/.19/.19/.05), scales
    14..18 in turn;
  - 24 Chung-Lu power-law graphs, n uniform in [10^5, 10^6], exponent 2.1,
    mean degree 30, no planted communities --
(graph i drawn with seed i, its parameters from stream (2, 0x5F), counter
i) and a Poisson stream of queries (graph uniform, k uniform in 3..12,
pivot with probability 1/2) at a given rate (stream (2, 0x5A)).
"""
from __future__ import annotations

import math
import os

import numpy as np

from . import synth


def ego_batch(count: int = 4096, n: int = 500_000, m: int = 20, size_min: int = 50, size_max: int = 5000):
    """(ego networks, k per query) of the batched workload."""
    ba = synth.barabasi_albert(n, m, seed=0)
    egos = synth.ego_networks(ba, count, size_min, size_max, seed=0)
    ks = 3 + np.floor(synth.uniform(synth.stream_key(1, 0xB3), np.arange(count, dtype=np.uint64)) * 6).astype(np.int64)
    return egos, ks


POOL_SIZE = 64


def serve_spec(i: int) -> tuple:
    """Kind and parameters of pool graph i."""
    u = synth.uniform(synth.stream_key(2, 0x5F), np.array([3 * i, 3 * i + 1, 3 * i + 2], dtype=np.uint64))
    if i < 16:
        n = 10_000 + int(u[0] * 90_000)
        deg = 8.0 + u[1] * 24.0
        return ("er", n, deg / (n - 1))
    if i < 40:
        return ("rmat", 14 + (i - 16) % 5)
    return ("chunglu", 100_000 + int(u[0] * 900_000))


def serve_graph(i: int) -> synth.CSRGraph:
    spec = serve_spec(i)
    if spec[0] == "er":
        g = synth.erdos_renyi(spec[1], spec[2], seed=i)
    elif spec[0] == "rmat":
        g = synth.rmat(spec[1], 16, seed=i)
    else:
        g = synth.chung_lu_planted(spec[1], 2.1, 30.0, 0, seed=i)
    g.name = f"pool{i}-{spec[0]}"
    return g


def serve_pool(processes: int | None = None) -> list[synth.CSRGraph]:
    """The 64 pool graphs, generated in parallel worker processes (spawned,
    so that no process forks a CUDA context)."""
    import concurrent.futures as cf
    import multiprocessing as mp

    procs = processes or min(16, os.cpu_count() or 1)
    if procs <= 1:
        return [serve_graph(i) for i in range(POOL_SIZE)]
    with cf.ProcessPoolExecutor(max_workers=procs, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(serve_graph, range(POOL_SIZE)))


def query_stream(rate: float, seconds: float, ngraphs: int = POOL_SIZE):
    """Arrival times (s), graph ids, k and pivot flags of a Poisson stream."""
    nmax = int(rate * seconds * 1.5) + 64
    key = synth.stream_key(2, 0x5A)
    c = np.arange(nmax, dtype=np.uint64)
    gaps = -np.log1p(-synth.uniform(key, 4 * c)) / rate
    t = np.cumsum(gaps)
    keep = t < seconds
    g = np.floor(synth.uniform(key, 4 * c + 1) * ngraphs).astype(np.int64)
    k = 3 + np.floor(synth.uniform(key, 4 * c + 2) * 10).astype(np.int64)
    p = synth.uniform(key, 4 * c + 3) < 0.5
    return t[keep], g[keep], k[keep], p[keep]
