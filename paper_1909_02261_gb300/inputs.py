"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module only draws random graphs and random initial weights; it holds
none of the coloring method's arithmetic.  Every generator uses numpy's
PCG64 stream, which gives the same values on every platform for a seed.

Graph shapes follow the random DIMACS graphs the paper evaluates on
(DSJC<n>.<p>: uniform random graphs of a given edge density), which are not
shipped here; G(n, p) with the same n and p stands in for them.
"""
from __future__ import annotations

import numpy as np


def _csr_from_upper(n: int, iu: np.ndarray, ju: np.ndarray):
    """Symmetric CSR (rowptr int32[n+1], colidx int32[2|E|], sorted rows)."""
    src = np.concatenate([iu, ju]).astype(np.int64)
    dst = np.concatenate([ju, iu]).astype(np.int64)
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    rowptr = np.zeros(n + 1, np.int64)
    np.add.at(rowptr, src + 1, 1)
    rowptr = np.cumsum(rowptr)
    return rowptr.astype(np.int32), dst.astype(np.int32)


def gnp(n: int, p: float, seed: int):
    """Erdos-Renyi G(n, p): each of the n(n-1)/2 pairs is an edge with prob. p.

    Returns (rowptr, colidx) as int32 CSR, symmetric, no self loops.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    iu, ju = np.triu_indices(n, k=1)
    keep = rng.random(iu.shape[0]) < p
    return _csr_from_upper(n, iu[keep], ju[keep])


def planted_partition(n: int, groups: int, p_inter: float, seed: int):
    """n vertices split into `groups` equal consecutive blocks (hidden colour
    = i * groups // n), no edge inside a block, and each pair of vertices in
    different blocks joined with probability p_inter.

    Returns (rowptr, colidx, hidden) with hidden an int32 colouring.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    hidden = (np.arange(n, dtype=np.int64) * groups // n).astype(np.int32)
    iu, ju = np.triu_indices(n, k=1)
    keep = (hidden[iu] != hidden[ju]) & (rng.random(iu.shape[0]) < p_inter)
    rowptr, colidx = _csr_from_upper(n, iu[keep], ju[keep])
    return rowptr, colidx, hidden


def from_edges(n: int, edges):
    """CSR from an explicit list of undirected edges (u, v), u != v."""
    e = np.asarray(list(edges), dtype=np.int64).reshape(-1, 2)
    lo = np.minimum(e[:, 0], e[:, 1])
    hi = np.maximum(e[:, 0], e[:, 1])
    uniq = np.unique(lo * n + hi)
    return _csr_from_upper(n, uniq // n, uniq % n)


def edge_list(rowptr, colidx):
    """Each undirected edge once, as (u, v) with u < v."""
    rowptr = np.asarray(rowptr)
    colidx = np.asarray(colidx)
    n = len(rowptr) - 1
    src = np.repeat(np.arange(n, dtype=np.int32), np.diff(rowptr))
    keep = src < colidx
    return src[keep], colidx[keep].astype(np.int32)


def dense(rowptr, colidx) -> np.ndarray:
    """n x n uint8 0/1 adjacency matrix."""
    n = len(rowptr) - 1
    A = np.zeros((n, n), np.uint8)
    src = np.repeat(np.arange(n), np.diff(rowptr))
    A[src, colidx] = 1
    return A


def init_weights(D: int, n: int, k: int, sigma0: float, seed: int) -> np.ndarray:
    """float32 D x n x k weights drawn from N(0, sigma0) (sigma0 = std)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return (rng.standard_normal((D, n, k)) * sigma0).astype(np.float32)


def one_hot_weights(colors: np.ndarray, k: int, hi: float = 1.0) -> np.ndarray:
    """float32 weights whose row argmax is `colors` (D x n): `hi` at the
    chosen colour, 0 elsewhere."""
    colors = np.asarray(colors)
    D, n = colors.shape
    W = np.zeros((D, n, k), np.float32)
    W[np.arange(D)[:, None], np.arange(n)[None, :], colors] = hi
    return W


def random_colors(D: int, n: int, k: int, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(0, k, size=(D, n), dtype=np.int64).astype(np.int32)


# Workload recipes (graph seed, n, p or planted shape, k, D) used by the
# parity tests and the benchmark.  Parameters follow Table 2 of the paper
# (GCP column unless noted), rho = 100 for the random graphs.
WORKLOADS = {
    "gnp125_k18_D20": dict(kind="gnp", n=125, p=0.5, graph_seed=1, k=18, D=20, w_seed=1,
                           problem=0),
    "gnp1000_k90_D200": dict(kind="gnp", n=1000, p=0.5, graph_seed=2, k=90, D=200, w_seed=2,
                             problem=0),
    "planted500_k20_D64": dict(kind="planted", n=500, groups=20, p=0.5, graph_seed=3, k=20,
                               D=64, w_seed=3, problem=0),
    "ecp_gnp1000p01_k25_D128": dict(kind="gnp", n=1000, p=0.1, graph_seed=4, k=25, D=128,
                                    w_seed=4, problem=1),
    "ecp_gnp1000p09_k230_D128": dict(kind="gnp", n=1000, p=0.9, graph_seed=5, k=230, D=128,
                                     w_seed=5, problem=1, alpha=1.5),
}


def batched_instances():
    """The batched workload: G(4000, 0.5) with k = 290, D = 100, plus 8
    instances of uneven n = 250, 500, ..., 2000 with p cycling 0.1 / 0.5 / 0.9
    and k = round(n / 50), round(n / 12), round(n / 4.5) by density (the
    ratios of the paper's DSJC1000.{1,5,9} colour counts), D = 100.  Graph
    seeds 10, 11, ..., weight seeds 110, 111, ... .  Returns a list of
    WORKLOADS-style dicts (kind "gnp", problem 0)."""
    out = [dict(kind="gnp", n=4000, p=0.5, graph_seed=10, k=290, D=100, w_seed=110, problem=0)]
    ratio = {0.1: 50.0, 0.5: 12.0, 0.9: 4.5}
    for q in range(8):
        n = 250 * (q + 1)
        p = (0.1, 0.5, 0.9)[q % 3]
        out.append(dict(kind="gnp", n=n, p=p, graph_seed=11 + q, k=max(2, int(round(n / ratio[p]))), D=100,
                        w_seed=111 + q, problem=0))
    return out


def workload_graph(name: str):
    w = WORKLOADS[name]
    if w["kind"] == "gnp":
        rp, ci = gnp(w["n"], w["p"], w["graph_seed"])
        return rp, ci, None
    return planted_partition(w["n"], w["groups"], w["p"], w["graph_seed"])
