"""Seeded synthetic graph generators (inputs only; none of the decomposition's arithmetic).

Every generator returns an undirected simple graph in CSR form: ``off`` (int64, n+1) and ``adj``
(int32, 2m), each neighbour list sorted ascending, with no self-loops and no duplicate edges.
These graphs stand in for the SNAP graphs of the paper's evaluation, which are not used here.
Randomness comes from numpy's PCG64 generator seeded explicitly, so a seed fixes the graph.

This module is shared by the tests, the benchmark and the oracle's callers; it must not import
the CUDA binding or the oracle.
"""
from __future__ import annotations

import math

import numpy as np


def csr_from_pairs(n: int, u, v):
    """Symmetrise, drop self-loops, de-duplicate and sort; returns (off, adj)."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    keep = u != v
    u, v = u[keep], v[keep]
    lo = np.minimum(u, v)
    hi = np.maximum(u, v)
    key = np.unique(lo * n + hi)
    lo = key // n
    hi = key - lo * n
    src = np.concatenate([lo, hi])
    dst = np.concatenate([hi, lo])
    k2 = np.sort(src * n + dst)
    src = k2 // n
    dst = (k2 - src * n).astype(np.int32)
    deg = np.bincount(src, minlength=n)
    off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=off[1:])
    return off, np.ascontiguousarray(dst)


def from_edges(n: int, edges):
    e = np.asarray(list(edges), dtype=np.int64).reshape(-1, 2)
    return csr_from_pairs(n, e[:, 0], e[:, 1])


def edge_list(off, adj):
    """Upper-triangular edge list (u < v) in lexicographic order."""
    n = len(off) - 1
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(off))
    m = adj > src
    return np.stack([src[m], adj[m].astype(np.int64)], axis=1)


def complete(n: int):
    iu = np.triu_indices(n, 1)
    return csr_from_pairs(n, iu[0], iu[1])


def disjoint_cliques(sizes):
    us, vs, base = [], [], 0
    for k in sizes:
        iu = np.triu_indices(k, 1)
        us.append(iu[0] + base)
        vs.append(iu[1] + base)
        base += k
    return csr_from_pairs(base, np.concatenate(us) if us else [], np.concatenate(vs) if vs else [])


def gnp(n: int, p: float, seed: int):
    """G(n, p) -- small random graphs for exhaustive tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    iu = np.triu_indices(n, 1)
    keep = rng.random(len(iu[0])) < p
    return csr_from_pairs(n, iu[0][keep], iu[1][keep])


def erdos_renyi(n: int, m: int, seed: int):
    """G(n, m): m distinct uniformly random vertex pairs, no self-loops."""
    rng = np.random.Generator(np.random.PCG64(seed))
    have = np.zeros(0, dtype=np.int64)
    while len(have) < m:
        k = int((m - len(have)) * 1.2) + 16
        a = rng.integers(0, n, size=k)
        b = rng.integers(0, n, size=k)
        ok = a != b
        key = np.minimum(a, b)[ok] * n + np.maximum(a, b)[ok]
        allk = np.concatenate([have, key])
        _, first = np.unique(allk, return_index=True)
        have = allk[np.sort(first)]
    have = have[:m]
    return csr_from_pairs(n, have // n, have % n)


def rmat(scale: int, edge_factor: int, seed: int, a: float = 0.57, b: float = 0.19, c: float = 0.19):
    """R-MAT: edge_factor * 2**scale sampled pairs; at every bit the quadrant is drawn with
    probabilities (a, b, c, 1-a-b-c); no noise, no vertex permutation; symmetrised and
    de-duplicated, self-loops dropped."""
    n = 1 << scale
    M = edge_factor * n
    rng = np.random.Generator(np.random.PCG64(seed))
    u = np.zeros(M, dtype=np.int64)
    v = np.zeros(M, dtype=np.int64)
    ab, abc = a + b, a + b + c
    for bit in range(scale - 1, -1, -1):
        x = rng.random(M, dtype=np.float32)
        ubit = x >= ab
        vbit = ((x >= a) & (x < ab)) | (x >= abc)
        u |= ubit.astype(np.int64) << bit
        v |= vbit.astype(np.int64) << bit
    return csr_from_pairs(n, u, v)


def planted_clique_pairs(n: int, groups: int, per_group: int, size_lo: int, size_hi: int, rng):
    """Nested groups of cliques: clique j+1 of a group reuses ceil(size/2) vertices of clique j,
    its other vertices uniform; returns (u, v) pair arrays."""
    us, vs = [], []
    for _ in range(groups):
        prev = None
        for _j in range(per_group):
            k = int(rng.integers(size_lo, size_hi + 1))
            if prev is None:
                verts = rng.choice(n, size=k, replace=False)
            else:
                reuse = min(int(math.ceil(k / 2)), len(prev))
                keep = rng.choice(prev, size=reuse, replace=False)
                fresh = rng.choice(n, size=k - reuse, replace=False)
                verts = np.unique(np.concatenate([keep, fresh]))
            iu = np.triu_indices(len(verts), 1)
            us.append(verts[iu[0]])
            vs.append(verts[iu[1]])
            prev = verts
    if not us:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    return np.concatenate(us), np.concatenate(vs)


def chung_lu(n: int, beta: float, mean_deg: float, seed: int, groups: int = 0, per_group: int = 5,
             size_lo: int = 10, size_hi: int = 60):
    """Chung-Lu power-law graph with weights w_i proportional to (i+1)^(-1/(beta-1)), scaled to
    the mean degree and capped at sqrt(sum w); n*mean_deg/2 endpoint pairs drawn proportional to
    w; plus ``groups`` x ``per_group`` planted nested cliques of sizes U[size_lo, size_hi]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w = (np.arange(n, dtype=np.float64) + 1.0) ** (-1.0 / (beta - 1.0))
    w *= mean_deg * n / w.sum()
    w = np.minimum(w, math.sqrt(w.sum()))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    E = int(n * mean_deg / 2)
    u = np.searchsorted(cdf, rng.random(E), side="right")
    v = np.searchsorted(cdf, rng.random(E), side="right")
    u = np.minimum(u, n - 1)
    v = np.minimum(v, n - 1)
    if groups:
        pu, pv = planted_clique_pairs(n, groups, per_group, size_lo, size_hi, rng)
        u = np.concatenate([u, pu])
        v = np.concatenate([v, pv])
    return csr_from_pairs(n, u, v)


def shared_hubs(commons, inner_deg: float, seed: int, extra: int = 0):
    """Adjacent hub pairs with long shared neighbourhoods: for each k in ``commons`` two new hub
    vertices, joined to each other and to the same k fresh vertices, whose k vertices get about
    k * inner_deg / 2 random edges among themselves; the hub edge then lies in k triangles and
    in one 4-clique per inner edge.  ``extra`` random vertices with the same inner density are
    attached to random shared vertices.  Exercises long per-edge triangle lists."""
    rng = np.random.Generator(np.random.PCG64(seed))
    us, vs = [], []
    base = 0
    for k in commons:
        a, b = base, base + 1
        W = np.arange(base + 2, base + 2 + k, dtype=np.int64)
        us += [np.array([a]), np.full(k, a), np.full(k, b)]
        vs += [np.array([b]), W, W]
        E = int(k * inner_deg / 2)
        us.append(rng.choice(W, size=E))
        vs.append(rng.choice(W, size=E))
        base += 2 + k
    n = base + extra
    if extra and base > 0:
        X = np.arange(base, n, dtype=np.int64)
        us.append(np.repeat(X, 3))
        vs.append(rng.integers(0, base, size=3 * extra))
    if not us:
        return csr_from_pairs(max(n, 1), [], [])
    return csr_from_pairs(n, np.concatenate(us), np.concatenate(vs))


def batch_member_shape(seed: int):
    """(n, mean degree, family) of one graph of the 512-graph batch, without building it."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = int(round(math.exp(rng.uniform(math.log(1e3), math.log(2e5)))))
    md = float(rng.uniform(8.0, 40.0))
    return n, md, seed % 3


def batch_member(seed: int):
    """One graph of the 512-graph batch: n log-uniform in [1e3, 2e5], mean degree U[8, 40],
    family by seed mod 3: Erdos-Renyi, R-MAT (scale ceil(log2 n), ids >= n dropped), Chung-Lu
    with max(1, n/2000) planted cliques."""
    n, md, fam = batch_member_shape(seed)
    if fam == 0:
        return erdos_renyi(n, int(n * md / 2), seed)
    if fam == 1:
        scale = int(math.ceil(math.log2(n)))
        ef = max(1, int(round(md / 2 * n / (1 << scale))))
        off, adj = rmat(scale, ef, seed)
        e = edge_list(off, adj)
        e = e[(e[:, 0] < n) & (e[:, 1] < n)]
        return csr_from_pairs(n, e[:, 0], e[:, 1])
    return chung_lu(n, 2.1, md, seed, groups=max(1, n // 2000), per_group=1)


def describe(off, adj) -> dict:
    deg = np.diff(off)
    return {"n": int(len(off) - 1), "m": int(len(adj) // 2), "max_deg": int(deg.max() if len(deg) else 0),
            "non_isolated": int((deg > 0).sum())}
