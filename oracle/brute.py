"""Brute force straight from the definitions, for graphs of at most ~12 vertices.

TEST INFRASTRUCTURE (part of the oracle).  No peeling order, no union-find, no bucket queue:

* an r-clique / s-clique is a vertex set whose pairs are all edges (§3);
* X_c is the largest set of r-cliques in which every member lies in at least c s-cliques whose
  r-subsets all belong to X_c -- computed as a fixpoint by repeated deletion;
* the (r,s)-clique core number of R is the largest c with R in X_c (X_0 = all r-cliques);
* the hierarchy node set is every connected component of size >= 2 of X_c (c >= 1), where two
  r-cliques are joined when one s-clique inside X_c contains both; a component is labelled by the
  largest c at which exactly that set is a component.

The "pairwise" variant joins two r-cliques of one s-clique at level c when both have core >= c,
whatever the other members of that s-clique are (the literal pair rule of Alg. 1 / Alg. 3).
"""
from __future__ import annotations

from itertools import combinations


def cliques(n: int, adjset: list[set[int]], k: int) -> list[tuple[int, ...]]:
    out = []
    for c in combinations(range(n), k):
        if all(b in adjset[a] for a, b in combinations(c, 2)):
            out.append(c)
    return out  # itertools yields lexicographic order


def brute_nucleus(n: int, edges, r: int, s: int, mode: str = "def"):
    adjset = [set() for _ in range(n)]
    for a, b in edges:
        adjset[a].add(b)
        adjset[b].add(a)
    rcl = cliques(n, adjset, r)
    rid = {c: i for i, c in enumerate(rcl)}
    scl = cliques(n, adjset, s)
    mem = [[rid[sub] for sub in combinations(S, r)] for S in scl]
    n_r = len(rcl)
    cnt = [0] * n_r
    for m in mem:
        for x in m:
            cnt[x] += 1
    # X_c by deletion fixpoint, for c = 1, 2, ... until empty
    X = {0: set(range(n_r))}
    c = 1
    while True:
        cur = set(X[c - 1])
        changed = True
        while changed:
            changed = False
            inside = [0] * n_r
            for m in mem:
                if all(x in cur for x in m):
                    for x in m:
                        inside[x] += 1
            drop = {x for x in cur if inside[x] < c}
            if drop:
                cur -= drop
                changed = True
        if not cur:
            break
        X[c] = cur
        c += 1
    kmax = c - 1
    core = [0] * n_r
    for lev in range(1, kmax + 1):
        for x in X[lev]:
            core[x] = lev
    nodes = components_by_level(n_r, mem, core, kmax, mode)
    return {"rcliques": rcl, "n_s": len(scl), "cnt": cnt, "core": core, "kmax": kmax, "nodes": nodes}


def brute_label_hierarchy(n: int, edges, r: int, s: int, labels) -> dict[frozenset, int]:
    """Hierarchy nodes of arbitrary per-r-clique labels (lexicographic r-clique ids), by the same
    definition with labels in place of core numbers."""
    adjset = [set() for _ in range(n)]
    for a, b in edges:
        adjset[a].add(b)
        adjset[b].add(a)
    rcl = cliques(n, adjset, r)
    rid = {c: i for i, c in enumerate(rcl)}
    mem = [[rid[sub] for sub in combinations(S, r)] for S in cliques(n, adjset, s)]
    labels = [int(x) for x in labels]
    return components_by_level(len(rcl), mem, labels, max(labels, default=0), "def")


def components_by_level(n_r: int, mem, core, kmax: int, mode: str) -> dict[frozenset, int]:
    """Every component of size >= 2 at every level c >= 1 (r-cliques of core >= c, joined by the
    s-cliques inside), labelled by the largest c at which it is a component."""
    nodes: dict[frozenset, int] = {}
    for lev in range(1, kmax + 1):
        par = list(range(n_r))

        def find(x):
            while par[x] != x:
                par[x] = par[par[x]]
                x = par[x]
            return x

        for m in mem:
            if mode == "def":
                if all(core[x] >= lev for x in m):
                    for x in m[1:]:
                        par[find(x)] = find(m[0])
            else:
                sel = [x for x in m if core[x] >= lev]
                for x in sel[1:]:
                    par[find(x)] = find(sel[0])
        comps: dict[int, set] = {}
        for x in range(n_r):
            if core[x] >= lev:
                comps.setdefault(find(x), set()).add(x)
        for comp in comps.values():
            if len(comp) >= 2:
                fs = frozenset(comp)
                nodes[fs] = max(nodes.get(fs, 0), lev)
    return nodes


def tree_to_nodes(leaf_node, node_parent, node_label) -> dict[frozenset, int]:
    """Hierarchy given as (leaf -> smallest node, node -> parent, node -> level) to the set of
    (leaf set, level) pairs."""
    nn = len(node_parent)
    leaves = [set() for _ in range(nn)]
    for R, N in enumerate(leaf_node):
        N = int(N)
        while N >= 0:
            leaves[N].add(R)
            N = int(node_parent[N])
    return {frozenset(leaves[N]): int(node_label[N]) for N in range(nn)}
