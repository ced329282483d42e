"""Pins of the CPU oracle against things other than itself (CPU only).

Each test fixes a part of the oracle to the paper's definitions, to closed forms, to
hand-derived examples (tests/golden), to textbook routines (networkx k-core / k-truss, scipy
triangle count) or to brute force on tiny graphs.
"""
import json
import os
from fractions import Fraction
from math import comb, ceil, floor, log

import numpy as np
import pytest

import oracle
from oracle.brute import brute_label_hierarchy, brute_nucleus, tree_to_nodes
from paper_2306_08623_gb300 import graphgen as gg

GOLD = os.path.join(os.path.dirname(__file__), "golden")
RS_SMALL = [(1, 2), (1, 3), (2, 3), (1, 4), (2, 4), (3, 4), (2, 5), (3, 5)]
# every other r < s <= 7 (the generic GPU path's pairs), with fewer trials each
RS_WIDE = [(r, s) for s in range(5, 8) for r in range(1, s) if (r, s) not in RS_SMALL]


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _hier(res):
    nodes = tree_to_nodes(res["leaf_node"], res["node_parent"], res["node_label"])
    assert len(nodes) == res["n_nodes"], "two nodes with the same leaf set"
    return nodes


# --------------------------------------------------------------------------------------------
# brute force on tiny graphs: counts, core numbers, both hierarchy readings, Alg. 3 + Alg. 5
# --------------------------------------------------------------------------------------------

@pytest.mark.parametrize("r,s", RS_SMALL)
def test_oracle_vs_brute_force(r, s):
    rng = np.random.default_rng(100 + 10 * r + s)
    for trial in range(40):
        n = int(rng.integers(4, 12))
        p = float(rng.uniform(0.35, 0.95))
        off, adj = gg.gnp(n, p, int(rng.integers(1 << 30)))
        edges = [tuple(e) for e in gg.edge_list(off, adj)]
        bf = brute_nucleus(n, edges, r, s, "def")
        bp = brute_nucleus(n, edges, r, s, "pair")
        res = oracle.nucleus(off, adj, r, s, hier="def")
        assert [tuple(t) for t in res["tuples"]] == bf["rcliques"]
        assert res["n_s"] == bf["n_s"]
        assert res["cnt"].tolist() == bf["cnt"]
        assert res["core"].tolist() == bf["core"], (n, edges)
        assert _hier(res) == bf["nodes"], (n, edges)
        assert _hier(oracle.nucleus(off, adj, r, s, hier="pair")) == bp["nodes"], (n, edges)
        assert _hier(oracle.nucleus(off, adj, r, s, hier="link_def")) == bf["nodes"], (n, edges)
        assert _hier(oracle.nucleus(off, adj, r, s, hier="link_pair")) == bp["nodes"], (n, edges)


@pytest.mark.parametrize("r,s", RS_WIDE)
def test_oracle_vs_brute_force_wide_pairs(r, s):
    """The same pins for the remaining pairs up to s = 7 on graphs with planted overlapping cliques
    (so that s-cliques and nuclei of several levels exist): tuples, counts, core numbers, both
    hierarchy readings, both hierarchy algorithms."""
    rng = np.random.default_rng(500 + 10 * r + s)
    with_nodes = 0
    for trial in range(12):
        # two or three overlapping planted cliques of s..s+2 vertices plus sparse random edges:
        # nuclei of several levels
        n = int(rng.integers(s + 2, 14))
        es = set()
        for _ in range(int(rng.integers(2, 4))):
            k = int(rng.integers(s, min(s + 3, n + 1)))
            vs = sorted(rng.choice(n, size=k, replace=False).tolist())
            es |= {(a, b) for i, a in enumerate(vs) for b in vs[i + 1:]}
        es |= {(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < 0.25}
        off, adj = gg.from_edges(n, sorted(es))
        edges = [tuple(e) for e in gg.edge_list(off, adj)]
        bf = brute_nucleus(n, edges, r, s, "def")
        bp = brute_nucleus(n, edges, r, s, "pair")
        res = oracle.nucleus(off, adj, r, s, hier="def")
        assert [tuple(t) for t in res["tuples"]] == bf["rcliques"]
        assert res["n_s"] == bf["n_s"]
        assert res["cnt"].tolist() == bf["cnt"]
        assert res["core"].tolist() == bf["core"], (n, edges)
        assert _hier(res) == bf["nodes"], (n, edges)
        assert _hier(oracle.nucleus(off, adj, r, s, hier="pair")) == bp["nodes"], (n, edges)
        assert _hier(oracle.nucleus(off, adj, r, s, hier="link_def")) == bf["nodes"], (n, edges)
        with_nodes += len(bf["nodes"]) > 1
    assert with_nodes >= 3  # the pins are not vacuous: several trials have multi-node hierarchies


def test_level_and_link_hierarchies_agree_medium():
    """Alg. 3 + Alg. 5 (sequential) and the level union-find give the same hierarchy on graphs
    too large for brute force."""
    for seed, (r, s) in [(1, (1, 2)), (2, (2, 3)), (3, (2, 4)), (4, (3, 4)), (5, (1, 3))]:
        off, adj = gg.rmat(8, 6, seed)
        a = _hier(oracle.nucleus(off, adj, r, s, hier="def"))
        b = _hier(oracle.nucleus(off, adj, r, s, hier="link_def"))
        assert a == b
        a = _hier(oracle.nucleus(off, adj, r, s, hier="pair"))
        b = _hier(oracle.nucleus(off, adj, r, s, hier="link_pair"))
        assert a == b


# --------------------------------------------------------------------------------------------
# closed forms and special cases
# --------------------------------------------------------------------------------------------

@pytest.mark.parametrize("n,r,s", [(5, 2, 3), (6, 3, 4), (10, 2, 4), (7, 1, 2), (8, 1, 3), (9, 3, 5), (6, 2, 5)])
def test_complete_graph_closed_form(n, r, s):
    """K_n: every r-clique lies in C(n-r, s-r) s-cliques, which is also its core number, and the
    hierarchy is one node holding every r-clique."""
    off, adj = gg.complete(n)
    res = oracle.nucleus(off, adj, r, s)
    k = comb(n - r, s - r)
    assert res["n_r"] == comb(n, r) and res["n_s"] == comb(n, s)
    assert (res["cnt"] == k).all() and (res["core"] == k).all()
    assert _hier(res) == {frozenset(range(comb(n, r))): k}


def test_disjoint_planted_cliques():
    sizes = [4, 7, 5, 9, 3, 6]
    off, adj = gg.disjoint_cliques(sizes)
    for r, s in [(1, 2), (2, 3), (2, 4), (3, 4)]:
        res = oracle.nucleus(off, adj, r, s)
        nodes = _hier(res)
        expect, base_ids = {}, 0
        tup = res["tuples"]
        starts = np.cumsum([0] + sizes)
        for i, k in enumerate(sizes):
            in_clique = (tup[:, 0] >= starts[i]) & (tup[:, 0] < starts[i + 1])
            ids = np.nonzero(in_clique)[0]
            assert len(ids) == comb(k, r)
            want = comb(k - r, s - r) if k >= s else 0
            assert (res["core"][ids] == want).all()
            if want >= 1:
                expect[frozenset(ids.tolist())] = want
        assert nodes == expect


def test_two_k4_bridge_golden():
    g = _gold("two_k4_bridge.json")
    off, adj = gg.from_edges(g["n"], g["edges"])
    name = lambda t: "%d-%d" % (t[0], t[1])
    for mode, key in [("def", "nodes_definitional"), ("pair", "nodes_pairwise"),
                      ("link_def", "nodes_definitional"), ("link_pair", "nodes_pairwise")]:
        res = oracle.nucleus(off, adj, g["r"], g["s"], hier=mode)
        names = [name(t) for t in res["tuples"]]
        assert {names[i]: int(c) for i, c in enumerate(res["core"])} == g["core"]
        got = {frozenset(names[i] for i in leaves): lab for leaves, lab in _hier(res).items()}
        want = {frozenset(x["edges"]): x["label"] for x in g[key]}
        assert got == want, mode


def test_sum_of_counts_and_cores():
    """sum_R cnt(R) = C(s,r) n_s; core <= cnt; sum of cores <= C(s,r) n_s (§5, proof of Thm. 1)."""
    off, adj = gg.rmat(9, 8, 11)
    for r, s in [(1, 2), (2, 3), (2, 4), (3, 4), (1, 3)]:
        res = oracle.nucleus(off, adj, r, s, hier=None)
        C = comb(s, r)
        assert int(res["cnt"].sum(dtype=np.int64)) == C * res["n_s"]
        assert (res["core"] <= res["cnt"]).all()
        assert int(res["core"].sum(dtype=np.int64)) <= C * res["n_s"]


def test_triangle_count_matches_trace_of_a_cubed():
    scipy = pytest.importorskip("scipy.sparse")
    off, adj = gg.rmat(10, 8, 5)
    n = len(off) - 1
    A = scipy.csr_matrix((np.ones(len(adj)), adj, off), shape=(n, n))
    tri = int(round((A @ A).multiply(A).sum() / 6))
    res = oracle.nucleus(off, adj, 2, 3, hier=None)
    assert res["n_s"] == tri
    assert int(res["cnt"].sum(dtype=np.int64)) == 3 * tri


def test_relabel_invariance():
    """Core numbers and hierarchy do not depend on vertex ids."""
    off, adj = gg.rmat(8, 8, 21)
    n = len(off) - 1
    perm = np.random.default_rng(3).permutation(n)
    e = gg.edge_list(off, adj)
    off2, adj2 = gg.csr_from_pairs(n, perm[e[:, 0]], perm[e[:, 1]])
    for r, s in [(1, 2), (2, 3), (3, 4)]:
        a = oracle.nucleus(off, adj, r, s)
        b = oracle.nucleus(off2, adj2, r, s)
        key_a = {tuple(sorted(perm[t])): c for t, c in zip(a["tuples"].tolist(), a["core"].tolist())}
        key_b = {tuple(t): c for t, c in zip(b["tuples"].tolist(), b["core"].tolist())}
        assert key_a == key_b
        name_a = [tuple(sorted(perm[t])) for t in a["tuples"].tolist()]
        name_b = [tuple(t) for t in b["tuples"].tolist()]
        ha = {frozenset(name_a[i] for i in L): c for L, c in _hier(a).items()}
        hb = {frozenset(name_b[i] for i in L): c for L, c in _hier(b).items()}
        assert ha == hb


# --------------------------------------------------------------------------------------------
# textbook routines: (1,2) = k-core, (2,3) = k-truss (§3)
# --------------------------------------------------------------------------------------------

def _nx_graph(off, adj):
    nx = pytest.importorskip("networkx")
    G = nx.Graph()
    G.add_nodes_from(range(len(off) - 1))
    G.add_edges_from(map(tuple, gg.edge_list(off, adj).tolist()))
    return nx, G


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_k_core_matches_networkx(seed):
    off, adj = gg.rmat(10, 8, seed)
    nx, G = _nx_graph(off, adj)
    res = oracle.nucleus(off, adj, 1, 2, hier="def")
    want = nx.core_number(G)
    assert res["core"].tolist() == [want[v] for v in range(len(off) - 1)]
    # hierarchy nodes of (1,2) are connected components of k-cores with at least 2 vertices
    nodes = _hier(res)
    expect = {}
    for k in range(1, res["kmax"] + 1):
        H = nx.k_core(G, k)
        for comp in nx.connected_components(H):
            if len(comp) >= 2:
                fs = frozenset(comp)
                expect[fs] = max(expect.get(fs, 0), k)
    assert nodes == expect


@pytest.mark.parametrize("seed", [4, 5])
def test_k_truss_matches_networkx(seed):
    """networkx k_truss(G, k): every edge in >= k-2 triangles; (2,3) core = truss - 2."""
    off, adj = gg.rmat(9, 8, seed)
    nx, G = _nx_graph(off, adj)
    res = oracle.nucleus(off, adj, 2, 3, hier=None)
    eid = {tuple(t): i for i, t in enumerate(res["tuples"].tolist())}
    truss = np.full(res["n_r"], 2, dtype=np.int64)
    k = 3
    while True:
        H = nx.k_truss(G, k)
        if H.number_of_edges() == 0:
            break
        for a, b in H.edges():
            truss[eid[(min(a, b), max(a, b))]] = k
        k += 1
    assert (res["core"].astype(np.int64) == truss - 2).all()


# --------------------------------------------------------------------------------------------
# §7.3 worked traces for link-efficient and construct-tree-efficient
# --------------------------------------------------------------------------------------------

def test_link_efficient_worked_trace():
    g = _gold("link_efficient_trace.json")
    ids = {name: i for i, name in enumerate(g["rcliques"])}
    n = len(ids)
    uf = np.arange(n, dtype=np.int32)
    L = np.full(n, -1, dtype=np.int32)
    for k, v in g["initial_L"].items():
        L[ids[k]] = ids[v]
    oracle.link_apply(np.array(g["core"], dtype=np.uint32), uf, L,
                      [(ids[a], ids[b]) for a, b in g["calls"]])
    root = {x: oracle.uf_find(uf, ids[x]) for x in ids}
    e = g["expect"]
    for a, b in e["same_component"]:
        assert root[a] == root[b]
    for x in e["singleton"]:
        assert sum(1 for y in ids if root[y] == root[x]) == 1
    for x, y in e["L_of_component"].items():
        assert L[root[x]] >= 0 and oracle.uf_find(uf, L[root[x]]) == root[y]
    for x, ys in e["L_of_component_one_of"].items():
        assert int(L[root[x]]) in {ids[y] for y in ys}
    for x in e["L_empty"]:
        assert L[root[x]] == -1


def test_construct_tree_worked_trace():
    g = _gold("construct_tree_trace.json")
    ids = {name: i for i, name in enumerate(g["rcliques"])}
    n = len(ids)
    uf = np.arange(n, dtype=np.int32)
    for k, v in g["uf"].items():
        uf[ids[k]] = ids[v]
    L = np.full(n, -1, dtype=np.int32)
    for k, v in g["L"].items():
        L[ids[k]] = ids[v]
    t = oracle.tree_from_uf(uf, L, np.array(g["core"], dtype=np.uint32))
    got = tree_to_nodes(t["leaf_node"], t["node_parent"], t["node_label"])
    want = {frozenset(ids[x] for x in nd["leaves"]): nd["label"] for nd in g["expect_nodes"]}
    assert got == want


# --------------------------------------------------------------------------------------------
# Alg. 2 (approximate core numbers)
# --------------------------------------------------------------------------------------------

def test_approx_thresholds_closed_form():
    """delta = 0.5: (C+delta)(1+delta)^(i+1) is exact in binary, so the FP64 recurrence must equal
    the exact rational floor; delta = 0.1, 1.0 checked against exact rational arithmetic on the
    same double."""
    for C in (2, 3, 4, 6):
        for delta in (0.5, 0.1, 1.0):
            t = oracle.approx_thresholds(C, delta, 10 ** 9)
            d = Fraction(delta)
            for i, ti in enumerate(t[:60].tolist()):
                assert ti == floor((C + d) * (1 + d) ** (i + 1)), (C, delta, i)
            assert (np.diff(t.astype(np.int64)) >= 0).all()


def test_approx_round_cap_formula():
    for C, delta, n_r in [(3, 0.1, 10 ** 6), (2, 0.5, 12), (4, 0.5, 424_000_000), (3, 1.0, 5)]:
        assert oracle.approx_round_cap(C, delta, n_r) == ceil(log(max(n_r, 2)) / log(1 + delta / C)) + 1


def test_approx_hand_worked_example():
    g = _gold("approx_k6_star.json")
    off, adj = gg.from_edges(g["n"], g["edges"])
    res = oracle.nucleus(off, adj, g["r"], g["s"], hier=None, approx_delta=g["delta"])
    assert oracle.approx_thresholds(2, g["delta"], 100)[:4].tolist() == g["thresholds_prefix"]
    assert res["thresholds"][-1] >= res["cnt"].max()
    assert res["approx_T"] == g["T"]
    assert res["approx"].tolist() == g["approx"]
    assert res["core"].tolist() == g["exact_core"]
    assert res["approx_rounds"] == g["rounds"]


@pytest.mark.parametrize("delta", [0.1, 0.5, 1.0])
def test_approx_bounds_random(delta):
    """Thm. 2: core <= approx <= (C(s,r)+delta)(1+delta) core; core 0 gives approx 0."""
    for seed, (r, s) in [(31, (1, 2)), (32, (2, 3)), (33, (2, 4)), (34, (3, 4)), (35, (1, 3))]:
        off, adj = gg.rmat(9, 10, seed)
        res = oracle.nucleus(off, adj, r, s, hier=None, approx_delta=delta)
        core = res["core"].astype(np.float64)
        ap = res["approx"].astype(np.float64)
        C = comb(s, r)
        assert (ap[core == 0] == 0).all()
        nz = core > 0
        assert (ap[nz] >= core[nz]).all()
        assert (ap[nz] <= (C + delta) * (1 + delta) * core[nz] + 1e-9).all()
        assert (ap <= res["cnt"]).all()


def test_approx_special_cases():
    # K_n: all counts equal -> everything peeled together at its own count = exact core
    off, adj = gg.complete(9)
    res = oracle.nucleus(off, adj, 2, 3, hier=None, approx_delta=0.5)
    assert (res["approx"] == res["core"]).all()
    # disjoint cliques: each clique peels as a block at its own count
    off, adj = gg.disjoint_cliques([4, 6, 9, 5])
    res = oracle.nucleus(off, adj, 2, 3, hier=None, approx_delta=0.1)
    assert (res["approx"] == res["core"]).all()
    # very large delta: one round peels everything at min(t_0, cnt) = cnt
    off, adj = gg.rmat(8, 8, 2)
    res = oracle.nucleus(off, adj, 2, 3, hier=None, approx_delta=1e4)
    assert (res["approx"] == res["cnt"]).all() and res["approx_rounds"] == 1


# --------------------------------------------------------------------------------------------
# the sampled local certificate used at sizes the full oracle cannot reach
# --------------------------------------------------------------------------------------------

def _sync_peel_rounds(off, adj, r, s, res):
    """Round stamps of the synchronous peel (each round removes every live r-clique of current
    count <= k, k the running maximum of the minimum), in plain Python, to feed the checker a
    valid peel order."""
    ids = {tuple(t): i for i, t in enumerate(res["tuples"].tolist())}
    from itertools import combinations
    mem = [[ids[c] for c in combinations(S, r)] for S in oracle.list_cliques(off, adj, s).tolist()]
    inc = [[] for _ in range(res["n_r"])]
    for j, m in enumerate(mem):
        for x in m:
            inc[x].append(j)
    cnt = res["cnt"].astype(np.int64).copy()
    rnd = np.zeros(res["n_r"], dtype=np.uint32)
    dead = [False] * len(mem)
    k, t = 0, 0
    while (rnd == 0).any():
        t += 1
        alive = np.nonzero(rnd == 0)[0]
        k = max(k, int(cnt[alive].min()))
        A = alive[cnt[alive] <= k]
        rnd[A] = t
        for R in A.tolist():
            for j in inc[R]:
                if dead[j]:
                    continue
                dead[j] = True
                for x in mem[j]:
                    if rnd[x] == 0:
                        cnt[x] -= 1
    return rnd


def test_check_sample_accepts_truth_and_rejects_planted_mistakes():
    off, adj = gg.rmat(8, 8, 7)
    r, s = 2, 3
    res = oracle.nucleus(off, adj, r, s, hier="def")
    n_r = res["n_r"]
    tuples = res["tuples"]
    sample = np.arange(n_r)
    # parent array in the GPU layout: leaves then nodes
    parent = np.concatenate([res["leaf_node"], res["node_parent"]]).astype(np.int32)
    label = res["node_label"]
    rnd = _sync_peel_rounds(off, adj, r, s, res)
    bad = oracle.check_sample(off, adj, r, s, tuples, sample, cnt=res["cnt"], core=res["core"],
                              rnd=rnd, parent=parent, label=label)
    assert bad.tolist() == [0, 0, 0, 0]
    # every r-clique in one round breaks the peel-order bound wherever cnt > core
    ones = np.ones(n_r, dtype=np.uint32)
    assert oracle.check_sample(off, adj, r, s, tuples, sample, core=res["core"], rnd=ones)[2] == \
        int((res["cnt"] > res["core"]).sum())
    # a wrong count
    cnt2 = res["cnt"].copy()
    cnt2[5] += 1
    assert oracle.check_sample(off, adj, r, s, tuples, sample, cnt=cnt2)[0] == 1
    # a core number one too high fails validity somewhere
    top = int(np.argmax(res["core"]))
    core2 = res["core"].copy()
    core2[top] += 1
    assert oracle.check_sample(off, adj, r, s, tuples, sample, core=core2)[1] >= 1
    # a hierarchy with two nodes' parents cut apart fails connectivity
    if res["n_nodes"] >= 2:
        child = int(np.nonzero(res["node_parent"] >= 0)[0][0])
        parent2 = parent.copy()
        parent2[n_r + child] = -1
        assert oracle.check_sample(off, adj, r, s, tuples, sample, core=res["core"], parent=parent2,
                                   label=label)[3] >= 1


# ---- hierarchy of arbitrary labels (the approximate hierarchy of §6 on Alg. 2's values) ----

def _edges(off, adj):
    return [(a, int(b)) for a in range(len(off) - 1) for b in adj[off[a]:off[a + 1]] if a < b]


@pytest.mark.parametrize("r,s", [(1, 2), (1, 3), (2, 3), (2, 4), (3, 4)])
def test_label_hierarchy_vs_brute_force(r, s):
    """Core numbers, random labels (r-cliques left alone at their own level occur) and Alg. 2's
    approximate values, against components taken level by level from the definition."""
    rng = np.random.default_rng(100 + 10 * r + s)
    n_cases = 0
    for _ in range(60):
        n = int(rng.integers(4, 10))
        off, adj = gg.gnp(n, float(rng.uniform(0.4, 0.95)), int(rng.integers(1 << 30)))
        o = oracle.nucleus(off, adj, r, s)
        if o["n_r"] == 0:
            continue
        for lab in (o["core"], rng.integers(0, 6, size=o["n_r"]).astype(np.uint32),
                    oracle.nucleus(off, adj, r, s, hier=None, approx_delta=0.5)["approx"]):
            res = oracle.label_hierarchy(off, adj, r, s, lab)
            got = tree_to_nodes(res["leaf_node"], res["node_parent"], res["node_label"])
            assert got == brute_label_hierarchy(n, _edges(off, adj), r, s, lab)
            n_cases += 1
    assert n_cases > 100


def test_label_hierarchy_of_cores_is_the_core_hierarchy():
    off, adj = gg.rmat(8, 8, 3)
    for r, s in [(1, 2), (2, 3), (2, 4), (3, 4)]:
        o = oracle.nucleus(off, adj, r, s)
        res = oracle.label_hierarchy(off, adj, r, s, o["core"])
        assert tree_to_nodes(res["leaf_node"], res["node_parent"], res["node_label"]) == \
            tree_to_nodes(o["leaf_node"], o["node_parent"], o["node_label"])


def test_label_hierarchy_singleton_waits_for_a_lower_level():
    """K3 with (1,2): vertex 0 labelled 2, the others 1.  At level 2 vertex 0 is alone (no edge
    has both ends labelled >= 2), so no node exists there; at level 1 all three join: one node
    {0,1,2} labelled 1, and vertex 0 is its leaf."""
    off, adj = gg.complete(3)
    res = oracle.label_hierarchy(off, adj, 1, 2, np.array([2, 1, 1], dtype=np.uint32))
    assert res["n_nodes"] == 1
    assert list(res["leaf_node"]) == [0, 0, 0]
    assert list(res["node_label"]) == [1]
    # a vertex whose label is never matched by any edge stays outside every node
    off, adj = gg.from_edges(4, [(0, 1), (1, 2)])
    res = oracle.label_hierarchy(off, adj, 1, 2, np.array([0, 3, 3, 5], dtype=np.uint32))
    assert tree_to_nodes(res["leaf_node"], res["node_parent"], res["node_label"]) == {frozenset({1, 2}): 3}
    assert res["leaf_node"][0] == -1 and res["leaf_node"][3] == -1


# ---- c-(r,s) nuclei by cutting the hierarchy (§8, dense subgraph discovery) ----

def _partition(labels):
    groups = {}
    for i, g in enumerate(labels):
        if g >= 0:
            groups.setdefault(int(g), set()).add(i)
    return {frozenset(v) for v in groups.values()}


@pytest.mark.parametrize("r,s", [(1, 2), (2, 3), (2, 4), (3, 4)])
def test_cut_hierarchy_gives_the_c_nuclei(r, s):
    """Cutting the tree at c equals the connected components, by definition, of the r-cliques of
    core >= c joined through the s-cliques all of whose members have core >= c."""
    rng = np.random.default_rng(300 + 10 * r + s)
    checked = 0
    for _ in range(25):
        n = int(rng.integers(5, 11))
        off, adj = gg.gnp(n, float(rng.uniform(0.4, 0.95)), int(rng.integers(1 << 30)))
        o = oracle.nucleus(off, adj, r, s)
        if o["n_r"] == 0:
            continue
        edges = _edges(off, adj)
        b = brute_nucleus(n, edges, r, s)
        for c in range(1, o["kmax"] + 1):
            comp = oracle.cut_hierarchy(o["leaf_node"], o["node_parent"], o["node_label"], c)
            # the components of X_c are the nodes of the brute-force hierarchy present at level c
            want = {X for X, lab in b["nodes"].items() if lab >= c}
            maximal = {X for X in want if not any(X < Y for Y in want)}
            assert _partition(comp) == maximal
            assert all((comp[R] >= 0) == (o["core"][R] >= c) for R in range(o["n_r"]))
            checked += 1
    assert checked > 20


def test_cut_hierarchy_of_cliques_sharing_a_vertex():
    """Two K5 sharing vertex 4 plus a separate K4.  (1,2): the K5 pair is one 4-nucleus (the
    shared vertex connects them), the K4 a 3-nucleus.  (2,3): no triangle spans the two K5, so
    at c = 3 they are two separate 3-nuclei of 10 edges each, and the K4's 6 edges a 2-nucleus."""
    e = [(a, b) for a in range(5) for b in range(a + 1, 5)]
    e += [(a, b) for a in range(4, 9) for b in range(a + 1, 9)]
    e += [(a, b) for a in range(10, 14) for b in range(a + 1, 14)]
    off, adj = gg.from_edges(14, sorted(set(e)))
    o = oracle.nucleus(off, adj, 1, 2)
    cut = lambda c: _partition(oracle.cut_hierarchy(o["leaf_node"], o["node_parent"], o["node_label"], c))
    assert cut(4) == {frozenset(range(9))}
    assert cut(3) == {frozenset(range(9)), frozenset(range(10, 14))}
    assert cut(5) == set()
    o = oracle.nucleus(off, adj, 2, 3)
    tup = [tuple(t) for t in o["tuples"]]
    edges_of = lambda vs: frozenset(i for i, (a, b) in enumerate(tup) if a in vs and b in vs)
    A, B, K = edges_of(set(range(5))), edges_of(set(range(4, 9))), edges_of(set(range(10, 14)))
    cut = lambda c: _partition(oracle.cut_hierarchy(o["leaf_node"], o["node_parent"], o["node_label"], c))
    assert len(A) == len(B) == 10 and len(K) == 6
    assert cut(3) == {A, B}
    assert cut(2) == {A, B, K}
