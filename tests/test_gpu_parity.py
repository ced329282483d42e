"""GPU path (through the C-ABI) against the CPU oracle, element by element.

Integer results: bit-exact.  r-clique ids, s-clique-degrees, exact core numbers and approximate
core numbers must be identical; hierarchies must be identical up to node numbering.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from helpers import compare_hierarchy, u32  # noqa: E402
from paper_2306_08623_gb300 import graphgen as gg  # noqa: E402

pytestmark = pytest.mark.gpu
SUPPORTED = [(1, 2), (1, 3), (2, 3), (2, 4), (3, 4)]
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def nc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2306_08623_gb300.nucleus as mod
    mod.lib()
    return mod


def to_dev(off, adj):
    return torch.from_numpy(np.ascontiguousarray(off)).cuda(), torch.from_numpy(np.ascontiguousarray(adj)).cuda()


def run_gpu(nc, off, adj, r, s, link_mode="def", deltas=()):
    d_off, d_adj = to_dev(off, adj)
    res = nc.hierarchy(d_off, d_adj, r, s, link_mode=link_mode, stats=True)
    out = {"n_r": res["n_r"], "n_s": res["n_s"], "cnt": u32(res["cnt"]), "core": u32(res["core"]),
           "round": u32(res["round"]), "parent": res["parent"].cpu().numpy(), "label": u32(res["label"]),
           "n_nodes": res["n_nodes"], "tuples": nc.rindex_tuples(res["rindex"]).cpu().numpy(),
           "stats": res["stats"]}
    for d in deltas:
        a = nc.approx_nucleus(res["oriented"], res["rindex"], s, d, res["cnt"], stats=True)
        out["approx_%g" % d] = u32(a["approx"])
        out["approx_stats_%g" % d] = a["stats"]
    return out


def check(nc, off, adj, r, s, link_mode="def", deltas=(), ref=None):
    g = run_gpu(nc, off, adj, r, s, link_mode, deltas)
    if ref is None:
        ref = oracle.nucleus(off, adj, r, s, hier=link_mode)
    assert g["n_r"] == ref["n_r"]
    assert g["n_s"] == ref["n_s"]
    assert np.array_equal(g["tuples"].reshape(-1, r), ref["tuples"])
    assert np.array_equal(g["cnt"], ref["cnt"])
    assert np.array_equal(g["core"], ref["core"])
    compare_hierarchy(g["parent"], g["label"], g["n_nodes"], ref["leaf_node"], ref["node_parent"],
                      ref["node_label"])
    for d in deltas:
        ra = oracle.nucleus(off, adj, r, s, hier=None, approx_delta=d)
        assert np.array_equal(g["approx_%g" % d], ra["approx"]), d
        assert g["approx_stats_%g" % d]["rounds"] == ra["approx_rounds"]
    return g, ref


# --------------------------------------------------------------------------------------------

@pytest.mark.parametrize("r,s", SUPPORTED)
def test_small_random_graphs(nc, r, s):
    rng = np.random.default_rng(7 + 10 * r + s)
    for trial in range(25):
        n = int(rng.integers(3, 16))
        off, adj = gg.gnp(n, float(rng.uniform(0.3, 0.95)), int(rng.integers(1 << 30)))
        check(nc, off, adj, r, s, "def", deltas=(0.1, 0.5))
        if trial % 3 == 0:
            check(nc, off, adj, r, s, "pair")


def test_er_2000_16000_23(nc):
    """Erdos-Renyi G(n=2000, m=16000), seed 1, exact (2,3) hierarchy and approximate cores."""
    off, adj = gg.erdos_renyi(2000, 16000, 1)
    check(nc, off, adj, 2, 3, "def", deltas=(0.1, 0.5))
    check(nc, off, adj, 2, 3, "pair")


@pytest.mark.parametrize("r,s", SUPPORTED)
def test_rmat_several_tiles(nc, r, s):
    """R-MAT scale 11: many warps, many rounds, hub vertices, ragged frontiers."""
    off, adj = gg.rmat(11, 8, 3)
    g, _ = check(nc, off, adj, r, s, "def", deltas=(0.1, 0.5))
    assert g["stats"]["rounds"] >= 2
    check(nc, off, adj, r, s, "pair")


@pytest.mark.parametrize("r,s", [(2, 3), (3, 4)])
def test_chung_lu_planted(nc, r, s):
    off, adj = gg.chung_lu(3000, 2.1, 10, 5, groups=6, per_group=5, size_lo=6, size_hi=14)
    check(nc, off, adj, r, s, "def", deltas=(0.5,))


def test_edge_cases(nc):
    cases = [
        gg.from_edges(5, []),                       # no edges: every count 0
        gg.from_edges(1, []),                       # one vertex
        gg.from_edges(2, [(0, 1)]),                 # one edge
        gg.from_edges(6, [(0, i) for i in range(1, 6)]),  # star: no triangles
        gg.complete(7),
        gg.disjoint_cliques([3, 5, 6, 4]),
        gg.from_edges(9, [(i, i + 1) for i in range(8)]),  # path
    ]
    for off, adj in cases:
        for r, s in SUPPORTED:
            check(nc, off, adj, r, s, "def", deltas=(0.5,))


def test_two_k4_bridge_both_readings(nc):
    g = json.load(open(os.path.join(GOLD, "two_k4_bridge.json")))
    off, adj = gg.from_edges(g["n"], g["edges"])
    check(nc, off, adj, 2, 3, "def")
    check(nc, off, adj, 2, 3, "pair")


def test_round_stamps_are_a_peel_certificate(nc):
    """The GPU's round stamps and core numbers satisfy the local certificate (every r-clique had
    at most core[R] live s-cliques when it was peeled; at least core[R] s-cliques inside the
    set of core >= core[R]); core numbers never decrease with the round."""
    off, adj = gg.rmat(10, 8, 9)
    for r, s in SUPPORTED:
        g = run_gpu(nc, off, adj, r, s)
        sample = np.arange(g["n_r"])
        bad = oracle.check_sample(off, adj, r, s, g["tuples"].reshape(-1, r), sample, cnt=g["cnt"],
                                  core=g["core"], rnd=g["round"], parent=g["parent"], label=g["label"])
        assert bad.tolist() == [0, 0, 0, 0], (r, s, bad)
        order = np.argsort(g["round"], kind="stable")
        assert (np.diff(g["core"][order].astype(np.int64)) >= 0).all()
        assert g["round"].min() >= 1 and g["round"].max() == g["stats"]["rounds"]


def test_repeatable(nc):
    off, adj = gg.rmat(10, 8, 4)
    a = run_gpu(nc, off, adj, 2, 3)
    b = run_gpu(nc, off, adj, 2, 3)
    assert np.array_equal(a["core"], b["core"]) and np.array_equal(a["round"], b["round"])
    ref = oracle.nucleus(off, adj, 2, 3)
    for g in (a, b):
        compare_hierarchy(g["parent"], g["label"], g["n_nodes"], ref["leaf_node"], ref["node_parent"],
                          ref["node_label"])


# --------------------------------------------------------------------------------------------
# link-efficient and construct-tree in isolation (§7.3 worked traces; concurrent stress)
# --------------------------------------------------------------------------------------------

def test_link_pairs_worked_trace(nc):
    g = json.load(open(os.path.join(GOLD, "link_efficient_trace.json")))
    ids = {name: i for i, name in enumerate(g["rcliques"])}
    n = len(ids)
    core = torch.tensor(g["core"], dtype=torch.int32, device="cuda")
    uf = torch.arange(n, dtype=torch.int32, device="cuda")
    L = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    for k, v in g["initial_L"].items():
        L[ids[k]] = ids[v]
    for a, b in g["calls"]:  # one call at a time: the trace is sequential
        nc.link_pairs(core, uf, L, torch.tensor([ids[a], ids[b]], dtype=torch.int32, device="cuda"))
    ufh, Lh = uf.cpu().numpy(), L.cpu().numpy()

    def root(x):
        while ufh[x] != x:
            x = ufh[x]
        return x
    rt = {x: root(ids[x]) for x in ids}
    e = g["expect"]
    for a, b in e["same_component"]:
        assert rt[a] == rt[b]
    for x in e["singleton"]:
        assert sum(1 for y in ids if rt[y] == rt[x]) == 1
    for x, y in e["L_of_component"].items():
        assert Lh[rt[x]] >= 0 and root(Lh[rt[x]]) == rt[y]
    for x, ys in e["L_of_component_one_of"].items():
        assert int(Lh[rt[x]]) in {ids[y] for y in ys}
    for x in e["L_empty"]:
        assert Lh[rt[x]] == -1


def test_construct_tree_worked_trace(nc):
    g = json.load(open(os.path.join(GOLD, "construct_tree_trace.json")))
    ids = {name: i for i, name in enumerate(g["rcliques"])}
    n = len(ids)
    uf = np.arange(n, dtype=np.int32)
    for k, v in g["uf"].items():
        uf[ids[k]] = ids[v]
    L = np.full(n, -1, dtype=np.int32)
    for k, v in g["L"].items():
        L[ids[k]] = ids[v]
    core = torch.tensor(g["core"], dtype=torch.int32, device="cuda")
    parent, label, nn = nc.construct_tree(core, torch.from_numpy(uf).cuda(), torch.from_numpy(L).cuda())
    from oracle.brute import tree_to_nodes
    p = parent.cpu().numpy()
    got = tree_to_nodes(p[:n], p[n:n + nn], u32(label))
    want = {frozenset(ids[x] for x in nd["leaves"]): nd["label"] for nd in g["expect_nodes"]}
    assert got == want


def test_construct_tree_rejects_cyclic_uf(nc):
    """A uf array with a cycle is no union-find forest: construct-tree reports NH_ERR_INVALID (its
    root walks are bounded by n_r steps) and a valid call afterwards still succeeds."""
    n = 5
    core = torch.ones(n, dtype=torch.int32, device="cuda")
    uf = torch.tensor([1, 2, 0, 3, 3], dtype=torch.int32, device="cuda")  # 0 -> 1 -> 2 -> 0
    L = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    with pytest.raises(nc.NucleusError) as ei:
        nc.construct_tree(core, uf, L)
    assert ei.value.status == 1  # NH_ERR_INVALID
    uf = torch.tensor([0, 0, 0, 3, 3], dtype=torch.int32, device="cuda")
    parent, label, nn = nc.construct_tree(core, uf, L)
    assert nn == 2 and sorted(u32(label).tolist()) == [1, 1]


def test_link_pairs_concurrent_matches_definition(nc):
    """All link calls of the definitional reading (each s-clique: its min-core member with every
    other member), shuffled and issued at once, then construct-tree: equals the oracle."""
    from itertools import combinations
    off, adj = gg.rmat(10, 10, 12)
    for r, s in [(1, 2), (2, 3), (3, 4)]:
        ref = oracle.nucleus(off, adj, r, s)
        tid = {tuple(t): i for i, t in enumerate(ref["tuples"].tolist())}
        core = ref["core"]
        pairs = []
        for S in oracle.list_cliques(off, adj, s).tolist():
            mem = [tid[c] for c in combinations(S, r)]
            m = min(mem, key=lambda x: core[x])
            pairs += [(m, x) for x in mem if x != m]
        pairs = np.array(pairs, dtype=np.int32)
        pairs = pairs[np.random.default_rng(1).permutation(len(pairs))]
        n = ref["n_r"]
        d_core = torch.from_numpy(core.view(np.int32)).cuda()
        uf = torch.arange(n, dtype=torch.int32, device="cuda")
        L = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        nc.link_pairs(d_core, uf, L, torch.from_numpy(pairs.reshape(-1)).cuda())
        parent, label, nn = nc.construct_tree(d_core, uf, L)
        compare_hierarchy(parent.cpu().numpy(), u32(label), nn, ref["leaf_node"], ref["node_parent"],
                          ref["node_label"])


def test_error_paths(nc):
    """Host-side argument checks return status codes; the context stays usable."""
    import ctypes
    lib = nc.lib()
    off, adj = gg.rmat(8, 4, 1)
    d_off, d_adj = to_dev(off, adj)
    o = nc.build_orientation(d_off, d_adj)
    ri = nc.index_r_cliques(o, 2)
    cnt, _ = nc.count_s_cliques(o, ri, 3)
    for bad_s in (8, 2, 1):  # s beyond 7, or not above r
        with pytest.raises(nc.NucleusError) as e:
            nc.count_s_cliques(o, ri, bad_s)
        assert e.value.status == 6
    with pytest.raises(nc.NucleusError) as e:
        nc.index_r_cliques(o, 7)  # r-clique index: r <= 6
    assert e.value.status == 1
    with pytest.raises(nc.NucleusError) as e:
        nc.approx_nucleus(o, ri, 3, -1.0, cnt)
    assert e.value.status == 1
    # unsorted / out of range / asymmetric CSR inputs are rejected before any kernel uses them
    bad_inputs = [
        (np.array([0, 2, 3, 4], np.int64), np.array([2, 1, 0, 0], np.int32)),   # unsorted list of 0
        (np.array([0, 1, 2], np.int64), np.array([1, 5], np.int32)),            # id out of range
        (np.array([0, 1, 2, 3, 4], np.int64), np.array([1, 2, 3, 0], np.int32)),  # directed cycle
        (np.array([0, 1, 1], np.int64), np.array([1], np.int32)),               # odd nnz
    ]
    for boff, badj in bad_inputs:
        with pytest.raises(nc.NucleusError) as e:
            nc.build_orientation(*to_dev(boff, badj))
        assert e.value.status == 1
    assert lib.nh_version() >= 100
    # still usable
    check(nc, off, adj, 2, 3)


@pytest.mark.parametrize("scale,r,s", [(12, 2, 4), (13, 2, 3), (13, 1, 2), (11, 3, 4), (12, 1, 3)])
def test_repeated_runs_deep_hierarchies(nc, scale, r, s):
    """Concurrent link-efficient is nondeterministic in its intermediate states; every repeat must
    still give the oracle's hierarchy (deep hierarchies: (2,4) on R-MAT 12 has 525 nodes over 993
    levels)."""
    off, adj = gg.rmat(scale, 16, 2)
    ref = oracle.nucleus(off, adj, r, s)
    for _ in range(4):
        check(nc, off, adj, r, s, ref=ref)


@pytest.mark.parametrize("r,s", SUPPORTED)
def test_two_phase_hierarchy(nc, r, s):
    """§7.4 two-phase hierarchy from the GPU core numbers equals the oracle's hierarchy."""
    graphs = [gg.rmat(11, 8, 3), gg.erdos_renyi(2000, 16000, 1), gg.complete(7), gg.from_edges(5, []),
              gg.chung_lu(3000, 2.1, 10, 5, groups=6, per_group=5, size_lo=6, size_hi=14)]
    rng = np.random.default_rng(99 + r + s)
    for _ in range(8):
        graphs.append(gg.gnp(int(rng.integers(4, 14)), float(rng.uniform(0.4, 0.95)), int(rng.integers(1 << 30))))
    for off, adj in graphs:
        d_off, d_adj = to_dev(off, adj)
        o = nc.build_orientation(d_off, d_adj)
        ri = nc.index_r_cliques(o, r)
        cnt, _ = nc.count_s_cliques(o, ri, s)
        pk = nc.peel_and_link(o, ri, s, cnt)
        parent, label, nn = nc.hierarchy_two_phase(o, ri, s, pk["core"])
        ref = oracle.nucleus(off, adj, r, s)
        compare_hierarchy(parent.cpu().numpy(), u32(label), nn, ref["leaf_node"], ref["node_parent"],
                          ref["node_label"])


@pytest.mark.parametrize("r,s", SUPPORTED)
@pytest.mark.parametrize("method", ["te", "auto"])
def test_hierarchy_methods(nc, r, s, method):
    """The cores-only peel (link mode 2, no union-find) gives the same cores and round stamps as the
    linking peel; the te/auto hierarchy from it equals the oracle's."""
    for off, adj in [gg.rmat(11, 8, 5), gg.chung_lu(3000, 2.1, 10, 6, groups=6, per_group=5, size_lo=6, size_hi=14),
                     gg.from_edges(4, []), gg.complete(6)]:
        d_off, d_adj = to_dev(off, adj)
        res = nc.hierarchy(d_off, d_adj, r, s, method=method, stats=True)
        ref = oracle.nucleus(off, adj, r, s)
        assert np.array_equal(u32(res["cnt"]), ref["cnt"])
        assert np.array_equal(u32(res["core"]), ref["core"])
        compare_hierarchy(res["parent"].cpu().numpy(), u32(res["label"]), res["n_nodes"], ref["leaf_node"],
                          ref["node_parent"], ref["node_label"])
        pk = nc.peel_cores(res["oriented"], res["rindex"], s, res["cnt"])
        assert np.array_equal(u32(pk["core"]), ref["core"])
        # the peel is round-synchronous, so its round stamps do not depend on linking
        assert np.array_equal(u32(pk["round"]), u32(res["round"]))


@pytest.mark.parametrize("r,s", SUPPORTED)
def test_tuning_knobs_do_not_change_results(nc, r, s):
    """Work-proportional tasks on or off, and any warp-group cap, give the oracle's cores, round
    stamps and hierarchy (both hierarchy methods; the approximate peel too)."""
    off, adj = gg.rmat(12, 16, 7)
    ref = oracle.nucleus(off, adj, r, s)
    ra = oracle.nucleus(off, adj, r, s, hier=None, approx_delta=0.5)
    d_off, d_adj = to_dev(off, adj)
    rounds = None
    try:
        for items, gmax in [(0, 1024), (0, 1), (4096, 1024), (64, 4), (1, 32), (-1, 1024)]:
            nc.set_peel_task_items(items)
            nc.set_peel_max_group(gmax)
            for method in ("el", "te"):
                res = nc.hierarchy(d_off, d_adj, r, s, method=method)
                assert np.array_equal(u32(res["core"]), ref["core"]), (items, gmax, method)
                compare_hierarchy(res["parent"].cpu().numpy(), u32(res["label"]), res["n_nodes"], ref["leaf_node"],
                                  ref["node_parent"], ref["node_label"])
                if rounds is None:
                    rounds = u32(res["round"])
                assert np.array_equal(u32(res["round"]), rounds)
            a = nc.approx_nucleus(res["oriented"], res["rindex"], s, 0.5, res["cnt"])
            assert np.array_equal(u32(a["approx"]), ra["approx"])
        with pytest.raises(nc.NucleusError):
            nc.set_peel_task_items(4097)
    finally:
        nc.set_peel_task_items(-1)
        nc.set_peel_max_group(1024)
