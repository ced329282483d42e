"""Every other (r,s) with r < s <= 7 (the generic path: r-clique index chain up to r = 6, counting by
recursive listing, round-by-round peel, hierarchy by link-efficient over every s-clique) and
link-basic (Alg. 4) for every pair, against the oracle: r-clique tuples, s-clique-degrees, core
numbers, approximate values and their round counts bit for bit, hierarchies after
canonicalisation."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from helpers import compare_hierarchy, u32  # noqa: E402
from paper_2306_08623_gb300 import graphgen as gg  # noqa: E402

pytestmark = pytest.mark.gpu

GENERIC = [(r, s) for s in range(4, 8) for r in range(1, s)
           if (r, s) not in ((2, 4), (3, 4))]
SPECIALISED = [(1, 2), (1, 3), (2, 3), (2, 4), (3, 4)]


@pytest.fixture(scope="module")
def nc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2306_08623_gb300.nucleus as mod
    mod.lib()
    return mod


def to_dev(off, adj):
    return torch.from_numpy(np.ascontiguousarray(off)).cuda(), torch.from_numpy(np.ascontiguousarray(adj)).cuda()


def check(nc, off, adj, r, s, method="el", link_mode="def", deltas=()):
    ref = oracle.nucleus(off, adj, r, s, hier=link_mode)
    d_off, d_adj = to_dev(off, adj)
    res = nc.hierarchy(d_off, d_adj, r, s, link_mode=link_mode, stats=True, method=method)
    assert res["n_r"] == ref["n_r"] and res["n_s"] == ref["n_s"]
    tup = nc.rindex_tuples(res["rindex"]).cpu().numpy().reshape(-1, r)
    assert np.array_equal(tup, ref["tuples"])
    assert np.array_equal(u32(res["cnt"]), ref["cnt"])
    assert np.array_equal(u32(res["core"]), ref["core"])
    compare_hierarchy(res["parent"].cpu().numpy(), u32(res["label"]), res["n_nodes"], ref["leaf_node"],
                      ref["node_parent"], ref["node_label"])
    for d in deltas:
        a = nc.approx_nucleus(res["oriented"], res["rindex"], s, d, res["cnt"], stats=True)
        ra = oracle.nucleus(off, adj, r, s, hier=None, approx_delta=d)
        assert np.array_equal(u32(a["approx"]), ra["approx"]), d
        assert a["stats"]["rounds"] == ra["approx_rounds"], d
    return res, ref


def dense_graphs(seed, count):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.integers(8, 19))
        out.append(gg.gnp(n, float(rng.uniform(0.55, 0.95)), int(rng.integers(1 << 30))))
    return out


@pytest.mark.parametrize("r,s", GENERIC)
def test_generic_pairs_small_dense(nc, r, s):
    for i, (off, adj) in enumerate(dense_graphs(100 + 10 * r + s, 6)):
        res, ref = check(nc, off, adj, r, s, "el", "def", deltas=(0.1, 0.5) if i < 3 else ())
        if i % 2 == 0:
            check(nc, off, adj, r, s, "te")
            check(nc, off, adj, r, s, "el", "pair")
        if i == 1:
            check(nc, off, adj, r, s, "bl")


@pytest.mark.parametrize("r,s", [(1, 4), (2, 5), (3, 5), (4, 5), (1, 5), (3, 6)])
def test_generic_rmat_hubs(nc, r, s):
    """R-MAT scale 9 with edge factor 16: hub vertices, many warps, many rounds."""
    off, adj = gg.rmat(9, 16, 4)
    res, ref = check(nc, off, adj, r, s, "el", "def", deltas=(0.5,))
    assert res["stats"]["rounds"] >= 2


@pytest.mark.parametrize("r,s", [(2, 5), (3, 6), (4, 7), (1, 7), (5, 6), (6, 7)])
def test_generic_closed_forms(nc, r, s):
    """K_9: every r-clique has core C(9-r, s-r) and the hierarchy is one node; disjoint cliques:
    one node per clique, C(k-r, s-r) each."""
    from math import comb
    off, adj = gg.complete(9)
    res, ref = check(nc, off, adj, r, s)
    assert (u32(res["core"]) == comb(9 - r, s - r)).all() and res["n_nodes"] == 1
    sizes = [s, s + 1, 8, 9]
    off, adj = gg.disjoint_cliques(sizes)
    res, ref = check(nc, off, adj, r, s)
    assert res["n_nodes"] == len(sizes)
    assert sorted(u32(res["label"]).tolist()) == sorted(comb(k - r, s - r) for k in sizes)


def test_generic_edge_cases(nc):
    cases = [gg.from_edges(5, []), gg.from_edges(1, []), gg.from_edges(2, [(0, 1)]),
             gg.from_edges(6, [(0, i) for i in range(1, 6)]), gg.from_edges(9, [(i, i + 1) for i in range(8)]),
             gg.complete(5)]
    for off, adj in cases:
        for r, s in [(2, 5), (4, 5), (1, 6), (6, 7)]:
            check(nc, off, adj, r, s, deltas=(0.5,))


@pytest.mark.parametrize("r,s", SPECIALISED)
def test_link_basic_specialised_pairs(nc, r, s):
    """Alg. 4 (per-level union-finds, construct-tree-basic) gives the definitional hierarchy."""
    off, adj = gg.rmat(10, 8, 5)
    res, _ = check(nc, off, adj, r, s, "bl")
    assert res["basic_unites"] > 0
    for off, adj in dense_graphs(200 + 10 * r + s, 4):
        check(nc, off, adj, r, s, "bl")


def test_generic_cut(nc):
    """c-nuclei of a generic pair's hierarchy equal the oracle's cut at every level."""
    from test_gpu_cut import same_partition
    off, adj = gg.chung_lu(600, 2.1, 8, 9, groups=3, per_group=3, size_lo=7, size_hi=11)
    res, ref = check(nc, off, adj, 2, 5)
    for c in range(0, int(ref["core"].max()) + 2):
        want = oracle.cut_hierarchy(ref["leaf_node"], ref["node_parent"], ref["node_label"], c)
        got, n = nc.cut_hierarchy(res["parent"], res["label"], res["n_r"], res["n_nodes"], c)
        assert same_partition(got.cpu().numpy(), want) and n == len(np.unique(want[want >= 0]))
