"""Batches run as one disjoint union: every graph's slice of the union result equals the oracle's
result for that graph alone."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from helpers import compare_hierarchy, u32  # noqa: E402
from paper_2306_08623_gb300 import graphgen as gg  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2306_08623_gb300.nucleus as mod
    mod.lib()
    return mod


def split_tree(parent, label, n_nodes, lo, hi, n_r):
    """the sub-forest of one graph: its leaves [lo, hi) and the nodes they reach"""
    leaf = parent[lo:hi]
    npar = parent[n_r:n_r + n_nodes]
    used = np.zeros(n_nodes, dtype=bool)
    stack = [int(x) for x in np.unique(leaf[leaf >= 0])]
    while stack:
        x = stack.pop()
        if used[x]:
            continue
        used[x] = True
        if npar[x] >= 0:
            stack.append(int(npar[x]))
    ids = np.nonzero(used)[0]
    remap = np.full(n_nodes, -1, dtype=np.int64)
    remap[ids] = np.arange(len(ids))
    sub_leaf = np.where(leaf >= 0, remap[np.maximum(leaf, 0)], -1)
    sub_par = np.where(npar[ids] >= 0, remap[np.maximum(npar[ids], 0)], -1)
    return np.concatenate([sub_leaf, sub_par]), label[ids], len(ids)


def test_union_batch_matches_each_graph(nc):
    graphs = [gg.batch_member(s) for s in (1000, 1001, 1002)]
    graphs += [gg.rmat(9, 6, 7), gg.complete(6), gg.from_edges(4, []), gg.erdos_renyi(500, 3000, 3)]
    dev = [(torch.from_numpy(o).cuda(), torch.from_numpy(a).cuda()) for o, a in graphs]
    off_u, adj_u, vbase = nc.batch_union(dev)
    assert vbase[-1] == sum(len(o) - 1 for o, _ in graphs)
    for r, s in [(2, 3), (3, 4)]:
        res = nc.hierarchy(off_u, adj_u, r, s)
        rb = nc.rindex_bases(res["rindex"], vbase)
        parent = res["parent"].cpu().numpy()
        label = u32(res["label"])
        cnt, core = u32(res["cnt"]), u32(res["core"])
        for g, (off, adj) in enumerate(graphs):
            ref = oracle.nucleus(off, adj, r, s)
            lo, hi = int(rb[g]), int(rb[g + 1])
            assert hi - lo == ref["n_r"]
            assert np.array_equal(cnt[lo:hi], ref["cnt"]) and np.array_equal(core[lo:hi], ref["core"])
            p, lab, nn = split_tree(parent, label, res["n_nodes"], lo, hi, res["n_r"])
            compare_hierarchy(p, lab, nn, ref["leaf_node"], ref["node_parent"], ref["node_label"])


def _graph_slice(parent, label, nbase, rbase, n_r, g):
    """graph g's part of a union tree: its leaves and its node range, renumbered from 0"""
    lo, hi, a, b = int(rbase[g]), int(rbase[g + 1]), int(nbase[g]), int(nbase[g + 1])
    leaf = parent[lo:hi].astype(np.int64)
    assert ((leaf < 0) | ((leaf >= a) & (leaf < b))).all(), "a leaf hangs from another graph's node"
    npar = parent[n_r + a:n_r + b].astype(np.int64)
    assert ((npar < 0) | ((npar >= a) & (npar < b))).all(), "a node's parent lies in another graph"
    return (np.concatenate([np.where(leaf >= 0, leaf - a, -1), np.where(npar >= 0, npar - a, -1)]),
            label[a:b], b - a)


def test_batch_handle_recipe_graphs(nc):
    """nh_batch_prepare / nh_batch_run on graphs of the 512-graph recipe (seeds 1000-1511): the 152
    with n <= 4000 for (2,3) and every sixth of them for (3,4), captured into one CUDA graph and
    replayed twice; every graph's counts, core numbers and hierarchy (node range from
    nh_batch_node_bases) equal the oracle's for that graph alone."""
    seeds = [1000 + i for i in range(512) if gg.batch_member_shape(1000 + i)[0] <= 4000]
    assert len(seeds) == 152
    for r, s, pick in [(2, 3, seeds), (3, 4, seeds[::6])]:
        graphs = [gg.batch_member(x) for x in pick]
        refs = [oracle.nucleus(off, adj, r, s) for off, adj in graphs]
        dev = [(torch.from_numpy(o).cuda(), torch.from_numpy(a).cuda()) for o, a in graphs]
        b = nc.Batch(dev, r)
        assert b.vbase[-1] == sum(len(o) - 1 for o, _ in graphs)
        buf = b.buffers()
        g = b.capture(s, buf)
        for rep in range(2):
            for t in buf.values():
                t.fill_(-1)
            g.replay()
            torch.cuda.synchronize()
            res = buf["res"].cpu().numpy()
            assert res[0] == 0, res
            nn = int(res[2])
            nb = b.node_bases(buf["parent"], nn)
            parent = buf["parent"].cpu().numpy()
            label = u32(buf["label"])
            cnt, core = u32(buf["cnt"]), u32(buf["core"])
            tot_s = 0
            for i, ref in enumerate(refs):
                lo, hi = int(b.rbase[i]), int(b.rbase[i + 1])
                assert hi - lo == ref["n_r"]
                assert np.array_equal(cnt[lo:hi], ref["cnt"]) and np.array_equal(core[lo:hi], ref["core"])
                p, lab, n_g = _graph_slice(parent, label, nb, b.rbase, b.n_r, i)
                compare_hierarchy(p, lab, n_g, ref["leaf_node"], ref["node_parent"], ref["node_label"])
                tot_s += ref["n_s"]
            assert int(res[1]) == tot_s
        del g, buf, b
