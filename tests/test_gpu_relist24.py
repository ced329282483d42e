"""The (2,4) re-listing over per-edge triangle lists (warp-staged, block-staged and multi-slab
candidate sets), the (2,3) re-listing over the same lists and the (3,4) re-listing over the
mirrored triangle lists, against the oracle and against the plain re-listing
(nh_set_peel_relist24(0)), through the C-ABI.

Graphs with hub edges whose triangle lists are longer than a warp's staging area (512) and than
a block's (4096) drive every branch; the exact core numbers and round stamps, the two-phase
hierarchy, the approximate values and the label hierarchy must equal the oracle's.
"""
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


GRAPHS = {
    "hubs": lambda: gg.shared_hubs([5000, 1500, 600, 90], 12.0, 11, extra=400),
    "hubs_dense": lambda: gg.shared_hubs([4500, 700], 30.0, 12),
    "rmat12": lambda: gg.rmat(12, 16, 7),
    "chung_lu": lambda: gg.chung_lu(4000, 2.1, 12, 8, groups=8, per_group=5, size_lo=8, size_hi=20),
}


def _run(nc, off, adj, r, s, on):
    nc.set_peel_relist24(on)
    try:
        d_off, d_adj = torch.from_numpy(off).cuda(), torch.from_numpy(adj).cuda()
        o = nc.build_orientation(d_off, d_adj)
        ri = nc.index_r_cliques(o, r)
        cnt, n_s = nc.count_s_cliques(o, ri, s)
        pk = nc.peel_cores(o, ri, s, cnt, stats=True)
        parent, label, nn = nc.hierarchy_two_phase(o, ri, s, pk["core"])
        out = {"n_s": n_s, "cnt": u32(cnt), "core": u32(pk["core"]), "round": u32(pk["round"]),
               "parent": parent.cpu().numpy(), "label": u32(label), "nn": nn, "stats": pk["stats"]}
        el = nc.peel_and_link(o, ri, s, cnt)  # the linking peel (the (3,4) builder of the benchmark)
        ep, elab, enn = nc.construct_tree(el["core"], el["uf"], el["L"])
        out["el"] = (u32(el["core"]), ep.cpu().numpy(), u32(elab), enn)
        for d in (0.1, 0.5):
            a = nc.approx_nucleus(o, ri, s, d, cnt, stats=True)
            out["approx_%g" % d] = u32(a["approx"])
            out["approx_rounds_%g" % d] = a["stats"]["rounds"]
            lp, ll, ln = nc.label_hierarchy(o, ri, s, a["approx"])
            out["lab_%g" % d] = (lp.cpu().numpy(), u32(ll), ln)
        torch.cuda.synchronize()
        return out
    finally:
        nc.set_peel_relist24(True)


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("r,s", [(2, 4), (2, 3), (3, 4)])
def test_triangle_list_relisting_matches_oracle(nc, name, r, s):
    off, adj = GRAPHS[name]()
    ref = oracle.nucleus(off, adj, r, s)
    g = _run(nc, off, adj, r, s, True)
    assert g["n_s"] == ref["n_s"]
    assert np.array_equal(g["cnt"], ref["cnt"])
    assert np.array_equal(g["core"], ref["core"])
    compare_hierarchy(g["parent"], g["label"], g["nn"], ref["leaf_node"], ref["node_parent"], ref["node_label"])
    ec, ep, elab, enn = g["el"]
    assert np.array_equal(ec, ref["core"])
    compare_hierarchy(ep, elab, enn, ref["leaf_node"], ref["node_parent"], ref["node_label"])
    rls = {}
    for d in (0.1, 0.5):
        ra = oracle.nucleus(off, adj, r, s, hier=None, approx_delta=d)
        assert np.array_equal(g["approx_%g" % d], ra["approx"]), d
        assert g["approx_rounds_%g" % d] == ra["approx_rounds"]
        rl = rls[d] = oracle.label_hierarchy(off, adj, r, s, g["approx_%g" % d])
        lp, ll, ln = g["lab_%g" % d]
        compare_hierarchy(lp, ll, ln, rl["leaf_node"], rl["node_parent"], rl["node_label"])
    # the other re-listing gives the same round stamps (the peel is round-synchronous)
    h = _run(nc, off, adj, r, s, False)
    assert np.array_equal(h["core"], g["core"]) and np.array_equal(h["round"], g["round"])
    for d in (0.1, 0.5):
        assert np.array_equal(h["approx_%g" % d], g["approx_%g" % d])
    if (r, s) == (3, 4):
        # the (edge, third vertex) table for the pruned peels (1) and everywhere (2) in place of
        # the default binary searches: the same results, the linking peel and the hierarchies
        # included
        for mode in (1, 2):
            nc.set_peel_list_hash(mode)
            try:
                b = _run(nc, off, adj, r, s, True)
            finally:
                nc.set_peel_list_hash(0)
            assert np.array_equal(b["core"], g["core"]) and np.array_equal(b["round"], g["round"])
            compare_hierarchy(b["parent"], b["label"], b["nn"], ref["leaf_node"], ref["node_parent"],
                              ref["node_label"])
            ec, ep, elab, enn = b["el"]
            assert np.array_equal(ec, ref["core"])
            compare_hierarchy(ep, elab, enn, ref["leaf_node"], ref["node_parent"], ref["node_label"])
            for d in (0.1, 0.5):
                assert np.array_equal(b["approx_%g" % d], g["approx_%g" % d])
                lp, ll, ln = b["lab_%g" % d]
                compare_hierarchy(lp, ll, ln, rls[d]["leaf_node"], rls[d]["node_parent"], rls[d]["node_label"])
            assert b["stats"]["hash_probes"] > 0  # the cores-only peel takes the table in both modes
        assert g["stats"]["hash_probes"] == 0


def test_long_lists_take_every_branch(nc):
    """The hub edges' triangle lists are longer than both staging areas."""
    off, adj = GRAPHS["hubs"]()
    e = gg.edge_list(off, adj)
    deg = np.diff(off)
    e = e[(deg[e[:, 0]] > 64) & (deg[e[:, 1]] > 64)]
    t = np.array([len(np.intersect1d(adj[off[a]:off[a + 1]], adj[off[b]:off[b + 1]])) for a, b in e])
    assert t.max() > 4096 and ((t > 512) & (t <= 4096)).sum() >= 2 and (t <= 512).any()


def test_relist24_knob_rejects_bad_values(nc):
    assert nc.lib().nh_set_peel_relist24(2) == 1
    assert nc.lib().nh_set_peel_relist24(1) == 0
    assert nc.lib().nh_set_peel_list_hash(3) == 1
    assert nc.lib().nh_set_peel_list_hash(-1) == 1
    assert nc.lib().nh_set_peel_list_hash(1) == 0
    assert nc.lib().nh_set_peel_list_hash(0) == 0  # back to the default
