"""Parity at the benchmark's full size: R-MAT scale 18, edge factor 16, seed 2, in the launch
configuration bench.py times.

(1,2) and (2,3): element-wise against the oracle (counts, core numbers, hierarchy).
(2,4) and (3,4): the oracle cannot enumerate 2.3e9 4-cliques in test time, so sampled r-cliques
are checked one by one with the oracle's local certificate (count from the definition; at least
core[R] s-cliques inside the set of core >= core[R]; at most core[R] live s-cliques when peeled;
every sampled s-clique's members meet in one hierarchy node at level c_S), plus properties that
hold at any size.  Approximate core numbers: Thm. 2's bound for every r-clique.
"""
from math import comb

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from helpers import compare_hierarchy, u32  # noqa: E402
from paper_2306_08623_gb300 import graphgen as gg  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def graph():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return gg.rmat(18, 16, 2)


@pytest.fixture(scope="module")
def gpu(graph):
    import paper_2306_08623_gb300.nucleus as nc
    off, adj = graph
    d_off = torch.from_numpy(off).cuda()
    d_adj = torch.from_numpy(adj).cuda()
    o = nc.build_orientation(d_off, d_adj)
    ris = {r: nc.index_r_cliques(o, r) for r in (1, 2, 3)}
    return nc, o, ris


def run_pair(gpu, r, s, deltas=()):
    nc, o, ris = gpu
    ri = ris[r]
    cnt, n_s = nc.count_s_cliques(o, ri, s)
    pk = nc.peel_and_link(o, ri, s, cnt, stats=True)
    parent, label, nn = nc.construct_tree(pk["core"], pk["uf"], pk["L"])
    out = {"n_r": ri.n_r, "n_s": n_s, "cnt": u32(cnt), "core": u32(pk["core"]), "round": u32(pk["round"]),
           "parent": parent.cpu().numpy(), "label": u32(label), "n_nodes": nn, "stats": pk["stats"]}
    for d in deltas:
        out["approx_%g" % d] = u32(nc.approx_nucleus(o, ri, s, d, cnt)["approx"])
    return out


def global_properties(g, r, s):
    C = comb(s, r)
    assert int(g["cnt"].sum(dtype=np.int64)) == C * g["n_s"]
    assert (g["core"] <= g["cnt"]).all()
    order = np.argsort(g["round"], kind="stable")
    assert (np.diff(g["core"][order].astype(np.int64)) >= 0).all()
    n_r, nn = g["n_r"], g["n_nodes"]
    leaf = g["parent"][:n_r]
    npar = g["parent"][n_r:n_r + nn]
    lab = g["label"][:nn].astype(np.int64)
    has = leaf >= 0
    assert ((g["core"] > 0) == has).all()
    assert (lab[leaf[has]] == g["core"][has]).all()          # a leaf's node is its own level
    ok = npar >= 0
    assert (lab[npar[ok]] < lab[ok]).all()                    # parents sit at lower levels


@pytest.mark.parametrize("r,s", [(1, 2), (2, 3)])
def test_full_parity(graph, gpu, r, s):
    off, adj = graph
    g = run_pair(gpu, r, s)
    ref = oracle.nucleus(off, adj, r, s, hier="def")
    assert g["n_r"] == ref["n_r"] and g["n_s"] == ref["n_s"]
    assert np.array_equal(g["cnt"], ref["cnt"])
    assert np.array_equal(g["core"], ref["core"])
    compare_hierarchy(g["parent"], g["label"], g["n_nodes"], ref["leaf_node"], ref["node_parent"],
                      ref["node_label"])
    global_properties(g, r, s)


@pytest.mark.parametrize("r,s", [(2, 4), (3, 4)])
def test_sampled_certificate(graph, gpu, r, s):
    off, adj = graph
    nc, o, ris = gpu
    g = run_pair(gpu, r, s)
    global_properties(g, r, s)
    tuples = nc.rindex_tuples(ris[r]).cpu().numpy().reshape(-1, r)
    rng = np.random.default_rng(2024 + r)
    n_r = g["n_r"]
    top = np.argsort(g["core"])[-300:]                        # the densest part, where ties are
    sample = np.unique(np.concatenate([rng.choice(n_r, size=1500, replace=False), top]))
    # the checker's lookups need the lexicographic r-clique table: the oracle builds its own
    rtab = oracle.list_cliques(off, adj, r) if r < 3 else tuples_from_oracle(off, adj)
    assert np.array_equal(rtab, tuples)
    bad = oracle.check_sample(off, adj, r, s, rtab, sample, cnt=g["cnt"], core=g["core"], rnd=g["round"],
                              parent=g["parent"], label=g["label"])
    assert bad.tolist() == [0, 0, 0, 0], bad


def tuples_from_oracle(off, adj):
    return oracle.list_cliques(off, adj, 3)


@pytest.mark.parametrize("r,s", [(2, 3), (3, 4)])
def test_approx_bound_full_size(graph, gpu, r, s):
    g = run_pair(gpu, r, s, deltas=(0.1, 0.5))
    C = comb(s, r)
    core = g["core"].astype(np.float64)
    nz = core > 0
    for d in (0.1, 0.5):
        ap = g["approx_%g" % d].astype(np.float64)
        assert (ap[~nz] == 0).all()
        assert (ap[nz] >= core[nz]).all()
        assert (ap[nz] <= (C + d) * (1 + d) * core[nz] + 1e-9).all()
        assert (ap <= g["cnt"]).all()


@pytest.mark.parametrize("r,s", [(1, 2), (2, 3), (2, 4)])
def test_two_phase_full_size(graph, gpu, r, s):
    """The bench builds these pairs with the two-phase hierarchy (cores-only peel, then §7.4):
    at full size its core numbers and round stamps equal the linking peel's, and its hierarchy
    equals the linking peel's tree, which the tests above tie to the oracle."""
    nc, o, ris = gpu
    ri = ris[r]
    cnt, _ = nc.count_s_cliques(o, ri, s)
    el = nc.peel_and_link(o, ri, s, cnt)
    p_el, l_el, nn_el = nc.construct_tree(el["core"], el["uf"], el["L"])
    te = nc.peel_cores(o, ri, s, cnt)
    assert torch.equal(te["core"], el["core"]) and torch.equal(te["round"], el["round"])
    p_te, l_te, nn_te = nc.hierarchy_two_phase(o, ri, s, te["core"])
    n_r = ri.n_r
    p_el = p_el.cpu().numpy()
    compare_hierarchy(p_te.cpu().numpy(), u32(l_te), nn_te, p_el[:n_r], p_el[n_r:n_r + nn_el], u32(l_el))
