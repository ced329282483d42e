"""Parity at the benchmark's full size: R-MAT scale 18, edge factor 16, seed 2, in the launch
configuration bench.py times.

(1,2) and (2,3): element-wise against the oracle (counts, core numbers, hierarchy) for both
hierarchy builders, and the approximate (2,3) values bit-exact against the oracle for delta 0.1
and 0.5.  The oracle runs in spawned host processes started with the module, beside the GPU work.
(2,4) and (3,4): the oracle cannot enumerate 2.3e9 4-cliques in test time; every r-clique and
every s-clique is checked with the oracle's full local certificate (oracle.certify: counts,
validity and peel order, which prove the core numbers; under- and over-merge, which prove the
hierarchy), for the hierarchy builders the benchmark uses ((2,4) two-phase, (3,4) linking peel)
and the other one for (3,4); plus properties that hold at any size.  Approximate (3,4) values:
Thm. 2's bound for every r-clique.
"""
import multiprocessing as mp
import os
from math import comb

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from helpers import compare_hierarchy, u32  # noqa: E402
from paper_2306_08623_gb300 import graphgen as gg  # noqa: E402

pytestmark = pytest.mark.gpu


def _oracle_job(job):
    """(kind, r, s, delta) -> the oracle's result on R-MAT 18 EF16 seed 2 (runs in a spawned process)."""
    import oracle as orc
    from paper_2306_08623_gb300 import graphgen as g
    kind, r, s, delta = job
    off, adj = g.rmat(18, 16, 2)
    if kind == "exact":
        return orc.nucleus(off, adj, r, s, hier="def")
    res = orc.nucleus(off, adj, r, s, hier=None, approx_delta=delta)
    return {"approx": res["approx"], "approx_rounds": res["approx_rounds"]}


JOBS = [("exact", 1, 2, None), ("exact", 2, 3, None), ("approx", 2, 3, 0.1), ("approx", 2, 3, 0.5)]


@pytest.fixture(scope="module")
def oracle_results():
    """The oracle's full-size results, computed in parallel host processes; a dict of futures."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    oracle.build()
    pool = mp.get_context("spawn").Pool(processes=len(JOBS))
    futures = {job: pool.apply_async(_oracle_job, (job,)) for job in JOBS}
    yield futures
    pool.terminate()
    pool.join()


@pytest.fixture(scope="module")
def graph():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return gg.rmat(18, 16, 2)


@pytest.fixture(scope="module")
def gpu(graph, oracle_results):
    import paper_2306_08623_gb300.nucleus as nc
    off, adj = graph
    d_off = torch.from_numpy(off).cuda()
    d_adj = torch.from_numpy(adj).cuda()
    o = nc.build_orientation(d_off, d_adj)
    ris = {r: nc.index_r_cliques(o, r) for r in (1, 2, 3)}
    return nc, o, ris


def run_pair(gpu, r, s, method, deltas=()):
    nc, o, ris = gpu
    ri = ris[r]
    cnt, n_s = nc.count_s_cliques(o, ri, s)
    if method == "el":
        pk = nc.peel_and_link(o, ri, s, cnt, stats=True)
        parent, label, nn = nc.construct_tree(pk["core"], pk["uf"], pk["L"])
    else:
        pk = nc.peel_cores(o, ri, s, cnt, stats=True)
        parent, label, nn = nc.hierarchy_two_phase(o, ri, s, pk["core"])
    out = {"n_r": ri.n_r, "n_s": n_s, "cnt": u32(cnt), "core": u32(pk["core"]), "round": u32(pk["round"]),
           "parent": parent.cpu().numpy(), "label": u32(label), "n_nodes": nn, "stats": pk["stats"]}
    for d in deltas:
        a = nc.approx_nucleus(o, ri, s, d, cnt, stats=True)
        out["approx_%g" % d] = u32(a["approx"])
        out["approx_rounds_%g" % d] = a["stats"]["rounds"]
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
def test_full_parity(graph, gpu, oracle_results, r, s):
    off, adj = graph
    ref = oracle_results[("exact", r, s, None)].get(timeout=1800)
    for method in ("te", "el"):
        g = run_pair(gpu, r, s, method)
        assert g["n_r"] == ref["n_r"] and g["n_s"] == ref["n_s"]
        assert np.array_equal(g["cnt"], ref["cnt"])
        assert np.array_equal(g["core"], ref["core"])
        compare_hierarchy(g["parent"], g["label"], g["n_nodes"], ref["leaf_node"], ref["node_parent"],
                          ref["node_label"])
        global_properties(g, r, s)


def test_approx_23_bit_exact_full_size(gpu, oracle_results):
    """Alg. 2 on the benchmark graph's (2,3): values and round counts equal the oracle's."""
    g = run_pair(gpu, 2, 3, "te", deltas=(0.1, 0.5))
    for d in (0.1, 0.5):
        ra = oracle_results[("approx", 2, 3, d)].get(timeout=1800)
        assert np.array_equal(g["approx_%g" % d], ra["approx"]), d
        assert g["approx_rounds_%g" % d] == ra["approx_rounds"]


def _tuples_match(nc, ris, r, off, adj):
    """the lexicographic r-clique order the certificate assumes is the GPU's"""
    got = nc.rindex_tuples(ris[r]).cpu().numpy().reshape(-1, r)
    if r == 2:
        assert np.array_equal(got, gg.edge_list(off, adj).astype(np.int32))
    else:
        assert (np.diff(got, axis=1) > 0).all()
        key = (got[:, 0].astype(np.int64) << 36) | (got[:, 1].astype(np.int64) << 18) | got[:, 2]
        assert (np.diff(key) > 0).all()


@pytest.mark.parametrize("r,s,method", [(2, 4, "te"), (3, 4, "el"), (3, 4, "te")])
def test_certified_on_every_r_clique(graph, gpu, r, s, method):
    """Every r-clique and every s-clique of the full-size (2,4) / (3,4) decomposition satisfies
    the local certificate: the core numbers are exact and the hierarchy is the definitional one."""
    off, adj = graph
    nc, o, ris = gpu
    g = run_pair(gpu, r, s, method)
    global_properties(g, r, s)
    _tuples_match(nc, ris, r, off, adj)
    cert = oracle.certify(off, adj, r, s, g["n_r"], cnt=g["cnt"], core=g["core"], rnd=g["round"],
                          parent=g["parent"][: g["n_r"] + g["n_nodes"]], label=g["label"][: g["n_nodes"]],
                          n_nodes=g["n_nodes"], threads=min(16, os.cpu_count() or 1))
    assert cert["hierarchy_checked"]
    assert cert["n_s"] == g["n_s"]
    bad = {k: cert[k] for k in ("count", "validity", "peel_order", "under_merge", "over_merge")}
    assert all(v == 0 for v in bad.values()), bad


def test_approx_bound_full_size_34(gpu):
    g = run_pair(gpu, 3, 4, "te", deltas=(0.1, 0.5))
    C = comb(4, 3)
    core = g["core"].astype(np.float64)
    nz = core > 0
    for d in (0.1, 0.5):
        ap = g["approx_%g" % d].astype(np.float64)
        assert (ap[~nz] == 0).all()
        assert (ap[nz] >= core[nz]).all()
        assert (ap[nz] <= (C + d) * (1 + d) * core[nz] + 1e-9).all()
        assert (ap <= g["cnt"]).all()
