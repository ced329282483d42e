"""c-(r,s) nuclei on the GPU (nh_cut_hierarchy): cutting the GPU's hierarchy at level c gives the
same partition of the r-cliques of core >= c as cutting the oracle's hierarchy, for every level."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2306_08623_gb300 import graphgen as gg  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2306_08623_gb300.nucleus as mod
    mod.lib()
    return mod


def same_partition(a, b) -> bool:
    """a, b: per-element group ids (-1 = in no group); equal up to renaming the groups"""
    a = np.asarray(a, dtype=np.int64)
    b = np.asarray(b, dtype=np.int64)
    if not np.array_equal(a < 0, b < 0):
        return False
    m = a >= 0
    pairs = np.unique(np.stack([a[m], b[m]], axis=1), axis=0)
    return len(pairs) == len(np.unique(a[m])) == len(np.unique(b[m]))


@pytest.mark.parametrize("r,s,method", [(1, 2, "te"), (2, 3, "el"), (2, 3, "te"), (2, 4, "te"), (3, 4, "el")])
def test_cut_matches_oracle_every_level(nc, r, s, method):
    for off, adj in [gg.rmat(10, 8, 21), gg.chung_lu(3000, 2.1, 10, 22, groups=4, per_group=3)]:
        ref = oracle.nucleus(off, adj, r, s)
        res = nc.hierarchy(torch.from_numpy(off).cuda(), torch.from_numpy(adj).cuda(), r, s, method=method)
        n_r, nn = res["n_r"], res["n_nodes"]
        assert n_r == ref["n_r"]
        kmax = int(ref["core"].max()) if n_r else 0
        levels = sorted(set(range(0, min(kmax, 40) + 2)) | set(np.unique(ref["node_label"]).tolist()))
        for c in levels:
            want = oracle.cut_hierarchy(ref["leaf_node"], ref["node_parent"], ref["node_label"], c)
            got, n_nuc = nc.cut_hierarchy(res["parent"], res["label"], n_r, nn, c)
            got = got.cpu().numpy()
            assert same_partition(got, want), "level %d" % c
            assert n_nuc == len(np.unique(want[want >= 0])), "level %d" % c


def test_cut_edge_cases(nc):
    # no nodes: every r-clique is outside every nucleus at any level
    parent = torch.full((4,), -1, dtype=torch.int32, device="cuda")
    label = torch.zeros(1, dtype=torch.int32, device="cuda")
    got, n = nc.cut_hierarchy(parent, label, 4, 0, 1)
    assert n == 0 and (got.cpu().numpy() == -1).all()
    # a chain of three nodes (levels 3 > 2 > 1) over leaves 0..3
    # leaf 0, 1 -> node 0 (level 3); leaf 2 -> node 1 (level 2); leaf 3 -> node 2 (level 1)
    par = torch.tensor([0, 0, 1, 2, 1, 2, -1], dtype=torch.int32, device="cuda")
    lab = torch.tensor([3, 2, 1], dtype=torch.int32, device="cuda")
    for c, want in [(1, [2, 2, 2, 2]), (2, [1, 1, 1, -1]), (3, [0, 0, -1, -1]), (4, [-1] * 4), (0, [2, 2, 2, 2])]:
        got, n = nc.cut_hierarchy(par, lab, 4, 3, c)
        assert got.cpu().numpy().tolist() == want, c
        assert n == (1 if c <= 3 else 0)
