"""Hierarchy of arbitrary labels on the GPU (nh_label_hierarchy) against the oracle: the
approximate hierarchy (Alg. 2's values as labels), random labels (r-cliques alone at their own
level), and core numbers (the exact hierarchy)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from helpers import compare_hierarchy, u32  # noqa: E402
from paper_2306_08623_gb300 import graphgen as gg  # noqa: E402

pytestmark = pytest.mark.gpu
SUPPORTED = [(1, 2), (1, 3), (2, 3), (2, 4), (3, 4)]


@pytest.fixture(scope="module")
def nc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2306_08623_gb300.nucleus as mod
    mod.lib()
    return mod


def _gpu_vs_oracle(nc, off, adj, r, s, o, ri, labels_dev):
    parent, label, nn = nc.label_hierarchy(o, ri, s, labels_dev)
    ref = oracle.label_hierarchy(off, adj, r, s, u32(labels_dev))
    compare_hierarchy(parent.cpu().numpy(), u32(label), nn, ref["leaf_node"], ref["node_parent"],
                      ref["node_label"])
    return nn


@pytest.mark.parametrize("r,s", SUPPORTED)
def test_approximate_hierarchy(nc, r, s):
    graphs = [gg.rmat(11, 8, 3), gg.chung_lu(3000, 2.1, 10, 5, groups=6, per_group=5, size_lo=6, size_hi=14),
              gg.complete(7), gg.from_edges(5, [])]
    for off, adj in graphs:
        d_off, d_adj = torch.from_numpy(off).cuda(), torch.from_numpy(adj).cuda()
        o = nc.build_orientation(d_off, d_adj)
        ri = nc.index_r_cliques(o, r)
        cnt, _ = nc.count_s_cliques(o, ri, s)
        for delta in (0.1, 0.5):
            a = nc.approx_nucleus(o, ri, s, delta, cnt)
            _gpu_vs_oracle(nc, off, adj, r, s, o, ri, a["approx"])


@pytest.mark.parametrize("r,s", SUPPORTED)
def test_random_labels_and_cores(nc, r, s):
    rng = np.random.default_rng(7 + 10 * r + s)
    graphs = [gg.rmat(10, 8, 4), gg.erdos_renyi(800, 6000, 3)]
    for _ in range(6):
        graphs.append(gg.gnp(int(rng.integers(5, 14)), float(rng.uniform(0.4, 0.95)), int(rng.integers(1 << 30))))
    for off, adj in graphs:
        d_off, d_adj = torch.from_numpy(off).cuda(), torch.from_numpy(adj).cuda()
        o = nc.build_orientation(d_off, d_adj)
        ri = nc.index_r_cliques(o, r)
        if ri.n_r == 0:
            continue
        for hi in (3, 40):
            lab = torch.from_numpy(rng.integers(0, hi, size=ri.n_r).astype(np.int32)).cuda()
            _gpu_vs_oracle(nc, off, adj, r, s, o, ri, lab)
        cnt, _ = nc.count_s_cliques(o, ri, s)
        pk = nc.peel_cores(o, ri, s, cnt)
        ref = oracle.nucleus(off, adj, r, s)
        parent, label, nn = nc.label_hierarchy(o, ri, s, pk["core"])
        compare_hierarchy(parent.cpu().numpy(), u32(label), nn, ref["leaf_node"], ref["node_parent"],
                          ref["node_label"])


def test_label_bound_is_checked(nc):
    off, adj = gg.complete(5)
    o = nc.build_orientation(torch.from_numpy(off).cuda(), torch.from_numpy(adj).cuda())
    ri = nc.index_r_cliques(o, 2)
    lab = torch.full((ri.n_r,), (1 << 30) + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(nc.NucleusError) as e:
        nc.label_hierarchy(o, ri, 3, lab)
    assert e.value.status == 1
