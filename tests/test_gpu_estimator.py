"""The learned work estimator (MLP) and the cost-balanced partition of the listing work.

Counting with any partition must give exactly the plain counts; the MLP inference kernel is
checked against a plain PyTorch fp32 evaluation of the same bf16 weights; training must lower
the loss.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from helpers import u32  # noqa: E402
from paper_2306_08623_gb300 import graphgen as gg  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2306_08623_gb300.nucleus as mod
    mod.lib()
    return mod


def _graph(nc, off, adj):
    o = nc.build_orientation(torch.from_numpy(off).cuda(), torch.from_numpy(adj).cuda())
    return o, {r: nc.index_r_cliques(o, r) for r in (1, 2, 3)}


def reference_mlp(feats, w16):
    """plain fp32 evaluation of the bf16 weights (torch CPU)"""
    w = w16.cpu().view(torch.bfloat16).float()
    F, H = 8, 64
    o = 0
    W1 = w[o:o + H * F].view(H, F); o += H * F
    b1 = w[o:o + H]; o += H
    W2 = w[o:o + H * H].view(H, H); o += H * H
    b2 = w[o:o + H]; o += H
    W3 = w[o:o + H]; o += H
    b3 = w[o]
    x = feats.cpu()
    h1 = torch.relu(x @ W1.T + b1)
    h2 = torch.relu(h1 @ W2.T + b2)
    return h2 @ W3 + b3


def test_partitioned_count_is_exact(nc):
    for off, adj in [gg.rmat(12, 8, 1), gg.chung_lu(20000, 2.1, 12, 3, groups=5, per_group=5),
                     gg.erdos_renyi(3000, 20000, 2)]:
        o, ris = _graph(nc, off, adj)
        for r, s in [(1, 3), (2, 3), (2, 4), (3, 4)]:
            cnt0, ns0 = nc.count_s_cliques(o, ris[r], s)
            want = u32(cnt0).copy()
            for cost in (nc.degree_cost(o, s), nc.listing_cost(o, ris[r], s),
                         torch.rand(o.n, device="cuda") * 100):
                cnt, ns = nc.count_s_cliques_partitioned(o, ris[r], s, cost)
                assert ns == ns0 and np.array_equal(u32(cnt), want)


def test_mlp_inference_matches_fp32_reference(nc):
    off, adj = gg.rmat(12, 8, 5)
    o, ris = _graph(nc, off, adj)
    feats = nc.vertex_features(o)
    cost = nc.listing_cost(o, ris[2], 3)
    w, loss = nc.mlp_train(feats, cost, n_train=4096, steps=50, lr=1e-2, seed=3)
    pred = nc.mlp_predict(feats, w).cpu()
    ref = reference_mlp(feats, w).clamp(0.0, 30.0)
    assert torch.allclose(torch.log1p(pred), ref, atol=2e-3, rtol=1e-3)


def test_mlp_training_lowers_loss(nc):
    off, adj = gg.chung_lu(50000, 2.1, 16, 7, groups=20, per_group=5)
    o, ris = _graph(nc, off, adj)
    feats = nc.vertex_features(o)
    cost = nc.listing_cost(o, ris[2], 3)
    assert float(cost.min()) >= 0.0 and float(cost.max()) > 0.0
    _, l1 = nc.mlp_train(feats, cost, n_train=8192, steps=1, lr=1e-2, seed=1)
    _, l2 = nc.mlp_train(feats, cost, n_train=8192, steps=300, lr=1e-2, seed=1)
    assert np.isfinite(l2) and l2 < 0.5 * l1
