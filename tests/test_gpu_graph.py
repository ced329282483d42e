"""Stream-ordered hierarchy (nh_hierarchy_enqueue): eager, and captured into a CUDA graph and
replayed, against the oracle."""
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


def _check(buf, ri, ref, n_s):
    res = buf["res"].cpu().numpy()
    n_r = ri.n_r
    assert res[0] == 0, res
    assert res[1] == n_s
    assert np.array_equal(u32(buf["cnt"][:n_r]), ref["cnt"])
    assert np.array_equal(u32(buf["core"][:n_r]), ref["core"])
    nn = int(res[2])
    compare_hierarchy(buf["parent"][: n_r + nn].cpu().numpy(), u32(buf["label"][:nn]), nn, ref["leaf_node"],
                      ref["node_parent"], ref["node_label"])


@pytest.mark.parametrize("r,s", SUPPORTED)
def test_enqueue_eager(nc, r, s):
    for off, adj in [gg.rmat(11, 8, 3), gg.complete(6), gg.erdos_renyi(500, 3000, 2)]:
        d_off, d_adj = torch.from_numpy(off).cuda(), torch.from_numpy(adj).cuda()
        o = nc.build_orientation(d_off, d_adj)
        ri = nc.index_r_cliques(o, r)
        buf = nc.hierarchy_buffers(ri)
        nc.hierarchy_enqueue(o, ri, s, buf)
        torch.cuda.synchronize()
        ref = oracle.nucleus(off, adj, r, s)
        _check(buf, ri, ref, ref["n_s"])


@pytest.mark.parametrize("r,s", [(2, 3), (2, 4), (3, 4)])
def test_enqueue_captured_and_replayed(nc, r, s):
    off, adj = gg.rmat(12, 16, 5)
    d_off, d_adj = torch.from_numpy(off).cuda(), torch.from_numpy(adj).cuda()
    o = nc.build_orientation(d_off, d_adj)
    ri = nc.index_r_cliques(o, r)
    buf = nc.hierarchy_buffers(ri)
    ref = oracle.nucleus(off, adj, r, s)
    nc.hierarchy_enqueue(o, ri, s, buf)  # warm-up outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    with torch.cuda.graph(g, stream=side, capture_error_mode="relaxed"):
        nc.hierarchy_enqueue(o, ri, s, buf)
    for _ in range(2):
        for t in buf.values():
            t.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        _check(buf, ri, ref, ref["n_s"])
