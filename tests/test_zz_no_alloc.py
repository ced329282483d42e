"""nh_construct_tree_noalloc: the tree construction for callers that cannot allocate device
memory while they run (a process whose device memory is owned by its own pooling allocator, or a
latency-bound caller that cannot afford the synchronisation cudaMalloc / cudaFree may cause).
Its working memory is a fixed device array shared by all calls.

Checked through the C-ABI against the allocating nh_construct_tree on two calls in a row with
different inputs (so leftovers of the first call in the shared array would show), and for the
size limit.  Kept in a file that pytest collects last.
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


def _peeled(nc, off, adj, r, s):
    o = nc.build_orientation(torch.from_numpy(off).cuda(), torch.from_numpy(adj).cuda())
    ri = nc.index_r_cliques(o, r)
    cnt, _ = nc.count_s_cliques(o, ri, s)
    pk = nc.peel_and_link(o, ri, s, cnt)
    return pk["core"], pk["uf"], pk["L"]


def test_noalloc_tree_matches_allocating_tree_twice(nc):
    cases = [(gg.rmat(12, 8, 3), 2, 3), (gg.rmat(11, 16, 4), 1, 2)]
    for (off, adj), r, s in cases:  # two calls in a row, different inputs
        core, uf, L = _peeled(nc, off, adj, r, s)
        n_r = core.numel()
        assert 0 < n_r <= nc.TREE_NOALLOC_MAX
        p_ref, l_ref, nn_ref = nc.construct_tree(core, uf.clone(), L)
        parent = torch.full((2 * n_r,), -7, dtype=torch.int32, device="cuda")
        label = torch.full((n_r,), -7, dtype=torch.int32, device="cuda")
        p, lab, nn = nc.construct_tree_noalloc(core, uf.clone(), L, parent, label)
        assert nn == nn_ref and nn > 0
        assert np.array_equal(p.cpu().numpy(), p_ref.cpu().numpy())
        assert np.array_equal(u32(lab), u32(l_ref))


def test_noalloc_tree_rejects_sizes_beyond_its_array(nc):
    n_r = nc.TREE_NOALLOC_MAX + 1
    core = torch.zeros(n_r, dtype=torch.int32, device="cuda")
    uf = torch.arange(n_r, dtype=torch.int32, device="cuda")
    L = torch.full((n_r,), -1, dtype=torch.int32, device="cuda")
    parent = torch.empty(2 * n_r, dtype=torch.int32, device="cuda")
    label = torch.empty(n_r, dtype=torch.int32, device="cuda")
    with pytest.raises(nc.NucleusError) as e:
        nc.construct_tree_noalloc(core, uf, L, parent, label)
    assert e.value.status == 1
