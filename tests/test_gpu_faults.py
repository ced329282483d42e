"""Error paths under host-side fault injection (include/nucleus_debug.h): a grid-barrier wait
limit too short for any round makes the persistent kernels give up and report NH_ERR_TIMEOUT; a
hash table too small reports NH_ERR_TABLE_FULL.  Nothing here faults, traps or hangs the GPU:
every wait is bounded, and each case is followed by a normal run checked against the oracle
(the context stays usable)."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from helpers import compare_hierarchy, u32  # noqa: E402
from paper_2306_08623_gb300 import graphgen as gg  # noqa: E402

pytestmark = pytest.mark.gpu
NH_INJECT_WAIT_NS, NH_INJECT_TABLE_CAP, NH_INJECT_COUNT_BASE = 1, 2, 3
NH_ERR_TABLE_FULL, NH_ERR_TIMEOUT, NH_ERR_COUNT_OVERFLOW = 3, 5, 9


@pytest.fixture(scope="module")
def nc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2306_08623_gb300.nucleus as mod
    lib = mod.lib()
    lib.nh_debug_inject.argtypes = [ctypes.c_int, ctypes.c_int64]
    lib.nh_debug_inject.restype = ctypes.c_int
    yield mod
    lib.nh_debug_inject(NH_INJECT_WAIT_NS, 0)
    lib.nh_debug_inject(NH_INJECT_TABLE_CAP, 0)
    lib.nh_debug_inject(NH_INJECT_COUNT_BASE, 0)


def _inject(nc, what, value):
    assert nc.lib().nh_debug_inject(what, value) == 0


def _normal_run_matches_oracle(nc, off, adj, r, s):
    d_off, d_adj = torch.from_numpy(off).cuda(), torch.from_numpy(adj).cuda()
    res = nc.hierarchy(d_off, d_adj, r, s)
    ref = oracle.nucleus(off, adj, r, s)
    assert np.array_equal(u32(res["core"]), ref["core"])
    compare_hierarchy(res["parent"].cpu().numpy(), u32(res["label"]), res["n_nodes"], ref["leaf_node"],
                      ref["node_parent"], ref["node_label"])


def test_barrier_wait_limit_reports_timeout(nc):
    off, adj = gg.rmat(12, 16, 2)  # about 1000 rounds, several grid barriers each
    d_off, d_adj = torch.from_numpy(off).cuda(), torch.from_numpy(adj).cuda()
    o = nc.build_orientation(d_off, d_adj)
    ri = nc.index_r_cliques(o, 2)
    cnt, _ = nc.count_s_cliques(o, ri, 3)
    core = nc.peel_cores(o, ri, 3, cnt)["core"]  # before the injection: the two-phase input
    _inject(nc, NH_INJECT_WAIT_NS, 1)
    try:
        with pytest.raises(nc.NucleusError) as e:
            nc.peel_and_link(o, ri, 3, cnt)
        assert e.value.status == NH_ERR_TIMEOUT
        with pytest.raises(nc.NucleusError) as e:
            nc.approx_nucleus(o, ri, 3, 0.5, cnt)
        assert e.value.status == NH_ERR_TIMEOUT
        with pytest.raises(nc.NucleusError) as e:
            nc.hierarchy_two_phase(o, ri, 3, core)
        assert e.value.status == NH_ERR_TIMEOUT
    finally:
        _inject(nc, NH_INJECT_WAIT_NS, 0)
    torch.cuda.synchronize()
    _normal_run_matches_oracle(nc, off, adj, 2, 3)


def test_small_tables_report_table_full(nc):
    off, adj = gg.rmat(10, 8, 4)
    d_off, d_adj = torch.from_numpy(off).cuda(), torch.from_numpy(adj).cuda()
    _inject(nc, NH_INJECT_TABLE_CAP, 16)
    try:
        with pytest.raises(nc.NucleusError) as e:
            nc.build_orientation(d_off, d_adj)  # edge table
        assert e.value.status == NH_ERR_TABLE_FULL
    finally:
        _inject(nc, NH_INJECT_TABLE_CAP, 0)
    o = nc.build_orientation(d_off, d_adj)
    _inject(nc, NH_INJECT_TABLE_CAP, 16)
    try:
        with pytest.raises(nc.NucleusError) as e:
            nc.index_r_cliques(o, 3)  # triangle table
        assert e.value.status == NH_ERR_TABLE_FULL
    finally:
        _inject(nc, NH_INJECT_TABLE_CAP, 0)
    _normal_run_matches_oracle(nc, off, adj, 3, 4)


@pytest.mark.parametrize("r,s", [(1, 3), (2, 3), (2, 4), (3, 4)])
def test_count_overflow_is_reported(nc, r, s):
    """Every r-clique of K_7 lies in C(7-r, s-r) >= 3 s-cliques: counts that start at 2^32 - 3
    wrap and counting reports NH_ERR_COUNT_OVERFLOW; started at 2^32 - 100 they end at the
    start plus the s-clique-degree, with no error."""
    from math import comb
    off, adj = gg.complete(7)
    d_off, d_adj = torch.from_numpy(off).cuda(), torch.from_numpy(adj).cuda()
    o = nc.build_orientation(d_off, d_adj)
    ri = nc.index_r_cliques(o, r)
    try:
        _inject(nc, NH_INJECT_COUNT_BASE, (1 << 32) - 3)
        with pytest.raises(nc.NucleusError) as e:
            nc.count_s_cliques(o, ri, s)
        assert e.value.status == NH_ERR_COUNT_OVERFLOW
        _inject(nc, NH_INJECT_COUNT_BASE, (1 << 32) - 100)
        cnt, n_s = nc.count_s_cliques(o, ri, s)
        assert n_s == comb(7, s)
        assert (u32(cnt).astype(np.int64) == (1 << 32) - 100 + comb(7 - r, s - r)).all()
    finally:
        _inject(nc, NH_INJECT_COUNT_BASE, 0)
    _normal_run_matches_oracle(nc, off, adj, r, s)
