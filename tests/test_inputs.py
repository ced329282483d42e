"""The seeded input recipes (paper_2306_08623_gb300/graphgen.py) on the CPU: every generator
yields a valid undirected simple CSR graph, deterministically from its seed, with the sizes the
documentation states for the benchmark graph."""
import math

import numpy as np
import pytest

from paper_2306_08623_gb300 import graphgen as gg


def _valid_simple_csr(off, adj):
    off = np.asarray(off)
    adj = np.asarray(adj)
    n = len(off) - 1
    assert off[0] == 0 and off[-1] == len(adj) and np.all(np.diff(off) >= 0)
    src = np.repeat(np.arange(n), np.diff(off))
    assert np.all((adj >= 0) & (adj < n))
    assert not np.any(src == adj), "self-loop"
    for v in range(n):
        row = adj[off[v]:off[v + 1]]
        assert np.all(np.diff(row) > 0), "row not strictly increasing (unsorted or duplicate)"
    pairs = set(zip(src.tolist(), adj.tolist()))
    assert all((b, a) in pairs for a, b in pairs), "not symmetric"
    return n, len(adj) // 2


@pytest.mark.parametrize("make", [
    lambda: gg.rmat(10, 8, 1),
    lambda: gg.erdos_renyi(500, 2000, 3),
    lambda: gg.gnp(20, 0.3, 5),
    lambda: gg.chung_lu(3000, 2.1, 10, 5, groups=6, per_group=5, size_lo=6, size_hi=14),
    lambda: gg.batch_member(1002),
    lambda: gg.batch_member(1003),
    lambda: gg.batch_member(1004),
])
def test_generators_give_valid_simple_graphs_deterministically(make):
    off, adj = make()
    _valid_simple_csr(off, adj)
    off2, adj2 = make()
    assert np.array_equal(off, off2) and np.array_equal(adj, adj2)


def test_closed_form_sizes():
    assert _valid_simple_csr(*gg.complete(6)) == (6, 15)
    assert _valid_simple_csr(*gg.disjoint_cliques([3, 4, 5])) == (12, 3 + 6 + 10)
    assert _valid_simple_csr(*gg.erdos_renyi(2000, 16000, 1)) == (2000, 16000)
    assert _valid_simple_csr(*gg.from_edges(5, [])) == (5, 0)


def test_seeds_matter():
    a = gg.rmat(10, 8, 1)[1]
    b = gg.rmat(10, 8, 2)[1]
    assert len(a) != len(b) or not np.array_equal(a, b)


def test_batch_member_recipe_ranges():
    for seed in range(1000, 1012):
        off, adj = gg.batch_member(seed)
        n = len(off) - 1
        assert 1000 <= n <= 200000
        # mean degree drawn from U[8, 40]; de-duplication and dropped ids only lower it
        assert 0 < len(adj) / n <= 40.0 + 1e-9


def test_rmat18_benchmark_graph_sizes():
    """R-MAT scale 18, edge factor 16, seed 2: the benchmark graph's stated sizes."""
    off, adj = gg.rmat(18, 16, 2)
    assert len(off) - 1 == 262144
    assert len(adj) // 2 == 3806903
    assert int(np.diff(off).max()) == 25260
    assert math.isclose(len(adj) / 2 / (16 * 262144), 3806903 / 4194304)
