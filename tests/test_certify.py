"""Pins of the full-size local certificate (oracle.certify, oracle/certify.c) on the CPU.

The certificate is what the full-size GPU tests rest on for (2,4) and (3,4), where the sequential
oracle cannot run.  It must (a) report no violation on the oracle's own exact decomposition, with
the oracle's removal order as rounds, (b) agree with the per-r-clique checker check_sample on every
r-clique, and (c) detect every planted mistake: a wrong count, any single wrong core number
(certificate plus core non-decreasing in round order), a leaf moved to another node, a node
re-parented, two nodes merged.
"""
import numpy as np
import pytest

import oracle
from paper_2306_08623_gb300 import graphgen as gg

PAIRS = [(1, 2), (1, 3), (2, 3), (2, 4), (3, 4)]


def _run(off, adj, r, s):
    ref = oracle.nucleus(off, adj, r, s)
    parent = np.concatenate([ref["leaf_node"], ref["node_parent"]]).astype(np.int32)
    return ref, parent


def _cert(off, adj, r, s, ref, parent, cnt=None, core=None, rnd=None, label=None):
    return oracle.certify(off, adj, r, s, ref["n_r"], cnt=ref["cnt"] if cnt is None else cnt,
                          core=ref["core"] if core is None else core, rnd=ref["removal"] if rnd is None else rnd,
                          parent=parent, label=ref["node_label"] if label is None else label,
                          n_nodes=len(ref["node_parent"]), threads=3)


def _violations(c):
    return c["count"] + c["validity"] + c["peel_order"] + max(c["under_merge"], 0) + c["over_merge"]


def _monotone(core, rnd):
    order = np.argsort(rnd, kind="stable")
    return bool((np.diff(core[order].astype(np.int64)) >= 0).all())


GRAPHS = [gg.rmat(10, 8, 9), gg.chung_lu(1500, 2.1, 10, 3, groups=4, per_group=4, size_lo=6, size_hi=12),
          gg.complete(8), gg.disjoint_cliques([5, 6, 4]), gg.from_edges(6, [])]


@pytest.mark.parametrize("r,s", PAIRS)
def test_oracle_decomposition_has_no_violation(r, s):
    rng = np.random.default_rng(3 + r + s)
    graphs = GRAPHS + [gg.gnp(int(rng.integers(5, 14)), float(rng.uniform(0.4, 0.9)), int(rng.integers(1 << 30)))
                       for _ in range(10)]
    for off, adj in graphs:
        ref, parent = _run(off, adj, r, s)
        c = _cert(off, adj, r, s, ref, parent)
        assert _violations(c) == 0, c
        assert c["hierarchy_checked"] and c["n_s"] == ref["n_s"]
        assert _monotone(ref["core"], ref["removal"])


@pytest.mark.parametrize("r,s", PAIRS)
def test_agrees_with_check_sample_on_every_r_clique(r, s):
    """Counts, validity and peel-order violations equal those of check_sample over all r-cliques,
    also after planting mistakes in counts, cores and rounds."""
    off, adj = gg.rmat(9, 8, 4)
    ref, parent = _run(off, adj, r, s)
    rng = np.random.default_rng(11)
    n_r = ref["n_r"]
    for trial in range(4):
        cnt, core, rnd = ref["cnt"].copy(), ref["core"].copy(), ref["removal"].copy()
        k = max(1, n_r // 50)
        idx = rng.choice(n_r, size=k, replace=False)
        if trial == 1:
            cnt[idx] += 1
        if trial == 2:
            core[idx] = np.maximum(core[idx].astype(np.int64) + rng.choice([-1, 1], size=k), 0).astype(np.uint32)
        if trial == 3:
            rnd = rng.permutation(rnd).astype(np.uint32)
        c = oracle.certify(off, adj, r, s, n_r, cnt=cnt, core=core, rnd=rnd, threads=2)
        b = oracle.check_sample(off, adj, r, s, ref["tuples"], np.arange(n_r), cnt=cnt, core=core, rnd=rnd)
        assert [c["count"], c["validity"], c["peel_order"]] == b[:3].tolist(), (trial, c, b)
        if trial in (1, 2):
            assert c["count"] + c["validity"] + c["peel_order"] > 0 or not _monotone(core, rnd)


@pytest.mark.parametrize("r,s", PAIRS)
def test_every_wrong_core_number_is_detected(r, s):
    """A core number raised or lowered by one, anywhere, trips the certificate or the round-order
    monotonicity (together they prove the core numbers)."""
    off, adj = gg.rmat(9, 8, 5)
    ref, parent = _run(off, adj, r, s)
    rng = np.random.default_rng(17)
    n_r = ref["n_r"]
    for R in rng.choice(n_r, size=min(n_r, 40), replace=False):
        for d in (-1, 1):
            if ref["core"][R] == 0 and d < 0:
                continue
            core = ref["core"].copy()
            core[R] = core[R] + d if d > 0 else core[R] - 1
            c = oracle.certify(off, adj, r, s, n_r, cnt=ref["cnt"], core=core, rnd=ref["removal"], threads=2)
            assert c["validity"] + c["peel_order"] > 0 or not _monotone(core, ref["removal"]), (R, d)


def test_wrong_counts_are_detected():
    off, adj = gg.rmat(9, 8, 6)
    for r, s in PAIRS:
        ref, parent = _run(off, adj, r, s)
        cnt = ref["cnt"].copy()
        cnt[len(cnt) // 2] += 1
        assert _cert(off, adj, r, s, ref, parent, cnt=cnt)["count"] == 1


@pytest.mark.parametrize("r,s", [(1, 2), (2, 3), (2, 4), (3, 4)])
def test_planted_hierarchy_mistakes_are_detected(r, s):
    off, adj = gg.chung_lu(2500, 2.1, 12, 7, groups=6, per_group=5, size_lo=6, size_hi=14)
    ref, parent = _run(off, adj, r, s)
    n_r = ref["n_r"]
    nn = len(ref["node_parent"])
    lab = ref["node_label"]
    rng = np.random.default_rng(23)
    assert nn >= 4
    detected = 0
    trials = 0
    # a leaf moved to another node of its own level
    leaves = np.nonzero(parent[:n_r] >= 0)[0]
    for R in rng.choice(leaves, size=min(10, len(leaves)), replace=False):
        others = [x for x in range(nn) if lab[x] == lab[parent[R]] and x != parent[R]]
        if not others:
            continue
        p = parent.copy()
        p[R] = others[0]
        trials += 1
        detected += _violations(_cert(off, adj, r, s, ref, p)) > 0
    # a node re-parented to another node of lower label that is not its parent
    for Y in range(nn):
        cands = [x for x in range(nn) if lab[x] < lab[Y] and x != parent[n_r + Y]]
        if not cands:
            continue
        p = parent.copy()
        p[n_r + Y] = cands[0]
        trials += 1
        detected += _violations(_cert(off, adj, r, s, ref, p)) > 0
        if trials > 25:
            break
    # two nodes of one level merged (the second keeps no part)
    for lv in np.unique(lab):
        xs = np.nonzero(lab == lv)[0]
        if len(xs) < 2:
            continue
        A, B = int(xs[0]), int(xs[1])
        p = parent.copy()
        p[:n_r][p[:n_r] == B] = A
        kids = np.nonzero(p[n_r:] == B)[0]
        p[n_r + kids] = A
        trials += 1
        c = _cert(off, adj, r, s, ref, p)
        detected += _violations(c) > 0
        assert c["single_part_nodes"] >= 1
    assert trials >= 5 and detected == trials, (detected, trials)
