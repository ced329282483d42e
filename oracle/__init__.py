"""Sequential CPU oracle for (r,s) nucleus decomposition -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline / reference leg of ``bench.py``
may import this package.  It shares no code with the CUDA library: the C file
``nucleus_oracle.c`` and the pure-Python brute force in ``brute.py`` are written from the paper
(Shi, Dhulipala, Shun, "Parallel Algorithms for Hierarchical Nucleus Decomposition") alone.

Parity status per function:
  * ``nucleus(..., hier='def')``  exact core numbers + definitional hierarchy -- pinned
    (brute force <= 12 vertices, networkx k-core / k-truss, K_n, planted cliques, hand-derived
    two-K4 example).
  * ``nucleus(..., hier='pair')`` literal pair rule of Alg. 1 / Alg. 3 -- pinned (brute force of
    the pair rule, hand-derived two-K4 example).
  * ``nucleus(..., hier='link_def' | 'link_pair')`` Alg. 3 + Alg. 5 run sequentially -- pinned
    (equal to the level hierarchies; §7.3 worked traces).
  * ``nucleus(..., approx_delta=d)`` Alg. 2 -- pinned by Thm. 2's bound, lower bound,
    special cases (K_n, huge delta, disjoint cliques) and a hand-worked example.
  * ``check_sample`` local certificate -- pinned by planting mistakes into oracle output.
  * ``certify`` local certificate over every r-clique and s-clique (certify.c), for full-size
    checks -- pinned against ``nucleus`` on random graphs (zero violations), against
    ``check_sample`` over all r-cliques, and by planting each kind of mistake.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from math import comb

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nucleus_oracle.c")
_SRC_CERT = os.path.join(_HERE, "certify.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

HIER_MODES = {None: 0, "def": 1, "pair": 2, "link_def": 3, "link_pair": 4}


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler into oracle/_build/liboracle.so."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    stale = not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(f) for f in (_SRC, _SRC_CERT))
    if force or stale:
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-pthread", "-shared", "-fPIC", "-o", tmp, _SRC, _SRC_CERT,
                               "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Result(ctypes.Structure):
    _fields_ = [
        ("r", ctypes.c_int32), ("s", ctypes.c_int32), ("C", ctypes.c_int32), ("status", ctypes.c_int32),
        ("n_r", ctypes.c_int64), ("n_s", ctypes.c_int64),
        ("tuples", ctypes.POINTER(ctypes.c_int32)),
        ("cnt", ctypes.POINTER(ctypes.c_uint32)),
        ("core", ctypes.POINTER(ctypes.c_uint32)),
        ("kmax", ctypes.c_uint32),
        ("n_nodes", ctypes.c_int64),
        ("leaf_node", ctypes.POINTER(ctypes.c_int32)),
        ("node_parent", ctypes.POINTER(ctypes.c_int32)),
        ("node_label", ctypes.POINTER(ctypes.c_uint32)),
        ("n_link_calls", ctypes.c_int64), ("n_unite_calls", ctypes.c_int64),
        ("approx", ctypes.POINTER(ctypes.c_uint32)),
        ("approx_rounds", ctypes.c_int64),
        ("approx_T", ctypes.c_uint32),
        ("n_thresholds", ctypes.c_int32),
        ("thresholds", ctypes.POINTER(ctypes.c_uint32)),
        ("removal", ctypes.POINTER(ctypes.c_uint32)),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.orc_nucleus.restype = ctypes.POINTER(_Result)
        lib.orc_nucleus.argtypes = [ctypes.c_int64, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_double]
        lib.orc_label_hierarchy.restype = ctypes.POINTER(_Result)
        lib.orc_label_hierarchy.argtypes = [ctypes.c_int64, P, P, ctypes.c_int, ctypes.c_int, P]
        lib.orc_tree_from_uf.restype = ctypes.POINTER(_Result)
        lib.orc_tree_from_uf.argtypes = [ctypes.c_int64, P, P, P]
        lib.orc_free.argtypes = [ctypes.POINTER(_Result)]
        lib.orc_count_cliques.restype = ctypes.c_int64
        lib.orc_count_cliques.argtypes = [ctypes.c_int64, P, P, ctypes.c_int]
        lib.orc_list_cliques.restype = ctypes.c_int64
        lib.orc_list_cliques.argtypes = [ctypes.c_int64, P, P, ctypes.c_int, P]
        lib.orc_link_apply.restype = ctypes.c_int
        lib.orc_link_apply.argtypes = [ctypes.c_int64, P, P, P, P, ctypes.c_int64]
        lib.orc_uf_find.restype = ctypes.c_int32
        lib.orc_uf_find.argtypes = [P, ctypes.c_int32]
        lib.orc_approx_thresholds.restype = ctypes.c_int
        lib.orc_approx_thresholds.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_uint32, P, ctypes.c_int]
        lib.orc_approx_round_cap.restype = ctypes.c_uint32
        lib.orc_approx_round_cap.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int64]
        lib.crt_certify.restype = ctypes.c_int
        lib.crt_certify.argtypes = [ctypes.c_int64, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int64, P, P, P, P, P,
                                    ctypes.c_int64, ctypes.c_int, P]
        lib.orc_check_sample.restype = ctypes.c_int
        lib.orc_check_sample.argtypes = [ctypes.c_int64, P, P, ctypes.c_int, ctypes.c_int, P, ctypes.c_int64,
                                         P, ctypes.c_int64, P, P, P, P, P, P]
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _csr(off, adj):
    off = np.ascontiguousarray(off, dtype=np.int64)
    adj = np.ascontiguousarray(adj, dtype=np.int32)
    return off, adj


def _copy(p, n, dtype):
    if n == 0 or not p:
        return np.zeros(0, dtype=dtype)
    return np.ctypeslib.as_array(p, shape=(n,)).astype(dtype, copy=True)


def list_cliques(off, adj, k: int) -> np.ndarray:
    """All k-cliques as an (n_k, k) int32 array of increasing vertex ids, lexicographic."""
    off, adj = _csr(off, adj)
    lib = _load()
    n = len(off) - 1
    cnt = lib.orc_count_cliques(n, _ptr(off), _ptr(adj), k)
    out = np.zeros((max(cnt, 1), k), dtype=np.int32)
    lib.orc_list_cliques(n, _ptr(off), _ptr(adj), k, _ptr(out))
    return out[:cnt]


def nucleus(off, adj, r: int, s: int, core: bool = True, hier: str | None = "def",
            approx_delta: float | None = None) -> dict:
    """Run the oracle.  Returns a dict with (as present):
    n_r, n_s, tuples (n_r, r), cnt, core, kmax, leaf_node, node_parent, node_label,
    n_link_calls, n_unite_calls, approx, approx_rounds, approx_T, thresholds, removal (1-based
    position of each r-clique in the exact peel's removal order)."""
    off, adj = _csr(off, adj)
    lib = _load()
    flags = (1 if core else 0) | (2 if approx_delta is not None else 0)
    p = lib.orc_nucleus(len(off) - 1, _ptr(off), _ptr(adj), r, s, flags, HIER_MODES[hier],
                        float(approx_delta or 0.0))
    if not p:
        raise MemoryError("oracle allocation failed")
    try:
        res = p.contents
        if res.status != 0:
            raise RuntimeError("oracle failed with status %d" % res.status)
        n_r = res.n_r
        out = {"n_r": n_r, "n_s": res.n_s, "C": res.C,
               "tuples": _copy(res.tuples, n_r * r, np.int32).reshape(n_r, r),
               "cnt": _copy(res.cnt, n_r, np.uint32)}
        if res.core:
            out["core"] = _copy(res.core, n_r, np.uint32)
            out["kmax"] = int(res.kmax)
        if res.removal:
            out["removal"] = _copy(res.removal, n_r, np.uint32)
        if hier is not None:
            nn = res.n_nodes
            out["n_nodes"] = nn
            out["leaf_node"] = _copy(res.leaf_node, n_r, np.int32)
            out["node_parent"] = _copy(res.node_parent, nn, np.int32)
            out["node_label"] = _copy(res.node_label, nn, np.uint32)
            out["n_link_calls"] = int(res.n_link_calls)
            out["n_unite_calls"] = int(res.n_unite_calls)
        if approx_delta is not None:
            out["approx"] = _copy(res.approx, n_r, np.uint32)
            out["approx_rounds"] = int(res.approx_rounds)
            out["approx_T"] = int(res.approx_T)
            out["thresholds"] = _copy(res.thresholds, res.n_thresholds, np.uint32)
        return out
    finally:
        lib.orc_free(p)


def label_hierarchy(off, adj, r: int, s: int, labels) -> dict:
    """Definitional hierarchy of arbitrary per-r-clique labels (lexicographic ids): leaf_node,
    node_parent, node_label, n_nodes (plus n_r, n_s, cnt)."""
    off, adj = _csr(off, adj)
    labels = np.ascontiguousarray(labels, dtype=np.uint32)
    lib = _load()
    n_r = lib.orc_count_cliques(len(off) - 1, _ptr(off), _ptr(adj), r)
    if len(labels) != n_r:
        raise ValueError("labels must have one entry per r-clique (%d), got %d" % (n_r, len(labels)))
    p = lib.orc_label_hierarchy(len(off) - 1, _ptr(off), _ptr(adj), r, s, _ptr(labels))
    if not p:
        raise MemoryError("oracle allocation failed")
    try:
        res = p.contents
        if res.status != 0:
            raise RuntimeError("oracle failed with status %d" % res.status)
        nn = res.n_nodes
        return {"n_r": res.n_r, "n_s": res.n_s, "cnt": _copy(res.cnt, res.n_r, np.uint32), "n_nodes": nn,
                "leaf_node": _copy(res.leaf_node, res.n_r, np.int32),
                "node_parent": _copy(res.node_parent, nn, np.int32),
                "node_label": _copy(res.node_label, nn, np.uint32)}
    finally:
        lib.orc_free(p)


def cut_hierarchy(leaf_node, node_parent, node_label, c: int) -> np.ndarray:
    """The c-(r,s) nuclei read off a hierarchy (§8, dense subgraphs): remove every node of label
    < c; each remaining subtree is one c-nucleus holding all its leaves.  Returns, per r-clique,
    the id of the top node of its c-nucleus, or -1 when its smallest node has label < c (core < c)
    or it has none."""
    leaf_node = np.asarray(leaf_node)
    node_parent = np.asarray(node_parent)
    node_label = np.asarray(node_label)
    top = {}

    def top_of(N):
        path = []
        while N not in top:
            path.append(N)
            P = int(node_parent[N])
            if P < 0 or node_label[P] < c:
                top[N] = N
                break
            N = P
        t = top[N]
        for x in path:
            top[x] = t
        return t

    out = np.full(len(leaf_node), -1, dtype=np.int64)
    for R, N in enumerate(leaf_node):
        N = int(N)
        if N >= 0 and node_label[N] >= c:
            out[R] = top_of(N)
    return out


def tree_from_uf(uf, L, core) -> dict:
    """construct-tree-efficient (Alg. 5) on given uf / L / core arrays."""
    lib = _load()
    uf = np.ascontiguousarray(uf, dtype=np.int32)
    L = np.ascontiguousarray(L, dtype=np.int32)
    core = np.ascontiguousarray(core, dtype=np.uint32)
    p = lib.orc_tree_from_uf(len(uf), _ptr(uf), _ptr(L), _ptr(core))
    try:
        res = p.contents
        if res.status != 0:
            raise RuntimeError("oracle failed with status %d" % res.status)
        nn = res.n_nodes
        return {"n_nodes": nn, "leaf_node": _copy(res.leaf_node, len(uf), np.int32),
                "node_parent": _copy(res.node_parent, nn, np.int32),
                "node_label": _copy(res.node_label, nn, np.uint32)}
    finally:
        lib.orc_free(p)


def link_apply(ND, uf, L, calls):
    """Apply link-efficient calls (list of (R, Q)) sequentially to uf / L (modified in place)."""
    lib = _load()
    ND = np.ascontiguousarray(ND, dtype=np.uint32)
    calls = np.ascontiguousarray(np.asarray(calls, dtype=np.int32).reshape(-1, 2))
    assert uf.dtype == np.int32 and L.dtype == np.int32 and uf.flags.c_contiguous and L.flags.c_contiguous
    rc = lib.orc_link_apply(len(ND), _ptr(ND), _ptr(uf), _ptr(L), _ptr(calls), len(calls))
    if rc != 0:
        raise RuntimeError("link_apply failed with status %d" % rc)


def uf_find(uf, x: int) -> int:
    return int(_load().orc_uf_find(_ptr(uf), int(x)))


def approx_thresholds(C: int, delta: float, max_cnt: int, cap: int = 1 << 16) -> np.ndarray:
    out = np.zeros(cap, dtype=np.uint32)
    k = _load().orc_approx_thresholds(C, float(delta), int(max_cnt), _ptr(out), cap)
    return out[:k]


def approx_round_cap(C: int, delta: float, n_r: int) -> int:
    return int(_load().orc_approx_round_cap(C, float(delta), int(n_r)))


def check_sample(off, adj, r: int, s: int, tuples, sample, cnt=None, core=None, rnd=None,
                 parent=None, label=None) -> np.ndarray:
    """Local certificate on sampled r-cliques (see orc_check_sample).  Returns the 4 counts of
    violations: [count, validity, peel-order bound, hierarchy connectivity]."""
    off, adj = _csr(off, adj)
    lib = _load()
    tuples = np.ascontiguousarray(tuples, dtype=np.int32)
    sample = np.ascontiguousarray(sample, dtype=np.int64)
    conv = lambda a, dt: None if a is None else np.ascontiguousarray(a, dtype=dt)
    cnt, core, rnd = conv(cnt, np.uint32), conv(core, np.uint32), conv(rnd, np.uint32)
    parent, label = conv(parent, np.int32), conv(label, np.uint32)
    bad = np.zeros(4, dtype=np.int64)
    rc = lib.orc_check_sample(len(off) - 1, _ptr(off), _ptr(adj), r, s, _ptr(tuples), len(tuples),
                              _ptr(sample), len(sample), _ptr(cnt), _ptr(core), _ptr(rnd),
                              _ptr(parent), _ptr(label), _ptr(bad))
    if rc != 0:
        raise RuntimeError("check_sample failed with status %d" % rc)
    return bad


def certify(off, adj, r: int, s: int, n_r: int, cnt=None, core=None, rnd=None, parent=None, label=None,
            n_nodes: int = 0, threads: int | None = None) -> dict:
    """Local certificate of a claimed exact decomposition over EVERY r-clique and s-clique
    (certify.c): count, validity and peel-order conditions (which prove the core numbers) and the
    hierarchy's under- and over-merge conditions (which prove it equals the definitional one).
    Returns the number of violations of each, whether the hierarchy was checked (trees up to
    16384 nodes with parents below their children's labels), and the s-cliques enumerated."""
    off, adj = _csr(off, adj)
    lib = _load()
    conv = lambda a, dt: None if a is None else np.ascontiguousarray(a, dtype=dt)
    cnt, core, rnd = conv(cnt, np.uint32), conv(core, np.uint32), conv(rnd, np.uint32)
    parent, label = conv(parent, np.int32), conv(label, np.uint32)
    out = np.zeros(8, dtype=np.int64)
    threads = threads or min(16, os.cpu_count() or 1)
    rc = lib.crt_certify(len(off) - 1, _ptr(off), _ptr(adj), r, s, int(n_r), _ptr(cnt), _ptr(core), _ptr(rnd),
                         _ptr(parent), _ptr(label), int(n_nodes), int(threads), _ptr(out))
    if rc != 0:
        raise RuntimeError("certify failed with status %d" % rc)
    return {"count": int(out[0]), "validity": int(out[1]), "peel_order": int(out[2]),
            "under_merge": int(out[3]), "over_merge": int(out[4]), "hierarchy_checked": bool(out[5]),
            "n_s": int(out[6]), "single_part_nodes": int(out[7])}


def binom(s: int, r: int) -> int:
    return comb(s, r)
