"""Thin Python binding of libnucleus (argument marshalling only; every step runs in the CUDA
library).  Device buffers are torch tensors; 32-bit unsigned outputs are returned in int32
tensors holding the same bit patterns (view them as uint32 on the host).

The binding fails loudly when the library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnucleus.so")

SPECIALISED = ((1, 2), (1, 3), (2, 3), (2, 4), (3, 4))  # persistent-peel pairs
SUPPORTED = tuple((r, s) for s in range(2, 8) for r in range(1, s))  # every r < s <= 7
LINK_MODES = {"def": 0, "pair": 1, "none": 2}


class NucleusError(RuntimeError):
    def __init__(self, where: str, status: int, text: str):
        super().__init__("%s failed: %s (status %d)" % (where, text, status))
        self.status = status


class PeelStats(ctypes.Structure):
    _fields_ = [
        ("rounds", ctypes.c_uint64), ("levels", ctypes.c_uint64), ("kmax", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32), ("s_cliques_listed", ctypes.c_uint64), ("decrements", ctypes.c_uint64),
        ("link_calls", ctypes.c_uint64), ("unites", ctypes.c_uint64), ("scan_elements", ctypes.c_uint64),
        ("hash_probes", ctypes.c_uint64), ("frontier_total", ctypes.c_uint64), ("overflow_links", ctypes.c_uint64),
        ("stamp_reads", ctypes.c_uint64),
    ]

    def as_dict(self) -> dict:
        return {name: int(getattr(self, name)) for name, _ in self._fields_ if name != "reserved"}


_lib = None
P = ctypes.c_void_p
I64 = ctypes.c_int64
I32 = ctypes.c_int


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libnucleus.so is not built (run __graft_entry__.build()); no CPU fallback exists")
        L = ctypes.CDLL(LIB_PATH)
        sig = {
            "nh_build_orientation": (I32, [I64, I64, P, P, ctypes.POINTER(P), P]),
            "nh_oriented_info": (I32, [P, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64),
                                       ctypes.POINTER(I64)]),
            "nh_oriented_free": (None, [P]),
            "nh_index_r_cliques": (I32, [P, I32, ctypes.POINTER(P), ctypes.POINTER(I64), P]),
            "nh_rindex_tuples": (I32, [P, P, P]),
            "nh_rindex_free": (None, [P]),
            "nh_count_s_cliques": (I32, [P, P, I32, P, ctypes.POINTER(ctypes.c_uint64), P]),
            "nh_peel_and_link": (I32, [P, P, I32, P, P, P, P, P, I32, ctypes.POINTER(PeelStats), P]),
            "nh_construct_tree": (I32, [I64, P, P, P, P, P, ctypes.POINTER(I64), P]),
            "nh_construct_tree_noalloc": (I32, [I64, P, P, P, P, P, ctypes.POINTER(I64), P]),
            "nh_hierarchy_two_phase": (I32, [P, P, I32, P, P, P, ctypes.POINTER(I64), P]),
            "nh_hierarchy_enqueue": (I32, [P, P, I32, P, P, P, P, P, P, P, P, P]),
            "nh_label_hierarchy": (I32, [P, P, I32, P, P, P, ctypes.POINTER(I64), P]),
            "nh_set_peel_max_group": (I32, [I32]),
            "nh_set_peel_task_items": (I32, [I32]),
            "nh_set_peel_relist24": (I32, [I32]),
            "nh_set_peel_list_hash": (I32, [I32]),
            "nh_set_relist_split": (I32, [ctypes.c_float, I32, I32, I32]),
            "nh_debug_round_log": (I32, [P, I64]),
            "nh_approx_nucleus": (I32, [P, P, I32, ctypes.c_double, P, P, P, ctypes.POINTER(PeelStats), P]),
            "nh_link_pairs": (I32, [I64, P, P, P, P, I64, P]),
            "nh_status_string": (ctypes.c_char_p, [I32]),
            "nh_version": (I32, []),
            "nh_kernel_launches": (I64, []),
            "nh_vertex_features": (I32, [P, P, P]),
            "nh_batch_union": (I32, [P, I32, P, P, P, P]),
            "nh_rindex_bases": (I32, [P, P, I32, P, P]),
            "nh_batch_prepare": (I32, [P, I32, I32, ctypes.POINTER(P), ctypes.POINTER(I64), P]),
            "nh_batch_bases": (I32, [P, P, P]),
            "nh_batch_run": (I32, [P, I32, P, P, P, P, P, P, P, P, P]),
            "nh_batch_node_bases": (I32, [P, P, I64, P, P]),
            "nh_batch_free": (None, [P]),
            "nh_cut_hierarchy": (I32, [I64, I64, P, P, ctypes.c_uint32, P, ctypes.POINTER(I64), P]),
            "nh_hierarchy_basic": (I32, [P, P, I32, P, P, P, ctypes.POINTER(I64), ctypes.POINTER(ctypes.c_uint64), P]),
            "nh_listing_cost": (I32, [P, P, I32, P, P]),
            "nh_degree_cost": (I32, [P, I32, P, P]),
            "nh_mlp_train": (I32, [P, P, I64, I64, I32, ctypes.c_float, ctypes.c_uint64, P,
                                   ctypes.POINTER(ctypes.c_float), P]),
            "nh_mlp_predict": (I32, [P, I64, P, P, P]),
            "nh_count_s_cliques_partitioned": (I32, [P, P, I32, P, P, ctypes.POINTER(ctypes.c_uint64), P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(where: str, rc: int):
    if rc != 0:
        raise NucleusError(where, rc, lib().nh_status_string(rc).decode())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return P(s.cuda_stream)


def _dptr(t: torch.Tensor | None):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "device tensors must be contiguous CUDA tensors"
    return P(t.data_ptr())


class Oriented:
    """Degree orientation of a CSR graph held on the device (keeps the CSR tensors alive)."""

    def __init__(self, handle, off, adj):
        self.handle = handle
        self.off, self.adj = off, adj
        n, m, mo, md = I64(), I64(), I64(), I64()
        _check("nh_oriented_info", lib().nh_oriented_info(handle, ctypes.byref(n), ctypes.byref(m),
                                                          ctypes.byref(mo), ctypes.byref(md)))
        self.n, self.m, self.max_out, self.max_deg = n.value, m.value, mo.value, md.value

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.nh_oriented_free(self.handle)
            self.handle = None


class RIndex:
    def __init__(self, handle, oriented: Oriented, r: int, n_r: int):
        self.handle, self.oriented, self.r, self.n_r = handle, oriented, r, n_r

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.nh_rindex_free(self.handle)
            self.handle = None


def build_orientation(off: torch.Tensor, adj: torch.Tensor, stream=None) -> Oriented:
    assert off.dtype == torch.int64 and adj.dtype == torch.int32
    h = P()
    n = off.numel() - 1
    _check("nh_build_orientation", lib().nh_build_orientation(n, adj.numel(), _dptr(off), _dptr(adj),
                                                              ctypes.byref(h), _stream(stream)))
    return Oriented(h, off, adj)


def index_r_cliques(o: Oriented, r: int, stream=None) -> RIndex:
    h = P()
    n_r = I64()
    _check("nh_index_r_cliques", lib().nh_index_r_cliques(o.handle, r, ctypes.byref(h), ctypes.byref(n_r),
                                                          _stream(stream)))
    return RIndex(h, o, r, n_r.value)


def rindex_tuples(ri: RIndex, stream=None) -> torch.Tensor:
    out = torch.empty((max(ri.n_r, 1), ri.r), dtype=torch.int32, device="cuda")
    _check("nh_rindex_tuples", lib().nh_rindex_tuples(ri.handle, _dptr(out), _stream(stream)))
    return out[: ri.n_r]


def count_s_cliques(o: Oriented, ri: RIndex, s: int, cnt: torch.Tensor | None = None, stream=None):
    if cnt is None:
        cnt = torch.empty(max(ri.n_r, 1), dtype=torch.int32, device="cuda")
    n_s = ctypes.c_uint64()
    _check("nh_count_s_cliques", lib().nh_count_s_cliques(o.handle, ri.handle, s, _dptr(cnt), ctypes.byref(n_s),
                                                          _stream(stream)))
    return cnt[: ri.n_r], int(n_s.value)


def peel_and_link(o: Oriented, ri: RIndex, s: int, cnt: torch.Tensor, link_mode: str = "def",
                  stats: bool = False, out: dict | None = None, stream=None) -> dict:
    n = max(ri.n_r, 1)
    out = out or {}
    for key in ("core", "round", "uf", "L"):
        if key not in out:
            out[key] = torch.empty(n, dtype=torch.int32, device="cuda")
    st = PeelStats() if stats else None
    _check("nh_peel_and_link", lib().nh_peel_and_link(
        o.handle, ri.handle, s, _dptr(cnt), _dptr(out["core"]), _dptr(out["round"]), _dptr(out["uf"]),
        _dptr(out["L"]), LINK_MODES[link_mode], ctypes.byref(st) if st is not None else None, _stream(stream)))
    res = {k: out[k][: ri.n_r] for k in ("core", "round", "uf", "L")}
    if st is not None:
        res["stats"] = st.as_dict()
    return res


def peel_cores(o: Oriented, ri: RIndex, s: int, cnt: torch.Tensor, stats: bool = False, stream=None) -> dict:
    """The exact peel without linking (core numbers and round stamps only; link mode 2)."""
    n = max(ri.n_r, 1)
    core = torch.empty(n, dtype=torch.int32, device="cuda")
    rnd = torch.empty(n, dtype=torch.int32, device="cuda")
    st = PeelStats() if stats else None
    _check("nh_peel_and_link", lib().nh_peel_and_link(o.handle, ri.handle, s, _dptr(cnt), _dptr(core), _dptr(rnd),
                                                      None, None, 2, ctypes.byref(st) if st is not None else None,
                                                      _stream(stream)))
    res = {"core": core[: ri.n_r], "round": rnd[: ri.n_r]}
    if st is not None:
        res["stats"] = st.as_dict()
    return res


def construct_tree(core: torch.Tensor, uf: torch.Tensor, L: torch.Tensor, parent: torch.Tensor | None = None,
                   label: torch.Tensor | None = None, stream=None):
    n_r = core.numel()
    if parent is None:
        parent = torch.empty(max(2 * n_r, 1), dtype=torch.int32, device="cuda")
    if label is None:
        label = torch.empty(max(n_r, 1), dtype=torch.int32, device="cuda")
    nn = I64()
    _check("nh_construct_tree", lib().nh_construct_tree(n_r, _dptr(core), _dptr(uf), _dptr(L), _dptr(parent),
                                                        _dptr(label), ctypes.byref(nn), _stream(stream)))
    return parent[: n_r + nn.value], label[: nn.value], nn.value


def hierarchy_two_phase(o: Oriented, ri: RIndex, s: int, core: torch.Tensor, stream=None):
    """§7.4 two-phase hierarchy from final core numbers; returns (parent, label, n_nodes) like
    construct_tree."""
    n_r = ri.n_r
    parent = torch.empty(max(2 * n_r, 1), dtype=torch.int32, device="cuda")
    label = torch.empty(max(n_r, 1), dtype=torch.int32, device="cuda")
    nn = I64()
    _check("nh_hierarchy_two_phase", lib().nh_hierarchy_two_phase(o.handle, ri.handle, s, _dptr(core), _dptr(parent),
                                                                  _dptr(label), ctypes.byref(nn), _stream(stream)))
    return parent[: n_r + nn.value], label[: nn.value], nn.value


def hierarchy_basic(o: Oriented, ri: RIndex, s: int, core: torch.Tensor, stream=None):
    """link-basic + construct-tree-basic (Alg. 4) from final core numbers; returns (parent, label,
    n_nodes, unites) with parent / label like construct_tree."""
    n_r = ri.n_r
    parent = torch.empty(max(2 * n_r, 1), dtype=torch.int32, device="cuda")
    label = torch.empty(max(n_r, 1), dtype=torch.int32, device="cuda")
    nn = I64()
    un = ctypes.c_uint64()
    _check("nh_hierarchy_basic", lib().nh_hierarchy_basic(o.handle, ri.handle, s, _dptr(core), _dptr(parent),
                                                          _dptr(label), ctypes.byref(nn), ctypes.byref(un),
                                                          _stream(stream)))
    return parent[: n_r + nn.value], label[: nn.value], nn.value, un.value


TREE_NOALLOC_MAX = 1 << 18


def label_hierarchy(o: Oriented, ri: RIndex, s: int, labels: torch.Tensor, stream=None):
    """Definitional hierarchy of arbitrary labels (e.g. approx_nucleus values: the approximate
    hierarchy); returns (parent, label, n_nodes) like construct_tree."""
    n_r = ri.n_r
    parent = torch.empty(max(2 * n_r, 1), dtype=torch.int32, device="cuda")
    label = torch.empty(max(n_r, 1), dtype=torch.int32, device="cuda")
    nn = I64()
    _check("nh_label_hierarchy", lib().nh_label_hierarchy(o.handle, ri.handle, s, _dptr(labels), _dptr(parent),
                                                          _dptr(label), ctypes.byref(nn), _stream(stream)))
    return parent[: n_r + nn.value], label[: nn.value], nn.value


def hierarchy_buffers(ri: RIndex) -> dict:
    """Device outputs of hierarchy_enqueue for one r-clique index."""
    n = max(ri.n_r, 1)
    i32 = dict(dtype=torch.int32, device="cuda")
    return {"cnt": torch.empty(n, **i32), "core": torch.empty(n, **i32), "round": torch.empty(n, **i32),
            "uf": torch.empty(n, **i32), "L": torch.empty(n, **i32), "parent": torch.empty(2 * n, **i32),
            "label": torch.empty(n, **i32), "res": torch.zeros(4, dtype=torch.int64, device="cuda")}


def hierarchy_enqueue(o: Oriented, ri: RIndex, s: int, buf: dict, stream=None):
    """Counts, peel with link-efficient and construct-tree in stream order with no host
    synchronisation (capturable into a CUDA graph); buf from hierarchy_buffers.  After the stream
    has run it, buf["res"] holds (status, n_s, n_nodes, rounds)."""
    _check("nh_hierarchy_enqueue", lib().nh_hierarchy_enqueue(
        o.handle, ri.handle, s, _dptr(buf["cnt"]), _dptr(buf["core"]), _dptr(buf["round"]), _dptr(buf["uf"]),
        _dptr(buf["L"]), _dptr(buf["parent"]), _dptr(buf["label"]), _dptr(buf["res"]), _stream(stream)))


def capture_hierarchy(o: Oriented, ri: RIndex, s: int, buf: dict):
    """hierarchy_enqueue captured into a CUDA graph (after one eager warm-up call): replaying the
    returned torch.cuda.CUDAGraph reruns counts, peel and construct-tree into buf."""
    hierarchy_enqueue(o, ri, s, buf)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    with torch.cuda.graph(g, stream=side, capture_error_mode="relaxed"):
        hierarchy_enqueue(o, ri, s, buf)
    return g


def cut_hierarchy(parent: torch.Tensor, label: torch.Tensor, n_r: int, n_nodes: int, c: int, stream=None):
    """c-(r,s) nuclei from a hierarchy: per r-clique the node id of the top of its c-nucleus (-1
    when its core is below c), and the number of c-nuclei."""
    out = torch.empty(max(n_r, 1), dtype=torch.int32, device="cuda")
    nn = I64()
    _check("nh_cut_hierarchy", lib().nh_cut_hierarchy(n_r, n_nodes, _dptr(parent), _dptr(label), int(c), _dptr(out),
                                                      ctypes.byref(nn), _stream(stream)))
    return out[:n_r], nn.value


def construct_tree_noalloc(core: torch.Tensor, uf: torch.Tensor, L: torch.Tensor, parent: torch.Tensor,
                           label: torch.Tensor, stream=None):
    """nh_construct_tree without device allocation (n_r <= TREE_NOALLOC_MAX): the outputs are the
    caller's tensors (parent: 2*n_r entries, label: n_r entries), the library's working memory is
    a fixed device array shared by all calls, so overlapping calls must not be issued."""
    n_r = core.numel()
    nn = I64()
    _check("nh_construct_tree_noalloc", lib().nh_construct_tree_noalloc(
        n_r, _dptr(core), _dptr(uf), _dptr(L), _dptr(parent), _dptr(label), ctypes.byref(nn), _stream(stream)))
    return parent[: n_r + nn.value], label[: nn.value], nn.value


def approx_nucleus(o: Oriented, ri: RIndex, s: int, delta: float, cnt: torch.Tensor, stats: bool = False,
                   stream=None) -> dict:
    n = max(ri.n_r, 1)
    approx = torch.empty(n, dtype=torch.int32, device="cuda")
    rnd = torch.empty(n, dtype=torch.int32, device="cuda")
    st = PeelStats() if stats else None
    _check("nh_approx_nucleus", lib().nh_approx_nucleus(o.handle, ri.handle, s, float(delta), _dptr(cnt),
                                                        _dptr(approx), _dptr(rnd),
                                                        ctypes.byref(st) if st is not None else None,
                                                        _stream(stream)))
    res = {"approx": approx[: ri.n_r], "round": rnd[: ri.n_r]}
    if st is not None:
        res["stats"] = st.as_dict()
    return res


def link_pairs(core: torch.Tensor, uf: torch.Tensor, L: torch.Tensor, pairs: torch.Tensor, stream=None):
    """link-efficient (Alg. 5) on a batch of (R, Q) calls; uf and L are updated in place."""
    pairs = pairs.to(torch.int32).contiguous()
    _check("nh_link_pairs", lib().nh_link_pairs(core.numel(), _dptr(core), _dptr(uf), _dptr(L), _dptr(pairs),
                                                pairs.numel() // 2, _stream(stream)))


MLP_FEATURES = 8
MLP_PARAMS = 4801


def vertex_features(o: Oriented, stream=None) -> torch.Tensor:
    """(n, 8) float32 work-estimator features per vertex."""
    f = torch.empty((max(o.n, 1), MLP_FEATURES), dtype=torch.float32, device="cuda")
    _check("nh_vertex_features", lib().nh_vertex_features(o.handle, _dptr(f), _stream(stream)))
    return f[: o.n]


def listing_cost(o: Oriented, ri: RIndex, s: int, stream=None) -> torch.Tensor:
    """Measured listing work per vertex of one counting pass (the estimator's training label)."""
    c = torch.empty(max(o.n, 1), dtype=torch.float32, device="cuda")
    _check("nh_listing_cost", lib().nh_listing_cost(o.handle, ri.handle, s, _dptr(c), _stream(stream)))
    return c[: o.n]


def degree_cost(o: Oriented, s: int, stream=None) -> torch.Tensor:
    c = torch.empty(max(o.n, 1), dtype=torch.float32, device="cuda")
    _check("nh_degree_cost", lib().nh_degree_cost(o.handle, s, _dptr(c), _stream(stream)))
    return c[: o.n]


def mlp_train(feats: torch.Tensor, cost: torch.Tensor, n_train: int = 16384, steps: int = 200, lr: float = 1e-2,
              seed: int = 1, stream=None):
    """Train the work estimator; returns (bf16 weights as an int16 tensor, final MSE on log1p cost)."""
    w = torch.empty(MLP_PARAMS, dtype=torch.int16, device="cuda")
    loss = ctypes.c_float()
    _check("nh_mlp_train", lib().nh_mlp_train(_dptr(feats.contiguous()), _dptr(cost.contiguous()), feats.shape[0],
                                              n_train, steps, float(lr), seed, _dptr(w), ctypes.byref(loss),
                                              _stream(stream)))
    return w, float(loss.value)


def mlp_predict(feats: torch.Tensor, weights: torch.Tensor, stream=None) -> torch.Tensor:
    out = torch.empty(max(feats.shape[0], 1), dtype=torch.float32, device="cuda")
    _check("nh_mlp_predict", lib().nh_mlp_predict(_dptr(feats.contiguous()), feats.shape[0], _dptr(weights),
                                                  _dptr(out), _stream(stream)))
    return out[: feats.shape[0]]


def count_s_cliques_partitioned(o: Oriented, ri: RIndex, s: int, vertex_cost: torch.Tensor,
                                cnt: torch.Tensor | None = None, stream=None):
    if cnt is None:
        cnt = torch.empty(max(ri.n_r, 1), dtype=torch.int32, device="cuda")
    n_s = ctypes.c_uint64()
    _check("nh_count_s_cliques_partitioned", lib().nh_count_s_cliques_partitioned(
        o.handle, ri.handle, s, _dptr(vertex_cost.contiguous()), _dptr(cnt), ctypes.byref(n_s), _stream(stream)))
    return cnt[: ri.n_r], int(n_s.value)


class GraphDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("off", ctypes.c_void_p), ("adj", ctypes.c_void_p)]


def batch_union(graphs, stream=None):
    """graphs: list of (off, adj) device tensors -> (off, adj, vbase list) of their disjoint union."""
    import numpy as np
    descs = (GraphDesc * len(graphs))()
    N = NNZ = 0
    for i, (off, adj) in enumerate(graphs):
        descs[i] = GraphDesc(off.numel() - 1, adj.numel(), off.data_ptr(), adj.data_ptr() if adj.numel() else None)
        N += off.numel() - 1
        NNZ += adj.numel()
    off_u = torch.empty(N + 1, dtype=torch.int64, device="cuda")
    adj_u = torch.empty(max(NNZ, 1), dtype=torch.int32, device="cuda")
    vbase = np.zeros(len(graphs) + 1, dtype=np.int64)
    _check("nh_batch_union", lib().nh_batch_union(descs, len(graphs), _dptr(off_u), _dptr(adj_u),
                                                  vbase.ctypes.data_as(P), _stream(stream)))
    return off_u, adj_u[:NNZ], vbase


def rindex_bases(ri: RIndex, vbase, stream=None):
    import numpy as np
    vbase = np.ascontiguousarray(vbase, dtype=np.int64)
    out = np.zeros(len(vbase), dtype=np.int64)
    _check("nh_rindex_bases", lib().nh_rindex_bases(ri.handle, vbase.ctypes.data_as(P), len(vbase) - 1,
                                                    out.ctypes.data_as(P), _stream(stream)))
    return out


class Batch:
    """A batch of graphs prepared as one disjoint union (nh_batch_prepare): its orientation and
    r-clique index live in the handle; run(s, buf) enqueues counts, the persistent peel and
    construct-tree over every graph at once (capturable).  vbase / rbase: the first vertex /
    r-clique of every graph in the union (n_graphs + 1 entries)."""

    def __init__(self, graphs, r: int, stream=None):
        import numpy as np
        descs = (GraphDesc * len(graphs))()
        for i, (off, adj) in enumerate(graphs):
            descs[i] = GraphDesc(off.numel() - 1, adj.numel(), off.data_ptr(), adj.data_ptr() if adj.numel() else None)
        h, n_r = P(), I64()
        _check("nh_batch_prepare", lib().nh_batch_prepare(descs, len(graphs), r, ctypes.byref(h), ctypes.byref(n_r),
                                                          _stream(stream)))
        self.handle, self.r, self.n_r, self.n_graphs = h, r, n_r.value, len(graphs)
        self.vbase = np.zeros(len(graphs) + 1, dtype=np.int64)
        self.rbase = np.zeros(len(graphs) + 1, dtype=np.int64)
        _check("nh_batch_bases", lib().nh_batch_bases(h, self.vbase.ctypes.data_as(P), self.rbase.ctypes.data_as(P)))

    def buffers(self) -> dict:
        return hierarchy_buffers(self)

    def run(self, s: int, buf: dict, stream=None):
        _check("nh_batch_run", lib().nh_batch_run(
            self.handle, s, _dptr(buf["cnt"]), _dptr(buf["core"]), _dptr(buf["round"]), _dptr(buf["uf"]),
            _dptr(buf["L"]), _dptr(buf["parent"]), _dptr(buf["label"]), _dptr(buf["res"]), _stream(stream)))

    def capture(self, s: int, buf: dict):
        """run(s, buf) captured into a CUDA graph after one eager call; replay() reruns it."""
        self.run(s, buf)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        with torch.cuda.graph(g, stream=side, capture_error_mode="relaxed"):
            self.run(s, buf)
        return g

    def node_bases(self, parent: torch.Tensor, n_nodes: int, stream=None):
        import numpy as np
        out = np.zeros(self.n_graphs + 1, dtype=np.int64)
        _check("nh_batch_node_bases", lib().nh_batch_node_bases(self.handle, _dptr(parent), int(n_nodes),
                                                                out.ctypes.data_as(P), _stream(stream)))
        return out

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.nh_batch_free(self.handle)
            self.handle = None


def set_peel_max_group(g: int):
    """Largest number of warps per frontier r-clique (power of two, 1..1024); results never
    depend on it."""
    _check("nh_set_peel_max_group", lib().nh_set_peel_max_group(int(g)))


def set_peel_task_items(n: int):
    """Largest frontier (or level) re-listed as work-proportional chunk tasks (0..4096, 0 = off,
    -1 = automatic); results never depend on it."""
    _check("nh_set_peel_task_items", lib().nh_set_peel_task_items(int(n)))


def set_peel_list_hash(mode: int):
    """(3,4) re-listing: find a candidate's other two list entries by binary search (0, the
    default), through the (edge, third vertex) table (2), or automatically (1: the table for the
    cores-only and approximate peels); results never depend on it."""
    _check("nh_set_peel_list_hash", lib().nh_set_peel_list_hash(int(mode)))


def set_peel_relist24(on: bool):
    """(2,4) without links: re-list each edge from its triangle list with candidates staged in
    shared memory (True, the default) or by the adjacency scans of the other pairs (False);
    results never depend on it."""
    _check("nh_set_peel_relist24", lib().nh_set_peel_relist24(int(bool(on))))


RELIST_SPLIT_DEFAULT = (1.0, 128, 1024, 0)


def set_relist_split(per_warp: float = 1.0, warp_grain: int = 128, block_grain: int = 1024, len_mult: int = 0):
    """Sub-task split of the (2,4) triangle-list re-listing (see nucleus.h); results never depend
    on it."""
    _check("nh_set_relist_split", lib().nh_set_relist_split(float(per_warp), int(warp_grain), int(block_grain),
                                                            int(len_mult)))


def debug_round_log(log: torch.Tensor | None):
    """Trace the rounds of the next peels into log (int64 device tensor of 8*cap entries): per
    round (frontier size << 32 | levels opened so far, device timer in ns at the round's end,
    out-list entries expanded, sub-tasks << 32 | block sub-tasks, then block 0's timer at the
    (2,4) re-listing's start, after its split, after its warp phase, at its end); None turns the
    trace off."""
    if log is None:
        _check("nh_debug_round_log", lib().nh_debug_round_log(None, 0))
    else:
        assert log.dtype == torch.int64 and log.is_cuda
        _check("nh_debug_round_log", lib().nh_debug_round_log(_dptr(log), log.numel() // 8))


def _cuda_timer(run) -> float:
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    run()
    b.record()
    b.synchronize()
    return a.elapsed_time(b)


def set_relist_split(per_warp: float = 1.0, warp_grain: int = 128, block_grain: int = 1024, len_mult: int = 0):
    """Sub-task size of the triangle-list re-listing ((2,4) without links): sub-tasks per warp of
    the grid a round aims at, and the least scan bound of a warp / block sub-task; results never
    depend on it."""
    _check("nh_set_relist_split", lib().nh_set_relist_split(float(per_warp), int(warp_grain), int(block_grain),
                                                            int(len_mult)))


def autotune_peel(run, max_groups=(16, 64, 256, 1024), task_items=(-1,), splits=(None,), repeats: int = 1,
                  timer=None) -> dict:
    """Grid search over the peel's scheduling knobs: time `run()` (one piece of device work, e.g.
    a whole hierarchy) under every (warps-per-r-clique cap, task-frontier size[, sub-tasks per
    warp]) combination, keep the fastest set, and return {"best": key, "times_ms": {key: ms}} with
    key = (cap, items) or, when splits are given, (cap, items, split).  The knobs change only the
    scheduling, never a result.  `timer(run) -> ms` defaults to CUDA events on the current
    stream."""
    timer = timer or _cuda_timer
    times = {}
    for g in max_groups:
        for t in task_items:
            for sp in splits:
                set_peel_max_group(g)
                set_peel_task_items(t)
                if sp is not None:
                    set_relist_split(sp)
                key = (g, t) if sp is None else (g, t, sp)
                times[key] = min(timer(run) for _ in range(max(1, repeats)))
    best = min(times, key=times.get)
    set_peel_max_group(best[0])
    set_peel_task_items(best[1])
    if len(best) > 2:
        set_relist_split(best[2])
    return {"best": best, "times_ms": times}


def autotune_peel_max_group(run, candidates=(16, 64, 256, 1024), repeats: int = 1, timer=None) -> dict:
    """autotune_peel over the warps-per-r-clique cap alone; returns {cap: ms}."""
    res = autotune_peel(run, max_groups=candidates, task_items=(-1,), repeats=repeats, timer=timer)
    return {g: ms for (g, _), ms in res["times_ms"].items()}


def kernel_launches() -> int:
    """CUDA kernels launched by the library in this process so far."""
    return int(lib().nh_kernel_launches())


def hierarchy(off: torch.Tensor, adj: torch.Tensor, r: int, s: int, link_mode: str = "def", stats: bool = False,
              method: str = "el", stream=None) -> dict:
    """The whole exact path on device tensors: orientation, r-clique index, s-clique counts, peel
    and hierarchy.  method "el": link-efficient interleaved with the peel, then construct-tree
    (Alg. 3 + Alg. 5); "te": core numbers, then the two-phase hierarchy (§7.4, definitional
    reading only); "bl": core numbers, then link-basic and construct-tree-basic (Alg. 4, the
    ablation); "auto": "te" for (1,2), (2,3), (2,4), where it is the faster builder on a GB300
    (R-MAT 18, peel + hierarchy), "el" for (3,4), where the two are level, and for the pair rule
    (link_mode "pair"), which only "el" follows.
    Pairs beyond (1,2), (1,3), (2,3), (2,4), (3,4) (any r < s <= 7) run the generic path, where
    "el" and "te" both link over every s-clique after the peel."""
    if method == "auto":
        method = "el" if (r, s) == (3, 4) or link_mode != "def" else "te"
    o = build_orientation(off, adj, stream)
    ri = index_r_cliques(o, r, stream)
    cnt, n_s = count_s_cliques(o, ri, s, stream=stream)
    if method == "bl":
        assert link_mode == "def", "link-basic follows the definition here"
        pk = peel_cores(o, ri, s, cnt, stats=stats, stream=stream)
        parent, label, nn, unites = hierarchy_basic(o, ri, s, pk["core"], stream=stream)
        pk["basic_unites"] = unites
    elif method == "te":
        assert link_mode == "def", "the two-phase hierarchy follows the definition"
        pk = peel_cores(o, ri, s, cnt, stats=stats, stream=stream)
        parent, label, nn = hierarchy_two_phase(o, ri, s, pk["core"], stream=stream)
    else:
        pk = peel_and_link(o, ri, s, cnt, link_mode=link_mode, stats=stats, stream=stream)
        parent, label, nn = construct_tree(pk["core"], pk["uf"], pk["L"], stream=stream)
    res = {"oriented": o, "rindex": ri, "n_r": ri.n_r, "n_s": n_s, "cnt": cnt, "parent": parent,
           "label": label, "n_nodes": nn}
    res.update(pk)
    return res
