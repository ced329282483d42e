"""Test-side helpers: run the GPU path through the binding and compare with the oracle.

These compare two independent results; they are neither part of the oracle nor of the CUDA path.
"""
import numpy as np


def u32(t):
    """int32 device tensor holding uint32 bit patterns -> numpy uint32"""
    return t.cpu().numpy().view(np.uint32)


def i32(t):
    return t.cpu().numpy().astype(np.int32)


def compare_hierarchy(parent, label, n_nodes, o_leaf, o_parent, o_label):
    """GPU tree (parent over leaves then nodes, label per node) against the oracle's tree
    (leaf -> smallest node, node -> parent, node -> level).  Node ids are arbitrary on both sides:
    nodes are matched through the r-cliques whose smallest node they are (every node has one),
    then labels and parents must agree under that matching."""
    n_r = len(o_leaf)
    parent = np.asarray(parent, dtype=np.int64)
    gl = parent[:n_r]
    gp = parent[n_r:n_r + n_nodes]
    glab = np.asarray(label, dtype=np.int64)[:n_nodes]
    o_leaf = np.asarray(o_leaf, dtype=np.int64)
    o_parent = np.asarray(o_parent, dtype=np.int64)
    o_label = np.asarray(o_label, dtype=np.int64)
    assert n_nodes == len(o_parent), "node count %d vs oracle %d" % (n_nodes, len(o_parent))
    assert ((gl < 0) == (o_leaf < 0)).all(), "r-cliques outside every node differ"
    m = gl >= 0
    if n_nodes == 0:
        return
    pairs = np.unique(np.stack([gl[m], o_leaf[m]], axis=1), axis=0)
    assert len(pairs) == n_nodes, "leaf-to-node maps are not one-to-one (%d pairs, %d nodes)" % (len(pairs), n_nodes)
    assert len(np.unique(pairs[:, 0])) == n_nodes and len(np.unique(pairs[:, 1])) == n_nodes
    g2o = np.full(n_nodes, -1, dtype=np.int64)
    g2o[pairs[:, 0]] = pairs[:, 1]
    assert (glab == o_label[g2o]).all(), "node labels differ"
    mapped = np.where(gp >= 0, g2o[np.maximum(gp, 0)], -1)
    assert (mapped == o_parent[g2o]).all(), "node parents differ"
