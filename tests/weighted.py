"""Checks of neighbourhood-weighted results (Section 4.2.4) node by node.

A weighted voxel's colour depends on the colours of the child voxels it
samples (8-bit, already rounded), so a mistake in a child also moves its
ancestors.  ``per_node_check`` recomputes every inner node with the oracle
from that node's own children *in the result being checked* (the leaf
children's points and the inner children's voxels), which locates a
difference at the node where it arises."""
from __future__ import annotations

import numpy as np

import oracle


def children(res, i):
    fc = int(res["first_child"][i])
    k = int(res["child_mask"][i])
    return [fc + r for r in range(bin(k).count("1"))]


def octant_of(res, parent, child):
    b = (res["min"][child] != res["min"][parent]).astype(np.int64)
    return int(4 * b[0] + 2 * b[1] + b[2])


def voxels_of(res, i):
    a, c = int(res["voxel_offset"][i]), int(res["voxel_count"][i])
    v = np.asarray(res["voxels"]).reshape(-1, 4)[a:a + c]
    return v[np.argsort(v[:, 0], kind="stable")]


def node_samples(res, i):
    """The samples node i takes from its children in ``res``."""
    pts, vox, octs = [], [], []
    for j in children(res, i):
        if res["flags"][j] & 1:
            a, c = int(res["point_offset"][j]), int(res["point_count"][j])
            pts.append(np.asarray(res["points"])[a:a + c])
        else:
            v = voxels_of(res, j)
            vox.append(v)
            octs.append(np.full(len(v), octant_of(res, i, j), np.uint8))
    P = np.concatenate(pts) if pts else np.zeros((0, 4), np.int32)
    V = np.concatenate(vox) if vox else np.zeros((0, 4), np.uint32)
    O = np.concatenate(octs) if octs else np.zeros(0, np.uint8)
    return P, V, O


def channels(rgba):
    u = np.asarray(rgba).astype(np.uint32)
    return np.stack([(u >> s) & 255 for s in (0, 8, 16, 24)], axis=1).astype(np.int64)


def per_node_check(res, tol: int = 1, nodes=None) -> tuple:
    """Every inner node's voxels against the oracle evaluated on the node's
    own children in ``res``: identical cells, counts and pick fields, alpha
    255, every colour channel within ``tol``.  Returns (channels compared,
    channels equal)."""
    inner = np.nonzero((np.asarray(res["flags"]) & 1) == 0)[0] if nodes is None else nodes
    total = exact = 0
    for i in inner:
        P, V, O = node_samples(res, i)
        want = oracle.weighted_node(P, V, O, res["min"][i], int(res["log2_size"][i]))
        have = voxels_of(res, i)
        assert have.shape == want.shape, f"node {i}: {len(have)} voxels, oracle {len(want)}"
        assert np.array_equal(have[:, [0, 2, 3]], want[:, [0, 2, 3]]), f"node {i}: cells / counts"
        d = np.abs(channels(have[:, 1]) - channels(want[:, 1]))
        assert d.max(initial=0) <= tol, f"node {i}: a channel differs by {d.max()}"
        total += d[:, :3].size
        exact += int((d[:, :3] == 0).sum())
    return total, exact
