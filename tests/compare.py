"""Bit-exact comparison of a GPU LOD result with the CPU oracle's.

* Node table: every field equal (voxel_offset excluded — it depends on where
  each side lays out its voxel blocks; both sides' voxel ranges are compared
  through their own offsets instead).
* Leaf points: identical multiset per leaf (order inside a leaf is free).
* Leaf indices: GPU points[i] == input[index[i]] and the index multiset per
  leaf equals the oracle's.
* Voxels: identical rows per node after sorting by cell (order is free).
"""
from __future__ import annotations

import numpy as np

NODE_KEYS = ("min", "level", "log2_size", "child_mask", "flags", "parent", "first_child",
             "point_offset", "point_count", "voxel_count")


def _seg_ids(offsets, counts, total):
    seg = np.full(total, -1, dtype=np.int64)
    order = np.argsort(offsets, kind="stable")
    ids = np.repeat(order, counts[order].astype(np.int64))
    pos = np.concatenate([np.arange(o, o + c) for o, c in zip(offsets[order], counts[order])]) if len(order) else np.zeros(0, np.int64)
    seg[pos] = ids
    return seg


def _sorted_rows(rows, seg):
    rows = np.asarray(rows).astype(np.int64)
    keys = [rows[:, j] for j in range(rows.shape[1] - 1, -1, -1)] + [seg]
    o = np.lexsort(keys)
    return np.concatenate([seg[o][:, None], rows[o]], axis=1)


def compare(got: dict, want: dict, inp: np.ndarray | None = None, check_index: bool = True) -> None:
    for k in NODE_KEYS:
        a, b = np.asarray(got[k]), np.asarray(want[k])
        assert a.shape == b.shape, f"node field {k}: shape {a.shape} != {b.shape}"
        if not np.array_equal(a, b):
            bad = np.nonzero(a != b)[0] if a.ndim == 1 else np.nonzero(np.any(a != b, axis=1))[0]
            raise AssertionError(f"node field {k} differs at {bad[:10].tolist()}: got {a[bad[:3]]} want {b[bad[:3]]}")
    leaf = (np.asarray(want["flags"]) & 1) == 1
    n = len(want["points"])
    off = np.asarray(want["point_offset"])[leaf].astype(np.int64)
    cnt = np.asarray(want["point_count"])[leaf].astype(np.int64)
    seg = _seg_ids(off, cnt, n)
    assert np.all(seg >= 0) or n == 0
    gp = np.asarray(got["points"]).reshape(-1, 4)
    wp = np.asarray(want["points"]).reshape(-1, 4)
    assert gp.shape == wp.shape
    if n:
        a = _sorted_rows(gp, seg)
        b = _sorted_rows(wp, seg)
        if not np.array_equal(a, b):
            bad = np.nonzero(np.any(a != b, axis=1))[0]
            raise AssertionError(f"leaf point multisets differ ({len(bad)} rows), first leaf {a[bad[0], 0]}")
    if check_index and got.get("index") is not None and n:
        gi = np.asarray(got["index"]).astype(np.int64)
        if inp is not None:
            assert np.array_equal(np.asarray(inp)[gi], gp), "points[i] != input[index[i]]"
        a = _sorted_rows(gi[:, None], seg)
        b = _sorted_rows(np.asarray(want["index"]).astype(np.int64)[:, None], seg)
        assert np.array_equal(a, b), "leaf index multisets differ"
    gv = np.asarray(got["voxels"]).reshape(-1, 4)
    wv = np.asarray(want["voxels"]).reshape(-1, 4)
    assert gv.shape == wv.shape, f"voxel totals differ: {gv.shape[0]} vs {wv.shape[0]}"
    nn = len(want["level"])
    vc = np.asarray(want["voxel_count"]).astype(np.int64)
    gseg = _seg_ids(np.asarray(got["voxel_offset"]).astype(np.int64), vc, len(gv))
    wseg = _seg_ids(np.asarray(want["voxel_offset"]).astype(np.int64), vc, len(wv))
    if len(gv):
        a = _sorted_rows(gv, gseg)
        b = _sorted_rows(wv, wseg)
        if not np.array_equal(a, b):
            bad = np.nonzero(np.any(a != b, axis=1))[0]
            raise AssertionError(f"voxels differ in {len(bad)} rows; first: got {a[bad[0]]} want {b[bad[0]]} (nodes {nn})")
