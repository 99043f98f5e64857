"""Bit-exact comparison of a GPU LOD result with the CPU oracle's.

* Node table: every field equal (voxel_offset excluded — it depends on where
  each side lays out its voxel blocks; both sides' voxel ranges are compared
  through their own offsets instead).
* Leaf points: identical multiset per leaf (order inside a leaf is free).
* Leaf indices: GPU points[i] == input[index[i]] and the index multiset per
  leaf equals the oracle's.
* Voxels: identical rows per node after sorting by cell (order is free).

Results of more than ``FAST_ROWS`` leaf points compare each leaf's point
and index multisets, and each node's voxel multiset, through an
order-independent fingerprint instead of a sort: the wrapping 64-bit sums,
over the segment's rows, of two different 64-bit mixes of each row (two
independent 64-bit sums, so two different multisets agree with probability
about 2^-128 per segment).  Node tables are always compared field by field.
"""
from __future__ import annotations

import numpy as np

NODE_KEYS = ("min", "level", "log2_size", "child_mask", "flags", "parent", "first_child",
             "point_offset", "point_count", "voxel_count")


FAST_ROWS = 8_000_000

_M1 = (np.uint64(0xBF58476D1CE4E5B9), np.uint64(0x94D049BB133111EB), np.uint64(0x9E3779B97F4A7C15))
_M2 = (np.uint64(0xFF51AFD7ED558CCD), np.uint64(0xC4CEB9FE1A85EC53), np.uint64(0xD6E8FEB86659FD93))


def _mix(v, m):
    """A 64-bit finalizer (xor-shift / multiply rounds) applied elementwise."""
    with np.errstate(over="ignore"):
        v = v + m[2]
        v = (v ^ (v >> np.uint64(30))) * m[0]
        v = (v ^ (v >> np.uint64(27))) * m[1]
        return v ^ (v >> np.uint64(31))


def _row_hashes(rows):
    """Two independent 64-bit hashes of every row of a 2-D integer array."""
    rows = np.asarray(rows)
    u = rows.astype(np.int64).view(np.uint64) if rows.dtype.kind == "i" else rows.astype(np.uint64)
    h1 = np.zeros(len(u), np.uint64)
    h2 = np.zeros(len(u), np.uint64)
    for j in range(u.shape[1]):
        h1 = _mix(h1 ^ u[:, j], _M1)
        h2 = _mix(h2 ^ u[:, j], _M2)
    return h1, h2


def _seg_fingerprints(rows, offsets, counts):
    """(n_segments, 2) wrapping sums of the row hashes over each segment
    [offsets[i], offsets[i] + counts[i]); empty segments give zeros."""
    h1, h2 = _row_hashes(rows)
    offsets = np.asarray(offsets).astype(np.int64)
    counts = np.asarray(counts).astype(np.int64)
    out = np.zeros((len(offsets), 2), np.uint64)
    c1 = np.concatenate([[np.uint64(0)], np.cumsum(h1, dtype=np.uint64)])
    c2 = np.concatenate([[np.uint64(0)], np.cumsum(h2, dtype=np.uint64)])
    with np.errstate(over="ignore"):
        out[:, 0] = c1[offsets + counts] - c1[offsets]
        out[:, 1] = c2[offsets + counts] - c2[offsets]
    return out


def _compare_fast(got, want, inp, check_index):
    leaf = (np.asarray(want["flags"]) & 1) == 1
    off = np.asarray(want["point_offset"])[leaf].astype(np.int64)
    cnt = np.asarray(want["point_count"])[leaf].astype(np.int64)
    gp = np.asarray(got["points"]).reshape(-1, 4)
    wp = np.asarray(want["points"]).reshape(-1, 4)
    assert gp.shape == wp.shape
    a = _seg_fingerprints(gp, off, cnt)
    b = _seg_fingerprints(wp, off, cnt)
    bad = np.nonzero(np.any(a != b, axis=1))[0]
    assert len(bad) == 0, f"leaf point multisets differ in {len(bad)} leaves, first leaf {np.nonzero(leaf)[0][bad[0]]}"
    if check_index and got.get("index") is not None:
        gi = np.asarray(got["index"]).astype(np.int64)
        if inp is not None:
            assert np.array_equal(np.asarray(inp)[gi], gp), "points[i] != input[index[i]]"
        a = _seg_fingerprints(gi[:, None], off, cnt)
        b = _seg_fingerprints(np.asarray(want["index"]).astype(np.int64)[:, None], off, cnt)
        assert np.array_equal(a, b), "leaf index multisets differ"
    gv = np.asarray(got["voxels"]).reshape(-1, 4)
    wv = np.asarray(want["voxels"]).reshape(-1, 4)
    assert gv.shape == wv.shape, f"voxel totals differ: {gv.shape[0]} vs {wv.shape[0]}"
    vc = np.asarray(want["voxel_count"]).astype(np.int64)
    a = _seg_fingerprints(gv, np.asarray(got["voxel_offset"]).astype(np.int64), vc)
    b = _seg_fingerprints(wv, np.asarray(want["voxel_offset"]).astype(np.int64), vc)
    bad = np.nonzero(np.any(a != b, axis=1))[0]
    assert len(bad) == 0, f"voxel sets differ in {len(bad)} nodes, first node {bad[0]}"


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
    if len(want["points"]) > FAST_ROWS:
        _compare_fast(got, want, inp, check_index)
        return
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
