"""Brute-force checker for tiny inputs, independent of the oracle's code.

Every quantity is recomputed from scratch per node by scanning ALL points
with a cube-membership test (no recursive partitioning), and the 128^3
projection uses floor division / multiplication instead of shifts.  It
checks a full LOD result (oracle's or the GPU's, as numpy arrays in the
oracle's dictionary layout) against the definitions:

* root cube = bbox min, edge = smallest power of two > largest extent;
* a node is a leaf iff it has <= T points, is a unit cube, or sits at
  max_depth; inner nodes list exactly their non-empty octants, in octant
  order k = 4*bx + 2*by + bz, breadth first, ascending path key;
* leaves tile the points: each leaf's range holds exactly the points of its
  cube; ranges follow depth-first (ascending Morton key of the min corner);
* every inner node's voxels are exactly the occupied 128^3 cells, with the
  exact count, the rounded-half-up mean colour (filtered), the member of
  minimal splitmix64(index) (pick) or the first member in input order
  (first come);
* random (Section 4.2.2, Listing 1): computed recursively here from its
  definition — an inner node's candidates in a cell are the points of its
  leaf children and the winners of its inner children's cells that lie in
  that cell; the winner is the candidate of largest 32-bit key (top 12
  bits of the high half of splitmix64(level << 32 | index) above the low
  20 index bits), the larger index on equal keys.
"""
from __future__ import annotations

import numpy as np

M64 = (1 << 64) - 1


def splitmix64_py(x: int) -> int:
    z = (x + 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def random_key_py(i: int, level: int) -> tuple:
    """Listing 1's key of sample i drawn while filling a node at ``level``,
    with the index as the tie-break: compare as a tuple."""
    r = splitmix64_py((level << 32) | i) >> 32
    return ((r >> 20) << 20) | (i & 0xFFFFF), i


def _morton(dx: int, dy: int, dz: int, bits: int) -> int:
    key = 0
    for b in range(bits - 1, -1, -1):
        key = (key << 3) | (((dx >> b) & 1) << 2) | (((dy >> b) & 1) << 1) | ((dz >> b) & 1)
    return key


def check(points: np.ndarray, res: dict, T: int, mode: int, max_depth: int) -> None:
    pts = np.asarray(points, dtype=np.int64).reshape(-1, 4)
    n = pts.shape[0]
    xyz = pts[:, :3]
    rgba = pts[:, 3] & 0xFFFFFFFF
    nn = len(res["level"])
    mins = res["min"].astype(np.int64)
    lvl = res["level"].astype(np.int64)
    lg = res["log2_size"].astype(np.int64)
    mask = res["child_mask"].astype(np.int64)
    flags = res["flags"].astype(np.int64)
    parent = res["parent"].astype(np.int64)
    fc = res["first_child"].astype(np.int64)
    poff = res["point_offset"].astype(np.int64)
    pcnt = res["point_count"].astype(np.int64)
    NONE = 0xFFFFFFFF

    # --- root cube
    if n == 0:
        assert nn == 1 and list(mins[0]) == [0, 0, 0] and lg[0] == 0 and pcnt[0] == 0
        assert flags[0] & 1
        return
    lo = xyz.min(axis=0)
    ext = int((xyz.max(axis=0) - lo).max())
    L = 0
    while 2 ** L <= ext:
        L += 1
    assert list(mins[0]) == list(lo), (mins[0], lo)
    assert lg[0] == L and lvl[0] == 0 and parent[0] == NONE

    # --- per-node counts, leaf rule, children
    expect_children_total = 0
    for i in range(nn):
        c = mins[i]
        s = 2 ** int(lg[i])
        inside = np.all((xyz >= c) & (xyz < c + s), axis=1)
        cnt = int(inside.sum())
        assert pcnt[i] == cnt, (i, pcnt[i], cnt)
        assert cnt > 0 or n == 0
        assert lvl[i] <= max_depth
        leaf = cnt <= T or lg[i] == 0 or lvl[i] == max_depth
        assert bool(flags[i] & 1) == leaf, (i, flags[i], cnt)
        assert bool(flags[i] & 2) == (leaf and cnt > T)
        if leaf:
            assert mask[i] == 0 and fc[i] == NONE
            continue
        h = s // 2
        want = []
        for k in range(8):
            cc = c + np.array([(k >> 2) & 1, (k >> 1) & 1, k & 1]) * h
            if np.any(np.all((xyz >= cc) & (xyz < cc + h), axis=1)):
                want.append((k, cc))
        assert mask[i] == sum(1 << k for k, _ in want)
        for r, (k, cc) in enumerate(want):
            j = fc[i] + r
            assert parent[j] == i and lvl[j] == lvl[i] + 1 and lg[j] == lg[i] - 1
            assert list(mins[j]) == list(cc)
        expect_children_total += len(want)
    assert nn == 1 + expect_children_total

    # --- breadth-first order, ascending path key within a level
    keys = [(_morton(*(int(v) for v in (mins[i] - mins[0]) >> lg[i]), int(lvl[i])) if lg[i] < 64 else 0)
            for i in range(nn)]
    order = sorted(range(nn), key=lambda i: (lvl[i], keys[i]))
    assert order == list(range(nn))

    # --- leaf ranges: depth-first layout, exact point multisets
    leaves = [i for i in range(nn) if flags[i] & 1]
    mk = {i: _morton(*(int(v) for v in mins[i] - mins[0]), L) for i in range(nn)}
    leaves_dfs = sorted(leaves, key=lambda i: mk[i])
    off = 0
    for i in leaves_dfs:
        assert poff[i] == off, (i, poff[i], off)
        off += pcnt[i]
    assert off == n
    for i in range(nn):
        before = sum(int(pcnt[j]) for j in leaves if mk[j] < mk[i])
        assert poff[i] == before
    lp = np.asarray(res["points"], dtype=np.int64).reshape(-1, 4)
    for i in leaves:
        got = lp[poff[i]:poff[i] + pcnt[i]]
        c = mins[i]
        s = 2 ** int(lg[i])
        inside = np.all((xyz >= c) & (xyz < c + s), axis=1)
        want = pts[inside]
        g = sorted(map(tuple, got.tolist()))
        w = sorted(map(tuple, want.tolist()))
        assert g == w
    if "index" in res and res["index"] is not None:
        idx = np.asarray(res["index"], dtype=np.int64)
        assert sorted(idx.tolist()) == list(range(n))
        assert np.array_equal(pts[idx], lp)

    # --- voxels of inner nodes
    vox = np.asarray(res["voxels"], dtype=np.int64).reshape(-1, 4)
    voff = res["voxel_offset"].astype(np.int64)
    vcnt = res["voxel_count"].astype(np.int64)

    def cell_of(p, node):
        c, s = mins[node], 2 ** int(lg[node])
        q = [((int(xyz[p, a]) - int(c[a])) * 128) // s for a in range(3)]
        return q[0] + 128 * q[1] + 16384 * q[2]

    winners = {}  # random mode: node -> {cell: winning input index}

    def random_winners(i):
        if i in winners:
            return winners[i]
        cand = {}
        for r in range(bin(int(mask[i])).count("1")):
            j = int(fc[i] + r)
            if flags[j] & 1:
                c, s = mins[j], 2 ** int(lg[j])
                pts_j = np.nonzero(np.all((xyz >= c) & (xyz < c + s), axis=1))[0].tolist()
            else:
                pts_j = list(random_winners(j).values())
            for p in pts_j:
                cand.setdefault(cell_of(p, i), []).append(p)
        winners[i] = {cell: max(ps, key=lambda p: random_key_py(p, int(lvl[i]))) for cell, ps in cand.items()}
        return winners[i]

    for i in range(nn):
        if flags[i] & 1:
            assert vcnt[i] == 0
            continue
        c = mins[i]
        s = 2 ** int(lg[i])
        inside = np.nonzero(np.all((xyz >= c) & (xyz < c + s), axis=1))[0]
        cells = {}
        for p in inside.tolist():
            q = [((int(xyz[p, a]) - int(c[a])) * 128) // s for a in range(3)]
            cells.setdefault(q[0] + 128 * q[1] + 16384 * q[2], []).append(p)
        got = vox[voff[i]:voff[i] + vcnt[i]]
        assert len(got) == len(cells), (i, len(got), len(cells))
        got = {int(r[0]): r for r in got}
        assert set(got) == set(cells)
        for cell, members in cells.items():
            r = got[cell]
            assert r[2] == len(members)
            if mode == 0:
                cnt = len(members)
                ch = []
                for sh in (0, 8, 16):
                    tot = sum((int(rgba[p]) >> sh) & 255 for p in members)
                    ch.append((2 * tot + cnt) // (2 * cnt))
                want_rgba = ch[0] | (ch[1] << 8) | (ch[2] << 16) | (255 << 24)
                assert r[1] == want_rgba and r[3] == NONE
            elif mode == 3:
                best = min(members)  # first come: the first member in input order
                assert r[3] == best and r[1] == int(rgba[best])
            elif mode == 4:
                best = random_winners(i)[cell]
                assert r[3] == best and r[1] == int(rgba[best])
            else:
                best = min(members, key=splitmix64_py)
                assert r[3] == best and r[1] == int(rgba[best])
