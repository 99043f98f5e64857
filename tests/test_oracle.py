"""CPU pins of the oracle: values and structures fixed by the paper's
definitions and by mathematics, not by the oracle itself.

* splitmix64: the published first output for seed 0 (Steele, Lea & Flood,
  OOPSLA 2014; the value every reference implementation prints).
* Hand-derived closed forms: root cube sizing, octant bit order, node order,
  rounding of the cell mean (Section 4.2.3), the unique minimal-hash pick,
  duplicate-point chains capped by unit cubes and max_depth (Section 4.1.5
  reading), complete lattices and a line with closed-form counts.
* An independent brute-force checker (tests/bruteforce.py) on random tiny
  clouds with small T (deep trees), in both modes.
* Cross-mode identities: identical cells and counts in both modes.
* Hand-worked examples under tests/golden/ (whole results in every mode
  each file states, each derivation written out in its file).
* First come (Section 4.2.1, oracle mode 3): the brute-force checker takes
  every cell's first point in input order.
* Random (Section 4.2.2 with Listing 1's key, oracle mode 4): the
  brute-force checker's recursive definition (children's winners compete
  again at every level with fresh random bits); the key's bit layout from
  the published splitmix64 outputs; cells and counts equal to the average
  mode's; the result differs from a single top-down draw.
* Neighbourhood-weighted average (Section 4.2.4, oracle mode 2): the mean
  of the corner samples on cubes of edge <= 128 (equal weights), cells and
  counts equal to the average mode's, constant colours exact, channels
  within the input's range.
"""
import numpy as np
import pytest

import golden
import oracle
from bruteforce import check, random_key_py, splitmix64_py
from paper_2302_14801_gb300 import synth

NONE = 0xFFFFFFFF


def P(rows):
    """Rows of (x, y, z, r, g, b) -> (N, 4) int32 points with alpha 255."""
    a = np.asarray(rows, dtype=np.int64).reshape(-1, 6)
    out = np.empty((len(a), 4), np.int32)
    out[:, :3] = a[:, :3]
    out[:, 3] = synth.pack_rgba(a[:, 3], a[:, 4], a[:, 5])
    return out


def test_splitmix64_published_seed0():
    # First output of splitmix64 seeded with 0 (the standard test vector).
    assert oracle.splitmix64(0) == 0xE220A8397B1DCDAF


def test_splitmix64_matches_generator_stream():
    # splitmix64(x) is the first output of a generator in state x, so the
    # second output of a generator seeded with 0 is splitmix64(golden).
    # The published second output for seed 0 is 0x6E789E6AA1B965F4.
    assert oracle.splitmix64(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4


def test_splitmix64_is_a_bijection_on_samples():
    # Invert with modular inverses derived here (Newton iteration), which is
    # independent of how the forward map is coded.
    def inv_mul(a):
        x = a
        for _ in range(6):
            x = (x * (2 - a * x)) & ((1 << 64) - 1)
        return x

    def unxorshift(y, s):
        x = y
        for _ in range(64 // s + 1):
            x = y ^ (x >> s)
        return x

    M = (1 << 64) - 1
    for x in [0, 1, 2, 12345, 2**32 - 1, 2**63 + 7]:
        h = oracle.splitmix64(x)
        z = unxorshift(h, 31)
        z = (z * inv_mul(0x94D049BB133111EB)) & M
        z = unxorshift(z, 27)
        z = (z * inv_mul(0xBF58476D1CE4E5B9)) & M
        z = unxorshift(z, 30)
        assert (z - 0x9E3779B97F4A7C15) & M == x


def test_empty_input():
    r = oracle.build(np.zeros((0, 4), np.int32), 10, 0)
    assert len(r["level"]) == 1
    assert list(r["min"][0]) == [0, 0, 0] and r["log2_size"][0] == 0
    assert r["flags"][0] == 1 and r["point_count"][0] == 0 and len(r["voxels"]) == 0


@pytest.mark.parametrize("ext,log2", [(0, 0), (1, 1), (3, 2), (4, 3), (5, 3), (7, 3), (8, 4),
                                      (2**31 - 1, 31), (2**31, 32), (2**32 - 1, 32)])
def test_root_cube_edge_is_smallest_power_of_two_above_extent(ext, log2):
    lo = -(2**31)
    hi = lo + ext
    pts = P([(lo, 5, 5, 1, 2, 3), (hi, 5, 5, 4, 5, 6)])
    r = oracle.build(pts, 10, 0)
    assert r["log2_size"][0] == log2
    assert list(r["min"][0]) == [lo, 5, 5]


def test_octant_bit_order_and_node_order():
    # Cube [0,8)^3 (extent 7).  One point in each of four octants; T = 1.
    # Octant k = 4*bx + 2*by + bz, so x-high is k=4, y-high k=2, z-high k=1.
    pts = P([(0, 0, 7, 10, 0, 0), (7, 0, 0, 20, 0, 0), (0, 0, 0, 30, 0, 0), (0, 7, 0, 40, 0, 0)])
    r = oracle.build(pts, 1, 0)
    assert r["log2_size"][0] == 3
    assert r["child_mask"][0] == (1 << 0) | (1 << 1) | (1 << 2) | (1 << 4)
    assert r["first_child"][0] == 1
    assert [list(m) for m in r["min"][1:]] == [[0, 0, 0], [0, 0, 4], [0, 4, 0], [4, 0, 0]]
    assert list(r["level"]) == [0, 1, 1, 1, 1]
    assert list(r["parent"]) == [NONE, 0, 0, 0, 0]
    # depth-first leaf layout follows the same octant order
    assert [int(v) for v in r["points"][:, 3] & 255] == [30, 10, 40, 20]
    assert list(r["point_offset"]) == [0, 0, 1, 2, 3]
    # root voxels: cube edge 8 < 128, so q = d * 16 per axis
    cells = sorted(int(c) for c in r["voxels"][:, 0])
    assert cells == sorted([0, 112 * 16384, 112, 112 * 128])


@pytest.mark.parametrize("reds,mean", [((1, 2), 2), ((1, 2, 2), 2), ((0, 1, 1, 1), 1),
                                       ((1, 1, 1, 2), 1), ((254, 255), 255), ((0, 1), 1),
                                       ((0, 0, 1), 0), ((3, 4, 4, 4), 4), ((100,), 100)])
def test_cell_mean_rounds_half_up(reds, mean):
    # All sample points share root cell 0 (cube edge 2^20, cells 2^13 wide);
    # a far point forces a split (T = len-1 ... ) so the root is inner.
    rows = [(i, 0, 0, r, 7, 200) for i, r in enumerate(reds)]
    rows.append((2**20 - 1, 0, 0, 0, 0, 0))
    pts = P(rows)
    r = oracle.build(pts, 1, 0)
    v = r["voxels"][r["voxel_offset"][0]:r["voxel_offset"][0] + r["voxel_count"][0]]
    v0 = v[v[:, 0] == 0][0]
    assert v0[2] == len(reds)
    assert v0[1] == mean | (7 << 8) | (200 << 16) | (255 << 24)
    assert v0[3] == NONE


def test_pick_is_unique_minimal_splitmix64():
    # Indices 0, 1, 2 in one cell.  Published hashes: h(1) = 0x910a2dec89025cc1
    # < h(2) = 0x975835de1c9756ce < h(0) = 0xe220a8397b1dcdaf, so index 1 wins.
    pts = P([(0, 0, 0, 11, 0, 0), (1, 0, 0, 22, 0, 0), (2, 0, 0, 33, 0, 0), (2**20 - 1, 0, 0, 44, 0, 0)])
    r = oracle.build(pts, 1, 1)
    v = r["voxels"][r["voxel_offset"][0]:r["voxel_offset"][0] + r["voxel_count"][0]]
    v0 = v[v[:, 0] == 0][0]
    assert v0[2] == 3 and v0[3] == 1 and (int(v0[1]) & 255) == 22


def test_single_leaf_when_n_at_most_T():
    pts = synth.sphere(500, seed=9)
    r = oracle.build(pts, 500, 0)
    assert len(r["level"]) == 1 and r["flags"][0] == 1 and len(r["voxels"]) == 0
    r = oracle.build(pts, 499, 0)
    assert r["flags"][0] == 0 and len(r["level"]) > 1


def test_all_identical_points_unit_cube_overfull():
    pts = P([(5, 5, 5, 1, 2, 3)] * 10)
    r = oracle.build(pts, 3, 0)
    assert len(r["level"]) == 1 and r["log2_size"][0] == 0 and r["flags"][0] == 3


@pytest.mark.parametrize("max_depth,expect_nodes,last_level", [(21, 12, 10), (5, 7, 5), (0, 1, 0)])
def test_duplicate_chain_capped(max_depth, expect_nodes, last_level):
    # 9 copies of the origin and one point at x = 1023: edge 1024 (log2 10).
    # The 9 copies descend a chain of single children until the unit cube at
    # level 10, or until max_depth; that last node is an overfull leaf.
    pts = P([(0, 0, 0, 1, 1, 1)] * 9 + [(1023, 0, 0, 2, 2, 2)])
    r = oracle.build(pts, 3, 0, max_depth)
    assert len(r["level"]) == expect_nodes
    deepest = int(np.argmax(r["level"]))
    assert r["level"][deepest] == last_level and r["point_count"][deepest] == (9 if max_depth else 10)
    assert r["flags"][deepest] == 3


@pytest.mark.parametrize("T,n_nodes,n_inner,n_vox", [(8, 73, 9, 512 + 8 * 64), (7, 585, 73, 512 + 512 + 64 * 8),
                                                     (64, 9, 1, 512), (512, 1, 0, 0)])
def test_complete_lattice_closed_form(T, n_nodes, n_inner, n_vox):
    g = np.stack(np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij"), -1).reshape(-1, 3)
    rows = np.concatenate([g, np.full((512, 3), 9)], axis=1)
    r = oracle.build(P(rows), T, 0)
    assert len(r["level"]) == n_nodes
    assert int(((r["flags"] & 1) == 0).sum()) == n_inner
    assert len(r["voxels"]) == n_vox
    assert np.all(r["voxels"][:, 2] == 1)  # edge <= 8 < 128: every point its own cell
    assert np.all(r["voxels"][:, 1] == (9 | (9 << 8) | (9 << 16) | (255 << 24)))


def test_line_closed_form_counts_and_means():
    # 1024 points (i, 0, 0), R = i mod 256.  Edge 1024 (log2 10), T = 100:
    # levels 0..3 inner (1+2+4+8 = 15 nodes), 16 leaves of 64 at level 4.
    # A level-l inner node spans 1024/2^l points in 128 cells of 8/2^l.
    n = 1024
    rows = [(i, 0, 0, i % 256, 0, 0) for i in range(n)]
    r = oracle.build(P(rows), 100, 0)
    assert len(r["level"]) == 31
    assert list(np.bincount(r["level"])) == [1, 2, 4, 8, 16]
    assert int((r["flags"] & 1).sum()) == 16
    assert len(r["voxels"]) == 15 * 128
    root = r["voxels"][r["voxel_offset"][0]:r["voxel_offset"][0] + 128]
    assert np.all(root[:, 2] == 8)
    for v in root:
        j = int(v[0])  # cell j holds x = 8j..8j+7, red = (8j mod 256) + 0..7
        assert int(v[1]) & 255 == (8 * j) % 256 + 4  # mean x.5 rounds up
    for lvl, cnt in [(1, 4), (2, 2), (3, 1)]:
        for i in np.nonzero(r["level"] == lvl)[0]:
            v = r["voxels"][r["voxel_offset"][i]:r["voxel_offset"][i] + r["voxel_count"][i]]
            assert len(v) == 128 and np.all(v[:, 2] == cnt)


def test_constant_colour_mean_exact():
    pts = synth.sphere(20000, seed=4)
    pts[:, 3] = synth.pack_rgba(np.full(20000, 17), np.full(20000, 99), np.full(20000, 250))
    r = oracle.build(pts, 1000, 0)
    assert len(r["voxels"]) > 0
    assert np.all(r["voxels"][:, 1] == (17 | (99 << 8) | (250 << 16) | (255 << 24)))


def _random_cloud(rng, n, spread_log2):
    kind = rng.integers(0, 3)
    if kind == 0:
        xyz = rng.integers(-(2**spread_log2), 2**spread_log2, size=(n, 3))
    elif kind == 1:  # clustered, with duplicates
        c = rng.integers(0, 2**spread_log2, size=(4, 3))
        xyz = c[rng.integers(0, 4, size=n)] + rng.integers(0, 3, size=(n, 3))
    else:  # points on a plane
        xyz = rng.integers(0, 2**spread_log2, size=(n, 3))
        xyz[:, 2] = 77
    out = np.empty((n, 4), np.int32)
    out[:, :3] = xyz
    out[:, 3] = rng.integers(-(2**31), 2**31, size=n)
    return out


@pytest.mark.parametrize("seed", range(12))
def test_bruteforce_random_tiny(seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(1, 400))
    T = int(rng.integers(1, 17))
    max_depth = int(rng.choice([21, 3, 1, 6]))
    pts = _random_cloud(rng, n, int(rng.integers(1, 24)))
    for mode in (0, 1, 3, 4):
        r = oracle.build(pts, T, mode, max_depth)
        check(pts, r, T, mode, max_depth)


def test_bruteforce_sphere_small():
    pts = synth.sphere(1500, seed=5)
    for mode in (0, 1, 3, 4):
        r = oracle.build(pts, 16, mode)
        check(pts, r, 16, mode, 21)


def test_cross_mode_identical_cells_and_counts():
    pts = synth.aerial(30000, seed=6, n_buildings=20)
    a = oracle.build(pts, 2000, 0)
    b = oracle.build(pts, 2000, 1)
    for k in ("min", "level", "log2_size", "child_mask", "flags", "parent", "first_child",
              "point_offset", "point_count", "voxel_count"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["voxels"][:, [0, 2]], b["voxels"][:, [0, 2]])


def test_invariants_medium():
    pts = synth.indoor(200000, seed=7, n_prims=64)
    r = oracle.build(pts, 5000, 1)
    leaf = (r["flags"] & 1) == 1
    assert int(r["point_count"][leaf].sum()) == len(pts)
    assert np.all(r["point_count"][leaf & ((r["flags"] & 2) == 0)] <= 5000)
    assert np.all(r["point_count"][~leaf] > 5000)
    # parent subtree count = sum of children
    for i in np.nonzero(~leaf)[0]:
        k = bin(int(r["child_mask"][i])).count("1")
        f = int(r["first_child"][i])
        assert int(r["point_count"][f:f + k].sum()) == int(r["point_count"][i])
        v = r["voxels"][r["voxel_offset"][i]:r["voxel_offset"][i] + r["voxel_count"][i]]
        assert int(v[:, 2].sum()) == int(r["point_count"][i])
    # each picked point lies in its cell with the minimal hash among its cell
    assert sorted(r["index"].tolist()) == list(range(len(pts)))


def test_parent_voxel_counts_are_sums_of_nested_child_cells():
    # A parent cell covers a 2x2x2 block of cells of the child in its octant.
    pts = synth.sphere(60000, seed=8)
    r = oracle.build(pts, 3000, 0)
    vox = r["voxels"]
    for i in np.nonzero((r["flags"] & 1) == 0)[0]:
        pv = vox[r["voxel_offset"][i]:r["voxel_offset"][i] + r["voxel_count"][i]]
        pc = {int(c): int(n) for c, n in zip(pv[:, 0], pv[:, 2])}
        acc = {}
        f = int(r["first_child"][i])
        k_list = [k for k in range(8) if r["child_mask"][i] >> k & 1]
        for rank, k in enumerate(k_list):
            j = f + rank
            ox, oy, oz = (k >> 2) & 1, (k >> 1) & 1, k & 1
            if r["flags"][j] & 1:
                # leaf child: project its points directly
                lp = r["points"][r["point_offset"][j]:r["point_offset"][j] + r["point_count"][j], :3]
                L = int(r["log2_size"][i])
                d = lp.astype(np.int64) - r["min"][i].astype(np.int64)
                q = d >> (L - 7) if L >= 7 else d << (7 - L)
                for c in (q[:, 0] | (q[:, 1] << 7) | (q[:, 2] << 14)).tolist():
                    acc[c] = acc.get(c, 0) + 1
                continue
            cv = vox[r["voxel_offset"][j]:r["voxel_offset"][j] + r["voxel_count"][j]]
            for c, n in zip(cv[:, 0].tolist(), cv[:, 2].tolist()):
                x, y, z = c & 127, (c >> 7) & 127, c >> 14
                pcell = (ox * 64 + (x >> 1)) | ((oy * 64 + (y >> 1)) << 7) | ((oz * 64 + (z >> 1)) << 14)
                acc[pcell] = acc.get(pcell, 0) + n
        assert acc == pc


def test_rejects_bad_arguments():
    pts = synth.sphere(10, seed=1)
    with pytest.raises(ValueError):
        oracle.build(pts, 0, 0)
    with pytest.raises(ValueError):
        oracle.build(pts, 10, 5)  # modes: 0 average, 1 pick, 2 weighted, 3 first come, 4 random
    with pytest.raises(ValueError):
        oracle.build(pts, 10, 0, 33)


def test_bruteforce_checker_catches_planted_mistakes():
    """The checker must fail on plausible oracle mistakes, planted here on
    the CPU in a copy of a correct result."""
    pts = synth.sphere(800, seed=11)
    good = oracle.build(pts, 12, 0)
    check(pts, good, 12, 0, 21)

    def mutated(fn):
        bad = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in good.items()}
        fn(bad)
        return bad

    plants = [
        lambda b: b["voxels"].__setitem__((0, 1), b["voxels"][0, 1] ^ 1),        # mean off by one
        lambda b: b["voxels"].__setitem__((0, 2), b["voxels"][0, 2] + 1),        # count
        lambda b: b["min"].__setitem__((1, 0), b["min"][1, 0] + 1),              # child min
        lambda b: b["point_offset"].__setitem__(-1, b["point_offset"][-1] + 1),  # layout
        lambda b: b["points"].__setitem__(slice(None), b["points"][::-1]),       # leaf contents
        lambda b: b["voxels"].__setitem__((0, 0), b["voxels"][0, 0] ^ 1),        # transposed cell bit
    ]
    for fn in plants:
        with pytest.raises(AssertionError):
            check(pts, mutated(fn), 12, 0, 21)


@pytest.mark.parametrize("mode", [1, 3, 4])
def test_bruteforce_pick_catches_wrong_argmin(mode):
    pts = synth.sphere(600, seed=12)
    good = oracle.build(pts, 10, mode)
    check(pts, good, 10, mode, 21)
    bad = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in good.items()}
    # find a voxel with >= 2 members and replace the pick by another member
    v = bad["voxels"]
    i = int(np.nonzero(v[:, 2] >= 2)[0][0])
    node = int(np.nonzero((bad["voxel_offset"] <= i) & (i < bad["voxel_offset"] + bad["voxel_count"]))[0][0])
    L = int(bad["log2_size"][node])
    d = pts[:, :3].astype(np.int64) - bad["min"][node].astype(np.int64)
    s = 1 << L
    inside = np.all((d >= 0) & (d < s), axis=1)
    q = (d * 128) // s
    cell = q[:, 0] + 128 * q[:, 1] + 16384 * q[:, 2]
    members = np.nonzero(inside & (cell == v[i, 0]))[0]
    other = [m for m in members.tolist() if m != v[i, 3]][0]
    v[i, 3] = other
    v[i, 1] = int(pts[other, 3]) & 0xFFFFFFFF
    with pytest.raises(AssertionError):
        check(pts, bad, 10, mode, 21)
    assert splitmix64_py(0) == 0xE220A8397B1DCDAF


def _in_cube(pts, mn, lg):
    d = pts[:, :3].astype(np.int64) - np.asarray(mn, np.int64)
    return np.all((d >= 0) & (d < (1 << int(lg))), axis=1)


@pytest.mark.parametrize("seed", range(6))
def test_cube_voxels_equals_every_inner_node(seed):
    # the single-cube entry point (used to check nodes of builds too large for
    # the whole-cloud oracle) gives each inner node's voxels from the points of
    # its cube and their input indices, in any row order
    rng = np.random.default_rng(2000 + seed)
    n = int(rng.integers(50, 600))
    pts = _random_cloud(rng, n, int(rng.integers(3, 20)))
    T = int(rng.integers(2, 30))
    for mode in (0, 1):
        r = oracle.build(pts, T, mode)
        inner = np.nonzero((r["flags"] & 1) == 0)[0]
        for i in inner:
            sel = np.nonzero(_in_cube(pts, r["min"][i], r["log2_size"][i]))[0]
            perm = rng.permutation(len(sel))
            got = oracle.cube_voxels(pts[sel[perm]], sel[perm], r["min"][i], r["log2_size"][i], mode)
            a, c = int(r["voxel_offset"][i]), int(r["voxel_count"][i])
            assert np.array_equal(got, r["voxels"][a:a + c]), (mode, i)


def test_cube_voxels_rejects_points_outside():
    pts = P([(0, 0, 0, 1, 2, 3), (8, 0, 0, 1, 2, 3)])
    with pytest.raises(ValueError):
        oracle.cube_voxels(pts, np.arange(2), (0, 0, 0), 3, 0)


# ------------------------------------------------------------------ golden
# Hand-derived worked examples (tests/golden/): the oracle reproduces every
# node, leaf and voxel in both modes.


@pytest.mark.parametrize("path,mode", golden.cases(),
                         ids=lambda v: v.rsplit("/", 1)[-1] if isinstance(v, str) else str(v))
def test_oracle_reproduces_hand_worked_examples(path, mode):
    fx = golden.load(path)
    res = oracle.build(fx["input"], fx["T"], mode, fx["max_depth"])
    golden.check(res, fx, mode)


def test_golden_check_catches_planted_mistakes():
    # a wrong rounding, a dropped count and a wrong pick are all caught
    fx = golden.load(golden.fixtures()[0])
    res = oracle.build(fx["input"], fx["T"], 0, fx["max_depth"])
    for mutate in (lambda v: v.__setitem__((0, 1), v[0, 1] + 1), lambda v: v.__setitem__((0, 2), v[0, 2] - 1),
                   lambda v: v.__setitem__((0, 3), 7)):
        bad = dict(res)
        bad["voxels"] = np.array(res["voxels"], copy=True).reshape(-1, 4)
        mutate(bad["voxels"])
        with pytest.raises(AssertionError):
            golden.check(bad, fx, 0)


# ----------------------------------------------- neighbourhood-weighted mode
# Pins of the oracle's neighbourhood-weighted average (Section 4.2.4, mode
# 2), beside the hand-worked examples above.


def clustered_corner_cloud(L, seed, n_clusters=8, per=60, box=6):
    """Points on integer positions of a cube of edge 2^L (L <= 7), in small
    clusters spread over all eight octants so that the root is inner and
    all its children are leaves (T = 100)."""
    rng = np.random.default_rng(seed)
    edge = 1 << L
    half = edge // 2
    rows = [(0, 0, 0), (edge - 1, edge - 1, edge - 1)]  # fix the cube
    for k in range(n_clusters):
        o = np.array([(k >> 2) & 1, (k >> 1) & 1, k & 1]) * half
        c = o + rng.integers(0, half - box, size=3)
        rows += [tuple(int(t) for t in c + rng.integers(0, box, size=3)) for _ in range(per)]
    xyz = np.array(rows, np.int64)
    col = rng.integers(0, 256, size=(len(rows), 3))
    return P(np.concatenate([xyz, col], axis=1))


def check_corner_means(pts, res, L):
    """The root's weighted voxels against the corner rule (see the test
    below): cells, colours (rounded half up; either neighbour on an exact
    half, where the double-precision sum may fall on either side) and
    counts.  Returns the number of cells with more than one sample."""
    scale = 1 << (7 - L)
    g = (pts[:, :3].astype(np.int64) - res["min"][0]) * scale
    rgb = np.stack([(pts[:, 3].view(np.uint32) >> s) & 255 for s in (0, 8, 16)], axis=1).astype(np.int64)
    by_pos = {}
    for pos, c in zip(map(tuple, g), rgb):
        by_pos.setdefault(pos, []).append(c)
    a, n = int(res["voxel_offset"][0]), int(res["voxel_count"][0])
    vox = res["voxels"][a:a + n]
    assert set(int(v) for v in vox[:, 0]) == {x | y << 7 | z << 14 for x, y, z in by_pos}
    multi = 0
    for cell, rgba, cnt, pick in vox:
        j = (int(cell) & 127, (int(cell) >> 7) & 127, int(cell) >> 14)
        samples = [c for d in np.ndindex(2, 2, 2) for c in by_pos.get(tuple(j[i] + d[i] for i in range(3)), [])]
        k = len(samples)
        multi += k > 1
        s = np.sum(samples, axis=0)
        got = [(int(rgba) >> sh) & 255 for sh in (0, 8, 16)]
        for ch in range(3):
            up = (2 * int(s[ch]) + k) // (2 * k)  # s / k rounded half up
            ok = {up, up - 1} if k > 1 and (2 * int(s[ch])) % (2 * k) == k else {up}
            assert got[ch] in ok, (j, ch, got[ch], s[ch], k)
        assert int(rgba) >> 24 == 255 and int(pick) == NONE
        assert int(cnt) == len(by_pos[j])
    return multi


@pytest.mark.parametrize("L", [7, 6])
def test_weighted_on_cell_corners_is_the_mean_of_the_corner_samples(L):
    """On a cube of edge <= 128 every point sits on a grid-cell corner, at
    distance sqrt(3)/2 from the centres of the eight cells sharing that
    corner (and farther than one cell from all others), so every weight is
    the same and an occupied cell's colour is the plain mean of the samples
    on its eight corners, rounded half up.  The cell a point lies in is the
    one whose lowest corner it is."""
    pts = clustered_corner_cloud(L, seed=40 + L)
    res = oracle.build(pts, 100, 2, 21)
    assert res["flags"][0] == 0 and np.all(res["flags"][1:] & 1 == 1)  # root inner, children leaves
    assert check_corner_means(pts, res, L) > 20  # the cloud does exercise shared corners


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_weighted_cells_and_counts_equal_the_average_modes(seed):
    """Occupancy and counts do not depend on the colour rule: an inner
    node's occupied cells are the cells holding its points (a child voxel's
    centre lies in the parent cell that nests the child cell), so every
    node's cells and counts equal those of the cell average, over trees
    several levels deep."""
    pts = synth.sphere(20_000, seed=seed, radius_log2=11)
    avg = oracle.build(pts, 300, 0, 21)
    wtd = oracle.build(pts, 300, 2, 21)
    assert avg["level"].max() >= 3
    for k in ("min", "level", "log2_size", "child_mask", "flags", "parent", "first_child",
              "point_offset", "point_count", "voxel_count"):
        assert np.array_equal(avg[k], wtd[k]), k
    for i in np.nonzero((avg["flags"] & 1) == 0)[0]:
        a, b = int(avg["voxel_offset"][i]), int(wtd["voxel_offset"][i])
        c = int(avg["voxel_count"][i])
        assert np.array_equal(avg["voxels"][a:a + c][:, [0, 2]], wtd["voxels"][b:b + c][:, [0, 2]])


def test_weighted_constant_colour_and_bounds():
    """A weighted mean of one colour is that colour at every level; with
    random colours every voxel channel stays within the input's range."""
    pts = synth.sphere(8_000, seed=9, radius_log2=9)
    const = pts.copy()
    const[:, 3] = synth.pack_rgba(np.full(len(pts), 17), np.full(len(pts), 200), np.full(len(pts), 93))
    res = oracle.build(const, 150, 2, 21)
    assert len(res["voxels"]) > 0 and np.all(res["voxels"][:, 1] == np.uint32(const[0, 3].view(np.uint32)))
    res = oracle.build(pts, 150, 2, 21)
    u = pts[:, 3].view(np.uint32)
    for sh in (0, 8, 16):
        ch = (res["voxels"][:, 1] >> sh) & 255
        src = (u >> sh) & 255
        assert ch.min() >= src.min() and ch.max() <= src.max()
    assert np.all(res["voxels"][:, 3] == NONE)


def test_weighted_check_catches_planted_mistakes():
    """The corner rule rejects plausible mistakes, planted in copies of a
    correct result: a colour off by one in a cell with several samples, a
    wrong count, a cell moved by one."""
    pts = clustered_corner_cloud(7, seed=47)
    res = oracle.build(pts, 100, 2, 21)
    a, n = int(res["voxel_offset"][0]), int(res["voxel_count"][0])
    g = pts[:, :3].astype(np.int64) - res["min"][0]  # edge 128: grid position = offset
    shared = []
    for r in range(a, a + n):
        c = int(res["voxels"][r, 0])
        j = np.array([c & 127, (c >> 7) & 127, c >> 14])
        if np.sum(np.all((g - j >= 0) & (g - j <= 1), axis=1)) > 1:
            shared.append(r)
    assert shared
    r = shared[0]
    for mutate in (lambda v: v.__setitem__((r, 1), v[r, 1] ^ 1), lambda v: v.__setitem__((r, 2), v[r, 2] + 1),
                   lambda v: v.__setitem__((r, 0), v[r, 0] ^ 1)):
        bad = dict(res)
        bad["voxels"] = np.array(res["voxels"], copy=True)
        mutate(bad["voxels"])
        with pytest.raises(AssertionError):
            check_corner_means(pts, bad, 7)


# ------------------------------------------------- random (Listing 1 key)

def test_random_key_layout_from_published_splitmix64():
    # Listing 1: key = (random & 0xfff00000) | (index & 0x000fffff).  The
    # random number of index i at level l is the high half of
    # splitmix64(l << 32 | i); for level 0 and i = 0 that is the published
    # seed-0 output 0xe220a8397b1dcdaf, whose high half 0xe220a839 keeps
    # 0xe22 as its top 12 bits.
    assert oracle.random_key(0, 0) == (0xE2200000 << 32) | 0
    # the high 12 bits come from the random number, the low 20 from the index
    # (which also breaks ties below the 32-bit key)
    i = (5 << 20) | 0x12345
    k = oracle.random_key(i, 7)
    assert (k >> 32) & 0xFFFFF == 0x12345 and k & 0xFFFFFFFF == i
    assert (k >> 52) == splitmix64_py((7 << 32) | i) >> 52


def test_random_cells_and_counts_equal_the_average_modes():
    pts = synth.indoor(60_000, seed=8, n_prims=16)
    a = oracle.build(pts, 700, 0)
    b = oracle.build(pts, 700, 4)
    for k in ("min", "level", "log2_size", "child_mask", "flags", "parent", "first_child",
              "point_offset", "point_count", "voxel_count"):
        assert np.array_equal(a[k], b[k]), k
    # per node (the bottom-up mode lays its node blocks out in another order)
    for i in np.nonzero(a["voxel_count"])[0]:
        va = a["voxels"][int(a["voxel_offset"][i]):][: int(a["voxel_count"][i])]
        vb = b["voxels"][int(b["voxel_offset"][i]):][: int(b["voxel_count"][i])]
        assert np.array_equal(va[:, [0, 2]], vb[:, [0, 2]]), i
    # every pick is a member point of its cell with that point's colour
    assert np.array_equal(b["voxels"][:, 1], pts[b["voxels"][:, 3].astype(np.int64), 3].view(np.uint32))


def test_random_is_drawn_bottom_up_not_top_down():
    # children's winners compete again with fresh random bits: on a tree a
    # few levels deep some cell of the root keeps another point than a
    # single draw over all of the cell's points would
    pts = synth.sphere(20_000, seed=9)
    r = oracle.build(pts, 200, 4)
    root = r["voxels"][int(r["voxel_offset"][0]):][: int(r["voxel_count"][0])]
    d = pts[:, :3].astype(np.int64) - r["min"][0].astype(np.int64)
    q = (d * 128) >> int(r["log2_size"][0])
    cell = q[:, 0] + 128 * q[:, 1] + 16384 * q[:, 2]
    differ = 0
    for row in root:
        members = np.nonzero(cell == row[0])[0]
        top_down = max(members.tolist(), key=lambda p: random_key_py(p, 0))
        differ += int(top_down != row[3])
    assert differ > 0


def test_random_checker_catches_a_top_down_draw():
    pts = synth.sphere(3000, seed=10)
    good = oracle.build(pts, 40, 4)
    check(pts, good, 40, 4, 21)
    bad = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in good.items()}
    d = pts[:, :3].astype(np.int64) - good["min"][0].astype(np.int64)
    q = (d * 128) >> int(good["log2_size"][0])
    cell = q[:, 0] + 128 * q[:, 1] + 16384 * q[:, 2]
    changed = 0
    o = int(good["voxel_offset"][0])  # the root's block (laid out last when filled bottom up)
    for j in range(o, o + int(good["voxel_count"][0])):
        members = np.nonzero(cell == bad["voxels"][j, 0])[0]
        top_down = max(members.tolist(), key=lambda p: random_key_py(p, 0))
        if top_down != bad["voxels"][j, 3]:
            bad["voxels"][j, 3] = top_down
            bad["voxels"][j, 1] = int(pts[top_down, 3]) & 0xFFFFFFFF
            changed += 1
    assert changed > 0
    with pytest.raises(AssertionError):
        check(pts, bad, 40, 4, 21)


# -------------------------------------- weighted average, one node at a time

@pytest.mark.parametrize("seed", [4, 5])
def test_weighted_node_entry_point_equals_every_inner_node(seed):
    # the per-node entry point (used to check CUDA results node by node on
    # their own children's samples) gives exactly the voxels the weighted
    # build computed for every inner node, on trees several levels deep
    import weighted
    pts = synth.sphere(15_000, seed=seed, radius_log2=12)
    res = oracle.build(pts, 200, 2, 21)
    assert res["level"].max() >= 3
    total, exact = weighted.per_node_check(res, tol=0)
    assert total > 0 and exact == total


def test_weighted_node_rejects_points_outside_the_cube():
    with pytest.raises(ValueError):
        oracle.weighted_node(P([(300, 0, 0, 1, 2, 3)]), np.zeros((0, 4), np.uint32), np.zeros(0, np.uint8),
                             [0, 0, 0], 8)
