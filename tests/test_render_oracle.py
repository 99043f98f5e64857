"""CPU pins of the rasteriser oracle (rendering of Section 5, oracle/
render_oracle.cpp): pixel positions and keys worked out by hand on cameras
whose arithmetic is exact (power-of-two scales), the depth test, clipping,
the node selection's closed form on an orthographic view, the child-octant
voxel discard, and a whole image against an independent numpy splat."""
import numpy as np
import pytest

import oracle
from paper_2302_14801_gb300 import camera, synth

ONE = np.float32(1.0).view(np.uint32)


def ortho_box(lo, size):
    """Orthographic view of the cube [lo, lo + size)^3 from +z (power-of-two
    size: every scale factor is exact)."""
    m, org = camera.orthographic(np.asarray(lo, float), np.asarray(lo, float) + size)
    return m, org


def single(points, cells=()):
    """A one-leaf 'octree' holding the given points (rows x, y, z, rgba)."""
    pts = np.asarray(points, dtype=np.int64).reshape(-1, 4).astype(np.uint32).view(np.int32)
    return {"min": np.zeros((1, 3), np.int32), "level": np.zeros(1, np.uint8), "log2_size": np.array([8], np.uint8),
            "child_mask": np.zeros(1, np.uint8), "flags": np.ones(1, np.uint8),
            "parent": np.array([0xFFFFFFFF], np.uint32), "first_child": np.array([0xFFFFFFFF], np.uint32),
            "point_offset": np.zeros(1, np.uint64), "point_count": np.array([len(pts)], np.uint64),
            "voxel_offset": np.zeros(1, np.uint64), "voxel_count": np.zeros(1, np.uint32),
            "voxels": np.zeros((0, 4), np.uint32), "points": pts}


def depth_bits(d):
    return int(np.float32(d).view(np.uint32))


def test_pixel_and_key_by_hand():
    # box [0, 256)^3 onto 128 x 128 pixels: one pixel = 2 units.  x = 75:
    # ndc = 75 * 2/256 - 1 = -0.4140625, pixel floor((ndc/2 + 1/2) * 128)
    # = floor(37.5) = 37; y = 200: ndc = 0.5625, pixel floor(100) = 100.
    # depth: z = 64 -> ndc z = -(64 * 2/256 - 1) = 0.5, depth 0.75.
    m, org = ortho_box([0, 0, 0], 256)
    fb, vis, drawn = oracle.render(single([(75, 200, 64, 0xFF112233)]), m, org, 128, 128)
    assert drawn == 1 and vis.tolist() == [1]
    want = (depth_bits(0.75) << 32) | 0xFF112233
    assert int(fb[100, 37]) == want
    assert int((fb != np.uint64(2**64 - 1)).sum()) == 1


def test_nearer_sample_wins_then_smaller_colour():
    m, org = ortho_box([0, 0, 0], 256)
    pts = [(10, 10, 100, 5), (10, 10, 120, 9), (11, 11, 120, 3), (40, 40, 7, 8), (40, 40, 7, 6)]
    fb, _, drawn = oracle.render(single(pts), m, org, 128, 128)
    assert drawn == 5
    # (10,10) and (11,11) share pixel (5, 5); z = 120 is nearer (smaller
    # depth 1 - 120/256, since ndc z = 1 - 2 * 120/256), colour 3 < 9
    assert int(fb[5, 5]) == (depth_bits(np.float32(1 - 120 / 256)) << 32) | 3
    assert int(fb[20, 20]) == (depth_bits(np.float32(1 - 7 / 256)) << 32) | 6


def test_points_outside_or_behind_are_dropped():
    m, org = ortho_box([0, 0, 0], 256)
    fb, _, drawn = oracle.render(single([(300, 10, 10, 1), (10, -5, 10, 2), (10, 10, 400, 3)]), m, org, 64, 64)
    assert drawn == 0 and np.all(fb == np.uint64(2**64 - 1))
    # a perspective camera looking along +x from x = 128: points behind it vanish
    m, org = camera.perspective((128, 128, 128), (1000, 128, 128), fovy_deg=90, aspect=1, near=1, far=1e4)
    fb, _, drawn = oracle.render(single([(50, 128, 128, 1), (200, 128, 128, 2)]), m, org, 32, 32)
    assert drawn == 1 and int(fb[16, 16]) & 0xFFFFFFFF == 2


def test_node_selection_closed_form():
    # an orthographic view of exactly the root cube on 1024 x 1024 pixels:
    # a node of level k spans 1024 / 2^k pixels, so with the threshold 100
    # levels 0-3 are refined (1024, 512, 256, 128 > 100) and level 4 (64)
    # is not: the drawn nodes are those of levels <= 4, and the samples
    # drawn are the level-4 inner nodes' voxels and the points of leaves at
    # levels <= 4 (refined nodes' voxels all lie in octants of drawn
    # children)
    pts = synth.sphere(60_000, seed=3, radius_log2=12)
    res = oracle.build(pts, 60, 0, 21)
    assert res["level"].max() >= 5  # some nodes lie below the drawn levels
    L = int(res["log2_size"][0])
    m, org = ortho_box(res["min"][0], 1 << L)
    fb, vis, drawn = oracle.render(res, m, org, 1024, 1024, 100.0)
    assert np.array_equal(vis.astype(bool), res["level"] <= 4)
    leaf = (res["flags"] & 1) == 1
    want = int(res["voxel_count"][(res["level"] == 4) & ~leaf].astype(np.int64).sum()) + \
        int(res["point_count"][(res["level"] <= 4) & leaf].astype(np.int64).sum())
    assert drawn == want


def test_octant_discard_keeps_voxels_of_undrawn_children():
    # a camera seeing only one octant of the root: the root is drawn and
    # refined, only its children inside the view are drawn, and the root's
    # voxels of the other octants are drawn in their place
    pts = synth.sphere(40_000, seed=4, radius_log2=12)
    res = oracle.build(pts, 2000, 0, 21)
    L = int(res["log2_size"][0])
    lo = res["min"][0].astype(np.int64)
    half = 1 << (L - 1)
    # the low-x, low-y quarter (a little inside it: a box touching the
    # frustum's side counts as inside)
    m, org = camera.orthographic(lo + [0, 0, 0], lo + [half - 2, half - 2, 2 * half])
    fb, vis, drawn = oracle.render(res, m, org, 256, 256, 100.0)
    kids = [int(res["first_child"][0]) + r for r in range(bin(int(res["child_mask"][0])).count("1"))]
    octs = [int(4 * (res["min"][k][0] != lo[0]) + 2 * (res["min"][k][1] != lo[1]) + (res["min"][k][2] != lo[2]))
            for k in kids]
    drawn_octs = {o for o, k in zip(octs, kids) if vis[k]}
    assert vis[0] and drawn_octs and drawn_octs <= {0, 1}
    assert all(not vis[k] for o, k in zip(octs, kids) if o not in (0, 1))


def numpy_splat(samples, rgba, m, org, w, h):
    """The projection written out with numpy float32 (each operation rounded
    on its own), independent of the oracle's code."""
    m = np.asarray(m, np.float32).reshape(4, 4)
    p = (samples.astype(np.int64) - np.asarray(org, np.int64)).astype(np.float32)
    c = []
    for i in range(4):
        s = m[i, 0] * p[:, 0]
        s = s + m[i, 1] * p[:, 1]
        s = s + m[i, 2] * p[:, 2]
        s = s + m[i, 3]
        c.append(s)
    x, y, z, ww = c
    ok = ww > 0
    nx, ny, nz = x / ww, y / ww, z / ww
    ok &= (nx >= -1) & (nx <= 1) & (ny >= -1) & (ny <= 1) & (nz >= -1) & (nz <= 1)
    px = np.minimum(np.floor((nx * np.float32(0.5) + np.float32(0.5)) * np.float32(w)), w - 1)
    py = np.minimum(np.floor((ny * np.float32(0.5) + np.float32(0.5)) * np.float32(h)), h - 1)
    dep = nz * np.float32(0.5) + np.float32(0.5)
    key = (dep.view(np.uint32).astype(np.uint64) << np.uint64(32)) | rgba.astype(np.uint64)
    fb = np.full(h * w, np.uint64(2**64 - 1))
    idx = (py[ok].astype(np.int64) * w + px[ok].astype(np.int64))
    np.minimum.at(fb, idx, key[ok])
    return fb.reshape(h, w), int(ok.sum())


def test_root_only_image_matches_numpy_splat():
    # threshold above the root's size: only the root is drawn, all its
    # voxels at their cell centres; a perspective camera
    pts = synth.sphere(30_000, seed=5, radius_log2=13)
    res = oracle.build(pts, 3000, 1, 21)
    L = int(res["log2_size"][0])
    c = res["min"][0].astype(np.int64) + (1 << (L - 1))
    m, org = camera.perspective(c + [3 << L, 1 << L, 2 << L], c, fovy_deg=40, aspect=1.25, near=1, far=1e7)
    fb, vis, drawn = oracle.render(res, m, org, 160, 128, 1e9)
    assert vis.sum() == 1 and vis[0]
    a, n = int(res["voxel_offset"][0]), int(res["voxel_count"][0])
    v = res["voxels"][a:a + n]
    q = np.stack([v[:, 0] & 127, (v[:, 0] >> 7) & 127, v[:, 0] >> 14], 1).astype(np.int64)
    # centres at min + (2 q + 1) 2^(L - 8): relative to the origin in float32
    lo = (res["min"][0].astype(np.int64) - org.astype(np.int64)).astype(np.float32)
    cen = lo + (2 * q + 1).astype(np.float32) * np.float32(2.0 ** (L - 8))
    # project the float centres directly (they are already relative to the origin)
    mm = np.asarray(m, np.float32).reshape(4, 4)
    cols = []
    for i in range(4):
        s = mm[i, 0] * cen[:, 0]
        s = s + mm[i, 1] * cen[:, 1]
        s = s + mm[i, 2] * cen[:, 2]
        s = s + mm[i, 3]
        cols.append(s)
    x, y, z, w = cols
    ok = w > 0
    nx, ny, nz = x / w, y / w, z / w
    ok &= (np.abs(nx) <= 1) & (np.abs(ny) <= 1) & (np.abs(nz) <= 1)
    px = np.minimum(np.floor((nx * np.float32(0.5) + np.float32(0.5)) * np.float32(160)), 159).astype(np.int64)
    py = np.minimum(np.floor((ny * np.float32(0.5) + np.float32(0.5)) * np.float32(128)), 127).astype(np.int64)
    dep = (nz * np.float32(0.5) + np.float32(0.5)).astype(np.float32)
    key = (dep.view(np.uint32).astype(np.uint64) << np.uint64(32)) | v[:, 1].astype(np.uint64)
    want = np.full(128 * 160, np.uint64(2**64 - 1))
    np.minimum.at(want, py[ok] * 160 + px[ok], key[ok])
    assert drawn == int(ok.sum()) > 1000
    assert np.array_equal(fb, want.reshape(128, 160))


def test_points_image_matches_numpy_splat():
    pts = synth.aerial(20_000, seed=6, n_buildings=5)
    res = single([])
    res["points"] = pts
    res["point_count"] = np.array([len(pts)], np.uint64)
    res["log2_size"] = np.array([25], np.uint8)
    res["min"] = pts[:, :3].min(axis=0).reshape(1, 3).astype(np.int32)
    c = pts[:, :3].astype(np.int64).mean(axis=0)
    m, org = camera.perspective(c + [0, -(1 << 24), 1 << 22], c, fovy_deg=50, aspect=1.5, near=10, far=1e9)
    fb, _, drawn = oracle.render(res, m, org, 300, 200, 100.0)
    want, n_ok = numpy_splat(pts[:, :3], pts[:, 3].view(np.uint32), m, org, 300, 200)
    assert drawn == n_ok > 1000
    assert np.array_equal(fb, want)
