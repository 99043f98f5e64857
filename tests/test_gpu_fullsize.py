"""GPU parity at the benchmark's full size: the 50M-point aerial cloud built
exactly as bench.py times it (lod.build on the current stream, T = 50k,
max_depth 21, default tuning), both modes, compared with the oracle over
the whole result (node table, every leaf's point multiset, indices, every
voxel), plus the size-independent invariants of the tree."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from compare import compare
from paper_2302_14801_gb300 import synth

pytestmark = pytest.mark.gpu

N = 50_000_000
T = 50_000


@pytest.fixture(scope="module")
def lod():
    import torch
    from paper_2302_14801_gb300 import _build_ext
    _build_ext.build()
    from paper_2302_14801_gb300 import lod as m
    torch.cuda.set_device(0)
    return m


@pytest.fixture(scope="module")
def aerial():
    return synth.aerial(N, seed=2)


def invariants(res, n):
    leaf = (res["flags"] & 1) == 1
    inner = ~leaf
    cnt = res["point_count"].astype(np.int64)
    # every point in exactly one leaf: leaf ranges tile [0, n)
    off = res["point_offset"].astype(np.int64)[leaf]
    o = np.argsort(off)
    ends = off[o] + cnt[leaf][o]
    assert off[o][0] == 0 and ends[-1] == n and np.array_equal(off[o][1:], ends[:-1])
    assert np.all((res["flags"][leaf & (cnt > T)] & 2) == 2)  # only capped leaves exceed T
    assert np.all(cnt[inner] > T)
    # a parent's points are its children's, and its voxels count them all
    par = res["parent"].astype(np.int64)
    sums = np.zeros(len(cnt), np.int64)
    np.add.at(sums, par[1:], cnt[1:])
    assert np.array_equal(sums[inner], cnt[inner])
    vox = res["voxels"].reshape(-1, 4)
    for i in np.nonzero(inner)[0][:64]:
        a, c = int(res["voxel_offset"][i]), int(res["voxel_count"][i])
        assert int(vox[a:a + c, 2].astype(np.int64).sum()) == cnt[i]


def test_aerial_50m_full_parity_all_modes(lod, aerial):
    # filtered, pick, first come and random, each against the whole-cloud
    # oracle (the oracle builds run side by side on the host cores)
    import torch
    modes = (0, 1, 3, 4)
    with ThreadPoolExecutor(len(modes)) as ex:
        futs = {m: ex.submit(oracle.build, aerial, T, m, 21) for m in modes}
        d = torch.from_numpy(aerial).cuda()
        for m in modes:
            r = lod.build(d, T, m, 21, stream=torch.cuda.current_stream())
            got = r.to_host()
            r.free()
            invariants(got, N)
            compare(got, futs[m].result(), inp=aerial)
        del d


# --------------------------------------------------------------------------
# Filtered colour sums of items whose cube holds more than 0xFFFFFFFF / 255
# = 16,843,009 points take 64-bit lanes in the voxel pass (32-bit lanes
# could overflow there).  17.5M points uniform in a 2^15 cube in one corner
# of a 2^22 root (a far point sets the extent) put all of them into one
# cell of the root's grid, whose channel sums exceed 2^32: with max_depth 1
# the item is an overfull leaf (points read directly), with max_depth 21 a
# chain of single-child inner nodes (child voxels merged with wide sums).

def wide_cloud():
    rng = np.random.default_rng(4242)
    n = 17_500_000
    pts = np.empty((n + 1, 4), np.int32)
    pts[:n, :3] = rng.integers(0, 1 << 15, size=(n, 3), dtype=np.int32)
    r = np.full(n, 255)
    g = 255 - rng.integers(0, 3, size=n)
    b = 200 + rng.integers(0, 56, size=n)
    pts[:n, 3] = synth.pack_rgba(r, g, b)
    pts[n] = (1 << 21, 1 << 21, 1 << 21, int(synth.pack_rgba(np.array([1]), np.array([2]), np.array([3]))[0]))
    return pts


@pytest.mark.parametrize("max_depth", [1, 21])
def test_filtered_wide_sums_against_oracle(lod, max_depth):
    import torch
    pts = wide_cloud()
    with ThreadPoolExecutor(1) as ex:
        fut = ex.submit(oracle.build, pts, T, 0, max_depth)
        d = torch.from_numpy(pts).cuda()
        r = lod.build(d, T, 0, max_depth, stream=torch.cuda.current_stream())
        got = r.to_host()
        r.free()
        want = fut.result()
    root = want["voxels"][: int(want["voxel_count"][0])]
    assert int(root[:, 2].max()) == len(pts) - 1  # one root cell holds all corner points
    compare(got, want, inp=pts)


# --------------------------------------------------------------------------
# A whole-cloud comparison beyond the 50M aerial cloud: 100M points of the
# indoor recipe (numpy generator), both modes, at the bench's settings.  Its
# log-normal clusters need refinement rounds and its deep volumetric levels
# hold more occupied cells per octant than one accumulate pass, so items take
# several rank ranges: the paths the 1B build takes.

@pytest.fixture(scope="module")
def indoor100m():
    return synth.indoor(100_000_000, seed=3)


def test_indoor_100m_full_parity_both_modes(lod, indoor100m):
    import torch
    pts = indoor100m
    with ThreadPoolExecutor(2) as ex:
        futs = {mode: ex.submit(oracle.build, pts, T, mode, 21) for mode in (0, 1)}
        d = torch.from_numpy(pts).cuda()
        got = {}
        for mode in (0, 1):
            r = lod.build(d, T, mode, 21, stream=torch.cuda.current_stream())
            got[mode] = r.to_host()
            r.free()
        del d
        for mode in (0, 1):
            invariants(got[mode], len(pts))
            compare(got[mode], futs[mode].result(), inp=pts)


# --------------------------------------------------------------------------
# The billion-point indoor scan (drawn on the device with the same recipe as
# synth.indoor), built exactly as the bench times it.  The whole-cloud oracle
# would take tens of minutes, so every node is checked against the tree's
# size-independent invariants and sampled nodes against the oracle one by
# one: inner nodes through the single-cube oracle (the cube's points and
# their input indices gathered on the device), leaves by their point
# multiset.

N1B = 1_000_000_000


@pytest.fixture(scope="module")
def indoor1b():
    from paper_2302_14801_gb300 import synth_gpu
    return synth_gpu.indoor(N1B, seed=3)


def cube_points(dev_pts, mn, lg):
    import torch
    lo = torch.tensor([int(v) for v in mn], dtype=torch.int64, device=dev_pts.device)
    d = dev_pts[:, :3].to(torch.int64) - lo
    inside = ((d >= 0) & (d < (1 << int(lg)))).all(dim=1)
    idx = torch.nonzero(inside).squeeze(1)
    return dev_pts[idx].cpu().numpy(), idx.cpu().numpy().astype(np.uint32)


def sorted_rows(a):
    a = np.asarray(a)
    return a[np.lexsort(a.T[::-1])]


def check_cube_nodes(got, dev_pts, mode, nodes):
    """Inner nodes of a large build against the single-cube oracle, several
    at a time (the oracle releases the GIL)."""
    vox = got["voxels"].reshape(-1, 4)
    jobs = []
    with ThreadPoolExecutor(4) as ex:
        for i in nodes:
            pts, idx = cube_points(dev_pts, got["min"][i], got["log2_size"][i])
            assert len(pts) == int(got["point_count"][i])
            jobs.append((i, ex.submit(oracle.cube_voxels, pts, idx, got["min"][i], got["log2_size"][i], mode)))
        for i, f in jobs:
            a, c = int(got["voxel_offset"][i]), int(got["voxel_count"][i])
            have = vox[a:a + c]
            have = have[np.argsort(have[:, 0], kind="stable")]
            assert np.array_equal(have, f.result()), f"node {i}"


def check_sampled_nodes(got, dev_pts, mode, rng, n_inner=6, n_leaf=6, max_pts=3_000_000):
    cnt = got["point_count"].astype(np.int64)
    leaf = (got["flags"] & 1) == 1
    inner_ok = np.nonzero(~leaf & (cnt <= max_pts))[0]
    leaf_ok = np.nonzero(leaf & (cnt > 0))[0]
    picks = list(rng.choice(inner_ok, size=min(n_inner, len(inner_ok)), replace=False))
    picks.append(int(inner_ok[np.argmax(cnt[inner_ok])]))  # the largest checkable inner node
    vox = got["voxels"].reshape(-1, 4)
    for i in picks:
        pts, idx = cube_points(dev_pts, got["min"][i], got["log2_size"][i])
        assert len(pts) == cnt[i]
        want = oracle.cube_voxels(pts, idx, got["min"][i], got["log2_size"][i], mode)
        a, c = int(got["voxel_offset"][i]), int(got["voxel_count"][i])
        have = vox[a:a + c]
        have = have[np.argsort(have[:, 0], kind="stable")]
        assert np.array_equal(have, want), f"node {i}"
    for i in rng.choice(leaf_ok, size=min(n_leaf, len(leaf_ok)), replace=False):
        pts, idx = cube_points(dev_pts, got["min"][i], got["log2_size"][i])
        a, c = int(got["point_offset"][i]), int(got["point_count"][i])
        assert np.array_equal(sorted_rows(got["points"][a:a + c]), sorted_rows(pts)), f"leaf {i}"
        if got.get("index") is not None:
            assert np.array_equal(np.sort(got["index"][a:a + c]), np.sort(idx)), f"leaf {i} indices"


@pytest.mark.parametrize("mode", [0, 1])
def test_indoor_1b_invariants_and_sampled_nodes(lod, indoor1b, mode):
    import torch
    r = lod.build(indoor1b, T, mode, 21, stream=torch.cuda.current_stream())
    got = r.to_host()
    r.free()
    invariants(got, N1B)
    check_sampled_nodes(got, indoor1b, mode, np.random.default_rng(77 + mode))
    # two level-1 nodes (each over 16.8M points: the filtered pass sums them
    # in 64-bit lanes): the smallest inner one and the largest
    lvl1 = np.nonzero((got["level"] == 1) & ((got["flags"] & 1) == 0))[0]
    cnt = got["point_count"][lvl1].astype(np.int64)
    pick = sorted({int(lvl1[np.argmin(cnt)]), int(lvl1[np.argmax(cnt)])})
    assert got["point_count"][pick].max() > 16_843_009
    check_cube_nodes(got, indoor1b, mode, pick)


# --------------------------------------------------------------------------
# Batched tiles as the bench builds them: the first wave (<= 1e9 points) of
# 2048 tiles with sizes log-uniform in [1e4, 2e7], each a sphere with its own
# seed and bbox, one lod_build_batched call, filtered mode.  Every tile of at
# most 3M points is compared with the whole-cloud oracle, every tile with
# the invariants.

def test_batched_first_wave_of_2048_tiles(lod):
    import torch
    from paper_2302_14801_gb300 import synth_gpu
    sizes = synth.tile_sizes(2048, 1e4, 2e7, seed=4)
    wave, acc = [], 0
    for t, m in enumerate(sizes):
        if wave and acc + int(m) > 1e9:
            break
        wave.append(t)
        acc += int(m)
    tiles = []
    for t in wave:
        off = np.random.default_rng((1000 + t) ^ 0x5EED).integers(0, (1 << 30) - (1 << 21), size=3)
        tiles.append(synth_gpu.sphere(int(sizes[t]), seed=1000 + t, offset=tuple(int(o) for o in off)))
    rs = lod.build_batched(tiles, T, 0, stream=torch.cuda.current_stream())
    check = [k for k in range(len(wave)) if sizes[wave[k]] <= 3_000_000]
    assert len(check) > 100
    with ThreadPoolExecutor(8) as ex:
        futs = {}
        for k in check:
            pts = tiles[k].cpu().numpy()
            futs[k] = (pts, ex.submit(oracle.build, pts, T, 0, 21))
        for k, r in enumerate(rs):
            got = r.to_host()
            r.free()
            invariants(got, int(sizes[wave[k]]))
            if k in futs:
                pts, f = futs.pop(k)
                compare(got, f.result(), inp=pts)


# --------------------------------------------------------------------------
# Serving at full request size: the 50M-point aerial cloud submitted while
# smaller requests are in flight gives the same octree as the plain call
# (which the full-size parity test above checks against the oracle).

def test_server_full_size_request_in_a_mix(lod, aerial):
    import torch
    d = torch.from_numpy(aerial).cuda()
    ref = lod.build(d, T, 1, 21)
    want = ref.to_host()
    ref.free()
    srv = lod.Server(120 * 10**9, 4)
    small = [d[:m] for m in (100_000, 2_000_000, 7_000_000)]
    tks = [srv.submit(x, T, 0) for x in small[:2]] + [srv.submit(d, T, 1)] + [srv.submit(small[2], T, 1)]
    res = [srv.wait(tk) for tk in tks]
    got = res[2].to_host()
    for r in res:
        r.free()
    srv.close()
    for k in ("min", "level", "log2_size", "child_mask", "flags", "parent", "first_child", "point_offset",
              "point_count", "voxel_count"):
        assert np.array_equal(got[k], want[k]), k
    compare(got, want, inp=aerial)
