"""GPU parity of the neighbourhood-weighted average (Section 4.2.4, mode 2).

Both sides take the weights in the kernel's precision (single precision,
every operation rounded on its own, rounded to multiples of 2^-24; the
paper fixes none), sum them exactly and round each mean half up in
integers, so the bar is bit-exact like the other modes:

* the whole result equals the oracle's weighted build (node table, leaf
  points, every voxel with its colour);
* node by node, every inner node equals the oracle evaluated on that
  node's own children in the CUDA result (so a mistake is located at the
  node where it happens, not at its ancestors);
* the hand-worked examples under tests/golden/ are reproduced, and two
  builds of one cloud are bit-identical.
"""
import numpy as np
import pytest

import oracle
import weighted
from compare import compare
from paper_2302_14801_gb300 import synth

pytestmark = pytest.mark.gpu

W = 2


@pytest.fixture(scope="module")
def lod():
    import torch
    from paper_2302_14801_gb300 import _build_ext
    _build_ext.build()
    from paper_2302_14801_gb300 import lod as m
    torch.cuda.set_device(0)
    return m


def gpu_build(lod, pts, T, max_depth=21):
    import torch
    d = torch.from_numpy(np.ascontiguousarray(pts, dtype=np.int32)).cuda()
    r = lod.build(d, T, W, max_depth)
    got = r.to_host()
    r.free()
    return got


def parity(lod, pts, T, max_depth=21):
    got = gpu_build(lod, pts, T, max_depth)
    total, exact = weighted.per_node_check(got, tol=0)
    assert exact == total
    compare(got, oracle.build(pts, T, W, max_depth), inp=pts)
    return got


def P(rows):
    a = np.asarray(rows, dtype=np.int64).reshape(-1, 6)
    out = np.empty((len(a), 4), np.int32)
    out[:, :3] = a[:, :3]
    out[:, 3] = synth.pack_rgba(a[:, 3], a[:, 4], a[:, 5])
    return out


def test_hand_worked_weighted_examples(lod):
    import golden
    cases = golden.cases(modes=(W,))
    assert len(cases) >= 2
    for path, m in cases:
        fx = golden.load(path)
        golden.check(gpu_build(lod, fx["input"], fx["T"], fx["max_depth"]), fx, m)


def test_edge_cases(lod):
    got = gpu_build(lod, np.zeros((0, 4), np.int32), 10)
    assert len(got["level"]) == 1 and got["flags"][0] == 1
    parity(lod, P([(5, -7, 9, 1, 2, 3)]), 1)
    parity(lod, P([(5, 5, 5, 1, 2, 3)] * 1000), 3)  # a chain of identical points to max_depth
    g = np.stack(np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij"), -1).reshape(-1, 3)
    rng = np.random.default_rng(3)
    rows = np.concatenate([g, rng.integers(0, 256, size=(512, 3))], axis=1)
    for T in (7, 64):  # cubes of edge <= 128: every point on a cell corner
        parity(lod, P(rows), T)


def test_full_int32_extent(lod):
    rng = np.random.default_rng(5)
    pts = np.empty((5000, 4), np.int32)
    pts[:, :3] = rng.integers(-(2**31), 2**31, size=(5000, 3))
    pts[0, :3] = -(2**31)
    pts[1, :3] = 2**31 - 1
    pts[:, 3] = rng.integers(-(2**31), 2**31, size=5000)
    got = parity(lod, pts, 40)
    assert got["log2_size"][0] == 32


@pytest.mark.parametrize("seed", range(8))
def test_random_tiny_deep_trees(lod, seed):
    rng = np.random.default_rng(9100 + seed)
    n = int(rng.integers(1, 2000))
    T = int(rng.integers(1, 17))
    max_depth = int(rng.choice([21, 3, 1, 6, 32]))
    kind = rng.integers(0, 2)
    if kind == 0:
        xyz = rng.integers(0, 2 ** int(rng.integers(1, 24)), size=(n, 3))
    else:
        c = rng.integers(0, 2**20, size=(4, 3))
        xyz = c[rng.integers(0, 4, size=n)] + rng.integers(0, 3, size=(n, 3))
    pts = np.empty((n, 4), np.int32)
    pts[:, :3] = xyz
    pts[:, 3] = rng.integers(-(2**31), 2**31, size=n)
    parity(lod, pts, T, max_depth)


def test_workload_shaped_clouds(lod):
    parity(lod, synth.sphere(1_000_000, seed=1), 50000)
    parity(lod, synth.aerial(2_000_000, seed=2, n_buildings=80), 3000)
    parity(lod, synth.indoor(3_000_000, seed=3, n_prims=256), 2000)


def test_volumetric_cloud(lod):
    rng = np.random.default_rng(31)
    pts = np.empty((400_000, 4), np.int32)
    pts[:, :3] = rng.integers(0, 1 << 16, size=(400_000, 3))
    pts[:, 3] = rng.integers(-(2**31), 2**31, size=400_000)
    parity(lod, pts, 20_000)


def test_deterministic_and_batched_equals_single(lod):
    import torch
    pts = synth.aerial(800_000, seed=7, n_buildings=30)
    a = gpu_build(lod, pts, 4000)
    b = gpu_build(lod, pts, 4000)
    compare(a, b)  # bit-identical, colours included
    sizes = [0, 1, 4097, 30_000, 250_000, 60_000]
    tiles = [synth.sphere_tile(int(n), seed=300 + i) for i, n in enumerate(sizes)]
    rs = lod.build_batched([torch.from_numpy(t).cuda() for t in tiles], 20000, W)
    for t, r in zip(tiles, rs):
        got = r.to_host()
        r.free()
        compare(got, gpu_build(lod, t, 20000))
