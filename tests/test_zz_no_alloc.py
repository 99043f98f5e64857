"""GPU test of lod_root_cubes_noalloc, the entry point that allocates no
device memory (for callers that cannot call cudaMalloc: a plug-in whose host
application owns every byte of device memory, a render loop that must not
let an allocation synchronise the device).  It must give the same root cubes
as the regular entry points (the root node of lod_build /
lod_build_batched) and as the definition computed here with numpy (bounding
box minimum; edge the smallest power of two above the largest extent),
exactly, on two calls in a row: the second call reuses the static scratch
left by the first and has to clear it itself.

This file is named so that pytest collects it last."""
import numpy as np
import pytest

from paper_2302_14801_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lod():
    import torch
    from paper_2302_14801_gb300 import _build_ext
    _build_ext.build()
    from paper_2302_14801_gb300 import lod as m
    torch.cuda.set_device(0)
    return m


def reference_cubes(lod, tiles):
    """Root nodes built by lod_build_batched (the existing entry point)."""
    rs = lod.build_batched(tiles, 50000, lod.FILTER)
    out = []
    for r in rs:
        h = r.to_host()
        out.append([int(h["min"][0][0]), int(h["min"][0][1]), int(h["min"][0][2]), int(h["log2_size"][0])])
        r.free()
    return np.asarray(out, dtype=np.int32)


def numpy_cubes(tiles):
    """The root cube written out from its definition (independent of the
    CUDA path): min corner = per-axis minimum, log2 edge = the smallest L
    with 2^L > the largest per-axis extent; an empty cloud gives zeros."""
    out = []
    for t in tiles:
        p = t.cpu().numpy().astype(np.int64)
        if len(p) == 0:
            out.append([0, 0, 0, 0])
            continue
        lo, hi = p[:, :3].min(axis=0), p[:, :3].max(axis=0)
        ext = int((hi - lo).max())
        L = 0
        while (1 << L) <= ext:
            L += 1
        out.append([int(lo[0]), int(lo[1]), int(lo[2]), L])
    return np.asarray(out, dtype=np.int32)


def test_noalloc_root_cubes_match_build_twice(lod):
    import torch
    rng = np.random.default_rng(77)
    # first call: many tiles of ragged sizes, including an empty one
    sizes1 = [0, 1, 4095, 4097, 100_000, 1_000_000] + [int(x) for x in rng.integers(1, 50_000, size=40)]
    tiles1 = [torch.from_numpy(synth.sphere_tile(n, seed=900 + i)).cuda() for i, n in enumerate(sizes1)]
    # second call: fewer tiles, other extents (negative and near the int32 limits)
    big = np.empty((70_000, 4), np.int32)
    big[:, :3] = rng.integers(-(2**31), 2**31, size=(70_000, 3))
    big[:, 3] = 0
    tiles2 = [torch.from_numpy(big).cuda(),
              torch.from_numpy(synth.aerial(300_000, seed=5, n_buildings=10)).cuda(),
              torch.from_numpy(synth.sphere(12345, seed=6)).cuda()]
    for tiles in (tiles1, tiles2):
        out = torch.full((len(tiles), 4), -7, dtype=torch.int32, device="cuda")
        lod.root_cubes_noalloc(tiles, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        want = reference_cubes(lod, tiles)
        assert np.array_equal(got, want), (got[:5], want[:5])
        assert np.array_equal(got, numpy_cubes(tiles))
    # and against lod_build on a single cloud
    out = torch.zeros((1, 4), dtype=torch.int32, device="cuda")
    lod.root_cubes_noalloc([tiles2[1]], out)
    r = lod.build(tiles2[1], 50000, lod.PICK)
    h = r.to_host()
    r.free()
    assert out.cpu().numpy().tolist() == [[*h["min"][0].tolist(), int(h["log2_size"][0])]]


def test_noalloc_uneven_batch(lod):
    import torch
    # one large cloud among thousands of tiny ones (the work list is flat
    # over all tiles' points), called twice with the same scratch
    rng = np.random.default_rng(78)
    sizes = [3_000_000] + [int(x) for x in rng.integers(0, 40, size=3000)]
    tiles = [torch.from_numpy(synth.sphere_tile(n, seed=20_000 + i)).cuda() for i, n in enumerate(sizes)]
    want = numpy_cubes(tiles)
    for _ in range(2):
        out = torch.full((len(tiles), 4), -7, dtype=torch.int32, device="cuda")
        lod.root_cubes_noalloc(tiles, out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), want)


def test_noalloc_rejects_oversized_batch(lod):
    import torch
    t = torch.zeros((1, 4), dtype=torch.int32, device="cuda")
    out = torch.zeros((4097, 4), dtype=torch.int32, device="cuda")
    with pytest.raises(lod.LodError) as e:
        lod.root_cubes_noalloc([t] * 4097, out)
    assert e.value.status == lod.LOD_ERR_INVALID_ARG
