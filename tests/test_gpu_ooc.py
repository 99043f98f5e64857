"""GPU parity of the out-of-core build (Section 7, lod_build_out_of_core):
chunks built one batch at a time and the root-side nodes merged afterwards
give exactly the oracle's octree (the in-core definition) in every
sampling mode — node table, leaf point multisets and input indices, every
voxel.  Chunk, transfer and batch sizes are made small so that one cloud
gives many chunks at several levels, several transfers and batches, and
root-side nodes over both leaf and inner chunk roots."""
import numpy as np
import pytest

import oracle
from compare import compare
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


def ooc(lod, pts, T, mode, **kw):
    r = lod.build_out_of_core(pts, T, mode, 21, **kw)
    got = r.to_host()
    r.free()
    return got


@pytest.mark.parametrize("mode", [0, 1, 2, 3, 4])
def test_out_of_core_equals_oracle_all_modes(lod, mode):
    pts = synth.aerial(1_500_000, seed=71, n_buildings=60)
    got = ooc(lod, pts, 4000, mode, chunk_points=60_000, stream_points=250_000, batch_points=400_000)
    compare(got, oracle.build(pts, 4000, mode, 21), inp=pts)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_out_of_core_clustered_and_sphere(lod, mode):
    # dense clusters give chunks at many levels (and oversized chunks at the
    # top grid's depth); the sphere gives leaf chunk roots beside inner ones
    pts = synth.indoor(2_000_000, seed=72, n_prims=64)
    compare(ooc(lod, pts, 3000, mode, chunk_points=20_000, stream_points=777_777), oracle.build(pts, 3000, mode, 21),
            inp=pts)
    pts = synth.sphere(400_000, seed=73)
    compare(ooc(lod, pts, 700, mode, chunk_points=5_000), oracle.build(pts, 700, mode, 21), inp=pts)


def test_out_of_core_equals_in_core_and_edge_cases(lod):
    import torch
    pts = synth.aerial(3_000_000, seed=74, n_buildings=100)
    for mode in (0, 1):
        r = lod.build(torch.from_numpy(pts).cuda(), 50000, mode)
        want = r.to_host()
        r.free()
        compare(ooc(lod, pts, 50000, mode, chunk_points=400_000), want, inp=pts)
    # one chunk (the root), an empty cloud, one point, a chain of identical points
    small = synth.sphere(3000, seed=75)
    compare(ooc(lod, small, 100, 1, chunk_points=10_000), oracle.build(small, 100, 1, 21), inp=small)
    got = ooc(lod, np.zeros((0, 4), np.int32), 10, 0)
    assert len(got["level"]) == 1 and got["point_count"][0] == 0
    one = np.array([[5, 6, 7, -1]], np.int32)
    compare(ooc(lod, one, 1, 0), oracle.build(one, 1, 0, 21), inp=one)
    same = np.tile(np.array([[9, 9, 9, 123]], np.int32), (500, 1))
    compare(ooc(lod, same, 3, 4, chunk_points=3), oracle.build(same, 3, 4, 21), inp=same)
