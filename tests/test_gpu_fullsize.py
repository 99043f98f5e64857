"""GPU parity at the benchmark's full size: the 50M-point aerial cloud built
exactly as bench.py times it (lod.build on the current stream, T = 50k,
max_depth 21, default tuning), both modes, compared with the oracle over
the whole result (node table, every leaf's point multiset, indices, every
voxel), plus the size-independent invariants of the tree."""
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


@pytest.mark.parametrize("mode", [0, 1])
def test_aerial_50m_full_parity(lod, aerial, mode):
    import torch
    d = torch.from_numpy(aerial).cuda()
    r = lod.build(d, T, mode, 21, stream=torch.cuda.current_stream())
    got = r.to_host()
    r.free()
    del d
    invariants(got, N)
    want = oracle.build(aerial, T, mode, 21)
    compare(got, want, inp=aerial)
