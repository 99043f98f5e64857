"""GPU parity of the LOD rasteriser (Section 5 restated as CUDA, lod_render):
every pixel key (depth bits << 32 | rgba), the drawn-node count and the
number of samples drawn equal the CPU oracle rasteriser's, bit for bit,
for cameras outside, above and inside the cloud, near and far.  The oracle
renders the oracle's own octree where the CUDA octree equals it exactly
(filtered and pick modes), and the CUDA octree itself for the weighted
mode."""
import numpy as np
import pytest

import oracle
from paper_2302_14801_gb300 import camera, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lod():
    import torch
    from paper_2302_14801_gb300 import _build_ext
    _build_ext.build()
    from paper_2302_14801_gb300 import lod as m
    torch.cuda.set_device(0)
    return m


def cameras(res, w, h):
    L = max(int(res["log2_size"][0]), 4)
    lo = res["min"][0].astype(np.int64)
    c = lo + (1 << (L - 1))
    out = {
        "overview": camera.perspective(c + [2 << L, -(1 << L), 1 << L], c, fovy_deg=50, aspect=w / h, near=1,
                                       far=1e9),
        "close": camera.perspective(c + [1 << (L - 3), 1 << (L - 4), 1 << (L - 3)], c, fovy_deg=70, aspect=w / h,
                                    near=1, far=1e9),
        "inside": camera.perspective(c, c + [1 << L, 3 << (L - 2), 0], fovy_deg=90, aspect=w / h, near=1, far=1e9),
        "top": camera.orthographic(lo, lo + (1 << L)),
        "away": camera.perspective(c + [4 << L, 0, 0], c + [8 << L, 0, 0], fovy_deg=30, aspect=w / h, near=1,
                                   far=1e9),
    }
    return out


def check_render(lod, r, res, w=640, h=360, thresholds=(100.0, 30.0)):
    for name, (m, org) in cameras(res, w, h).items():
        for thr in thresholds:
            fb, st = lod.render(r, m, org, w, h, thr, stats=True)
            got = fb.cpu().numpy().view(np.uint64)
            want, vis, drawn = oracle.render(res, m, org, w, h, thr)
            assert st["visible_nodes"] == int(vis.sum()), (name, thr)
            assert st["samples_drawn"] == drawn, (name, thr)
            bad = np.nonzero(got != want)
            assert len(bad[0]) == 0, f"{name} thr {thr}: {len(bad[0])} pixels differ, first {bad[0][0]},{bad[1][0]}"
            if name == "away":
                assert drawn == 0
            elif name in ("overview", "top"):
                assert drawn > 0


@pytest.mark.parametrize("mode", [0, 1])
def test_render_equals_oracle_on_the_oracles_octree(lod, mode):
    import torch
    pts = synth.aerial(2_000_000, seed=61, n_buildings=60)
    want = oracle.build(pts, 5000, mode, 21)
    r = lod.build(torch.from_numpy(pts).cuda(), 5000, mode)
    check_render(lod, r, want)
    r.free()


def test_render_weighted_and_sphere(lod):
    import torch
    pts = synth.sphere(1_000_000, seed=62)
    r = lod.build(torch.from_numpy(pts).cuda(), 20000, 2)
    check_render(lod, r, r.to_host())
    r.free()


def test_render_tiny_and_full_hd(lod):
    import torch
    # a single point, a small sphere, and a full-HD frame of a 3M indoor cloud
    for pts in (np.array([[5, 6, 7, -1]], np.int32), synth.sphere(3000, seed=63)):
        r = lod.build(torch.from_numpy(pts).cuda(), 100, 0)
        check_render(lod, r, oracle.build(pts, 100, 0, 21), 64, 48, (100.0,))
        r.free()
    pts = synth.indoor(3_000_000, seed=64, n_prims=128)
    r = lod.build(torch.from_numpy(pts).cuda(), 50000, 1)
    check_render(lod, r, oracle.build(pts, 50000, 1, 21), 1920, 1080, (100.0,))
    r.free()


def test_render_rejects_bad_arguments(lod):
    import ctypes

    import torch
    r = lod.build(torch.from_numpy(synth.sphere(1000, seed=65)).cuda(), 100, 0)
    fb = torch.empty((10, 10), dtype=torch.int64, device="cuda")
    m, org = camera.orthographic([0, 0, 0], [1 << 20] * 3)
    L = lod.lib()
    for w, h, thr in ((0, 10, 100.0), (10, 0, 100.0), (10, 10, -1.0), (1 << 16, 1 << 16, 100.0)):
        cam = lod.make_camera(m, org, w, h, thr)
        assert L.lod_render(r.handle, ctypes.byref(cam), fb.data_ptr(), None, None) == lod.LOD_ERR_INVALID_ARG
    cam = lod.make_camera(m, org, 10, 10, 100.0)
    assert L.lod_render(r.handle, ctypes.byref(cam), fb.data_ptr() + 4, None, None) == lod.LOD_ERR_INVALID_ARG
    bad = lod.make_camera(np.full(16, np.inf, np.float32), org, 10, 10, 100.0)
    assert L.lod_render(r.handle, ctypes.byref(bad), fb.data_ptr(), None, None) == lod.LOD_ERR_INVALID_ARG
    assert L.lod_render(r.handle, ctypes.byref(cam), fb.data_ptr(), None, None) == lod.LOD_OK
    torch.cuda.synchronize()
    r.free()
