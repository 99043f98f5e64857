"""CPU checks of the C ABI: the library builds, loads and exports every
entry point declared in include/lod.h; host-side argument validation works
without touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lodmod():
    from paper_2302_14801_gb300 import _build_ext
    _build_ext.build()
    from paper_2302_14801_gb300 import lod
    return lod


def declared_functions():
    text = open(os.path.join(ROOT, "include", "lod.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lod_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("lod_build", "lod_build_batched", "lod_submit", "lod_poll", "lod_free", "lod_result_view"):
        assert must in names


def test_library_exports_every_declared_symbol(lodmod):
    lib = ctypes.CDLL(lodmod.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert sorted(lodmod.EXPORTED) == declared_functions()


def test_struct_layouts(lodmod):
    assert ctypes.sizeof(lodmod.Node) == 56
    assert ctypes.sizeof(lodmod.Params) == 16
    assert ctypes.sizeof(lodmod.View) == 64


def test_params_defaults_and_error_strings(lodmod):
    p = lodmod.Params()
    assert lodmod.lib().lod_params_init(ctypes.byref(p)) == 0
    assert (p.leaf_threshold, p.mode, p.max_depth, p.flags) == (50000, 0, 21, 0)
    assert lodmod.error_string(0) == "ok"
    assert "budget" in lodmod.error_string(lodmod.LOD_ERR_BUDGET)


def test_invalid_arguments_rejected_on_host(lodmod):
    L = lodmod.lib()
    h = ctypes.c_void_p()
    p = lodmod.make_params()
    assert L.lod_build(None, 10, ctypes.byref(p), None, None) == lodmod.LOD_ERR_INVALID_ARG
    assert L.lod_build_batched(None, None, 0, None, None, None) == lodmod.LOD_ERR_INVALID_ARG
    bad = lodmod.make_params(leaf_threshold=0)
    assert L.lod_build_from_host(None, 0, ctypes.byref(bad), None, ctypes.byref(h)) == lodmod.LOD_ERR_INVALID_ARG
    assert L.lod_result_view(None, None) == lodmod.LOD_ERR_INVALID_ARG
    L.lod_free(None)  # no-op
    cfg = lodmod.ServerConfig(0, 1, 0)
    assert L.lod_server_create(ctypes.byref(cfg), ctypes.byref(h)) == lodmod.LOD_ERR_INVALID_ARG
    # checked before any device work: alignment, point count, parameters
    dev = ctypes.c_void_p(1 << 20)  # never dereferenced: every call below fails its checks first
    odd = ctypes.c_void_p((1 << 20) + 8)
    assert L.lod_build(odd, 1, ctypes.byref(p), None, ctypes.byref(h)) == lodmod.LOD_ERR_INVALID_ARG
    assert L.lod_build(dev, 1 << 32, ctypes.byref(p), None, ctypes.byref(h)) == lodmod.LOD_ERR_INVALID_ARG
    for bad in (lodmod.make_params(mode=5), lodmod.make_params(max_depth=33), lodmod.make_params(leaf_threshold=0)):
        assert L.lod_build(dev, 1, ctypes.byref(bad), None, ctypes.byref(h)) == lodmod.LOD_ERR_INVALID_ARG
    tiles = (ctypes.c_void_p * 2)(dev, odd)
    ns = (ctypes.c_uint64 * 2)(5, 5)
    outs = (ctypes.c_void_p * 2)()
    assert L.lod_build_batched(tiles, ns, 2, ctypes.byref(p), None, outs) == lodmod.LOD_ERR_INVALID_ARG
    assert L.lod_root_cubes_noalloc(tiles, ns, 2, dev, None) == lodmod.LOD_ERR_INVALID_ARG  # tile 1 misaligned
    assert L.lod_root_cubes_noalloc(tiles, ns, 0, dev, None) == lodmod.LOD_ERR_INVALID_ARG
    assert L.lod_root_cubes_noalloc(tiles, ns, 1, ctypes.c_void_p((1 << 20) + 2), None) == lodmod.LOD_ERR_INVALID_ARG
    assert L.lod_autotune(None, 10, None, None, None, None) == lodmod.LOD_ERR_INVALID_ARG
    cam = lodmod.make_camera(np.eye(4, dtype=np.float32), [0, 0, 0], 8, 8)
    assert L.lod_render(None, ctypes.byref(cam), dev, None, None) == lodmod.LOD_ERR_INVALID_ARG
    assert L.lod_result_voxel_points(None, None) == lodmod.LOD_ERR_INVALID_ARG
    assert L.lod_build_out_of_core(None, 5, ctypes.byref(p), None, None, ctypes.byref(h)) == \
        lodmod.LOD_ERR_INVALID_ARG  # no points
    small_chunk = lodmod.OocConfig(10, 0, 0)  # chunks smaller than T
    pts = np.zeros((5, 4), np.int32)
    assert L.lod_build_out_of_core(pts.ctypes.data, 5, ctypes.byref(p), ctypes.byref(small_chunk), None,
                                   ctypes.byref(h)) == lodmod.LOD_ERR_INVALID_ARG
    fp = lodmod.make_params(mode=1, full_precision=True)
    assert L.lod_build_out_of_core(pts.ctypes.data, 5, ctypes.byref(fp), None, None, ctypes.byref(h)) == \
        lodmod.LOD_ERR_INVALID_ARG
    assert L.lod_result_copy_voxel_points_to_host(None, None, None) == lodmod.LOD_ERR_INVALID_ARG
    assert L.lod_profile_read(None, 0, None) == lodmod.LOD_ERR_INVALID_ARG


def test_tuning_is_checked_and_restorable(lodmod):
    L = lodmod.lib()
    before = lodmod.get_tuning()
    for bad in ((9, 0), (0, 9), (0, 0, 100), (0, 0, 0, 4097), (0, 0, 0, 0, 2), (0, 0, 0, 0, 0, 0, (1 << 18) + 1)):
        assert L.lod_set_tuning(ctypes.byref(lodmod.Tuning(*bad))) == lodmod.LOD_ERR_INVALID_ARG
    assert lodmod.get_tuning() == before  # a rejected setting changes nothing
    try:
        lodmod.set_tuning(root_depth=5, stream_ctas_per_sm=3, dense_bins_max=512, vox_queue_ranges=7,
                          vox_range_cells=1000)
        assert lodmod.get_tuning() == {"root_depth": 5, "stream_ctas_per_sm": 3, "dense_bins_max": 512,
                                       "vox_queue_ranges": 7, "graph_voxel_levels": 0, "vox_no_merge": 0,
                                       "vox_range_cells": 1000}
    finally:
        lodmod.set_tuning(**before)
    assert lodmod.get_tuning() == before
    assert L.lod_get_tuning(None) == lodmod.LOD_ERR_INVALID_ARG


def test_binding_rejects_malformed_point_arrays(lodmod):
    # the binding checks shapes and types before any call into the library
    import numpy as np
    torch = pytest.importorskip("torch")
    for bad in (np.zeros((4, 3), np.int32), np.zeros(16, np.int32), torch.zeros((4, 3), dtype=torch.int32),
                torch.zeros((4, 4), dtype=torch.int64), [[0, 0, 0, 0]]):
        with pytest.raises(TypeError):
            lodmod.build_from_host(bad)
    for bad in (np.zeros((4, 4), np.int32), torch.zeros((4, 4), dtype=torch.int32)):
        with pytest.raises(TypeError):  # lod_build wants device memory
            lodmod.build(bad)
    with pytest.raises(TypeError):
        lodmod.build_batched([np.zeros((4, 4), np.int32)])
