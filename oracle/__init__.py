"""CPU oracle for the LOD construction — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
reference leg of ``bench.py`` may import this package.  The library under
``paper_2302_14801_gb300`` never imports it and shares no code with it.

``build(points, T, mode, max_depth)`` runs the plain single-threaded C++
restatement in ``lod_oracle.cpp`` (see its header for the passages of the
paper each step follows) and returns its output as numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lod_oracle.cpp")
_SRCS = [_SRC, os.path.join(_HERE, "render_oracle.cpp")]
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

FILTER = 0
PICK = 1
WEIGHTED = 2  # neighbourhood-weighted average (Section 4.2.4)
FIRST = 3     # first come in input order (Section 4.2.1)
RANDOM = 4    # random pick with the key of Listing 1 (Section 4.2.2), bottom up


def compile_oracle(force: bool = False) -> str:
    """Compile the oracle with g++ (plain -O2, no target-specific flags, no
    floating-point contraction: the rasteriser's pixel decisions depend on
    every single-precision operation being rounded on its own)."""
    newest = max(os.path.getmtime(f) for f in _SRCS + [os.path.abspath(__file__)])
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-o", tmp,
                               *_SRCS])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(compile_oracle())
        u8p = ctypes.POINTER(ctypes.c_uint8)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        i32p = ctypes.POINTER(ctypes.c_int32)
        lib.oracle_build.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32,
                                     ctypes.c_uint32, ctypes.c_uint32,
                                     ctypes.POINTER(ctypes.c_void_p)]
        lib.oracle_build.restype = ctypes.c_int
        lib.oracle_n_nodes.argtypes = [ctypes.c_void_p]
        lib.oracle_n_nodes.restype = ctypes.c_uint64
        lib.oracle_n_voxels.argtypes = [ctypes.c_void_p]
        lib.oracle_n_voxels.restype = ctypes.c_uint64
        lib.oracle_get_nodes.argtypes = [ctypes.c_void_p, i32p, u8p, u8p, u8p, u8p, u32p, u32p,
                                         u64p, u64p, u64p, u32p]
        lib.oracle_get_nodes.restype = None
        lib.oracle_get_voxels.argtypes = [ctypes.c_void_p, u32p]
        lib.oracle_get_voxels.restype = None
        lib.oracle_get_points.argtypes = [ctypes.c_void_p, i32p, u32p]
        lib.oracle_get_points.restype = None
        lib.oracle_free.argtypes = [ctypes.c_void_p]
        lib.oracle_free.restype = None
        lib.oracle_splitmix64.argtypes = [ctypes.c_uint64]
        lib.oracle_splitmix64.restype = ctypes.c_uint64
        lib.oracle_weighted_node.argtypes = [ctypes.c_void_p, ctypes.c_uint64, u32p, u8p, ctypes.c_uint64, i32p,
                                             ctypes.c_uint32, u32p]
        lib.oracle_weighted_node.restype = ctypes.c_int64
        f32p = ctypes.POINTER(ctypes.c_float)
        lib.oracle_render.argtypes = [ctypes.c_uint32, i32p, u8p, u8p, u8p, u32p, u32p, u64p, u64p, u64p, u32p,
                                      u32p, i32p, f32p, i32p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_float,
                                      u64p, u8p]
        lib.oracle_render.restype = ctypes.c_int64
        lib.oracle_random_key.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
        lib.oracle_random_key.restype = ctypes.c_uint64
        lib.oracle_cube_voxels.argtypes = [ctypes.c_void_p, u32p, ctypes.c_uint64, i32p, ctypes.c_uint32,
                                           ctypes.c_uint32, u32p]
        lib.oracle_cube_voxels.restype = ctypes.c_int64
        _lib = lib
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def splitmix64(x: int) -> int:
    return int(_load().oracle_splitmix64(ctypes.c_uint64(x)))


def random_key(i: int, level: int) -> int:
    """The oracle's 64-bit random-strategy key: Listing 1's 32-bit key above
    the index (the larger wins)."""
    return int(_load().oracle_random_key(ctypes.c_uint32(i), ctypes.c_uint32(level)))


def build(points: np.ndarray, leaf_threshold: int = 50000, mode: int = FILTER,
          max_depth: int = 21) -> dict:
    """Run the oracle on an (N, 4) int32 point array; return numpy arrays.

    ``mode``: FILTER (cell average), PICK (minimal-hash sample), WEIGHTED
    (neighbourhood-weighted average, computed bottom-up as the paper does),
    FIRST (the cell's first point in input order) or RANDOM (largest key of
    Listing 1 among the children's samples, bottom up).

    Keys: ``min`` (n,3) int32, ``level``, ``log2_size``, ``child_mask``,
    ``flags`` (uint8), ``parent``, ``first_child`` (uint32),
    ``point_offset``, ``point_count``, ``voxel_offset`` (uint64),
    ``voxel_count`` (uint32); ``points`` (N,4) int32 and ``index`` (N,)
    uint32 in leaf layout order; ``voxels`` (V,4) uint32 rows of
    (cell, rgba, count, pick_index), each node's voxels sorted by cell.
    """
    lib = _load()
    pts = np.ascontiguousarray(points, dtype=np.int32).reshape(-1, 4)
    n = pts.shape[0]
    h = ctypes.c_void_p()
    rc = lib.oracle_build(pts.ctypes.data if n else None, n, leaf_threshold, mode, max_depth,
                          ctypes.byref(h))
    if rc != 0:
        raise ValueError(f"oracle_build failed with status {rc}")
    try:
        nn = int(lib.oracle_n_nodes(h))
        nv = int(lib.oracle_n_voxels(h))
        out = {
            "min": np.empty((nn, 3), np.int32),
            "level": np.empty(nn, np.uint8),
            "log2_size": np.empty(nn, np.uint8),
            "child_mask": np.empty(nn, np.uint8),
            "flags": np.empty(nn, np.uint8),
            "parent": np.empty(nn, np.uint32),
            "first_child": np.empty(nn, np.uint32),
            "point_offset": np.empty(nn, np.uint64),
            "point_count": np.empty(nn, np.uint64),
            "voxel_offset": np.empty(nn, np.uint64),
            "voxel_count": np.empty(nn, np.uint32),
            "voxels": np.empty((nv, 4), np.uint32),
            "points": np.empty((n, 4), np.int32),
            "index": np.empty(n, np.uint32),
        }
        lib.oracle_get_nodes(h, _ptr(out["min"], ctypes.c_int32), _ptr(out["level"], ctypes.c_uint8),
                             _ptr(out["log2_size"], ctypes.c_uint8),
                             _ptr(out["child_mask"], ctypes.c_uint8),
                             _ptr(out["flags"], ctypes.c_uint8), _ptr(out["parent"], ctypes.c_uint32),
                             _ptr(out["first_child"], ctypes.c_uint32),
                             _ptr(out["point_offset"], ctypes.c_uint64),
                             _ptr(out["point_count"], ctypes.c_uint64),
                             _ptr(out["voxel_offset"], ctypes.c_uint64),
                             _ptr(out["voxel_count"], ctypes.c_uint32))
        lib.oracle_get_voxels(h, _ptr(out["voxels"], ctypes.c_uint32))
        lib.oracle_get_points(h, _ptr(out["points"], ctypes.c_int32), _ptr(out["index"], ctypes.c_uint32))
    finally:
        lib.oracle_free(h)
    return out


def cube_voxels(points: np.ndarray, index: np.ndarray, cube_min, log2_size: int, mode: int = FILTER) -> np.ndarray:
    """Voxels of one cube from every input point inside it (rows of
    (cell, rgba, count, pick_index), sorted by cell); ``index`` holds the
    points' input indices.  Used to check single nodes of builds too large
    for ``build``."""
    lib = _load()
    pts = np.ascontiguousarray(points, dtype=np.int32).reshape(-1, 4)
    idx = np.ascontiguousarray(index, dtype=np.uint32)
    assert len(idx) == len(pts)
    mn = np.ascontiguousarray(np.asarray(cube_min, dtype=np.int32).reshape(3))
    out = np.empty((max(len(pts), 1), 4), np.uint32)
    nv = lib.oracle_cube_voxels(pts.ctypes.data if len(pts) else None, _ptr(idx, ctypes.c_uint32), len(pts),
                                _ptr(mn, ctypes.c_int32), int(log2_size), int(mode), _ptr(out, ctypes.c_uint32))
    if nv < 0:
        raise ValueError("oracle_cube_voxels: invalid arguments (a point outside the cube?)")
    return out[:nv].copy()


def weighted_node(points: np.ndarray, voxels: np.ndarray, octants: np.ndarray, cube_min, log2_size: int) -> np.ndarray:
    """Neighbourhood-weighted voxels (Section 4.2.4) of one inner node from
    its children's samples: ``points`` (the leaf children's points, (n, 4)
    int32) and ``voxels`` (the inner children's voxels, (m, 4) rows of cell,
    rgba, count, pick_index) with ``octants`` (m,) giving each voxel's child
    octant.  Rows of (cell, rgba, count, pick_index) sorted by cell."""
    lib = _load()
    pts = np.ascontiguousarray(points, dtype=np.int32).reshape(-1, 4)
    vox = np.ascontiguousarray(voxels, dtype=np.uint32).reshape(-1, 4)
    octs = np.ascontiguousarray(octants, dtype=np.uint8).reshape(-1)
    assert len(octs) == len(vox)
    mn = np.ascontiguousarray(np.asarray(cube_min, dtype=np.int32).reshape(3))
    out = np.empty((max(len(pts) + len(vox), 1), 4), np.uint32)
    nv = lib.oracle_weighted_node(pts.ctypes.data if len(pts) else None, len(pts),
                                  _ptr(vox, ctypes.c_uint32) if len(vox) else None,
                                  _ptr(octs, ctypes.c_uint8) if len(vox) else None, len(vox),
                                  _ptr(mn, ctypes.c_int32), int(log2_size), _ptr(out, ctypes.c_uint32))
    if nv < 0:
        raise ValueError("oracle_weighted_node: invalid arguments")
    return out[:nv].copy()


def render(res: dict, view_proj, origin, width: int, height: int, threshold: float = 100.0):
    """Rasterise an LOD octree (a result dictionary as ``build`` returns it)
    into a headless framebuffer (rendering of Section 5, see
    render_oracle.cpp).  Returns (framebuffer (height, width) uint64 keys of
    the bits of depth (z/w / 2 + 1/2) << 32 | rgba, ~0 where nothing was
    drawn; drawn node flags; samples drawn)."""
    lib = _load()
    n = len(res["level"])
    m = np.ascontiguousarray(np.asarray(view_proj, dtype=np.float32).reshape(16))
    org = np.ascontiguousarray(np.asarray(origin, dtype=np.int32).reshape(3))
    fb = np.empty((height, width), np.uint64)
    vis = np.zeros(n, np.uint8)
    arr = {k: np.ascontiguousarray(res[k]) for k in ("min", "log2_size", "child_mask", "flags", "parent",
                                                     "first_child", "point_offset", "point_count",
                                                     "voxel_offset", "voxel_count")}
    vox = np.ascontiguousarray(np.asarray(res["voxels"], dtype=np.uint32).reshape(-1, 4))
    pts = np.ascontiguousarray(np.asarray(res["points"], dtype=np.int32).reshape(-1, 4))
    if len(vox) == 0:
        vox = np.zeros((1, 4), np.uint32)
    if len(pts) == 0:
        pts = np.zeros((1, 4), np.int32)
    drawn = lib.oracle_render(n, _ptr(arr["min"], ctypes.c_int32), _ptr(arr["log2_size"], ctypes.c_uint8),
                              _ptr(arr["child_mask"], ctypes.c_uint8), _ptr(arr["flags"], ctypes.c_uint8),
                              _ptr(arr["parent"], ctypes.c_uint32), _ptr(arr["first_child"], ctypes.c_uint32),
                              _ptr(arr["point_offset"], ctypes.c_uint64), _ptr(arr["point_count"], ctypes.c_uint64),
                              _ptr(arr["voxel_offset"], ctypes.c_uint64), _ptr(arr["voxel_count"], ctypes.c_uint32),
                              _ptr(vox, ctypes.c_uint32), _ptr(pts, ctypes.c_int32), _ptr(m, ctypes.c_float),
                              _ptr(org, ctypes.c_int32), int(width), int(height), float(threshold),
                              _ptr(fb, ctypes.c_uint64), _ptr(vis, ctypes.c_uint8))
    if drawn < 0:
        raise ValueError("oracle_render: invalid arguments")
    return fb, vis, int(drawn)
