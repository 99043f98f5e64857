"""Thin ctypes binding of the C ABI in include/lod.h.

Argument marshalling only: every step of the build runs in the CUDA
library liblod.so.  There is no CPU fallback; importing this module on a
machine without the built library raises immediately.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblod.so")

LOD_OK = 0
LOD_NOT_READY = 1
LOD_ERR_INVALID_ARG = 2
LOD_ERR_OOM = 3
LOD_ERR_BUDGET = 4
LOD_ERR_CUDA = 5
LOD_ERR_TIMEOUT = 6
LOD_ERR_INTERNAL = 7

FILTER = 0
PICK = 1
WEIGHTED = 2
FIRST = 3
RANDOM = 4
MODES = {"filter": FILTER, "filtered": FILTER, "pick": PICK, "weighted": WEIGHTED, "first": FIRST, "random": RANDOM}
FLAG_LEAF_INDEX = 1
FLAG_FULL_PRECISION = 2
NODE_LEAF = 1
NODE_OVERFULL = 2

EXPORTED = [
    "lod_params_init", "lod_build", "lod_build_from_host", "lod_build_batched", "lod_result_view",
    "lod_result_copy_to_host", "lod_result_device_bytes", "lod_free", "lod_error_string",
    "lod_server_create", "lod_submit", "lod_poll", "lod_wait", "lod_server_bytes_in_use",
    "lod_server_destroy", "lod_profile_enable", "lod_profile_reset", "lod_profile_read", "lod_launch_count",
    "lod_root_cubes_noalloc", "lod_set_tuning", "lod_get_tuning", "lod_autotune", "lod_scratch_bytes",
    "lod_trim", "lod_result_voxel_points", "lod_result_copy_voxel_points_to_host", "lod_render",
    "lod_build_out_of_core",
]


class Params(ctypes.Structure):
    _fields_ = [("leaf_threshold", ctypes.c_uint32), ("mode", ctypes.c_uint32),
                ("max_depth", ctypes.c_uint32), ("flags", ctypes.c_uint32)]


class Node(ctypes.Structure):
    _fields_ = [("min", ctypes.c_int32 * 3), ("level", ctypes.c_uint8), ("log2_size", ctypes.c_uint8),
                ("child_mask", ctypes.c_uint8), ("flags", ctypes.c_uint8), ("parent", ctypes.c_uint32),
                ("first_child", ctypes.c_uint32), ("point_offset", ctypes.c_uint64),
                ("point_count", ctypes.c_uint64), ("voxel_offset", ctypes.c_uint64),
                ("voxel_count", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class View(ctypes.Structure):
    _fields_ = [("nodes", ctypes.c_void_p), ("n_nodes", ctypes.c_uint32), ("n_levels", ctypes.c_uint32),
                ("points", ctypes.c_void_p), ("point_index", ctypes.c_void_p), ("n_points", ctypes.c_uint64),
                ("voxels", ctypes.c_void_p), ("n_voxels", ctypes.c_uint64), ("mode", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("max_inflight", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


class Tuning(ctypes.Structure):
    _fields_ = [("root_depth", ctypes.c_uint32), ("stream_ctas_per_sm", ctypes.c_uint32),
                ("dense_bins_max", ctypes.c_uint32), ("vox_queue_ranges", ctypes.c_uint32),
                ("graph_voxel_levels", ctypes.c_uint32), ("vox_no_merge", ctypes.c_uint32),
                ("vox_range_cells", ctypes.c_uint32), ("reserved", ctypes.c_uint32 * 1)]


class Camera(ctypes.Structure):
    _fields_ = [("view_proj", ctypes.c_float * 16), ("origin", ctypes.c_int32 * 3), ("width", ctypes.c_uint32),
                ("height", ctypes.c_uint32), ("lod_pixels", ctypes.c_float), ("reserved", ctypes.c_uint32 * 2)]


class RenderStats(ctypes.Structure):
    _fields_ = [("visible_nodes", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("samples_drawn", ctypes.c_uint64)]


class OocConfig(ctypes.Structure):
    _fields_ = [("chunk_points", ctypes.c_uint64), ("stream_points", ctypes.c_uint64),
                ("batch_points", ctypes.c_uint64)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_uint64), ("total_ms", ctypes.c_double),
                ("alg_bytes", ctypes.c_double)]


NODE_DTYPE = np.dtype([("min", "<i4", (3,)), ("level", "u1"), ("log2_size", "u1"), ("child_mask", "u1"),
                       ("flags", "u1"), ("parent", "<u4"), ("first_child", "<u4"), ("point_offset", "<u8"),
                       ("point_count", "<u8"), ("voxel_offset", "<u8"), ("voxel_count", "<u4"),
                       ("reserved", "<u4")])
assert NODE_DTYPE.itemsize == ctypes.sizeof(Node) == 56


class LodError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {error_string(status)} (status {status})")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
    lib = ctypes.CDLL(LIB_PATH, mode=ctypes.RTLD_GLOBAL)
    vp, u32, u64, i = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    P = ctypes.POINTER
    sig = {
        "lod_params_init": (i, [P(Params)]),
        "lod_build": (i, [vp, u64, P(Params), vp, P(vp)]),
        "lod_build_from_host": (i, [vp, u64, P(Params), vp, P(vp)]),
        "lod_build_batched": (i, [P(vp), P(u64), u32, P(Params), vp, P(vp)]),
        "lod_result_view": (i, [vp, P(View)]),
        "lod_result_copy_to_host": (i, [vp, vp, vp, vp, vp, vp]),
        "lod_result_device_bytes": (u64, [vp]),
        "lod_free": (None, [vp]),
        "lod_error_string": (ctypes.c_char_p, [i]),
        "lod_server_create": (i, [P(ServerConfig), P(vp)]),
        "lod_submit": (i, [vp, vp, u64, P(Params), P(u64)]),
        "lod_poll": (i, [vp, u64, P(vp)]),
        "lod_wait": (i, [vp, u64, u32, P(vp)]),
        "lod_server_bytes_in_use": (u64, [vp]),
        "lod_server_destroy": (i, [vp]),
        "lod_profile_enable": (i, [i]),
        "lod_profile_reset": (i, []),
        "lod_profile_read": (i, [P(KernelStat), u32, P(u32)]),
        "lod_launch_count": (u64, []),
        "lod_root_cubes_noalloc": (i, [P(vp), P(u64), u32, vp, vp]),
        "lod_set_tuning": (i, [P(Tuning)]),
        "lod_get_tuning": (i, [P(Tuning)]),
        "lod_autotune": (i, [vp, u64, P(Params), vp, P(Tuning), P(ctypes.c_float)]),
        "lod_scratch_bytes": (u64, [vp]),
        "lod_trim": (i, [vp]),
        "lod_result_voxel_points": (i, [vp, P(vp)]),
        "lod_render": (i, [vp, P(Camera), vp, vp, P(RenderStats)]),
        "lod_build_out_of_core": (i, [vp, u64, P(Params), P(OocConfig), vp, P(vp)]),
        "lod_result_copy_voxel_points_to_host": (i, [vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = _load()
    return _lib


def error_string(status: int) -> str:
    return lib().lod_error_string(status).decode()


def make_params(leaf_threshold=50000, mode=FILTER, max_depth=21, keep_index=False, full_precision=False) -> Params:
    if isinstance(mode, str):
        mode = MODES[mode]
    flags = (FLAG_LEAF_INDEX if keep_index else 0) | (FLAG_FULL_PRECISION if full_precision else 0)
    return Params(int(leaf_threshold), int(mode), int(max_depth), flags)


def _check(rc, what):
    if rc != LOD_OK:
        raise LodError(rc, what)


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def profile_enable(on: bool = True) -> None:
    _check(lib().lod_profile_enable(1 if on else 0), "lod_profile_enable")


def profile_reset() -> None:
    _check(lib().lod_profile_reset(), "lod_profile_reset")


def profile_read() -> dict:
    """{kernel name: {"launches", "total_ms", "alg_bytes"}} accumulated so far."""
    n = ctypes.c_uint32()
    _check(lib().lod_profile_read(None, 0, ctypes.byref(n)), "lod_profile_read")
    arr = (KernelStat * max(n.value, 1))()
    _check(lib().lod_profile_read(arr, n.value, ctypes.byref(n)), "lod_profile_read")
    return {arr[i].name.decode(): {"launches": int(arr[i].launches), "total_ms": float(arr[i].total_ms),
                                   "alg_bytes": float(arr[i].alg_bytes)} for i in range(n.value)}


def set_tuning(root_depth: int = 0, stream_ctas_per_sm: int = 0, dense_bins_max: int = 0,
               vox_queue_ranges: int = 0, graph_voxel_levels: int = 0, vox_no_merge: int = 0,
               vox_range_cells: int = 0) -> None:
    """Process-wide speed knobs (never change results); 0 = default."""
    t = Tuning(int(root_depth), int(stream_ctas_per_sm), int(dense_bins_max), int(vox_queue_ranges),
               int(graph_voxel_levels), int(vox_no_merge), int(vox_range_cells))
    _check(lib().lod_set_tuning(ctypes.byref(t)), "lod_set_tuning")


def get_tuning() -> dict:
    t = Tuning()
    _check(lib().lod_get_tuning(ctypes.byref(t)), "lod_get_tuning")
    return {"root_depth": t.root_depth, "stream_ctas_per_sm": t.stream_ctas_per_sm,
            "dense_bins_max": t.dense_bins_max, "vox_queue_ranges": t.vox_queue_ranges,
            "graph_voxel_levels": t.graph_voxel_levels, "vox_no_merge": t.vox_no_merge,
            "vox_range_cells": t.vox_range_cells}


def autotune(points, leaf_threshold=50000, mode=FILTER, max_depth=21, stream=None) -> dict:
    """lod_autotune on a CUDA int32 (N, 4) tensor: applies and returns the
    fastest tuning (``root_depth``, ``stream_ctas_per_sm``, ``ms``)."""
    ptr, n = _dev_ptr(points)
    p = make_params(leaf_threshold, mode, max_depth, False)
    t = Tuning()
    ms = ctypes.c_float()
    _check(lib().lod_autotune(ptr if n else None, n, ctypes.byref(p), _stream_handle(stream), ctypes.byref(t),
                              ctypes.byref(ms)), "lod_autotune")
    return {"root_depth": t.root_depth, "stream_ctas_per_sm": t.stream_ctas_per_sm,
            "dense_bins_max": t.dense_bins_max, "vox_queue_ranges": t.vox_queue_ranges,
            "graph_voxel_levels": t.graph_voxel_levels, "vox_no_merge": t.vox_no_merge,
            "vox_range_cells": t.vox_range_cells, "ms": ms.value}


def launch_count() -> int:
    return int(lib().lod_launch_count())


def scratch_bytes(stream=None) -> int:
    """Device bytes of build scratch kept for ``stream`` (lod_scratch_bytes)."""
    return int(lib().lod_scratch_bytes(_stream_handle(stream)))


def trim(stream=None) -> None:
    """lod_trim: wait for ``stream``, free its kept scratch and return the
    pool's unused memory to the device; results stay valid."""
    _check(lib().lod_trim(_stream_handle(stream)), "lod_trim")


class _DevArray:
    """Zero-copy device array exposed through __cuda_array_interface__."""

    def __init__(self, ptr, shape, typestr, owner):
        self._owner = owner
        self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


class Result:
    """An LOD octree living in device memory (owned by the library)."""

    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)

    @property
    def handle(self):
        return self._h

    def view(self) -> View:
        v = View()
        _check(lib().lod_result_view(self._h, ctypes.byref(v)), "lod_result_view")
        return v

    def device_bytes(self) -> int:
        return int(lib().lod_result_device_bytes(self._h))

    def tensors(self):
        """Zero-copy torch views: nodes (n,14) int32 (the 56-byte node
        records), points (N,4) int32, index (N,) int32 or None — valid while
        this Result is alive.  Voxels: ``view().voxels`` is the device base
        that the nodes' voxel_offset indexes; ``to_host()`` gathers them."""
        import torch
        v = self.view()
        out = {}
        dev = torch.device("cuda", torch.cuda.current_device())
        out["nodes"] = torch.as_tensor(_DevArray(v.nodes, (v.n_nodes, 14), "<i4", self), device=dev)
        out["points"] = torch.as_tensor(_DevArray(v.points, (v.n_points, 4), "<i4", self), device=dev)
        out["index"] = (torch.as_tensor(_DevArray(v.point_index, (v.n_points,), "<i4", self), device=dev)
                        if v.point_index else None)
        return out

    def to_host(self, stream=None, out=None) -> dict:
        """Copy to host; returns numpy arrays keyed like the CPU oracle.

        ``out`` may hold preallocated host arrays (page-locked ones make the
        copy run at full link speed): ``nodes`` (NODE_DTYPE), ``points``
        ((N, 4) int32), ``index`` (uint32) and ``voxels`` ((V, 4) uint32), each
        at least as long as the result; their leading parts are filled."""
        v = self.view()
        out = out or {}
        nodes = out["nodes"][:v.n_nodes] if "nodes" in out else np.empty(v.n_nodes, NODE_DTYPE)
        pts = out["points"][:v.n_points] if "points" in out else np.empty((v.n_points, 4), np.int32)
        idx = None
        if v.point_index:
            idx = out["index"][:v.n_points] if "index" in out else np.empty(v.n_points, np.uint32)
        vox = out["voxels"][:v.n_voxels] if "voxels" in out else np.empty((v.n_voxels, 4), np.uint32)
        for a in (nodes, pts, vox) + ((idx,) if idx is not None else ()):
            if not a.flags.c_contiguous:
                raise ValueError("to_host: output arrays must be contiguous")
        _check(lib().lod_result_copy_to_host(
            self._h, nodes.ctypes.data, pts.ctypes.data if v.n_points else None,
            idx.ctypes.data if (idx is not None and v.n_points) else None,
            vox.ctypes.data if v.n_voxels else None, _stream_handle(stream)), "lod_result_copy_to_host")
        return {
            "min": np.ascontiguousarray(nodes["min"]), "level": nodes["level"].copy(),
            "log2_size": nodes["log2_size"].copy(), "child_mask": nodes["child_mask"].copy(),
            "flags": nodes["flags"].copy(), "parent": nodes["parent"].copy(),
            "first_child": nodes["first_child"].copy(), "point_offset": nodes["point_offset"].copy(),
            "point_count": nodes["point_count"].copy(), "voxel_offset": nodes["voxel_offset"].copy(),
            "voxel_count": nodes["voxel_count"].copy(), "points": pts, "index": idx, "voxels": vox,
        }

    def voxel_points_host(self, stream=None) -> np.ndarray:
        """lod_result_copy_voxel_points_to_host: the full-precision picked
        points ((V, 4) int32), in the voxel order of ``to_host()``."""
        v = self.view()
        out = np.empty((v.n_voxels, 4), np.int32)
        _check(lib().lod_result_copy_voxel_points_to_host(self._h, out.ctypes.data if v.n_voxels else None,
                                                          _stream_handle(stream)),
               "lod_result_copy_voxel_points_to_host")
        return out

    def free(self):
        if self._h:
            lib().lod_free(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _dev_ptr(points):
    """Device pointer and point count of a CUDA int32 tensor shaped (N, 4)."""
    import torch
    if not (isinstance(points, torch.Tensor) and points.is_cuda):
        raise TypeError("points must be a CUDA tensor")
    if points.dtype != torch.int32 or points.dim() != 2 or points.shape[1] != 4 or not points.is_contiguous():
        raise TypeError("points must be a contiguous int32 tensor of shape (N, 4)")
    return points.data_ptr(), points.shape[0]


def build(points, leaf_threshold=50000, mode=FILTER, max_depth=21, keep_index=False, stream=None,
          full_precision=False) -> Result:
    """lod_build on a CUDA int32 (N, 4) tensor of (x, y, z, rgba) rows."""
    ptr, n = _dev_ptr(points)
    p = make_params(leaf_threshold, mode, max_depth, keep_index, full_precision)
    h = ctypes.c_void_p()
    _check(lib().lod_build(ptr if n else None, n, ctypes.byref(p), _stream_handle(stream), ctypes.byref(h)),
           "lod_build")
    return Result(h.value)


def make_camera(view_proj, origin, width: int, height: int, lod_pixels: float = 100.0) -> Camera:
    m = np.ascontiguousarray(np.asarray(view_proj, dtype=np.float32).reshape(16))
    c = Camera()
    c.view_proj[:] = [float(x) for x in m]
    c.origin[:] = [int(x) for x in np.asarray(origin).reshape(3)]
    c.width, c.height, c.lod_pixels = int(width), int(height), float(lod_pixels)
    return c


def render(result: "Result", view_proj, origin, width: int, height: int, lod_pixels: float = 100.0, out=None,
           stream=None, stats: bool = False):
    """lod_render: rasterise ``result`` into a CUDA int64 tensor (height,
    width) of keys (bits of depth in [0, 1] << 32 | rgba; -1 where nothing
    was drawn).
    With ``stats`` returns (framebuffer, {"visible_nodes", "samples_drawn"})."""
    import torch
    if out is None:
        out = torch.empty((height, width), dtype=torch.int64, device="cuda")
    if not (isinstance(out, torch.Tensor) and out.is_cuda and out.dtype == torch.int64 and out.is_contiguous()
            and tuple(out.shape) == (height, width)):
        raise TypeError("out must be a contiguous CUDA int64 tensor of shape (height, width)")
    cam = make_camera(view_proj, origin, width, height, lod_pixels)
    st = RenderStats()
    _check(lib().lod_render(result.handle, ctypes.byref(cam), out.data_ptr(), _stream_handle(stream),
                            ctypes.byref(st) if stats else None), "lod_render")
    if stats:
        return out, {"visible_nodes": int(st.visible_nodes), "samples_drawn": int(st.samples_drawn)}
    return out


def build_from_host(points, leaf_threshold=50000, mode=FILTER, max_depth=21, keep_index=False,
                    stream=None) -> Result:
    """lod_build_from_host on host memory: a numpy array or a (pinned) CPU tensor."""
    if isinstance(points, np.ndarray):
        if points.ndim != 2 or points.shape[1] != 4:
            raise TypeError("host points must have shape (N, 4)")
        arr = np.ascontiguousarray(points, dtype=np.int32)
        ptr, n, keep = arr.ctypes.data, arr.shape[0], arr
    else:
        import torch
        if not isinstance(points, torch.Tensor) or points.is_cuda or points.dtype != torch.int32 \
                or points.dim() != 2 or points.shape[1] != 4 or not points.is_contiguous():
            raise TypeError("host points must be a numpy array or a contiguous int32 CPU tensor of shape (N, 4)")
        ptr, n, keep = points.data_ptr(), points.shape[0], points
    p = make_params(leaf_threshold, mode, max_depth, keep_index)
    h = ctypes.c_void_p()
    _check(lib().lod_build_from_host(ptr if n else None, n, ctypes.byref(p), _stream_handle(stream),
                                     ctypes.byref(h)), "lod_build_from_host")
    del keep
    return Result(h.value)


def _host_ptr(points):
    """Pointer and length of host points: a numpy array or a CPU int32 tensor shaped (N, 4)."""
    if isinstance(points, np.ndarray):
        if points.ndim != 2 or points.shape[1] != 4:
            raise TypeError("host points must have shape (N, 4)")
        arr = np.ascontiguousarray(points, dtype=np.int32)
        return arr.ctypes.data, arr.shape[0], arr
    import torch
    if not isinstance(points, torch.Tensor) or points.is_cuda or points.dtype != torch.int32 \
            or points.dim() != 2 or points.shape[1] != 4 or not points.is_contiguous():
        raise TypeError("host points must be a numpy array or a contiguous int32 CPU tensor of shape (N, 4)")
    return points.data_ptr(), points.shape[0], points


def build_out_of_core(points, leaf_threshold=50000, mode=FILTER, max_depth=21, keep_index=False,
                      chunk_points=0, stream_points=0, batch_points=0, stream=None) -> Result:
    """lod_build_out_of_core: the octree of host points built chunk by
    chunk (0 selects each size's default)."""
    ptr, n, keep = _host_ptr(points)
    p = make_params(leaf_threshold, mode, max_depth, keep_index)
    cfg = OocConfig(int(chunk_points), int(stream_points), int(batch_points))
    h = ctypes.c_void_p()
    _check(lib().lod_build_out_of_core(ptr if n else None, n, ctypes.byref(p), ctypes.byref(cfg),
                                       _stream_handle(stream), ctypes.byref(h)), "lod_build_out_of_core")
    del keep
    return Result(h.value)


def build_batched(tiles, leaf_threshold=50000, mode=FILTER, max_depth=21, keep_index=False,
                  stream=None) -> list:
    """lod_build_batched over a list of CUDA int32 (N_t, 4) tensors."""
    nt = len(tiles)
    ptrs = (ctypes.c_void_p * nt)()
    ns = (ctypes.c_uint64 * nt)()
    for t, x in enumerate(tiles):
        ptr, n = _dev_ptr(x)
        ptrs[t] = ptr if n else None
        ns[t] = n
    p = make_params(leaf_threshold, mode, max_depth, keep_index)
    outs = (ctypes.c_void_p * nt)()
    _check(lib().lod_build_batched(ptrs, ns, nt, ctypes.byref(p), _stream_handle(stream), outs),
           "lod_build_batched")
    return [Result(outs[t]) for t in range(nt)]


def root_cubes_noalloc(tiles, out, stream=None) -> None:
    """lod_root_cubes_noalloc: root cube (min x, y, z, log2 edge) of every
    CUDA int32 (N_t, 4) tensor in ``tiles`` into the caller's CUDA int32
    tensor ``out`` of shape (len(tiles), 4).  The library allocates no device
    memory for this call (its scratch is a static device array)."""
    import torch
    nt = len(tiles)
    if not (isinstance(out, torch.Tensor) and out.is_cuda and out.dtype == torch.int32
            and tuple(out.shape) == (nt, 4) and out.is_contiguous()):
        raise TypeError("out must be a contiguous CUDA int32 tensor of shape (n_tiles, 4)")
    ptrs = (ctypes.c_void_p * max(nt, 1))()
    ns = (ctypes.c_uint64 * max(nt, 1))()
    for t, x in enumerate(tiles):
        ptr, n = _dev_ptr(x)
        ptrs[t] = ptr if n else None
        ns[t] = n
    _check(lib().lod_root_cubes_noalloc(ptrs, ns, nt, out.data_ptr(), _stream_handle(stream)),
           "lod_root_cubes_noalloc")


class Server:
    """Serving loop: lod_server_create / lod_submit / lod_poll / lod_wait."""

    def __init__(self, hbm_budget_bytes: int, max_inflight: int = 4):
        cfg = ServerConfig(int(hbm_budget_bytes), int(max_inflight), 0)
        h = ctypes.c_void_p()
        _check(lib().lod_server_create(ctypes.byref(cfg), ctypes.byref(h)), "lod_server_create")
        self._h = h
        self._inputs = {}

    def submit(self, points, leaf_threshold=50000, mode=FILTER, max_depth=21, keep_index=False) -> int:
        ptr, n = _dev_ptr(points)
        p = make_params(leaf_threshold, mode, max_depth, keep_index)
        t = ctypes.c_uint64()
        _check(lib().lod_submit(self._h, ptr if n else None, n, ctypes.byref(p), ctypes.byref(t)), "lod_submit")
        self._inputs[t.value] = points  # keep the input alive until the result is taken
        return t.value

    def poll(self, ticket: int):
        h = ctypes.c_void_p()
        rc = lib().lod_poll(self._h, ticket, ctypes.byref(h))
        if rc == LOD_NOT_READY:
            return None
        self._inputs.pop(ticket, None)
        _check(rc, "lod_poll")
        return Result(h.value)

    def wait(self, ticket: int, timeout_ms: int = 600000) -> Result:
        h = ctypes.c_void_p()
        rc = lib().lod_wait(self._h, ticket, timeout_ms, ctypes.byref(h))
        if rc != LOD_ERR_TIMEOUT:
            self._inputs.pop(ticket, None)
        _check(rc, "lod_wait")
        return Result(h.value)

    def bytes_in_use(self) -> int:
        return int(lib().lod_server_bytes_in_use(self._h))

    def close(self):
        if self._h:
            _check(lib().lod_server_destroy(self._h), "lod_server_destroy")
            self._h = ctypes.c_void_p(0)
            self._inputs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
