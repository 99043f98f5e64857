"""Camera matrices for ``lod.render`` (host-side helpers, not part of the
build): a row-major 4x4 ``view_proj`` applied to positions relative to an
integer ``origin``, as ``lod_camera_t`` in include/lod.h expects.  Matrices
are formed in double precision and stored as float32."""
from __future__ import annotations

import numpy as np


def _normalize(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


def perspective(eye, target, up=(0.0, 0.0, 1.0), fovy_deg: float = 60.0, aspect: float = 16 / 9,
                near: float = 1.0, far: float = 1e8):
    """Look-at perspective camera (OpenGL conventions: clip w = distance in
    front of the eye).  Returns (view_proj float32 (4, 4), origin int32 (3,)),
    the origin being the eye rounded to integers."""
    eye = np.asarray(eye, dtype=np.float64)
    origin = np.round(eye).astype(np.int64)
    e = eye - origin
    f = _normalize(np.asarray(target, dtype=np.float64) - eye)
    s = _normalize(np.cross(f, up))
    u = np.cross(s, f)
    view = np.eye(4)
    view[0, :3], view[1, :3], view[2, :3] = s, u, -f
    view[0, 3], view[1, 3], view[2, 3] = -s @ e, -u @ e, f @ e
    t = 1.0 / np.tan(np.radians(fovy_deg) / 2)
    proj = np.zeros((4, 4))
    proj[0, 0] = t / aspect
    proj[1, 1] = t
    proj[2, 2] = (far + near) / (near - far)
    proj[2, 3] = 2 * far * near / (near - far)
    proj[3, 2] = -1.0
    return (proj @ view).astype(np.float32), origin.astype(np.int32)


def orthographic(lo, hi):
    """Axis-aligned orthographic camera looking down -z onto the box
    [lo, hi] (x to the right, y up, w = 1).  Returns (view_proj, origin)."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    origin = np.floor(lo).astype(np.int64)
    a, b = lo - origin, hi - origin
    m = np.zeros((4, 4))
    for i in range(3):
        m[i, i] = 2.0 / (b[i] - a[i])
        m[i, 3] = -(b[i] + a[i]) / (b[i] - a[i])
    m[2, 2], m[2, 3] = -m[2, 2], -m[2, 3]  # nearer (larger z) gives smaller depth
    m[3, 3] = 1.0
    return m.astype(np.float32), origin.astype(np.int32)
