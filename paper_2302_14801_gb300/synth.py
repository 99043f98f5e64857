"""Seeded synthetic point clouds shaped like the paper's evaluation workloads.

The paper evaluates on four scanned data sets (Section 6, Figure 4 and
Table 1: Retz, Palmyra, Saint Roman, CA21 Bunds) that are not available
here.  These generators stand in for them.  They hold none of the LOD
construction's arithmetic: they only draw points.  Both the CUDA path and
the CPU oracle consume the very same byte buffers produced here.

Every cloud is returned as an ``(N, 4)`` int32 array whose rows are
``x, y, z, rgba`` (RGBA8 packed with R in the low byte, A in the high
byte), i.e. the 16-byte point record of the library.  All draws use
``numpy.random.default_rng(seed)`` (PCG64), which yields the same stream on
every platform.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "pack_rgba",
    "sphere",
    "aerial",
    "indoor",
    "tile_sizes",
    "sphere_tile",
    "poisson_arrivals",
]

_CHUNK = 1 << 22


def pack_rgba(r, g, b, a=255):
    """Pack 8-bit channels (any int arrays, clamped to 0..255) into int32."""
    r = np.clip(r, 0, 255).astype(np.uint32)
    g = np.clip(g, 0, 255).astype(np.uint32)
    b = np.clip(b, 0, 255).astype(np.uint32)
    a = np.clip(np.broadcast_to(a, r.shape), 0, 255).astype(np.uint32)
    return (r | (g << 8) | (b << 16) | (a << 24)).view(np.int32)


def _gradient_color(rng, xyz, lo, hi):
    """Linear position gradient (x->R, y->G, z->B over [lo, hi]) + U[-16,16]."""
    span = float(max(hi - lo, 1))
    t = (xyz.astype(np.float64) - lo) * (255.0 / span)
    noise = rng.integers(-16, 17, size=xyz.shape)
    c = np.rint(t).astype(np.int64) + noise
    return pack_rgba(c[:, 0], c[:, 1], c[:, 2])


def sphere(n: int, seed: int = 1, radius_log2: int = 19, offset=(0, 0, 0)) -> np.ndarray:
    """Points uniform on a sphere of radius 2^r centred in a 2^(r+1) cube.

    With the defaults this is the 1M-point sphere workload: radius 2^19,
    centre (2^19)^3, coordinates clamped into [0, 2^20).  ``offset`` shifts
    the whole cloud (used for independent tiles with their own bbox).
    """
    rng = np.random.default_rng(seed)
    out = np.empty((n, 4), dtype=np.int32)
    r = float(1 << radius_log2)
    hi = (1 << (radius_log2 + 1)) - 1
    off = np.asarray(offset, dtype=np.int64)
    for s in range(0, n, _CHUNK):
        m = min(_CHUNK, n - s)
        d = rng.standard_normal((m, 3))
        d /= np.maximum(np.linalg.norm(d, axis=1, keepdims=True), 1e-300)
        p = np.clip(np.rint(r + r * d), 0, hi).astype(np.int64)
        out[s:s + m, 3] = _gradient_color(rng, p, 0, hi)
        out[s:s + m, :3] = p + off
    return out


class _ValueNoise2D:
    """Smooth 2-D value noise on a square lattice of random values in [0, 1)."""

    def __init__(self, rng, cells: int):
        self.cells = cells
        self.table = rng.random((cells + 2, cells + 2))

    def __call__(self, u, v):
        # u, v in lattice units, 0 <= u, v < cells
        iu = np.floor(u).astype(np.int64)
        iv = np.floor(v).astype(np.int64)
        fu = u - iu
        fv = v - iv
        fu = fu * fu * (3.0 - 2.0 * fu)
        fv = fv * fv * (3.0 - 2.0 * fv)
        t = self.table
        a = t[iu, iv]
        b = t[iu + 1, iv]
        c = t[iu, iv + 1]
        d = t[iu + 1, iv + 1]
        return (a * (1 - fu) + b * fu) * (1 - fv) + (c * (1 - fu) + d * fu) * fv


class _Fbm:
    """6-octave fBm of value noise: lacunarity 2, gain 1/2, peak amplitude ``amp``."""

    def __init__(self, rng, domain_log2: int, amp: float, octaves: int = 6, base_cells: int = 4):
        self.domain = float(1 << domain_log2)
        self.layers = []
        norm = sum(0.5 ** o for o in range(octaves))
        for o in range(octaves):
            cells = base_cells << o
            self.layers.append((cells, amp * (0.5 ** o) / norm, _ValueNoise2D(rng, cells)))

    def __call__(self, x, y):
        z = np.zeros(x.shape, dtype=np.float64)
        for cells, a, noise in self.layers:
            s = cells / self.domain
            z += a * noise(x * s, y * s)
        return z


def _height_color(rng, z, zlo, zhi):
    t = np.clip((z.astype(np.float64) - zlo) / max(zhi - zlo, 1.0), 0.0, 1.0)
    noise = rng.integers(-16, 17, size=(z.shape[0], 3))
    r = np.rint(255.0 * t).astype(np.int64) + noise[:, 0]
    g = np.rint(255.0 * (1.0 - np.abs(2.0 * t - 1.0))).astype(np.int64) + noise[:, 1]
    b = np.rint(255.0 * (1.0 - t)).astype(np.int64) + noise[:, 2]
    return pack_rgba(r, g, b)


def aerial(n: int, seed: int = 2, n_buildings: int = 2000) -> np.ndarray:
    """Aerial-LiDAR-like cloud (stand-in for CA21 Bunds).

    90 % terrain: x, y ~ U[0, 2^24), z = 6-octave fBm heightfield with
    amplitude 2^18 plus N(0, 64) noise.  10 % on the walls and roofs of
    vertical boxes ("buildings"): footprint log-uniform in [2^8, 2^12],
    height U[2^10, 2^14], standing on the terrain.  RGBA8 = height ramp +
    U[-16, 16] noise, A = 255.
    """
    rng = np.random.default_rng(seed)
    amp = float(1 << 18)
    fbm = _Fbm(rng, 24, amp)
    dom = 1 << 24
    n_b = n // 10 if n_buildings > 0 else 0
    n_t = n - n_b
    out = np.empty((n, 4), dtype=np.int32)
    zlo, zhi = 0.0, amp + float(1 << 14)
    for s in range(0, n_t, _CHUNK):
        m = min(_CHUNK, n_t - s)
        x = rng.integers(0, dom, size=m)
        y = rng.integers(0, dom, size=m)
        z = np.rint(fbm(x.astype(np.float64), y.astype(np.float64)) + rng.normal(0.0, 64.0, size=m))
        out[s:s + m, 0] = x
        out[s:s + m, 1] = y
        out[s:s + m, 2] = z.astype(np.int64)
        out[s:s + m, 3] = _height_color(rng, z, zlo, zhi)
    if n_b:
        cx = rng.integers(0, dom, size=n_buildings).astype(np.float64)
        cy = rng.integers(0, dom, size=n_buildings).astype(np.float64)
        wx = np.exp(rng.uniform(np.log(2.0 ** 8), np.log(2.0 ** 12), size=n_buildings))
        wy = np.exp(rng.uniform(np.log(2.0 ** 8), np.log(2.0 ** 12), size=n_buildings))
        h = rng.uniform(2.0 ** 10, 2.0 ** 14, size=n_buildings)
        z0 = fbm(cx, cy)
        # faces: 0 roof, 1/2 walls at x0/x1 (area wy*h), 3/4 walls at y0/y1 (area wx*h)
        area = np.stack([wx * wy, wy * h, wy * h, wx * h, wx * h], axis=1)
        per_b = rng.multinomial(n_b, (area.sum(1) / area.sum()))
        s = n_t
        for i in range(n_buildings):
            m = int(per_b[i])
            if m == 0:
                continue
            face = rng.choice(5, size=m, p=area[i] / area[i].sum())
            u = rng.random(m)
            v = rng.random(m)
            x0, x1 = cx[i] - wx[i] / 2, cx[i] + wx[i] / 2
            y0, y1 = cy[i] - wy[i] / 2, cy[i] + wy[i] / 2
            px = np.where(face == 1, x0, np.where(face == 2, x1, x0 + u * wx[i]))
            py = np.where(face == 3, y0, np.where(face == 4, y1,
                          np.where(face == 0, y0 + v * wy[i], y0 + u * wy[i])))
            py = np.where((face == 1) | (face == 2), y0 + u * wy[i], py)
            pz = np.where(face == 0, z0[i] + h[i], z0[i] + v * h[i])
            px = np.clip(np.rint(px), 0, dom - 1).astype(np.int64)
            py = np.clip(np.rint(py), 0, dom - 1).astype(np.int64)
            pz = np.rint(pz + rng.normal(0.0, 64.0, size=m)).astype(np.int64)
            out[s:s + m, 0] = px
            out[s:s + m, 1] = py
            out[s:s + m, 2] = pz
            out[s:s + m, 3] = _height_color(rng, pz, zlo, zhi)
            s += m
        assert s == n
    return out


def indoor(n: int, seed: int = 3, n_prims: int = 4096, cube_log2: int = 22,
           sigma: float = 1.5) -> np.ndarray:
    """Indoor-scan-like cloud (stand-in for Saint Roman / Palmyra).

    ``n_prims`` primitives inside a 2^22 cube: half finite planes with a
    random orientation, half axis-aligned box surfaces, sizes log-uniform
    in [2^10, 2^20].  Point shares are log-normal (exp(sigma * Z)), rounded
    by largest remainder so that they sum to exactly ``n``; N(0, 32) noise
    along the surface normal; coordinates clamped into the cube.  Colours:
    position gradient + U[-16, 16].
    """
    rng = np.random.default_rng(seed)
    hi = (1 << cube_log2) - 1
    w = np.exp(sigma * rng.standard_normal(n_prims))
    share = w / w.sum() * n
    cnt = np.floor(share).astype(np.int64)
    rest = n - int(cnt.sum())
    if rest:
        cnt[np.argsort(-(share - cnt), kind="stable")[:rest]] += 1
    size = np.exp(rng.uniform(np.log(2.0 ** 10), np.log(2.0 ** 20), size=(n_prims, 3)))
    centre = rng.uniform(0, hi, size=(n_prims, 3))
    out = np.empty((n, 4), dtype=np.int32)
    s = 0
    for i in range(n_prims):
        m_total = int(cnt[i])
        # finite plane: one random orthonormal frame (t1, t2, normal) per primitive
        q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
        t1, t2, nrm = q[:, 0], q[:, 1], q[:, 2]
        done = 0
        while done < m_total:
            m = min(_CHUNK, m_total - done)
            if i % 2 == 0:
                u = (rng.random(m) - 0.5) * size[i, 0]
                v = (rng.random(m) - 0.5) * size[i, 1]
                p = centre[i] + u[:, None] * t1 + v[:, None] * t2
                p += rng.normal(0.0, 32.0, size=m)[:, None] * nrm
            else:
                # axis-aligned box surface: pick a face by area, uniform on it
                sx, sy, sz = size[i]
                areas = np.array([sy * sz, sy * sz, sx * sz, sx * sz, sx * sy, sx * sy])
                face = rng.choice(6, size=m, p=areas / areas.sum())
                uvw = rng.random((m, 3)) - 0.5
                axis = face // 2
                side = (face % 2) - 0.5
                uvw[np.arange(m), axis] = side
                uvw[np.arange(m), axis] += rng.normal(0.0, 32.0, size=m) / size[i, axis]
                p = centre[i] + uvw * size[i]
            p = np.clip(np.rint(p), 0, hi).astype(np.int64)
            out[s:s + m, :3] = p
            out[s:s + m, 3] = _gradient_color(rng, p, 0, hi)
            s += m
            done += m
    assert s == n
    return out


def tile_sizes(n_tiles: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """Tile point counts, log-uniform in [lo, hi] (int64)."""
    rng = np.random.default_rng(seed)
    return np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_tiles))).astype(np.int64)


def sphere_tile(n: int, seed: int) -> np.ndarray:
    """One independent tile: the sphere generator with its own seed and bbox offset."""
    rng = np.random.default_rng(seed ^ 0x5EED)
    off = rng.integers(0, (1 << 30) - (1 << 21), size=3)
    return sphere(n, seed=seed, offset=tuple(int(o) for o in off))


def poisson_arrivals(n: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Arrival times (seconds, ascending) of a Poisson process."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))
