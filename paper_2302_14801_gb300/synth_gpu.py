"""Device-side generators for the benchmark's largest workloads.

The same recipes as ``synth.sphere`` and ``synth.indoor`` (see there), drawn
with a seeded ``torch.Generator`` on the GPU instead of numpy: a billion
points take seconds here instead of minutes on the host.  The random
streams differ from the numpy ones, so these clouds are used for timing
only; parity tests use ``synth`` (whose clouds the CPU oracle also reads).
Like ``synth``, this module holds none of the LOD construction's arithmetic.

Clouds are ``(N, 4)`` int32 CUDA tensors with rows ``x, y, z, rgba``.
"""
from __future__ import annotations

import math

import torch

__all__ = ["sphere", "indoor", "pack_rgba"]


def pack_rgba(r: torch.Tensor, g: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """RGBA8 (A = 255) packed into int32, R in the low byte; channels clamped."""
    r = r.clamp(0, 255).to(torch.int64)
    g = g.clamp(0, 255).to(torch.int64)
    b = b.clamp(0, 255).to(torch.int64)
    v = r | (g << 8) | (b << 16) | (255 << 24)
    return (v - (1 << 32)).to(torch.int32)  # the top byte is 255: always >= 2^31


def _gradient(gen, p: torch.Tensor, hi: int) -> torch.Tensor:
    t = p.to(torch.float32) * (255.0 / float(max(hi, 1)))
    noise = torch.randint(-16, 17, p.shape, generator=gen, device=p.device)
    c = torch.round(t).to(torch.int64) + noise
    return pack_rgba(c[:, 0], c[:, 1], c[:, 2])


def sphere(n: int, seed: int = 1, radius_log2: int = 19, offset=(0, 0, 0), out=None,
           device="cuda") -> torch.Tensor:
    """Points uniform on a sphere of radius 2^r centred in a 2^(r+1) cube,
    shifted by ``offset``; colour = position gradient + U[-16, 16]."""
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    if out is None:
        out = torch.empty((n, 4), dtype=torch.int32, device=device)
    r = float(1 << radius_log2)
    hi = (1 << (radius_log2 + 1)) - 1
    off = torch.tensor(list(offset), dtype=torch.int64, device=device)
    chunk = 1 << 24
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        d = torch.randn((m, 3), generator=gen, device=device, dtype=torch.float32)
        d = d / d.norm(dim=1, keepdim=True).clamp_min(1e-30)
        p = torch.clamp(torch.round(r + r * d), 0, hi).to(torch.int64)
        out[s:s + m, 3] = _gradient(gen, p, hi)
        out[s:s + m, :3] = (p + off).to(torch.int32)
    return out


def indoor(n: int, seed: int = 3, n_prims: int = 4096, cube_log2: int = 22, sigma: float = 1.5,
           device="cuda") -> torch.Tensor:
    """Indoor-scan-like cloud: ``n_prims`` primitives in a 2^22 cube, half
    finite planes of random orientation, half axis-aligned box surfaces,
    sizes log-uniform in [2^10, 2^20], log-normal point shares (largest
    remainder, summing to n), N(0, 32) noise along the normal, clamped into
    the cube; colour = position gradient + U[-16, 16]."""
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    hi = (1 << cube_log2) - 1
    f64 = dict(device=device, dtype=torch.float64)
    w = torch.exp(sigma * torch.randn(n_prims, generator=gen, **f64))
    share = w / w.sum() * n
    cnt = torch.floor(share).to(torch.int64)
    rest = n - int(cnt.sum())
    if rest:
        order = torch.argsort(-(share - cnt.to(torch.float64)), stable=True)
        cnt[order[:rest]] += 1
    size = torch.exp(torch.empty((n_prims, 3), **f64).uniform_(math.log(2.0 ** 10), math.log(2.0 ** 20),
                                                                generator=gen))
    centre = torch.empty((n_prims, 3), **f64).uniform_(0, hi, generator=gen)
    out = torch.empty((n, 4), dtype=torch.int32, device=device)
    counts = cnt.tolist()
    sizes = size.tolist()
    s = 0
    chunk = 1 << 24
    for i in range(n_prims):
        # a random orthonormal frame: Gram-Schmidt on two Gaussian vectors
        # (plain tensor arithmetic, no linear-algebra library)
        g2 = torch.randn((2, 3), generator=gen, **f64)
        t1 = g2[0] / g2[0].norm()
        t2 = g2[1] - (g2[1] @ t1) * t1
        t2 = t2 / t2.norm()
        nrm = torch.stack([t1[1] * t2[2] - t1[2] * t2[1], t1[2] * t2[0] - t1[0] * t2[2],
                           t1[0] * t2[1] - t1[1] * t2[0]])
        done = 0
        while done < counts[i]:
            m = min(chunk, counts[i] - done)
            if i % 2 == 0:
                u = (torch.rand(m, generator=gen, **f64) - 0.5) * sizes[i][0]
                v = (torch.rand(m, generator=gen, **f64) - 0.5) * sizes[i][1]
                p = centre[i] + u[:, None] * t1 + v[:, None] * t2
                p = p + torch.randn(m, generator=gen, **f64)[:, None] * 32.0 * nrm
            else:
                sx, sy, sz = sizes[i]
                areas = torch.tensor([sy * sz, sy * sz, sx * sz, sx * sz, sx * sy, sx * sy], **f64)
                face = torch.multinomial(areas / areas.sum(), m, replacement=True, generator=gen)
                uvw = torch.rand((m, 3), generator=gen, **f64) - 0.5
                axis = face // 2
                side = (face % 2).to(torch.float64) - 0.5
                ar = torch.arange(m, device=device)
                uvw[ar, axis] = side
                sz_axis = size[i][axis]
                uvw[ar, axis] += torch.randn(m, generator=gen, **f64) * 32.0 / sz_axis
                p = centre[i] + uvw * size[i]
            p = torch.clamp(torch.round(p), 0, hi).to(torch.int64)
            out[s:s + m, :3] = p.to(torch.int32)
            out[s:s + m, 3] = _gradient(gen, p, hi)
            s += m
            done += m
    assert s == n
    return out
