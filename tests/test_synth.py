"""The seeded input generators follow their stated recipes (shapes, bounds,
shares, determinism).  They hold none of the method's arithmetic; these
checks make sure the workloads the benchmark and the parity tests draw are
the ones their docstrings and the benchmark's config describe.  The
device-side generators run here on the CPU device of torch."""
import numpy as np
import pytest

from paper_2302_14801_gb300 import synth


def channels(rgba):
    u = np.asarray(rgba).view(np.uint32)
    return u & 255, (u >> 8) & 255, (u >> 16) & 255, u >> 24


def test_pack_rgba_layout_and_clamp():
    v = synth.pack_rgba(np.array([1, -5, 300]), np.array([2, 0, 0]), np.array([3, 0, 0]))
    r, g, b, a = channels(v)
    assert list(r) == [1, 0, 255] and list(g) == [2, 0, 0] and list(b) == [3, 0, 0]
    assert np.all(a == 255)
    assert v.dtype == np.int32


def test_sphere_radius_bounds_and_seed():
    n, rl = 20_000, 12
    p = synth.sphere(n, seed=5, radius_log2=rl)
    assert p.shape == (n, 4) and p.dtype == np.int32
    xyz = p[:, :3].astype(np.float64)
    assert xyz.min() >= 0 and xyz.max() <= (1 << (rl + 1)) - 1
    d = np.linalg.norm(xyz - float(1 << rl), axis=1)
    assert np.all(np.abs(d - (1 << rl)) <= 1.0)  # rounding moves a point by at most sqrt(3)/2
    assert np.all(channels(p[:, 3])[3] == 255)
    # colour follows position: R rises with x
    assert np.corrcoef(xyz[:, 0], channels(p[:, 3])[0])[0, 1] > 0.95
    assert np.array_equal(p, synth.sphere(n, seed=5, radius_log2=rl))
    assert not np.array_equal(p, synth.sphere(n, seed=6, radius_log2=rl))


def test_sphere_tile_offset_stays_in_int32():
    for seed in (1000, 1001, 1777):
        t = synth.sphere_tile(5000, seed)
        lo = t[:, :3].min(axis=0)
        hi = t[:, :3].max(axis=0)
        assert np.all(lo >= 0) and np.all(hi < (1 << 30) + (1 << 20))
        assert np.all(hi - lo <= (1 << 20))


def test_aerial_terrain_and_buildings():
    n = 50_000
    p = synth.aerial(n, seed=2, n_buildings=50)
    assert p.shape == (n, 4)
    terrain, bld = p[: n - n // 10], p[n - n // 10:]
    assert terrain[:, :2].min() >= 0 and terrain[:, :2].max() < (1 << 24)
    # x, y uniform over the 2^24 square: each quarter holds about a quarter
    q = (terrain[:, 0] >> 23) * 2 + (terrain[:, 1] >> 23)
    assert np.all(np.abs(np.bincount(q, minlength=4) / len(terrain) - 0.25) < 0.02)
    # heights: fBm of amplitude 2^18 plus noise, buildings up to 2^14 above
    assert np.abs(terrain[:, 2]).max() < 2 * (1 << 18)
    assert bld[:, :2].min() >= 0 and bld[:, :2].max() < (1 << 24)
    assert np.all(channels(p[:, 3])[3] == 255)
    assert np.array_equal(p, synth.aerial(n, seed=2, n_buildings=50))


def test_indoor_bounds_and_exact_count():
    n = 30_000
    p = synth.indoor(n, seed=3, n_prims=64)
    assert p.shape == (n, 4)
    assert p[:, :3].min() >= 0 and p[:, :3].max() <= (1 << 22) - 1
    assert np.array_equal(p, synth.indoor(n, seed=3, n_prims=64))


def test_tile_sizes_log_uniform():
    s = synth.tile_sizes(4000, 1e4, 2e7, seed=4)
    assert s.min() >= 1e4 and s.max() <= 2e7
    lg = np.log(s.astype(np.float64))
    a, b = np.log(1e4), np.log(2e7)
    assert abs(lg.mean() - (a + b) / 2) < 0.05 * (b - a)
    assert abs(lg.std() - (b - a) / np.sqrt(12)) < 0.05 * (b - a)


def test_poisson_arrivals_rate():
    t = synth.poisson_arrivals(20_000, 200.0, seed=5)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert abs(gaps.mean() - 1 / 200.0) < 0.03 / 200.0


def test_device_generators_follow_the_same_recipes():
    torch = pytest.importorskip("torch")
    from paper_2302_14801_gb300 import synth_gpu
    p = synth_gpu.sphere(20_000, seed=7, radius_log2=12, device="cpu").numpy()
    xyz = p[:, :3].astype(np.float64)
    assert xyz.min() >= 0 and xyz.max() <= (1 << 13) - 1
    d = np.linalg.norm(xyz - float(1 << 12), axis=1)
    assert np.all(np.abs(d - (1 << 12)) <= 1.0)
    assert np.all(channels(p[:, 3])[3] == 255)
    q = synth_gpu.indoor(20_000, seed=3, n_prims=32, device="cpu").numpy()
    assert q.shape == (20_000, 4)
    assert q[:, :3].min() >= 0 and q[:, :3].max() <= (1 << 22) - 1
    assert np.array_equal(q, synth_gpu.indoor(20_000, seed=3, n_prims=32, device="cpu").numpy())
    assert torch.equal(synth_gpu.pack_rgba(torch.tensor([1]), torch.tensor([2]), torch.tensor([3])),
                       torch.from_numpy(synth.pack_rgba(np.array([1]), np.array([2]), np.array([3]))))
