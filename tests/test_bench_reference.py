"""The reference arm of bench.py (the CPU oracle, timed on the host) keeps
the benchmark's JSON contract, on CPU: one line with the same metric, unit
and direction as the GPU arm and the keys the driver reads; under a
multi-rank launch only rank 0 prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e")


def run(env_extra, *args):
    env = dict(os.environ, **env_extra)
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--workload", "sphere1m", "--steps", "2",
           "--warmup", "3", *args]
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    p = run({})
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in KEYS:
        assert k in d, k
    assert d["impl"] == "reference" and d["higher_is_better"] is True and d["unit"] == "M points/s"
    assert d["steps"] == 2 and d["warmup"] == 3 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] == 1 and d["cpu_baseline"]["host_cores"] >= 1
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_reference_arm_other_ranks_exit_quietly():
    p = run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert p.returncode == 0, p.stderr[-2000:]
    assert not [l for l in p.stdout.splitlines() if l.strip().startswith("{")]


def test_oracle_sample_is_one_definition():
    # the cpu_baseline leg and the reference arm time the oracle on the
    # same sample: the smallest lower-corner x-y window (1/4096, 1/2048, ...
    # of the area) that holds at least the requested number of points
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    rng = np.random.default_rng(3)
    pts = np.zeros((200_000, 4), np.int32)
    pts[:, :3] = rng.integers(0, 1 << 20, size=(200_000, 3))
    s, frac = bench.oracle_sample(pts, min_points=5_000)
    assert frac == 1.0 / 32 and len(s) >= 5_000
    side = int(np.floor(np.sqrt(frac) * ((1 << 20) - 1 - 0 + 1)))
    lo = pts[:, :2].min(axis=0)
    assert np.all((s[:, :2] >= lo) & (s[:, :2] < lo + side))
    inside = np.all((pts[:, :2] >= lo) & (pts[:, :2] < lo + side), axis=1)
    assert len(s) == int(inside.sum())
    s2, frac2 = bench.oracle_sample(pts, min_points=10**9)
    assert frac2 == 1.0 and len(s2) == len(pts)


def test_roofline_object_of_the_dominant_kernel():
    sys.path.insert(0, ROOT)
    import bench
    prof = {"scatter": {"launches": 4, "total_ms": 4.0, "alg_bytes": 4 * 1.6e9},
            "voxelize": {"launches": 24, "total_ms": 4.8, "alg_bytes": 24 * 1.9e8},
            "bbox": {"launches": 4, "total_ms": 0.5, "alg_bytes": 4 * 8e8}}
    pk = {"hbm_gbs": 6785.9, "source": "measured"}
    r = bench.roofline_of(prof, "indoor1b", pk)
    assert r["kernel"] == "voxelize" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - 24 * 1.9e8 / 4.8e-3 / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved"] / 6785.9) < 1e-12
    assert abs(r["avg_launch_ms"] - 0.2) < 1e-12 and r["alg_bytes_per_launch"] == 1.9e8
    assert isinstance(r["traffic"], int) and r["traffic"] > 0  # from profiles/traffic.json
    assert "shared-memory" in r["limiter"]
    assert bench.roofline_of({}, "indoor1b", pk) is None
    assert bench.roofline_of(prof, "sphere1m", pk)["traffic"] is None  # no capture of that workload
