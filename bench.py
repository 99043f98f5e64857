#!/usr/bin/env python3
"""LOD build benchmark (one JSON line on stdout).

Workload (default): the billion-point indoor-scan-like cloud (4096 planes
and box surfaces with log-normal point shares in a 2^22 cube, int32 xyz +
RGBA8, 16 GB, drawn on the device), leaf threshold T = 50k, 128^3 voxel
grid.  ``--workload aerial50m`` selects the 50M-point aerial-LiDAR-like
cloud instead.  One step = one colour-filtered build plus one sample-pick
build of that cloud, with the input resident in HBM; ``value`` is points
built per second over both builds (M points/s).  Inputs are larger than
L2, so no flush is needed between steps.

Reported beside it: per-build latency p50/p99, the build's fraction of the
HBM roofline (algorithmic bytes 64 N + 16 V + 16 (V - V_root)), the
dominant kernel's live roofline (CUDA events on the launching stream), an
end-to-end figure through the host-buffer C-ABI call (input H2D and the
whole octree D2H inside the timed region), SM clocks sampled during the
timed region, and the CPU oracle timed on a bounded sample.

``--impl reference`` times the CPU oracle (the plain restatement of the
method in oracle/) on the same workload and metric instead, on the same
bounded sample as the cpu_baseline leg (``oracle_sample``).
Multi-GPU (torchrun): every rank builds its own replica (the method has no
exchange step); ``value`` is all ranks' points over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    # name: (generator, n, seed, T)
    "aerial50m": ("aerial", 50_000_000, 2, 50000),
    "sphere1m": ("sphere", 1_000_000, 1, 50000),
    "indoor100m": ("indoor", 100_000_000, 3, 50000),
    # small cases (inputs still larger than L2) for profiler captures
    "aerial12m": ("aerial", 12_000_000, 2, 50000),
    "indoor20m": ("indoor", 20_000_000, 3, 50000),
    # the billion-point indoor scan, drawn on the device (same recipe, torch RNG)
    "indoor1b": ("indoor_gpu", 1_000_000_000, 3, 50000),
}
METRIC = "LOD build M points/s (filtered & sample-pick), % HBM roofline; tile p50/p99 ms"


def gen(name: str, seed_offset: int = 0) -> np.ndarray:
    """Seeded workload; LOD_BENCH_CACHE=<dir> keeps a copy between runs
    (generation is outside every timed region)."""
    cache = os.environ.get("LOD_BENCH_CACHE")
    if cache:
        path = os.path.join(cache, f"{name}_{seed_offset}.npy")
        if os.path.exists(path):
            return np.load(path)
        pts = _gen(name, seed_offset)
        os.makedirs(cache, exist_ok=True)
        np.save(path, pts)
        return pts
    return _gen(name, seed_offset)


def on_device(name: str) -> bool:
    return WORKLOADS[name][0].endswith("_gpu")


def gen_device(name: str, seed_offset: int = 0, device: str = "cuda"):
    """Device-drawn workloads (their random stream is torch's, not numpy's)."""
    from paper_2302_14801_gb300 import synth_gpu
    g, n, seed, _ = WORKLOADS[name]
    if g == "indoor_gpu":
        return synth_gpu.indoor(n, seed=seed + seed_offset, device=device)
    return synth_gpu.sphere(n, seed=seed + seed_offset, device=device)


def _gen(name: str, seed_offset: int) -> np.ndarray:
    from paper_2302_14801_gb300 import synth
    g, n, seed, _ = WORKLOADS[name]
    if g == "aerial":
        return synth.aerial(n, seed=seed + seed_offset)
    if g == "sphere":
        return synth.sphere(n, seed=seed + seed_offset)
    return synth.indoor(n, seed=seed + seed_offset)


def peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [r.split(", ") for r in open(self.f.name).read().strip().splitlines() if r.count(",") >= 9]
        os.unlink(self.f.name)
        if self.uuid:
            mine = [r for r in rows if self.uuid in r[1]]
            rows = mine or rows
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[6 + j].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def b_alg(n_points: int, n_voxels: int, root_voxels: int) -> float:
    """Algorithmic bytes of one build: 64 B per point (bounding box read,
    one counting read, scatter read + write) + 16 B per voxel written + 16 B
    per non-root voxel read by its parent."""
    return 64.0 * n_points + 16.0 * n_voxels + 16.0 * (n_voxels - root_voxels)


def oracle_sample(cloud, min_points: int = 3_000_000) -> np.ndarray:
    """The bounded sample of a workload that the CPU oracle is timed on
    (the cpu_baseline leg and the reference arm use this one definition):
    the points inside the square x-y window at the cloud's lower x-y corner
    whose area is the smallest of 1/4096, 1/2048, 1/1024, ... of the cloud's
    x-y extent that holds at least ``min_points`` points (the same density and
    structure as the full cloud, at a size the oracle builds in seconds).
    ``cloud`` is an (N, 4) int32 numpy array or CUDA tensor."""
    is_np = isinstance(cloud, np.ndarray)
    if is_np:
        xy = cloud[:, :2].astype(np.int64)
        lo, hi = xy.min(axis=0), xy.max(axis=0)
    else:
        import torch
        xy = cloud[:, :2].to(torch.int64)
        lo = xy.min(dim=0).values.cpu().numpy()
        hi = xy.max(dim=0).values.cpu().numpy()
    frac = 1.0 / 4096
    while True:
        side = np.floor(np.sqrt(frac) * (hi - lo + 1)).astype(np.int64)
        if is_np:
            sel = np.all((xy >= lo) & (xy < lo + side), axis=1)
            cnt = int(sel.sum())
        else:
            import torch
            lo_t = torch.as_tensor(lo, device=xy.device)
            sel = ((xy >= lo_t) & (xy < lo_t + torch.as_tensor(side, device=xy.device))).all(dim=1)
            cnt = int(sel.sum().item())
        if cnt >= min_points or frac >= 1.0:
            break
        frac = min(1.0, frac * 2)
    out = np.ascontiguousarray(cloud[sel]) if is_np else cloud[sel].cpu().numpy()
    return out, frac


def time_oracle_pair(sample: np.ndarray, T: int) -> float:
    """Seconds for one filtered + one pick oracle build of ``sample``."""
    import oracle
    t0 = time.perf_counter()
    oracle.build(sample, T, 0, 21)
    oracle.build(sample, T, 1, 21)
    return time.perf_counter() - t0


def cpu_oracle_sample(cloud, T: int, budget_s: float = 12.0) -> dict:
    """The oracle (as it stands) on the bounded sample of ``oracle_sample``,
    repeated until about budget_s seconds of CPU work have run."""
    import oracle
    oracle.compile_oracle()
    sample, frac = oracle_sample(cloud)
    times = [time_oracle_pair(sample, T)]
    while sum(times) < budget_s and len(times) < 20:
        times.append(time_oracle_pair(sample, T))
    dt = statistics.median(times)
    n = len(sample)
    return {"value": 2.0 * n / dt / 1e6, "unit": "M points/s", "cores": 1, "host_cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"{n} points in the x-y corner window covering {frac * 100:.3g}% of the cloud's area; "
                      f"one filtered + one pick build per repetition, single-threaded, median of "
                      f"{len(times)} repetitions ({dt:.2f} s each)"}


# What the ncu captures in profiles/ show limiting each kernel that can be
# the dominant one (the roofline below stays HBM: the path has no dense
# contraction and no other measured peak applies).
LIMITERS = {
    "voxelize": "shared-memory pipe, over half of it atomics (ncu: short-scoreboard stalls, 0.6-0.7 shared "
                "wavefronts per active SM cycle, DRAM 3-6 % on the 20M cut)",
    "scatter": "scattered stores and load latency (ncu: long-scoreboard stalls, DRAM 45 %, 36 % L2 write hits)",
    "count": "instruction issue (ncu: 68 % issue active, DRAM 41 %)",
    "bbox": "HBM bandwidth",
}


def roofline_of(prof: dict, name: str, pk: dict):
    """The roofline object of the kernel with the largest share of the
    timed region: its algorithmic bytes per launch over its CUDA-event
    launch time against the measured HBM peak, with the DRAM traffic per
    launch from the committed ncu launch list when it covers this
    workload and kernel."""
    if not prof:
        return None
    dom = max(prof, key=lambda k: prof[k]["total_ms"])
    s = prof[dom]
    if not s["launches"] or not s["total_ms"]:
        return None
    ach = s["alg_bytes"] / (s["total_ms"] * 1e-3) / 1e9
    traffic = None
    tp = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tp):
        traffic = json.load(open(tp)).get(f"{name}:{dom}")
    return {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": ach / pk["hbm_gbs"], "traffic": traffic, "peak_source": pk["source"],
            "avg_launch_ms": s["total_ms"] / s["launches"], "alg_bytes_per_launch": s["alg_bytes"] / s["launches"],
            "limiter": LIMITERS.get(dom)}


def max_over_ranks(x: float, dist) -> float:
    """The slowest rank's time (all ranks call this with their own)."""
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_points_per_s(world: int, n_per_rank: int, ms_step: float) -> float:
    """Whole-job throughput (M points/s): every rank builds its own replica of
    n points in both modes per step; the step takes the slowest rank's time."""
    return world * 2.0 * n_per_rank / (ms_step * 1e-3) / 1e6


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    import oracle
    oracle.compile_oracle()
    name = args.workload
    _, n, _, T = WORKLOADS[name]
    if on_device(name):
        # drawn with the device generator (input preparation only; the timed
        # work below runs on the host cores)
        import torch
        cloud = gen_device(name) if torch.cuda.is_available() else gen_device(name, device="cpu")
    else:
        cloud = gen(name)
    sample, frac = oracle_sample(cloud)
    del cloud
    ns = len(sample)
    for _ in range(args.warmup):
        time_oracle_pair(sample, T)
    times = [time_oracle_pair(sample, T) for _ in range(args.steps)]
    t = sum(times) / len(times)
    value = 2.0 * ns / t / 1e6
    what = f"{ns} points in the x-y corner window covering {frac * 100:.3g}% of the cloud's area"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "M points/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32/u64", "data": "synthetic",
        "config": {"workload": f"{name}: {n} points, T={T}, 128^3 grid, filtered + pick; "
                               f"CPU oracle on {what}"},
        "cpu_baseline": {"value": value, "unit": "M points/s", "cores": 1, "host_cores": os.cpu_count(),
                         "kind": "oracle", "sample": f"{what}; one filtered + one pick build per step"},
        "e2e": {"value": value, "unit": "M points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _tile_offsets(n_tiles: int, seed0: int) -> list:
    """bbox offset of every tile (each tile is a sphere with its own seed and offset)."""
    out = []
    for t in range(n_tiles):
        rng = np.random.default_rng((seed0 + t) ^ 0x5EED)
        out.append(tuple(int(o) for o in rng.integers(0, (1 << 30) - (1 << 21), size=3)))
    return out


def apply_tuning(args):
    """The --tuning knobs (lod_set_tuning), if any."""
    tuning = {k: int(v) for k, v in (kv.split("=") for kv in args.tuning.split(",") if kv)}
    if tuning:
        from paper_2302_14801_gb300 import lod
        lod.set_tuning(**tuning)


def run_batched(args):
    """Many independent tiles (point counts log-uniform in [1e4, tile_max],
    each a sphere with its own seed and bbox), filtered mode, built with one
    lod_build_batched call per wave of about wave_points points; compared
    with building the same tiles one lod_build call after another."""
    import torch
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2302_14801_gb300 import lod, synth, synth_gpu
    apply_tuning(args)
    T = 50000
    sizes = synth.tile_sizes(args.tiles, 1e4, args.tile_max, seed=4 + rank)
    offs = _tile_offsets(args.tiles, 1000 + 100000 * rank)
    waves, cur, acc = [], [], 0
    for t, m in enumerate(sizes):
        if cur and acc + int(m) > args.wave_points:
            waves.append(cur)
            cur, acc = [], 0
        cur.append(t)
        acc += int(m)
    if cur:
        waves.append(cur)
    cap = max(sum(int(sizes[t]) for t in w) for w in waves)
    buf = torch.empty((cap, 4), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    def load(w):
        views, o = [], 0
        for t in w:
            m = int(sizes[t])
            synth_gpu.sphere(m, seed=1000 + t + 100000 * rank, offset=offs[t], out=buf[o:o + m])
            views.append(buf[o:o + m])
            o += m
        torch.cuda.synchronize()
        return views

    def timed(fn):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        rs = fn()
        b.record(stream)
        torch.cuda.synchronize()
        for r in rs:
            r.free()
        return a.elapsed_time(b)

    # warm-up on the first wave (fills the stream's scratch workspace)
    views = load(waves[0])
    for _ in range(max(1, args.warmup - 2)):
        timed(lambda: lod.build_batched(views, T, lod.FILTER, stream=stream))
        timed(lambda: [lod.build(v, T, lod.FILTER, stream=stream) for v in views])
    t_batch, t_single, wave_ms = 0.0, 0.0, []
    launches0 = lod.launch_count()
    for w in waves:
        views = load(w)
        ms = timed(lambda: lod.build_batched(views, T, lod.FILTER, stream=stream))
        wave_ms.append(ms)
        t_batch += ms
    launches = lod.launch_count() - launches0
    for w in waves:
        views = load(w)
        t_single += timed(lambda: [lod.build(v, T, lod.FILTER, stream=stream) for v in views])
    total = int(sizes.sum())
    if rank == 0:
        line = {
            "metric": METRIC, "suite": "batched", "value": world * total / (t_batch * 1e-3) / 1e6,
            "unit": "M points/s", "n_gpus": world, "steps": 1, "warmup": args.warmup,
            "ms_per_step": t_batch, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32/u64", "data": "synthetic (drawn on the device)",
            "config": {"workload": f"{args.tiles} tiles, sizes log-uniform in [1e4, {args.tile_max:.0e}] "
                                   f"({total} points), spheres with their own seed and bbox, T={T}, filtered; "
                                   f"{len(waves)} waves of <= {args.wave_points:.0e} points, one "
                                   "lod_build_batched call per wave", "replicas": world},
            "single_calls": {"value": total / (t_single * 1e-3) / 1e6, "unit": "M points/s",
                             "ms": t_single, "what": "the same tiles, one lod_build call each"},
            "batched_vs_single_calls": t_single / t_batch,
            "wave_ms": wave_ms, "gpu_launches": launches, "tuning": lod.get_tuning(),
        }
        print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    """Poisson stream of build requests through the serving loop
    (lod_submit / lod_poll): sizes log-uniform in [1e5, 5e7] points,
    alternately a sphere cloud and an aerial cloud (prefixes of shuffled
    50M-point clouds held on the device), both modes alternating by request,
    admitted by an HBM budget; reports submit->ready latency p50/p99 and
    points/s per arrival rate, against the same requests built one
    lod_build call after another."""
    import torch
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2302_14801_gb300 import lod, synth, synth_gpu
    apply_tuning(args)
    T = 50000
    n_max = 50_000_000
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    base = [synth_gpu.sphere(n_max, seed=1), torch.from_numpy(gen("aerial50m")).cuda()]
    base = [b[torch.randperm(n_max, generator=g, device="cuda")].contiguous() for b in base]
    torch.cuda.synchronize()
    rates = [float(r) for r in args.rates.split(",") if r]
    stream = torch.cuda.current_stream()
    results = []
    for ri, rate in enumerate(rates):
        n_req = args.requests
        warm = min(20, n_req)
        sizes = synth.tile_sizes(warm + n_req, 1e5, 5e7, seed=5000 + ri)
        arrive = synth.poisson_arrivals(warm + n_req, rate, seed=5 + ri)
        srv = lod.Server(int(args.budget_gb * 1e9), args.inflight)
        pend = {}  # ticket -> (k, arrival)
        lat, done_pts, first, last = [], 0, None, None
        k = 0
        t0 = time.perf_counter()
        while k < len(sizes) or pend:
            now = time.perf_counter() - t0
            while k < len(sizes) and arrive[k] <= now:
                m = int(sizes[k])
                tk = srv.submit(base[k % 2][:m], T, lod.FILTER if (k // 2) % 2 == 0 else lod.PICK)
                pend[tk] = (k, arrive[k], m)
                k += 1
            for tk in list(pend):
                r = srv.poll(tk)
                if r is None:
                    continue
                kk, arr, m = pend.pop(tk)
                t_ready = time.perf_counter() - t0
                r.free()
                if kk >= warm:
                    lat.append((t_ready - arr) * 1e3)
                    done_pts += m
                    first = arr if first is None else min(first, arr)
                    last = t_ready if last is None else max(last, t_ready)
            if k < len(sizes) and not pend:
                time.sleep(max(0.0, min(arrive[k] - (time.perf_counter() - t0), 0.002)))
            else:
                time.sleep(0.0002)
        srv.close()
        lat.sort()
        results.append({"rate_per_s": rate, "requests": n_req, "p50_ms": statistics.median(lat),
                        "p99_ms": lat[min(len(lat) - 1, int(round(0.99 * (len(lat) - 1))))],
                        "mpts_per_s": done_pts / max(last - first, 1e-9) / 1e6,
                        "offered_mpts_per_s": float(sizes[warm:].mean()) * rate / 1e6})
    # the same request mix built one after another with the plain call
    sizes = synth.tile_sizes(args.requests, 1e5, 5e7, seed=5000)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for kk, m in enumerate(sizes):
        r = lod.build(base[kk % 2][:int(m)], T, lod.FILTER if (kk // 2) % 2 == 0 else lod.PICK, stream=stream)
        r.free()
    b.record(stream)
    torch.cuda.synchronize()
    single = float(sizes.sum()) / (a.elapsed_time(b) * 1e-3) / 1e6
    if rank == 0:
        best = max(results, key=lambda x: x["mpts_per_s"])
        line = {
            "metric": METRIC, "suite": "serve", "value": best["mpts_per_s"], "unit": "M points/s",
            "n_gpus": world, "steps": args.requests, "warmup": 20, "ms_per_step": None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32/u64",
            "data": "synthetic (sphere drawn on the device, aerial from the seeded generator)",
            "config": {"workload": "Poisson arrivals, sizes log-uniform in [1e5, 5e7] points, sphere / aerial "
                                   "alternating, filtered / pick alternating, T=50000",
                       "hbm_budget_gb": args.budget_gb, "max_inflight": args.inflight},
            "rates": results, "single_calls_mpts_per_s": single,
        }
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="indoor1b", choices=sorted(WORKLOADS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra-modes", action="store_true", help="skip timing the weighted / first / random modes")
    ap.add_argument("--no-render", action="store_true", help="skip timing the rasteriser")
    ap.add_argument("--tuning", default="", help="lod_set_tuning knobs for this run, e.g. "
                    "'vox_queue_ranges=1,dense_bins_max=512' (default: the library's defaults)")
    ap.add_argument("--suite", default="single", choices=["single", "batched", "serve"],
                    help="single: the headline line; batched: many independent tiles per launch "
                         "(lod_build_batched); serve: Poisson request stream through lod_submit/lod_poll")
    ap.add_argument("--tiles", type=int, default=2048, help="batched: number of tiles")
    ap.add_argument("--tile-max", type=float, default=2e7, help="batched: largest tile size (points)")
    ap.add_argument("--wave-points", type=float, default=1e9, help="batched: points built per wave")
    ap.add_argument("--rates", default="10,20,50,100,200,500,1000,2000", help="serve: arrival rates (requests/s)")
    ap.add_argument("--requests", type=int, default=200, help="serve: timed requests per rate")
    ap.add_argument("--budget-gb", type=float, default=120.0, help="serve: HBM budget")
    ap.add_argument("--inflight", type=int, default=8, help="serve: concurrent builds")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.suite == "batched":
        return run_batched(args)
    if args.suite == "serve":
        return run_serve(args)

    import torch
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    import __graft_entry__
    __graft_entry__.build()
    from paper_2302_14801_gb300 import lod
    apply_tuning(args)

    name = args.workload
    _, n, _, T = WORKLOADS[name]
    if on_device(name):
        d = gen_device(name, seed_offset=rank)
        pts = None  # host copy only if the e2e leg or the CPU baseline asks for it
    else:
        pts = gen(name, seed_offset=rank)
        d = torch.from_numpy(pts).cuda()
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()

    def step(timings=None):
        rs = []
        for mode in (lod.FILTER, lod.PICK):
            if timings is not None:
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
            r = lod.build(d, T, mode, 21, stream=stream)
            if timings is not None:
                b.record(stream)
                timings[mode].append((a, b))
            rs.append(r)
        return rs

    # warm-up (also yields the voxel counts for the algorithmic bytes)
    info = {}
    for _ in range(args.warmup):
        rs = step()
        for mode, r in zip((lod.FILTER, lod.PICK), rs):
            v = r.view()
            h = r.to_host() if mode not in info else None
            if h is not None:
                root_vox = int(h["voxel_count"][0])
                info[mode] = {"voxels": int(v.n_voxels), "root_voxels": root_vox, "nodes": int(v.n_nodes),
                              "levels": int(v.n_levels)}
            r.free()
    torch.cuda.synchronize()

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    lod.profile_reset()
    lod.profile_enable(True)
    timings = {lod.FILTER: [], lod.PICK: []}
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = lod.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        for r in step(timings):
            r.free()
    e1.record(stream)
    torch.cuda.synchronize()
    launches = lod.launch_count() - launches0
    if dist:
        dist.barrier()
    clk = clocks.stop()
    lod.profile_enable(False)
    prof = lod.profile_read()
    ms_step = e0.elapsed_time(e1) / args.steps
    if dist:
        ms_step = max_over_ranks(ms_step, dist)
    value = job_points_per_s(world, n, ms_step)

    pk = peaks()
    per_mode = {}
    for mode, key in ((lod.FILTER, "filtered"), (lod.PICK, "pick")):
        lat = sorted(a.elapsed_time(b) for a, b in timings[mode])
        med = statistics.median(lat)
        p99 = lat[min(len(lat) - 1, int(round(0.99 * (len(lat) - 1))))]
        ba = b_alg(n, info[mode]["voxels"], info[mode]["root_voxels"])
        per_mode[key] = {"ms_p50": med, "ms_p99": p99, "mpts_per_s": n / (med * 1e-3) / 1e6,
                         "voxels": info[mode]["voxels"], "nodes": info[mode]["nodes"],
                         "levels": info[mode]["levels"], "alg_bytes": ba,
                         "hbm_frac": (ba / (med * 1e-3) / 1e9) / pk["hbm_gbs"]}

    # dominant kernel (largest total time) and its live roofline
    kern = {}
    for k, s in prof.items():
        if s["launches"]:
            kern[k] = {"launches": s["launches"], "avg_ms": s["total_ms"] / s["launches"],
                       "share": None, "alg_gbs": (s["alg_bytes"] / (s["total_ms"] * 1e-3) / 1e9) if s["total_ms"] else 0}
    tot = sum(s["total_ms"] for s in prof.values()) or 1.0
    for k in kern:
        kern[k]["share"] = prof[k]["total_ms"] / tot
    roof = roofline_of(prof, name, pk)

    # the other sampling modes, timed one build at a time outside the step
    # (weighted average, first come, random with Listing 1's key)
    extra = {}
    if not args.no_extra_modes:
        for mode, key in ((2, "weighted"), (3, "first"), (4, "random")):
            lat = []
            vox = root_vox = None
            for it in range(4):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                r = lod.build(d, T, mode, 21, stream=stream)
                b.record(stream)
                torch.cuda.synchronize()
                if it == 0:
                    vv = r.view()
                    vox = int(vv.n_voxels)
                    root_vox = int(r.tensors()["nodes"][0, 12].item())  # voxel_count of the root
                else:
                    lat.append(a.elapsed_time(b))
                r.free()
            med = statistics.median(lat)
            ba = b_alg(n, vox, root_vox)
            extra[key] = {"ms_p50": med, "mpts_per_s": n / (med * 1e-3) / 1e6, "voxels": vox, "alg_bytes": ba,
                          "hbm_frac": (ba / (med * 1e-3) / 1e9) / pk["hbm_gbs"], "builds_timed": len(lat),
                          "in_step": False}
    # rendering (Section 5): full-HD frames of the pick-mode octree
    render = None
    if not args.no_render:
        from paper_2302_14801_gb300 import camera
        r = lod.build(d, T, lod.PICK, 21, stream=stream)
        hn = r.to_host()
        L = int(hn["log2_size"][0])
        lo = hn["min"][0].astype(np.int64)
        c = lo + (1 << (L - 1))
        cams = {"overview": camera.perspective(c + [2 << L, -(1 << L), 1 << L], c, fovy_deg=50, aspect=16 / 9,
                                               near=1, far=1e9),
                "close": camera.perspective(c + [1 << (L - 4), 1 << (L - 5), 1 << (L - 4)], c, fovy_deg=70,
                                            aspect=16 / 9, near=1, far=1e9)}
        fb = torch.empty((1080, 1920), dtype=torch.int64, device="cuda")
        render = {"width": 1920, "height": 1080, "lod_pixels": 100.0}
        for cname, (m, org) in cams.items():
            _, stt = lod.render(r, m, org, 1920, 1080, 100.0, out=fb, stream=stream, stats=True)
            times = []
            for _ in range(10):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                lod.render(r, m, org, 1920, 1080, 100.0, out=fb, stream=stream)
                b.record(stream)
                torch.cuda.synchronize()
                times.append(a.elapsed_time(b))
            render[cname] = {"ms_p50": statistics.median(times), "visible_nodes": stt["visible_nodes"],
                             "samples_drawn": stt["samples_drawn"]}
        r.free()

    # end to end through the host-buffer call: H2D of the input + build + D2H of the octree
    e2e = None
    if not args.no_e2e:
        hp = (d.cpu() if pts is None else torch.from_numpy(pts)).pin_memory()
        # page-locked result buffers, sized by the warm-up builds
        vmax = max(i["voxels"] for i in info.values())
        nmax = max(i["nodes"] for i in info.values())
        hout = {"points": torch.empty((n, 4), dtype=torch.int32, pin_memory=True).numpy(),
                "index": torch.empty(n, dtype=torch.int32, pin_memory=True).numpy().view(np.uint32),
                "voxels": torch.empty((vmax, 4), dtype=torch.int32, pin_memory=True).numpy().view(np.uint32),
                "nodes": torch.empty(nmax * lod.NODE_DTYPE.itemsize, dtype=torch.uint8,
                                     pin_memory=True).numpy().view(lod.NODE_DTYPE)}
        h2d = d2h = 0
        t_e2e = []
        for it in range(args.warmup + max(1, args.steps // 2)):
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            bytes_out = 0
            for mode in (lod.FILTER, lod.PICK):
                r = lod.build_from_host(hp, T, mode, 21, stream=stream)
                h = r.to_host(stream=stream, out=hout)
                bytes_out += sum(x.nbytes for x in (h["points"], h["voxels"]) if x is not None)
                bytes_out += (h["index"].nbytes if h["index"] is not None else 0) + len(h["level"]) * 56
                r.free()
            b.record(stream)
            torch.cuda.synchronize()
            if it >= args.warmup:
                t_e2e.append(a.elapsed_time(b))
                h2d, d2h = 2 * n * 16, bytes_out
        me = statistics.median(t_e2e)
        e2e = {"value": world * 2.0 * n / (me * 1e-3) / 1e6, "unit": "M points/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": me}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(d if pts is None else pts, T)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "M points/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32/u64", "data": "synthetic",
            "config": {"workload": f"{name}: {n} points (seeded synthetic"
                                   f"{', drawn on the device' if on_device(name) else ''}), T={T}, 128^3 grid; "
                                   "step = 1 filtered + 1 pick build, input resident in HBM",
                       "l2": f"inputs ({n * 16 / 1e6:.0f} MB) larger than L2; no flush", "replicas": world,
                       "tuning": lod.get_tuning()},
            "modes": per_mode, "modes_extra": extra, "render": render, "roofline": roof, "kernels": kern,
            "gpu_launches": launches,
            "clocks": clk, "e2e": e2e, "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
