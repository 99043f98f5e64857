"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle,
bit-exact, on seeded synthetic inputs spanning many chunks and ragged
tails, the edge cases of the method, and the batched / host-input /
serving entry points.  Modes: 0 cell-wise average (filtered), 1 minimal
splitmix64 pick, 3 first come, 4 random with Listing 1's key."""
import numpy as np
import pytest

import oracle
from bruteforce import check
from compare import compare
from paper_2302_14801_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lod():
    import torch
    from paper_2302_14801_gb300 import _build_ext
    _build_ext.build()
    from paper_2302_14801_gb300 import lod as m
    torch.cuda.set_device(0)
    return m


def gpu_build(lod, pts, T, mode, max_depth=21, keep_index=False):
    import torch
    d = torch.from_numpy(np.ascontiguousarray(pts, dtype=np.int32)).cuda()
    r = lod.build(d, T, mode, max_depth, keep_index)
    got = r.to_host()
    r.free()
    return got


def parity(lod, pts, T, mode, max_depth=21, keep_index=False):
    got = gpu_build(lod, pts, T, mode, max_depth, keep_index)
    want = oracle.build(pts, T, mode, max_depth)
    compare(got, want, inp=pts)
    return got


def P(rows):
    a = np.asarray(rows, dtype=np.int64).reshape(-1, 6)
    out = np.empty((len(a), 4), np.int32)
    out[:, :3] = a[:, :3]
    out[:, 3] = synth.pack_rgba(a[:, 3], a[:, 4], a[:, 5])
    return out


# ------------------------------------------------------------- edge cases

@pytest.mark.parametrize("mode", [0, 1, 3, 4])
def test_empty(lod, mode):
    got = gpu_build(lod, np.zeros((0, 4), np.int32), 10, mode)
    assert len(got["level"]) == 1 and got["flags"][0] == 1 and got["point_count"][0] == 0
    assert list(got["min"][0]) == [0, 0, 0] and got["log2_size"][0] == 0


@pytest.mark.parametrize("mode", [0, 1, 3, 4])
def test_single_point_and_leaf_root(lod, mode):
    parity(lod, P([(5, -7, 9, 1, 2, 3)]), 1, mode)
    parity(lod, synth.sphere(3000, seed=3), 3000, mode)


@pytest.mark.parametrize("mode", [0, 1, 3, 4])
def test_identical_points_and_chains(lod, mode):
    parity(lod, P([(5, 5, 5, 1, 2, 3)] * 1000), 3, mode)
    pts = P([(0, 0, 0, 1, 1, 1)] * 9 + [(1023, 0, 0, 2, 2, 2)])
    for md in (21, 5, 1, 0):
        parity(lod, pts, 3, mode, md)


@pytest.mark.parametrize("mode", [0, 1, 3, 4])
def test_full_int32_extent(lod, mode):
    rng = np.random.default_rng(5)
    xyz = rng.integers(-(2**31), 2**31, size=(5000, 3))
    xyz[0] = [-(2**31)] * 3
    xyz[1] = [2**31 - 1] * 3
    pts = np.empty((5000, 4), np.int32)
    pts[:, :3] = xyz
    pts[:, 3] = rng.integers(-(2**31), 2**31, size=5000)
    got = parity(lod, pts, 40, mode)
    assert got["log2_size"][0] == 32


@pytest.mark.parametrize("mode", [0, 1, 3, 4])
def test_lattices(lod, mode):
    g = np.stack(np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij"), -1).reshape(-1, 3)
    rows = np.concatenate([g, np.full((512, 3), 9)], axis=1)
    for T in (7, 8, 64):
        parity(lod, P(rows), T, mode)
    parity(lod, P([(i, 0, 0, i % 256, 0, 0) for i in range(1024)]), 100, mode)


@pytest.mark.parametrize("n", [4095, 4096, 4097, 3 * 4096 + 1])
def test_chunk_boundaries(lod, n):
    pts = synth.sphere(n, seed=n)
    for mode in (0, 1, 3, 4):
        parity(lod, pts, 200, mode)


def _random_cloud(rng, n, spread_log2):
    kind = rng.integers(0, 3)
    if kind == 0:
        xyz = rng.integers(-(2**spread_log2), 2**spread_log2, size=(n, 3))
    elif kind == 1:
        c = rng.integers(0, 2**spread_log2, size=(4, 3))
        xyz = c[rng.integers(0, 4, size=n)] + rng.integers(0, 3, size=(n, 3))
    else:
        xyz = rng.integers(0, 2**spread_log2, size=(n, 3))
        xyz[:, 2] = 77
    out = np.empty((n, 4), np.int32)
    out[:, :3] = xyz
    out[:, 3] = rng.integers(-(2**31), 2**31, size=n)
    return out


@pytest.mark.parametrize("seed", range(16))
def test_random_tiny_deep_trees(lod, seed):
    rng = np.random.default_rng(7000 + seed)
    n = int(rng.integers(1, 2000))
    T = int(rng.integers(1, 17))
    max_depth = int(rng.choice([21, 3, 1, 6, 32]))
    pts = _random_cloud(rng, n, int(rng.integers(1, 31)))
    for mode in (0, 1, 3, 4):
        got = parity(lod, pts, T, mode, max_depth)
        if n <= 600:
            check(pts, got, T, mode, max_depth)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("extra", [0, 1])
def test_threshold_boundary(lod, mode, extra):
    # exactly T points stay one leaf; T + 1 points split (leaf iff n <= T)
    T = 5000
    pts = synth.sphere(T + extra, seed=11)
    got = parity(lod, pts, T, mode)
    assert (len(got["level"]) == 1) == (extra == 0)


@pytest.mark.parametrize("mode", [0, 1])
def test_tuning_never_changes_results(lod, mode):
    # root depth and CTAs per SM are speed knobs: every setting gives the
    # oracle's result (a shallow first grid forces refinement rounds, a deep
    # one a sparse first grid)
    pts = synth.aerial(600_000, seed=12, n_buildings=40)
    want = oracle.build(pts, 5000, mode, 21)
    try:
        # (ranges of 300 or 1000 cells make most items take several
        # accumulate passes, in their own CTA (queue 1) or handed to others)
        for rd, cps, bins, queue, merge, cells in ((1, 1, 8, 1, 1, 300), (3, 0, 64, 0, 0, 0),
                                                   (5, 3, 512, 2, 1, 1000), (8, 2, 4096, 4096, 0, 0)):
            lod.set_tuning(rd, cps, bins, queue, 0, merge, cells)
            compare(gpu_build(lod, pts, 5000, mode), want, inp=pts)
    finally:
        lod.set_tuning(0, 0)


def test_autotune_picks_a_candidate_and_keeps_results(lod):
    import torch
    pts = synth.aerial(400_000, seed=13, n_buildings=30)
    d = torch.from_numpy(pts).cuda()
    try:
        best = lod.autotune(d, 5000, 0)
        assert best["stream_ctas_per_sm"] in (0, 2, 3, 4) and best["ms"] > 0
        assert best["vox_queue_ranges"] in (0, 1, 2) and best["dense_bins_max"] in (0, 512)
        assert lod.get_tuning()["stream_ctas_per_sm"] == best["stream_ctas_per_sm"]
        compare(gpu_build(lod, pts, 5000, 0), oracle.build(pts, 5000, 0, 21), inp=pts)
    finally:
        lod.set_tuning(0, 0)


# --------------------------------------------------- workload-shaped inputs

@pytest.mark.parametrize("mode", [0, 1, 3, 4])
def test_sphere_1m_default_T(lod, mode):
    parity(lod, synth.sphere(1_000_000, seed=1), 50000, mode)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("T", [50000, 3000])
def test_aerial_2m(lod, mode, T):
    parity(lod, synth.aerial(2_000_000, seed=2, n_buildings=80), T, mode)


@pytest.mark.parametrize("mode", [0, 1, 3, 4])
@pytest.mark.parametrize("T", [50000, 2000])
def test_indoor_dense_clusters_refinement(lod, mode, T):
    # log-normal densities put millions of points into single first-grid
    # cells: exercises several refinement rounds
    parity(lod, synth.indoor(3_000_000, seed=3, n_prims=256), T, mode)


@pytest.mark.parametrize("mode", [0, 1, 3, 4])
def test_volumetric_octants_overflow_tables(lod, mode):
    # 400k points uniform in a cube with T = 150k: every child octant of the
    # root holds ~50k distinct cells, more than one accumulate pass can hold,
    # so items take several rank ranges (handed to other SMs at the default
    # setting).
    rng = np.random.default_rng(31)
    pts = np.empty((400_000, 4), np.int32)
    pts[:, :3] = rng.integers(0, 1 << 16, size=(400_000, 3))
    pts[:, 3] = rng.integers(-(2**31), 2**31, size=400_000)
    parity(lod, pts, 150_000, mode)
    parity(lod, pts, 20_000, mode)


@pytest.mark.parametrize("mode", [0, 1, 3, 4])
def test_rank_ranges_all_modes(lod, mode):
    # accumulate ranges of 97 or 500 cells: nearly every item is taken in
    # several ranges, all in its own CTA (queue setting 1) or handed to the
    # partition kernel (2), and the top levels' up-front split units each
    # hold several ranges too
    pts = synth.indoor(300_000, seed=21, n_prims=64)
    want = oracle.build(pts, 5000, mode, 21)
    try:
        for queue, cells in ((1, 97), (2, 500), (3, 97)):
            lod.set_tuning(vox_queue_ranges=queue, vox_range_cells=cells)
            compare(gpu_build(lod, pts, 5000, mode), want, inp=pts)
    finally:
        lod.set_tuning()


def test_keep_index_filtered(lod):
    pts = synth.sphere(200_000, seed=12)
    got = gpu_build(lod, pts, 5000, 0, keep_index=True)
    assert got["index"] is not None
    want = oracle.build(pts, 5000, 0)
    compare(got, want, inp=pts)


# ----------------------------------------------------------- other entry points

def test_build_from_host(lod):
    pts = synth.aerial(300_000, seed=21, n_buildings=10)
    r = lod.build_from_host(pts, 4000, 1)
    got = r.to_host()
    r.free()
    compare(got, oracle.build(pts, 4000, 1, 21), inp=pts)


def test_trim_frees_scratch_and_keeps_results(lod):
    import torch
    pts = synth.aerial(400_000, seed=23, n_buildings=10)
    want = oracle.build(pts, 5000, 0, 21)
    st = torch.cuda.Stream()
    d = torch.from_numpy(pts).cuda()
    torch.cuda.synchronize()
    r = lod.build(d, 5000, 0, stream=st)
    assert lod.scratch_bytes(st) > 0  # the stream keeps its workspace
    lod.trim(st)
    assert lod.scratch_bytes(st) == 0
    compare(r.to_host(stream=st), want, inp=pts)  # a result outlives the trim
    r.free()
    r = lod.build(d, 5000, 0, stream=st)  # the next build allocates again
    assert lod.scratch_bytes(st) > 0
    compare(r.to_host(stream=st), want, inp=pts)
    r.free()
    lod.trim(st)
    assert lod.scratch_bytes(st) == 0


@pytest.mark.parametrize("mode", [0, 1, 3, 4])
def test_batched_equals_single(lod, mode):
    import torch
    sizes = [0, 1, 17, 4096, 4097, 30_000, 250_000, 1_000_000, 60_000, 5]
    tiles = [synth.sphere_tile(int(n), seed=100 + i) for i, n in enumerate(sizes)]
    dts = [torch.from_numpy(t).cuda() for t in tiles]
    rs = lod.build_batched(dts, 20000, mode)
    for t, r in zip(tiles, rs):
        got = r.to_host()
        compare(got, oracle.build(t, 20000, mode, 21), inp=t)
    for r in rs:
        r.free()


def test_server_alone_and_in_mix_identical(lod):
    import torch
    tiles = [synth.sphere_tile(int(n), seed=500 + i) for i, n in
             enumerate([300_000, 20_000, 1_200_000, 5_000, 700_000, 90_000])]
    dts = [torch.from_numpy(t).cuda() for t in tiles]
    torch.cuda.synchronize()
    srv = lod.Server(hbm_budget_bytes=8 << 30, max_inflight=4)
    try:
        tickets = [srv.submit(d, 30000, 1) for d in dts]
        mixed = [srv.wait(tk).to_host() for tk in tickets]
        alone = []
        for d in dts:
            tk = srv.submit(d, 30000, 1)
            alone.append(srv.wait(tk).to_host())
    finally:
        srv.close()
    for t, a, b in zip(tiles, alone, mixed):
        want = oracle.build(t, 30000, 1, 21)
        compare(a, want, inp=t)
        compare(b, want, inp=t)


def test_server_budget_rejects_oversized(lod):
    import torch
    srv = lod.Server(hbm_budget_bytes=1 << 20, max_inflight=1)
    try:
        d = torch.from_numpy(synth.sphere(100_000, seed=2)).cuda()
        with pytest.raises(lod.LodError) as e:
            srv.submit(d, 1000, 0)
        assert e.value.status == lod.LOD_ERR_BUDGET
    finally:
        srv.close()


# ---------------------------------------------------------------- golden

@pytest.mark.parametrize("mode", [0, 1, 3, 4])
def test_hand_worked_examples(lod, mode):
    import golden
    for path, m in golden.cases(modes=(mode,)):
        fx = golden.load(path)
        got = gpu_build(lod, fx["input"], fx["T"], m, fx["max_depth"])
        golden.check(got, fx, m)


# ------------------------------------------------------------ failure paths

def _pool_used_bytes():
    """Bytes in use in the current device's default stream-ordered pool (the
    pool the library's results and pool buffers come from), read through the
    CUDA runtime the library is linked against."""
    import ctypes

    import torch
    try:
        rt = ctypes.CDLL("libcudart.so.13")
    except OSError:
        pytest.skip("CUDA runtime library not found by name")
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), torch.cuda.current_device()) == 0
    val = ctypes.c_uint64()
    used_mem_current = 7  # cudaMemPoolAttrUsedMemCurrent
    assert rt.cudaMemPoolGetAttribute(pool, used_mem_current, ctypes.byref(val)) == 0
    return val.value


@pytest.mark.parametrize("mode", [0, 1])
def test_injected_allocation_failure_fails_cleanly(lod, mode, monkeypatch):
    # the k-th device allocation of a build fails (on the host side, never
    # asked of CUDA): the build returns LOD_ERR_OOM, holds no pool memory
    # afterwards, and the next build is correct
    import torch
    pts = synth.indoor(400_000, seed=41, n_prims=64)
    d = torch.from_numpy(pts).cuda()
    st = torch.cuda.current_stream()
    r = lod.build(d, 3000, mode, stream=st)  # warm: workspace and pool set up
    r.free()
    torch.cuda.synchronize()
    base = _pool_used_bytes()
    failed = 0
    for k in range(1, 400):
        monkeypatch.setenv("LOD_INJECT_OOM_AT", str(k))
        try:
            r = lod.build(d, 3000, mode, stream=st)
        except lod.LodError as e:
            assert e.status == lod.LOD_ERR_OOM, e
            failed += 1
            torch.cuda.synchronize()
            assert _pool_used_bytes() == base, f"pool memory held after failing allocation {k}"
            continue
        r.free()
        break
    else:
        raise AssertionError("every injected failure point failed the build")
    assert failed >= 10
    monkeypatch.delenv("LOD_INJECT_OOM_AT")
    torch.cuda.synchronize()
    assert _pool_used_bytes() == base
    compare(gpu_build(lod, pts, 3000, mode), oracle.build(pts, 3000, mode, 21), inp=pts)


def test_wait_times_out_and_the_request_still_completes(lod):
    import torch
    big = torch.from_numpy(synth.aerial(20_000_000, seed=42, n_buildings=200)).cuda()
    small_np = synth.sphere(500_000, seed=43)
    small = torch.from_numpy(small_np).cuda()
    torch.cuda.synchronize()
    srv = lod.Server(hbm_budget_bytes=64 << 30, max_inflight=1)
    try:
        t_big = srv.submit(big, 50000, 0)
        t_small = srv.submit(small, 20000, 1)  # queued behind the big build (one slot)
        with pytest.raises(lod.LodError) as e:
            srv.wait(t_small, timeout_ms=0)
        assert e.value.status == lod.LOD_ERR_TIMEOUT
        got = srv.wait(t_small).to_host()  # the ticket is still valid and completes
        srv.wait(t_big).free()
    finally:
        srv.close()
    compare(got, oracle.build(small_np, 20000, 1, 21), inp=small_np)


# ------------------------------------------- full-precision variant (Section 7)

@pytest.mark.parametrize("mode", [1, 3, 4])
def test_full_precision_voxel_points(lod, mode):
    # each voxel also carries the input point it picked, unquantised: the
    # input record at its pick_index, lying inside the voxel's cell
    import torch
    pts = synth.aerial(500_000, seed=44, n_buildings=20)
    d = torch.from_numpy(pts).cuda()
    r = lod.build(d, 5000, mode, full_precision=True)
    got = r.to_host()
    vp = r.voxel_points_host()
    r.free()
    compare(got, oracle.build(pts, 5000, mode, 21), inp=pts)
    vox = got["voxels"]
    assert np.array_equal(vp, pts[vox[:, 3].astype(np.int64)])
    for i in np.nonzero(got["voxel_count"])[0]:
        a, c = int(got["voxel_offset"][i]), int(got["voxel_count"][i])
        dd = vp[a:a + c, :3].astype(np.int64) - got["min"][i].astype(np.int64)
        L = int(got["log2_size"][i])
        q = (dd >> (L - 7)) if L >= 7 else (dd << (7 - L))
        assert np.array_equal(q[:, 0] | (q[:, 1] << 7) | (q[:, 2] << 14), vox[a:a + c, 0].astype(np.int64))
    for m in (0, 2):  # the averaging modes have no single picked point
        with pytest.raises(lod.LodError) as e:
            lod.build(d, 5000, m, full_precision=True)
        assert e.value.status == lod.LOD_ERR_INVALID_ARG


# ------------------------------------------------- CUDA-graph voxel levels

def test_graph_captured_voxel_levels_equal_oracle(lod):
    # with graph_voxel_levels every build launches its voxel levels as one
    # captured CUDA graph: single and batched builds, every mode
    import torch
    pts = synth.aerial(700_000, seed=45, n_buildings=30)
    sizes = [0, 1, 5000, 70_000, 300_000]
    tiles = [synth.sphere_tile(int(m), seed=600 + i) for i, m in enumerate(sizes)]
    before = lod.get_tuning()
    try:
        lod.set_tuning(graph_voxel_levels=1)
        for mode in (0, 1, 2, 3, 4):
            compare(gpu_build(lod, pts, 5000, mode), oracle.build(pts, 5000, mode, 21), inp=pts)
        rs = lod.build_batched([torch.from_numpy(t).cuda() for t in tiles], 20000, 0)
        for t, r in zip(tiles, rs):
            compare(r.to_host(), oracle.build(t, 20000, 0, 21), inp=t)
            r.free()
    finally:
        lod.set_tuning(**before)
