// Out-of-core build (Section 7 of the paper): the cloud stays in host
// memory and the device holds at most one batch of chunks under
// construction at a time, plus the output.
//
//  1. Stream the points through the device: bounding box -> root cube.
//  2. Stream again: counts over a top grid of 8^D cells (D <= 8).
//  3. On the host, the top of the octree from those counts: a node is a
//     chunk root when it holds at most `chunk_points` points, when it is a
//     leaf of the octree (at most T points, a unit cube or at max_depth), or
//     when it lies at the grid's depth D (then the chunk may be larger);
//     every other node is a root-side node, split into its octants.
//  4. Stream again: every point goes to its chunk's run in host memory,
//     with its input index (the pick rules and the reported indices use it).
//  5. Chunks are built in batches with the in-core engine, each with its
//     root cube, its level (the random strategy draws per level) and its
//     points' input indices; their results stay on the device.
//  6. The root-side nodes are filled bottom-up from their children's
//     samples (k_merge), the same sampling the in-core voxel passes do.
//  7. Nodes of all chunks and the root side are merged into one breadth-
//     first table; points are laid out chunk after chunk in depth-first
//     order, so the result equals the in-core build of the same cloud.
#include <algorithm>
#include <array>
#include <climits>
#include <cstring>
#include <map>
#include <memory>
#include <vector>

#include "engine.h"
#include "kernels.h"
#include "result.h"
#include "wgrid.cuh"

namespace lodk {

namespace {

#define OOC_CK(x)                                                          \
  do {                                                                     \
    cudaError_t e_ = (x);                                                  \
    if (e_ != cudaSuccess) {                                               \
      (void)cudaGetLastError();                                            \
      return e_ == cudaErrorMemoryAllocation ? LOD_ERR_OOM : LOD_ERR_CUDA; \
    }                                                                      \
  } while (0)

// Stream-ordered device buffer freed on destruction.
struct Dev {
  void* p = nullptr;
  cudaStream_t st = nullptr;
  explicit Dev(cudaStream_t s) : st(s) {}
  Dev(const Dev&) = delete;
  ~Dev() {
    if (p) cudaFreeAsync(p, st);
  }
  cudaError_t alloc(size_t b) {
    if (p) cudaFreeAsync(p, st);
    p = nullptr;
    return cudaMallocAsync(&p, b ? b : 16, st);
  }
  template <class T>
  T* as() const {
    return static_cast<T*>(p);
  }
  void* take() {
    void* q = p;
    p = nullptr;
    return q;
  }
};

// Pinned host memory freed on destruction.
struct Pinned {
  void* p = nullptr;
  ~Pinned() {
    if (p) cudaFreeHost(p);
  }
  cudaError_t alloc(size_t b) { return cudaMallocHost(&p, b ? b : 16); }
  template <class T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

int sms_of_device() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

// A node of the top of the octree: root-side (split further here) or a
// chunk root (built by the engine).
struct TopNode {
  int32_t min[3];
  uint32_t level, log2;
  uint64_t count;
  int32_t parent = -1;       // top node index
  uint32_t cell = 0;         // cell index at its level in the count pyramid
  bool chunk = false;
  uint32_t child_mask = 0;
  int32_t children[8];       // top node index per octant (-1 none)
  int32_t chunk_id = -1;
};

// Morton order of two cubes of the same size: compare the most significant
// differing bit over the three axes, x before y before z on ties (octant
// k = 4 bx + 2 by + bz).
bool morton_less(const uint32_t a[3], const uint32_t b[3]) {
  int axis = 0;
  uint32_t best = a[0] ^ b[0];
  for (int k = 1; k < 3; ++k) {
    const uint32_t d = a[k] ^ b[k];
    if (best < d && best < (best ^ d)) {  // d has a higher most significant bit
      axis = k;
      best = d;
    }
  }
  return a[axis] < b[axis];
}

}  // namespace

int build_out_of_core(const lod_point_t* h, uint64_t n, const lod_params_t& prm, const lod_ooc_config_t& cfg,
                      cudaStream_t st, std::shared_ptr<SharedBuffers>* sh_out, TileResult* tr_out) {
  if (!valid_params(prm) || (prm.flags & LOD_FLAG_FULL_PRECISION)) return LOD_ERR_INVALID_ARG;
  if (n > 0xFFFFFFFEull || (n && !h)) return LOD_ERR_INVALID_ARG;
  const uint32_t T = prm.leaf_threshold;
  const uint64_t C = cfg.chunk_points ? cfg.chunk_points : 10000000ull;
  const uint64_t B = std::min<uint64_t>(std::max<uint64_t>(n, 1), cfg.stream_points ? cfg.stream_points : (16ull << 20));
  const uint64_t batch_cap = cfg.batch_points ? cfg.batch_points : (256ull << 20);
  if (C < T) return LOD_ERR_INVALID_ARG;
  const bool want_idx = keeps_index(prm);
  const bool filt = prm.mode == LOD_FILTER;
  const int sms = sms_of_device();
  if (n == 0) {  // the empty cloud: one empty root leaf
    TileInput ti{nullptr, 0};
    std::vector<TileResult> trs;
    const int rc = run_build(&ti, 1, prm, st, sh_out, &trs, nullptr);
    if (rc == LOD_OK) *tr_out = trs[0];
    return rc;
  }

  // ---- 1. bounding box -> root cube
  Dev d_blk(st), d_box(st);
  OOC_CK(d_blk.alloc(B * 16));
  OOC_CK(d_box.alloc(24));
  const int box_init[6] = {INT_MAX, INT_MAX, INT_MAX, INT_MIN, INT_MIN, INT_MIN};
  OOC_CK(cudaMemcpyAsync(d_box.p, box_init, 24, cudaMemcpyHostToDevice, st));
  for (uint64_t off = 0; off < n; off += B) {
    const uint64_t m = std::min(B, n - off);
    OOC_CK(cudaMemcpyAsync(d_blk.p, h + off, m * 16, cudaMemcpyHostToDevice, st));
    OOC_CK(launch_ooc_bbox(d_blk.as<int4>(), m, d_box.as<int>(), sms, st));
  }
  int box[6];
  OOC_CK(cudaMemcpyAsync(box, d_box.p, 24, cudaMemcpyDeviceToHost, st));
  OOC_CK(cudaStreamSynchronize(st));
  OocGrid g;
  int64_t ext = 0;
  for (int a = 0; a < 3; ++a) {
    g.min[a] = box[a];
    ext = std::max<int64_t>(ext, (int64_t)box[3 + a] - (int64_t)box[a]);
  }
  uint32_t L = 0;
  while ((int64_t(1) << L) <= ext) ++L;  // smallest power of two above the extent
  g.L = L;
  g.D = std::min<uint32_t>(std::min<uint32_t>(8u, L), prm.max_depth);
  const uint32_t D = g.D;
  const uint64_t cells = 1ull << (3 * D);

  // ---- 2. top-grid counts and their pyramid (level j: x | y << j | z << 2j)
  Dev d_cnt(st);
  OOC_CK(d_cnt.alloc(cells * 4));
  OOC_CK(cudaMemsetAsync(d_cnt.p, 0, cells * 4, st));
  for (uint64_t off = 0; off < n; off += B) {
    const uint64_t m = std::min(B, n - off);
    OOC_CK(cudaMemcpyAsync(d_blk.p, h + off, m * 16, cudaMemcpyHostToDevice, st));
    OOC_CK(launch_ooc_count(d_blk.as<int4>(), m, g, d_cnt.as<unsigned int>(), sms, st));
  }
  std::vector<uint32_t> cnt(cells);
  OOC_CK(cudaMemcpyAsync(cnt.data(), d_cnt.p, cells * 4, cudaMemcpyDeviceToHost, st));
  OOC_CK(cudaStreamSynchronize(st));
  std::vector<std::vector<uint64_t>> pyr(D + 1);
  pyr[D].assign(cnt.begin(), cnt.end());
  for (int j = (int)D - 1; j >= 0; --j) {
    pyr[j].assign(1ull << (3 * j), 0);
    const uint32_t jj = (uint32_t)j + 1, mask = (1u << jj) - 1;
    for (uint64_t c = 0; c < pyr[jj].size(); ++c) {
      if (!pyr[jj][c]) continue;
      const uint32_t x = (uint32_t)c & mask, y = (uint32_t)(c >> jj) & mask, z = (uint32_t)(c >> (2 * jj));
      pyr[j][(x >> 1) | ((uint64_t)(y >> 1) << j) | ((uint64_t)(z >> 1) << (2 * j))] += pyr[jj][c];
    }
  }

  // ---- 3. the top of the octree, breadth first; chunk roots in depth-first order
  std::vector<TopNode> top(1);
  for (int a = 0; a < 3; ++a) top[0].min[a] = g.min[a];
  top[0].level = 0;
  top[0].log2 = L;
  top[0].count = pyr[0][0];
  for (size_t i = 0; i < top.size(); ++i) {
    std::fill(top[i].children, top[i].children + 8, -1);
    const bool leaf = top[i].count <= T || top[i].log2 == 0 || top[i].level >= prm.max_depth;
    if (leaf || top[i].count <= C || top[i].level >= D) {
      top[i].chunk = true;
      continue;
    }
    const uint32_t j = top[i].level, cm = (1u << j) - 1;
    const uint32_t x = top[i].cell & cm, y = (top[i].cell >> j) & cm, z = top[i].cell >> (2 * j);
    for (uint32_t k = 0; k < 8; ++k) {
      const uint32_t bx = (k >> 2) & 1u, by = (k >> 1) & 1u, bz = k & 1u;
      const uint64_t cc = (uint64_t)(2 * x + bx) | ((uint64_t)(2 * y + by) << (j + 1)) |
                          ((uint64_t)(2 * z + bz) << (2 * (j + 1)));
      const uint64_t c_n = pyr[j + 1][cc];
      if (!c_n) continue;
      TopNode ch;
      const int64_t half = int64_t(1) << (top[i].log2 - 1);
      ch.min[0] = (int32_t)(top[i].min[0] + bx * half);
      ch.min[1] = (int32_t)(top[i].min[1] + by * half);
      ch.min[2] = (int32_t)(top[i].min[2] + bz * half);
      ch.level = j + 1;
      ch.log2 = top[i].log2 - 1;
      ch.count = c_n;
      ch.parent = (int32_t)i;
      ch.cell = (uint32_t)cc;
      top[i].child_mask |= 1u << k;
      top[i].children[k] = (int32_t)top.size();
      top.push_back(ch);
    }
  }
  std::vector<int32_t> chunks;  // top node of each chunk, depth first (the final point layout order)
  {
    std::vector<int32_t> stack{0};
    while (!stack.empty()) {
      const int32_t i = stack.back();
      stack.pop_back();
      if (top[i].chunk) {
        top[i].chunk_id = (int32_t)chunks.size();
        chunks.push_back(i);
        continue;
      }
      for (int k = 7; k >= 0; --k)
        if (top[i].children[k] >= 0) stack.push_back(top[i].children[k]);
    }
  }
  const uint32_t nc = (uint32_t)chunks.size();
  std::vector<uint64_t> c_off(nc + 1, 0);
  for (uint32_t c = 0; c < nc; ++c) c_off[c + 1] = c_off[c] + top[chunks[c]].count;
  if (c_off[nc] != n) return LOD_ERR_INTERNAL;
  std::vector<uint32_t> cell_chunk(cells, 0xFFFFFFFFu);
  for (uint32_t c = 0; c < nc; ++c) {
    const TopNode& t = top[chunks[c]];
    const uint32_t j = t.level, cm = (1u << j) - 1, sh = D - j;
    const uint32_t x0 = (t.cell & cm) << sh, y0 = ((t.cell >> j) & cm) << sh, z0 = (t.cell >> (2 * j)) << sh;
    for (uint32_t z = z0; z < z0 + (1u << sh); ++z)
      for (uint32_t y = y0; y < y0 + (1u << sh); ++y)
        for (uint32_t x = x0; x < x0 + (1u << sh); ++x)
          cell_chunk[(uint64_t)x | ((uint64_t)y << D) | ((uint64_t)z << (2 * D))] = c;
  }

  // ---- 4. partition into the chunks' runs in host memory
  Pinned h_pts, h_idx;
  OOC_CK(h_pts.alloc(n * 16));
  OOC_CK(h_idx.alloc(n * 4));
  {
    Dev d_cc(st), d_of(st), d_hist(st), d_cur(st), d_part(st), d_pidx(st), d_err(st);
    OOC_CK(d_cc.alloc(cells * 4));
    OOC_CK(cudaMemcpyAsync(d_cc.p, cell_chunk.data(), cells * 4, cudaMemcpyHostToDevice, st));
    OOC_CK(d_of.alloc(B * 4));
    OOC_CK(d_hist.alloc(nc * 4));
    OOC_CK(d_cur.alloc(nc * 4));
    OOC_CK(d_part.alloc(B * 16));
    OOC_CK(d_pidx.alloc(B * 4));
    OOC_CK(d_err.alloc(4));
    OOC_CK(cudaMemsetAsync(d_err.p, 0, 4, st));
    std::vector<uint64_t> fill(c_off.begin(), c_off.end() - 1);
    std::vector<uint32_t> hist(nc), cur(nc);
    for (uint64_t off = 0; off < n; off += B) {
      const uint64_t m = std::min(B, n - off);
      OOC_CK(cudaMemcpyAsync(d_blk.p, h + off, m * 16, cudaMemcpyHostToDevice, st));
      OOC_CK(cudaMemsetAsync(d_hist.p, 0, nc * 4, st));
      OOC_CK(launch_ooc_chunk_of(d_blk.as<int4>(), m, g, d_cc.as<uint32_t>(), nc, d_of.as<uint32_t>(),
                                 d_hist.as<unsigned int>(), d_err.as<unsigned int>(), sms, st));
      OOC_CK(cudaMemcpyAsync(hist.data(), d_hist.p, nc * 4, cudaMemcpyDeviceToHost, st));
      OOC_CK(cudaStreamSynchronize(st));
      uint64_t acc = 0;
      for (uint32_t c = 0; c < nc; ++c) {
        cur[c] = (uint32_t)acc;
        acc += hist[c];
      }
      if (acc != m) return LOD_ERR_INTERNAL;  // a point outside every chunk
      OOC_CK(cudaMemcpyAsync(d_cur.p, cur.data(), nc * 4, cudaMemcpyHostToDevice, st));
      OOC_CK(launch_ooc_partition(d_blk.as<int4>(), m, (uint32_t)off, d_of.as<uint32_t>(), nc,
                                  d_cur.as<unsigned int>(), d_part.as<int4>(), d_pidx.as<uint32_t>(), sms, st));
      for (uint32_t c = 0; c < nc; ++c) {
        if (!hist[c]) continue;
        if (fill[c] + hist[c] > c_off[c + 1]) return LOD_ERR_INTERNAL;
        OOC_CK(cudaMemcpyAsync(h_pts.as<int4>() + fill[c], d_part.as<int4>() + cur[c], (size_t)hist[c] * 16,
                               cudaMemcpyDeviceToHost, st));
        OOC_CK(cudaMemcpyAsync(h_idx.as<uint32_t>() + fill[c], d_pidx.as<uint32_t>() + cur[c], (size_t)hist[c] * 4,
                               cudaMemcpyDeviceToHost, st));
        fill[c] += hist[c];
      }
    }
    unsigned int err = 0;
    OOC_CK(cudaMemcpyAsync(&err, d_err.p, 4, cudaMemcpyDeviceToHost, st));
    OOC_CK(cudaStreamSynchronize(st));
    if (err) return LOD_ERR_INTERNAL;
    for (uint32_t c = 0; c < nc; ++c)
      if (fill[c] != c_off[c + 1]) return LOD_ERR_INTERNAL;
  }
  cudaFreeAsync(d_blk.take(), st);

  // ---- 5. chunk builds, in batches of chunks of one level (max_depth and
  // the random draws depend on the level)
  struct ChunkOut {
    uint32_t batch = 0;
    TileResult tr;
    std::vector<lod_node_t> nodes;  // the chunk's node table (levels relative to its root)
  };
  std::vector<ChunkOut> co(nc);
  std::vector<std::shared_ptr<SharedBuffers>> bsh;
  {
    std::vector<uint32_t> order(nc);
    for (uint32_t c = 0; c < nc; ++c) order[c] = c;
    std::stable_sort(order.begin(), order.end(),
                     [&](uint32_t a, uint32_t b) { return top[chunks[a]].level < top[chunks[b]].level; });
    size_t i0 = 0;
    while (i0 < nc) {
      const uint32_t lvl = top[chunks[order[i0]]].level;
      size_t i1 = i0;
      uint64_t pts = 0;
      while (i1 < nc && top[chunks[order[i1]]].level == lvl &&
             (i1 == i0 || pts + top[chunks[order[i1]]].count <= batch_cap)) {
        pts += top[chunks[order[i1]]].count;
        ++i1;
      }
      const uint32_t k = (uint32_t)(i1 - i0);
      Dev d_cp(st), d_ci(st);
      OOC_CK(d_cp.alloc(pts * 16));
      OOC_CK(d_ci.alloc(pts * 4));
      std::vector<TileInput> ti(k);
      std::vector<std::array<int32_t, 4>> cubes(k);
      uint64_t bo = 0;
      for (uint32_t q = 0; q < k; ++q) {
        const uint32_t c = order[i0 + q];
        const TopNode& t = top[chunks[c]];
        const uint64_t m = t.count;
        OOC_CK(cudaMemcpyAsync(d_cp.as<int4>() + bo, h_pts.as<int4>() + c_off[c], m * 16, cudaMemcpyHostToDevice, st));
        OOC_CK(cudaMemcpyAsync(d_ci.as<uint32_t>() + bo, h_idx.as<uint32_t>() + c_off[c], m * 4,
                               cudaMemcpyHostToDevice, st));
        cubes[q] = {t.min[0], t.min[1], t.min[2], (int32_t)t.log2};
        ti[q].d_points = reinterpret_cast<const lod_point_t*>(d_cp.as<int4>() + bo);
        ti[q].n = m;
        ti[q].d_index = d_ci.as<uint32_t>() + bo;
        ti[q].index_bound = (uint32_t)n;
        ti[q].cube = cubes[q].data();
        ti[q].level0 = lvl;
        bo += m;
      }
      lod_params_t pb = prm;
      pb.max_depth = prm.max_depth - lvl;
      BuildOptions opt;
      opt.keep_root_sums = filt;
      std::shared_ptr<SharedBuffers> sh;
      std::vector<TileResult> trs;
      const int rc = run_build(ti.data(), k, pb, st, &sh, &trs, nullptr, true, opt);
      if (rc != LOD_OK) return rc;
      for (uint32_t q = 0; q < k; ++q) {
        const uint32_t c = order[i0 + q];
        co[c].batch = (uint32_t)bsh.size();
        co[c].tr = trs[q];
        co[c].nodes.resize(trs[q].n_nodes);
        OOC_CK(cudaMemcpyAsync(co[c].nodes.data(), static_cast<const lod_node_t*>(sh->nodes) + trs[q].node_base,
                               trs[q].n_nodes * sizeof(lod_node_t), cudaMemcpyDeviceToHost, st));
      }
      bsh.push_back(sh);
      OOC_CK(cudaStreamSynchronize(st));
      i0 = i1;
    }
  }

  // ---- 6. root-side nodes, deepest level first
  struct TopOut {
    const int4* recs = nullptr;
    const ulonglong2* sums = nullptr;
    uint64_t count = 0;
  };
  std::vector<TopOut> tout(top.size());
  std::vector<std::unique_ptr<Dev>> keep;  // merge outputs (part of the result until assembled)
  {
    uint32_t max_lvl = 0, max_jobs = 0;
    std::map<uint32_t, std::vector<int32_t>> by_level;
    for (size_t i = 0; i < top.size(); ++i)
      if (!top[i].chunk) by_level[top[i].level].push_back((int32_t)i);
    for (auto& kv : by_level) {
      max_lvl = std::max(max_lvl, kv.first);
      max_jobs = std::max<uint32_t>(max_jobs, (uint32_t)kv.second.size());
    }
    Dev d_grid(st);
    const uint32_t G = std::max<uint32_t>(1, std::min<uint32_t>(max_jobs, (uint32_t)sms));
    if (max_jobs) {
      OOC_CK(d_grid.alloc((size_t)G * kGridCells * 40));
      OOC_CK(cudaMemsetAsync(d_grid.p, 0, (size_t)G * kGridCells * 36, st));
    }
    for (auto it = by_level.rbegin(); it != by_level.rend(); ++it) {
      const uint32_t lvl = it->first;
      const std::vector<int32_t>& jobs_i = it->second;
      std::vector<MergeJob> jobs;
      std::vector<MergeSeg> segs;
      uint64_t cap = 0;
      for (int32_t i : jobs_i) {
        MergeJob J;
        std::memset(&J, 0, sizeof(J));
        for (int a = 0; a < 3; ++a) J.min[a] = top[i].min[a];
        J.log2 = top[i].log2;
        J.level = lvl;
        J.seg0 = (uint32_t)segs.size();
        uint64_t samples = 0;
        for (uint32_t k = 0; k < 8; ++k) {
          const int32_t c = top[i].children[k];
          if (c < 0) continue;
          MergeSeg S;
          std::memset(&S, 0, sizeof(S));
          S.octant = k;
          if (!top[c].chunk) {
            S.recs = tout[c].recs;
            S.sums = tout[c].sums;
            S.n = (uint32_t)tout[c].count;
            S.kind = 1;
          } else {
            const ChunkOut& o = co[top[c].chunk_id];
            const SharedBuffers& b = *bsh[o.batch];
            const lod_node_t& root = o.nodes[0];
            if (root.flags & LOD_NODE_LEAF) {
              S.recs = static_cast<const int4*>(b.points) + o.tr.pt_base;
              S.idx = b.index ? static_cast<const uint32_t*>(b.index) + o.tr.pt_base : nullptr;
              S.n = (uint32_t)root.point_count;
              S.kind = 0;
            } else {
              S.recs = static_cast<const int4*>(b.voxels) + root.voxel_offset;
              S.sums = b.root_sums ? static_cast<const ulonglong2*>(b.root_sums) + root.voxel_offset : nullptr;
              S.n = root.voxel_count;
              S.kind = 1;
            }
            if (prm.mode != LOD_FILTER && prm.mode != LOD_WEIGHTED && S.kind == 0 && !S.idx) return LOD_ERR_INTERNAL;
            if (prm.mode == LOD_FILTER && S.kind == 1 && !S.sums) return LOD_ERR_INTERNAL;
          }
          samples += S.n;
          segs.push_back(S);
        }
        J.nseg = (uint32_t)segs.size() - J.seg0;
        cap += std::min<uint64_t>(samples, kGridCells);
        jobs.push_back(J);
      }
      const uint32_t nj = (uint32_t)jobs.size();
      keep.emplace_back(new Dev(st));
      Dev& out = *keep.back();
      keep.emplace_back(new Dev(st));
      Dev& out_sums = *keep.back();
      Dev d_jobs(st), d_segs(st), d_res(st), d_ctr(st);
      OOC_CK(out.alloc(cap * 16));
      if (filt) OOC_CK(out_sums.alloc(cap * 16));
      OOC_CK(d_jobs.alloc(nj * sizeof(MergeJob)));
      OOC_CK(d_segs.alloc(segs.size() * sizeof(MergeSeg)));
      OOC_CK(d_res.alloc(nj * 16));
      OOC_CK(d_ctr.alloc(16));  // used (8), job head (4), error (4)
      OOC_CK(cudaMemcpyAsync(d_jobs.p, jobs.data(), nj * sizeof(MergeJob), cudaMemcpyHostToDevice, st));
      OOC_CK(cudaMemcpyAsync(d_segs.p, segs.data(), segs.size() * sizeof(MergeSeg), cudaMemcpyHostToDevice, st));
      OOC_CK(cudaMemsetAsync(d_ctr.p, 0, 16, st));
      MergeOut mo;
      mo.grid = d_grid.as<unsigned long long>();
      mo.cnt = reinterpret_cast<uint32_t*>(d_grid.as<char>() + (size_t)G * kGridCells * 32);
      mo.touched = reinterpret_cast<uint32_t*>(d_grid.as<char>() + (size_t)G * kGridCells * 36);
      mo.used = d_ctr.as<unsigned long long>();
      mo.job_head = reinterpret_cast<unsigned int*>(d_ctr.as<char>() + 8);
      mo.error = reinterpret_cast<unsigned int*>(d_ctr.as<char>() + 12);
      mo.recs = out.as<int4>();
      mo.sums = filt ? out_sums.as<ulonglong2>() : nullptr;
      mo.cap = cap;
      mo.result = d_res.as<ulonglong2>();
      OOC_CK(launch_merge(prm.mode, d_jobs.as<MergeJob>(), nj, d_segs.as<MergeSeg>(), mo,
                          (int)std::min<uint32_t>(G, nj), st));
      std::vector<ulonglong2> res(nj);
      unsigned int err = 0;
      OOC_CK(cudaMemcpyAsync(res.data(), d_res.p, nj * 16, cudaMemcpyDeviceToHost, st));
      OOC_CK(cudaMemcpyAsync(&err, d_ctr.as<char>() + 12, 4, cudaMemcpyDeviceToHost, st));
      OOC_CK(cudaStreamSynchronize(st));
      if (err) return LOD_ERR_INTERNAL;
      for (uint32_t q = 0; q < nj; ++q) {
        const int32_t i = jobs_i[q];
        tout[i].recs = out.as<int4>() + res[q].x;
        tout[i].sums = filt ? out_sums.as<ulonglong2>() + res[q].x : nullptr;
        tout[i].count = res[q].y;
      }
    }
  }

  // ---- 7. one breadth-first node table: root-side nodes and every chunk's
  // nodes, ordered by level, then by path (Morton order of the cube)
  struct Ref {
    int32_t top = -1;    // a root-side node
    int32_t chunk = -1;  // or node `local` of a chunk
    uint32_t local = 0;
    uint32_t level = 0;
    uint32_t q[3];       // (min - root min) >> log2
  };
  std::vector<Ref> refs;
  auto make_ref = [&](Ref r, const int32_t mn[3], uint32_t lg) {
    for (int a = 0; a < 3; ++a) r.q[a] = (uint32_t)(((int64_t)mn[a] - (int64_t)g.min[a]) >> lg);
    refs.push_back(r);
  };
  for (size_t i = 0; i < top.size(); ++i)
    if (!top[i].chunk) {
      Ref r;
      r.top = (int32_t)i;
      r.level = top[i].level;
      make_ref(r, top[i].min, top[i].log2);
    }
  for (uint32_t c = 0; c < nc; ++c) {
    const uint32_t l0 = top[chunks[c]].level;
    for (uint32_t j = 0; j < co[c].nodes.size(); ++j) {
      const lod_node_t& nd = co[c].nodes[j];
      Ref r;
      r.chunk = (int32_t)c;
      r.local = j;
      r.level = nd.level + l0;
      make_ref(r, nd.min, nd.log2_size);
    }
  }
  std::vector<uint32_t> ord(refs.size());
  for (uint32_t i = 0; i < ord.size(); ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](uint32_t a, uint32_t b) {
    if (refs[a].level != refs[b].level) return refs[a].level < refs[b].level;
    return morton_less(refs[a].q, refs[b].q);
  });
  const uint32_t nn = (uint32_t)ord.size();
  std::vector<uint32_t> fin_top(top.size(), kNone);
  std::vector<std::vector<uint32_t>> fin_chunk(nc);
  for (uint32_t c = 0; c < nc; ++c) fin_chunk[c].assign(co[c].nodes.size(), kNone);
  for (uint32_t f = 0; f < nn; ++f) {
    const Ref& r = refs[ord[f]];
    if (r.top >= 0) fin_top[r.top] = f;
    else fin_chunk[r.chunk][r.local] = f;
  }
  auto fin_of_top_child = [&](int32_t c) -> uint32_t {
    return top[c].chunk ? fin_chunk[top[c].chunk_id][0] : fin_top[c];
  };
  std::vector<lod_node_t> fn(nn);
  uint32_t max_level = 0;
  for (uint32_t f = 0; f < nn; ++f) {
    const Ref& r = refs[ord[f]];
    lod_node_t& d = fn[f];
    std::memset(&d, 0, sizeof(d));
    if (r.chunk >= 0) {
      const lod_node_t& s0 = co[r.chunk].nodes[r.local];
      d = s0;
      d.level = (uint8_t)r.level;
      if (r.local == 0) {
        const int32_t p = top[chunks[r.chunk]].parent;
        d.parent = p >= 0 ? fin_top[p] : kNone;
      } else {
        d.parent = fin_chunk[r.chunk][s0.parent];
      }
      d.first_child = s0.first_child == kNone ? kNone : fin_chunk[r.chunk][s0.first_child];
      d.point_offset = c_off[r.chunk] + s0.point_offset;
    } else {
      const TopNode& t = top[r.top];
      for (int a = 0; a < 3; ++a) d.min[a] = t.min[a];
      d.level = (uint8_t)t.level;
      d.log2_size = (uint8_t)t.log2;
      d.child_mask = (uint8_t)t.child_mask;
      d.flags = 0;
      d.parent = t.parent >= 0 ? fin_top[t.parent] : kNone;
      for (uint32_t k = 0; k < 8 && d.first_child == 0; ++k)
        if (t.children[k] >= 0) d.first_child = fin_of_top_child(t.children[k]);
      d.point_count = t.count;
    }
    max_level = std::max<uint32_t>(max_level, r.level);
  }
  // a root-side node's subtree starts where its first child's does
  for (uint32_t f = nn; f-- > 0;) {
    const Ref& r = refs[ord[f]];
    if (r.top >= 0) fn[f].point_offset = fn[fn[f].first_child].point_offset;
  }
  // voxels: root-side nodes' from the merge, chunks' gathered per chunk
  std::vector<std::vector<uint64_t>> chunk_new_off(nc);
  for (uint32_t c = 0; c < nc; ++c) chunk_new_off[c].assign(co[c].nodes.size(), 0);
  uint64_t V = 0;
  for (uint32_t f = 0; f < nn; ++f) {
    const Ref& r = refs[ord[f]];
    if (r.top >= 0) {
      fn[f].voxel_offset = V;
      fn[f].voxel_count = (uint32_t)tout[r.top].count;
    } else {
      chunk_new_off[r.chunk][r.local] = V;
      fn[f].voxel_offset = V;
    }
    V += fn[f].voxel_count;
  }
  auto sh = std::make_shared<SharedBuffers>();
  OOC_CK(cudaGetDevice(&sh->device));
  Dev d_pts(st), d_idx(st), d_nodes(st), d_vox(st);
  OOC_CK(d_pts.alloc(n * 16));
  if (want_idx) OOC_CK(d_idx.alloc(n * 4));
  OOC_CK(d_nodes.alloc((size_t)nn * sizeof(lod_node_t)));
  OOC_CK(d_vox.alloc(std::max<uint64_t>(V, 1) * 16));
  OOC_CK(cudaMemcpyAsync(d_nodes.p, fn.data(), (size_t)nn * sizeof(lod_node_t), cudaMemcpyHostToDevice, st));
  for (uint32_t f = 0; f < nn; ++f) {
    const Ref& r = refs[ord[f]];
    if (r.top >= 0 && tout[r.top].count)
      OOC_CK(cudaMemcpyAsync(d_vox.as<int4>() + fn[f].voxel_offset, tout[r.top].recs, tout[r.top].count * 16,
                             cudaMemcpyDeviceToDevice, st));
  }
  {
    std::vector<Dev*> offs;
    for (uint32_t c = 0; c < nc; ++c) {
      const SharedBuffers& b = *bsh[co[c].batch];
      const TileResult& tr = co[c].tr;
      OOC_CK(cudaMemcpyAsync(d_pts.as<int4>() + c_off[c], static_cast<const int4*>(b.points) + tr.pt_base,
                             tr.n_points * 16, cudaMemcpyDeviceToDevice, st));
      if (want_idx)
        OOC_CK(cudaMemcpyAsync(d_idx.as<uint32_t>() + c_off[c], static_cast<const uint32_t*>(b.index) + tr.pt_base,
                               tr.n_points * 4, cudaMemcpyDeviceToDevice, st));
      if (tr.n_voxels) {
        keep.emplace_back(new Dev(st));
        Dev& d_off = *keep.back();
        OOC_CK(d_off.alloc(co[c].nodes.size() * 8));
        OOC_CK(cudaMemcpyAsync(d_off.p, chunk_new_off[c].data(), co[c].nodes.size() * 8, cudaMemcpyHostToDevice, st));
        OOC_CK(launch_gather_voxels(static_cast<const lod_node_t*>(b.nodes) + tr.node_base, tr.n_nodes,
                                    d_off.as<uint64_t>(), static_cast<const int4*>(b.voxels), d_vox.as<int4>(), st));
      }
    }
  }
  OOC_CK(cudaStreamSynchronize(st));
  sh->bytes = n * 16 + (want_idx ? n * 4 : 0) + (uint64_t)nn * sizeof(lod_node_t) + std::max<uint64_t>(V, 1) * 16;
  sh->points = d_pts.take();
  sh->index = want_idx ? d_idx.take() : nullptr;
  sh->nodes = d_nodes.take();
  sh->voxels = d_vox.take();
  *sh_out = sh;
  TileResult tr;
  tr.pt_base = 0;
  tr.n_points = n;
  tr.node_base = 0;
  tr.n_nodes = nn;
  tr.n_levels = max_level + 1;
  tr.n_voxels = V;
  *tr_out = tr;
  return LOD_OK;
}

}  // namespace lodk

extern "C" int lod_build_out_of_core(const lod_point_t* h_points, uint64_t n, const lod_params_t* params,
                                     const lod_ooc_config_t* cfg, void* stream, lod_result_t** out) {
  if (!out) return LOD_ERR_INVALID_ARG;
  lod_params_t p;
  lod_params_init(&p);
  if (params) p = *params;
  lod_ooc_config_t c;
  std::memset(&c, 0, sizeof(c));
  if (cfg) c = *cfg;
  std::shared_ptr<lodk::SharedBuffers> sh;
  lodk::TileResult tr;
  const int rc = lodk::build_out_of_core(h_points, n, p, c, static_cast<cudaStream_t>(stream), &sh, &tr);
  if (rc != LOD_OK) return rc;
  lod_result_t* r = make_result(sh, tr, p.mode, sh->bytes);
  if (!r) return LOD_ERR_OOM;
  *out = r;
  return LOD_OK;
}
