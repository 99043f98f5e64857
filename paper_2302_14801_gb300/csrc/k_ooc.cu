// Device kernels of the out-of-core build (Section 7 of the paper: large
// clouds are split into chunks that are built on the GPU one batch at a
// time, and the coarsest nodes above the chunks are filled afterwards).
//
// The host streams the input through the device in blocks: a bounding-box
// pass, a count over a top grid of 8^D cells, and a partition of every
// point into the chunk whose root cube holds it (with its input index).
// After the chunks are built, k_merge fills the root-side nodes bottom-up:
// each top node samples its children exactly as the voxel passes do — the
// points of leaf children, the voxels of inner children (with their exact
// colour sums in filtered mode) — into a dense 128^3 grid in global memory,
// one grid per CTA, cleared again by the extraction.
#include <climits>

#include "common.cuh"
#include "kernels.h"
#include "wgrid.cuh"

namespace lodk {

namespace {

__device__ __forceinline__ uint32_t top_cell(const int4& p, const int32_t mn[3], uint32_t L, uint32_t D) {
  const uint32_t sh = L - D;  // D <= L
  const uint32_t qx = ((uint32_t)p.x - (uint32_t)mn[0]) >> sh;
  const uint32_t qy = ((uint32_t)p.y - (uint32_t)mn[1]) >> sh;
  const uint32_t qz = ((uint32_t)p.z - (uint32_t)mn[2]) >> sh;
  return qx | (qy << D) | (qz << (2 * D));
}

}  // namespace

// Bounding box of one block of points: six atomics per warp.
__global__ void __launch_bounds__(256) k_ooc_bbox(const int4* __restrict__ pts, uint64_t n, int* __restrict__ box) {
  int v[6] = {INT_MAX, INT_MAX, INT_MAX, INT_MIN, INT_MIN, INT_MIN};
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const int4 p = __ldcs(pts + i);
    v[0] = min(v[0], p.x);
    v[1] = min(v[1], p.y);
    v[2] = min(v[2], p.z);
    v[3] = max(v[3], p.x);
    v[4] = max(v[4], p.y);
    v[5] = max(v[5], p.z);
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    v[k] = __reduce_min_sync(0xFFFFFFFFu, v[k]);
    v[k + 3] = __reduce_max_sync(0xFFFFFFFFu, v[k + 3]);
  }
  const uint32_t lane = threadIdx.x & 31u;
  if (lane < 3) atomicMin(&box[lane], v[lane]);
  else if (lane < 6) atomicMax(&box[lane], v[lane]);
}

// Points per top-grid cell (cell = x | y << D | z << 2D at depth D below the
// root cube); lanes of a warp in one cell add once.
__global__ void __launch_bounds__(256) k_ooc_count(const int4* __restrict__ pts, uint64_t n, OocGrid g,
                                                   unsigned int* __restrict__ counts) {
  for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x; b < n; b += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = b + threadIdx.x;
    const bool v = i < n;
    const uint32_t c = v ? top_cell(__ldcs(pts + i), g.min, g.L, g.D) : 0xFFFFFFFFu;
    const unsigned act = __ballot_sync(0xFFFFFFFFu, v);
    if (!v) continue;
    const unsigned peers = __match_any_sync(act, c);
    if ((int)(threadIdx.x & 31u) == __ffs(peers) - 1) atomicAdd(&counts[c], (unsigned)__popc(peers));
  }
}

// Chunk of every point of a block (through the cell -> chunk map) and the
// number of the block's points per chunk; a point in no chunk (which the
// counting pass rules out) raises *err and is left out.
__global__ void __launch_bounds__(256) k_ooc_chunk_of(const int4* __restrict__ pts, uint64_t n, OocGrid g,
                                                      const uint32_t* __restrict__ cell_chunk, uint32_t n_chunks,
                                                      uint32_t* __restrict__ chunk_of,
                                                      unsigned int* __restrict__ hist, unsigned int* __restrict__ err) {
  for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x; b < n; b += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = b + threadIdx.x;
    uint32_t c = i < n ? cell_chunk[top_cell(__ldcs(pts + i), g.min, g.L, g.D)] : 0xFFFFFFFFu;
    if (i < n && c >= n_chunks) {
      atomicOr(err, 1u);
      chunk_of[i] = 0xFFFFFFFFu;
    }
    const bool v = i < n && c < n_chunks;
    const unsigned act = __ballot_sync(0xFFFFFFFFu, v);
    if (!v) continue;
    chunk_of[i] = c;
    const unsigned peers = __match_any_sync(act, c);
    if ((int)(threadIdx.x & 31u) == __ffs(peers) - 1) atomicAdd(&hist[c], (unsigned)__popc(peers));
  }
}

// Partition of a block by chunk: every point (and its input index, the
// block's first index plus its position) goes to its chunk's run, whose
// cursor the host set from the histogram.  Order inside a run is free.
__global__ void __launch_bounds__(256) k_ooc_partition(const int4* __restrict__ pts, uint64_t n, uint32_t first,
                                                       const uint32_t* __restrict__ chunk_of, uint32_t n_chunks,
                                                       unsigned int* __restrict__ cursor, int4* __restrict__ out,
                                                       uint32_t* __restrict__ out_idx) {
  for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x; b < n; b += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = b + threadIdx.x;
    const uint32_t c = i < n ? chunk_of[i] : 0xFFFFFFFFu;
    const bool v = c < n_chunks;
    const unsigned act = __ballot_sync(0xFFFFFFFFu, v);
    if (!v) continue;
    const unsigned peers = __match_any_sync(act, c);
    const int leader = __ffs(peers) - 1;
    unsigned base = 0;
    if ((int)(threadIdx.x & 31u) == leader) base = atomicAdd(&cursor[c], (unsigned)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    const uint32_t pos = base + __popc(peers & ((1u << (threadIdx.x & 31u)) - 1u));
    out[pos] = __ldcs(pts + i);
    out_idx[pos] = first + (uint32_t)i;
  }
}

// Voxels of the root-side nodes of one level, one node per CTA iteration.
template <int MODE>
__global__ void __launch_bounds__(1024, 1) k_merge(const MergeJob* __restrict__ jobs, uint32_t n_jobs,
                                                   const MergeSeg* __restrict__ segs, MergeOut o) {
  __shared__ uint32_t s_job, s_touched, s_occ, s_cur;
  __shared__ unsigned long long s_base;
  constexpr bool PICKLIKE = MODE == LOD_PICK || MODE == LOD_FIRST || MODE == LOD_RANDOM;
  unsigned long long* grid = o.grid + (uint64_t)blockIdx.x * 4ull * kGridCells;
  uint32_t* cnt = o.cnt + (uint64_t)blockIdx.x * kGridCells;
  uint32_t* touched = o.touched + (uint64_t)blockIdx.x * kGridCells;
  for (;;) {
    if (threadIdx.x == 0) {
      s_job = atomicAdd(o.job_head, 1u);
      s_touched = s_occ = s_cur = 0;
    }
    __syncthreads();
    const uint32_t j = s_job;
    if (j >= n_jobs) break;
    const MergeJob J = jobs[j];
    // accumulate every sample of the node's children
    for (uint32_t sgi = 0; sgi < J.nseg; ++sgi) {
      const MergeSeg S = segs[J.seg0 + sgi];
      for (uint32_t i = threadIdx.x; i < S.n; i += blockDim.x) {
        const int4 r = S.recs[i];
        uint32_t own, count, rgba, idx = 0;
        if (S.kind == 0) {  // a point
          own = grid_coord((uint32_t)r.x - (uint32_t)J.min[0], J.log2) |
                (grid_coord((uint32_t)r.y - (uint32_t)J.min[1], J.log2) << 7) |
                (grid_coord((uint32_t)r.z - (uint32_t)J.min[2], J.log2) << 14);
          count = 1;
          rgba = (uint32_t)r.w;
          if (PICKLIKE) idx = S.idx[i];
          if (MODE == LOD_WEIGHTED) {
            int64_t P[3];
            uint32_t s;
            w_point_pos(r, J.min, J.log2, P, &s, &own);
            w_sample(grid, cnt, touched, &s_touched, P, s, own, rgba, 1u);
            continue;
          }
        } else {  // a child voxel: its cell nests in one cell of this node
          const uint32_t cell = (uint32_t)r.x, k = S.octant;
          own = ((((k >> 2) & 1u) << 6) | ((cell & 127u) >> 1)) | (((((k >> 1) & 1u) << 6) | (((cell >> 7) & 127u) >> 1)) << 7) |
                ((((k & 1u) << 6) | ((cell >> 14) >> 1)) << 14);
          count = (uint32_t)r.z;
          rgba = (uint32_t)r.y;
          idx = (uint32_t)r.w;
          if (MODE == LOD_WEIGHTED) {
            int64_t P[3];
            w_voxel_pos(cell, k, P, &own);
            w_sample(grid, cnt, touched, &s_touched, P, 1u, own, rgba, count);
            continue;
          }
        }
        unsigned long long* e = grid + 4ull * own;
        if (MODE == LOD_FILTER) {
          uint64_t sr, sg, sb;
          if (S.kind == 0) {
            sr = rgba & 255u;
            sg = (rgba >> 8) & 255u;
            sb = (rgba >> 16) & 255u;
          } else {
            const ulonglong2 sm = S.sums[i];
            sr = sm.x & ((1ull << 40) - 1);
            sg = (sm.x >> 40) | ((sm.y & 0xFFFFull) << 24);
            sb = sm.y >> 16;
          }
          atomicAdd(e + 0, (unsigned long long)sr);
          atomicAdd(e + 1, (unsigned long long)sg);
          atomicAdd(e + 2, (unsigned long long)sb);
        } else if (PICKLIKE) {
          atomicMax(e + 0, ~pick_key<MODE>(idx, J.level));  // the largest complement is the smallest key
        }
        if (atomicAdd(&cnt[own], count) == 0u) touched[atomicAdd(&s_touched, 1u)] = own;
      }
    }
    __syncthreads();
    if (PICKLIKE) {
      // the winner of each cell (keys are unique) leaves its colour and index
      for (uint32_t sgi = 0; sgi < J.nseg; ++sgi) {
        const MergeSeg S = segs[J.seg0 + sgi];
        for (uint32_t i = threadIdx.x; i < S.n; i += blockDim.x) {
          const int4 r = S.recs[i];
          uint32_t own, idx;
          if (S.kind == 0) {
            own = grid_coord((uint32_t)r.x - (uint32_t)J.min[0], J.log2) |
                  (grid_coord((uint32_t)r.y - (uint32_t)J.min[1], J.log2) << 7) |
                  (grid_coord((uint32_t)r.z - (uint32_t)J.min[2], J.log2) << 14);
            idx = S.idx[i];
          } else {
            const uint32_t cell = (uint32_t)r.x, k = S.octant;
            own = ((((k >> 2) & 1u) << 6) | ((cell & 127u) >> 1)) |
                  (((((k >> 1) & 1u) << 6) | (((cell >> 7) & 127u) >> 1)) << 7) |
                  ((((k & 1u) << 6) | ((cell >> 14) >> 1)) << 14);
            idx = (uint32_t)r.w;
          }
          unsigned long long* e = grid + 4ull * own;
          if (__ldcg(e) == ~pick_key<MODE>(idx, J.level))
            __stcg(e + 1, (unsigned long long)(uint32_t)(S.kind == 0 ? r.w : r.y) | ((unsigned long long)idx << 32));
        }
      }
      __syncthreads();
    }
    // extraction of the occupied cells
    const uint32_t m = s_touched;
    uint32_t mine = 0;
    for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) mine += __ldcg(cnt + touched[i]) ? 1u : 0u;
    mine = __reduce_add_sync(0xFFFFFFFFu, mine);
    if ((threadIdx.x & 31u) == 0 && mine) atomicAdd(&s_occ, mine);
    __syncthreads();
    if (threadIdx.x == 0) {
      s_base = atomicAdd(o.used, (unsigned long long)s_occ);
      const bool ok = s_base + s_occ <= o.cap;
      if (!ok) atomicOr(o.error, 1u);
      o.result[j] = make_ulonglong2(ok ? s_base : 0ull, ok ? s_occ : 0ull);
    }
    __syncthreads();
    const bool ok = s_base + s_occ <= o.cap;
    for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) {
      const uint32_t cell = touched[i];
      unsigned long long* e = grid + 4ull * cell;
      const uint32_t n = __ldcg(cnt + cell);
      if (n && ok) {
        const ulonglong2 ab = __ldcg(reinterpret_cast<const ulonglong2*>(e));
        const ulonglong2 cd = __ldcg(reinterpret_cast<const ulonglong2*>(e) + 1);
        const uint64_t p = s_base + atomicAdd(&s_cur, 1u);
        int4 rec;
        rec.x = (int)cell;
        rec.z = (int)n;
        if (MODE == LOD_FILTER) {
          rec.y = (int)mean_rgba(ab.x, ab.y, cd.x, n);
          rec.w = (int)kNone;
          o.sums[p] = make_ulonglong2(ab.x | (ab.y << 40), (ab.y >> 24) | (cd.x << 16));
        } else if (MODE == LOD_WEIGHTED) {
          rec.y = (int)(w_round(ab.x, cd.y) | (w_round(ab.y, cd.y) << 8) | (w_round(cd.x, cd.y) << 16) | 0xFF000000u);
          rec.w = (int)kNone;
        } else {
          rec.y = (int)(uint32_t)ab.y;
          rec.w = (int)(uint32_t)(ab.y >> 32);
        }
        o.recs[p] = rec;
      }
      __stcg(reinterpret_cast<ulonglong2*>(e), make_ulonglong2(0ull, 0ull));
      __stcg(reinterpret_cast<ulonglong2*>(e) + 1, make_ulonglong2(0ull, 0ull));
      __stcg(cnt + cell, 0u);
    }
    __syncthreads();
  }
}

cudaError_t launch_ooc_bbox(const int4* pts, uint64_t n, int* box, int sms, cudaStream_t st) {
  if (!n) return cudaSuccess;
  const uint64_t want = (n + 255) / 256;
  k_ooc_bbox<<<(unsigned)(want < (uint64_t)(4 * sms) ? want : (uint64_t)(4 * sms)), 256, 0, st>>>(pts, n, box);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_ooc_count(const int4* pts, uint64_t n, const OocGrid& g, unsigned int* counts, int sms,
                             cudaStream_t st) {
  if (!n) return cudaSuccess;
  const uint64_t want = (n + 255) / 256;
  k_ooc_count<<<(unsigned)(want < (uint64_t)(8 * sms) ? want : (uint64_t)(8 * sms)), 256, 0, st>>>(pts, n, g, counts);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_ooc_chunk_of(const int4* pts, uint64_t n, const OocGrid& g, const uint32_t* cell_chunk,
                                uint32_t n_chunks, uint32_t* chunk_of, unsigned int* hist, unsigned int* err, int sms,
                                cudaStream_t st) {
  if (!n) return cudaSuccess;
  const uint64_t want = (n + 255) / 256;
  k_ooc_chunk_of<<<(unsigned)(want < (uint64_t)(8 * sms) ? want : (uint64_t)(8 * sms)), 256, 0, st>>>(
      pts, n, g, cell_chunk, n_chunks, chunk_of, hist, err);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_ooc_partition(const int4* pts, uint64_t n, uint32_t first, const uint32_t* chunk_of,
                                 uint32_t n_chunks, unsigned int* cursor, int4* out, uint32_t* out_idx, int sms,
                                 cudaStream_t st) {
  if (!n) return cudaSuccess;
  const uint64_t want = (n + 255) / 256;
  k_ooc_partition<<<(unsigned)(want < (uint64_t)(8 * sms) ? want : (uint64_t)(8 * sms)), 256, 0, st>>>(
      pts, n, first, chunk_of, n_chunks, cursor, out, out_idx);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_merge(uint32_t mode, const MergeJob* jobs, uint32_t n_jobs, const MergeSeg* segs,
                         const MergeOut& o, int ctas, cudaStream_t st) {
  if (!n_jobs) return cudaSuccess;
  switch (mode) {
    case LOD_FILTER: k_merge<LOD_FILTER><<<ctas, 1024, 0, st>>>(jobs, n_jobs, segs, o); break;
    case LOD_PICK: k_merge<LOD_PICK><<<ctas, 1024, 0, st>>>(jobs, n_jobs, segs, o); break;
    case LOD_WEIGHTED: k_merge<LOD_WEIGHTED><<<ctas, 1024, 0, st>>>(jobs, n_jobs, segs, o); break;
    case LOD_FIRST: k_merge<LOD_FIRST><<<ctas, 1024, 0, st>>>(jobs, n_jobs, segs, o); break;
    default: k_merge<LOD_RANDOM><<<ctas, 1024, 0, st>>>(jobs, n_jobs, segs, o); break;
  }
  note_launch();
  return cudaGetLastError();
}

}  // namespace lodk
