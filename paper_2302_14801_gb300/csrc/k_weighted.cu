// Neighbourhood-weighted average voxel sampling (Section 4.2.4 of the paper).
//
// An inner node's samples are its children's samples: the points of leaf
// children, and the voxels of inner children, each taken as one sample at
// the centre of its cell with its stored 8-bit colour.  A sample adds
// weight w = max(0, 1 - distance to the cell centre, in cells) times its
// colour to each cell of the 2x2x2 block around it (the cells whose centres
// are within one cell width along every axis), and marks the cell it lies
// in as occupied; only occupied cells become voxels, coloured by their
// weighted sum over their weight sum, rounded half up, alpha 255.  Counts
// are the cell's original points, as in the other modes.
//
// A sample's 2x2x2 block can reach into the neighbouring child octant, so
// a parent node is the unit of work here, not a (parent, octant) item: one
// persistent CTA per SM takes parents from a counter and accumulates into
// its own dense 128^3 grid in global memory (one 32-byte sector per cell:
// fixed-point sums of w*R, w*G, w*B and w, plus a count), appending every
// cell it touches for the first time to a list, so that extraction and
// clearing cost the touched cells only.  Weights are fp32 1 - sqrt(d^2)
// rounded to 24 fractional bits and summed exactly in 64-bit integers: the
// result does not depend on the order of the atomics.  Occupied cells go to
// staging grouped by child octant, so each child receives its block of the
// parent's voxels exactly as in the other modes (the level scan and the
// copy into the voxel array are shared).
#include "common.cuh"
#include "kernels.h"
#include "wgrid.cuh"

namespace lodk {

namespace {

// Shared state of one weighted CTA.
struct WShared {
  uint32_t touched;
  uint32_t occ[8], cur[8], base8[8];
  unsigned long long base;
  uint32_t parent_ok;
};

__device__ __forceinline__ uint32_t find_in_prefix(const uint32_t* prefix, uint32_t n_tiles, uint32_t x) {
  uint32_t lo = 0, hi = n_tiles;  // largest t with prefix[t] <= x
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (prefix[mid] <= x) lo = mid;
    else hi = mid;
  }
  return lo;
}

}  // namespace

// Parents at level v.level, taken in order by persistent CTAs.
__global__ void __launch_bounds__(kBlock, 1) k_wvox(BuildArgs a, VoxLevel v, DevCounters* __restrict__ ctr) {
  __shared__ WShared S;
  __shared__ uint32_t s_par;
  unsigned long long* grid = v.wgrid + (uint64_t)blockIdx.x * 4ull * kGridCells;
  uint32_t* cnt = v.wcnt + (uint64_t)blockIdx.x * kGridCells;
  uint32_t* touched = v.wtouch + (uint64_t)blockIdx.x * kGridCells;
  for (;;) {
    if (threadIdx.x == 0) s_par = atomicAdd(&ctr->item_head, 1u);
    __syncthreads();
    const uint32_t ip = s_par;
    __syncthreads();
    if (ip >= v.n_parents) break;
    const uint32_t t = find_in_prefix(v.parent_prefix, a.n_tiles, ip);
    const TileDesc& td = a.tiles[t];
    const uint64_t g = td.node_base + v.lvl_start[(uint64_t)t * (kMaxLevels + 1) + v.level] + (ip - v.parent_prefix[t]);
    const lod_node_t P = v.nodes[g];
    if (P.flags & LOD_NODE_LEAF) continue;  // uniform over the CTA
    if (threadIdx.x == 0) S.touched = 0;
    if (threadIdx.x < 8) S.occ[threadIdx.x] = S.cur[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t L = P.log2_size;
    const uint64_t fc = td.node_base + P.first_child;
    uint32_t r = 0;
    for (uint32_t k = 0; k < 8; ++k) {
      if (!(P.child_mask & (1u << k))) continue;
      const uint64_t cg = fc + r++;
      const lod_node_t& c = v.nodes[cg];
      if (c.flags & LOD_NODE_LEAF) {
        // leaf child: its points
        const uint64_t pbase = td.pt_base + c.point_offset;
        for (uint64_t i = threadIdx.x; i < c.point_count; i += blockDim.x) {
          int4 q;
          if (a.wide) {
            uint32_t x;
            ld_wide(a.wide + 2 * (pbase + i), q, x);
            a.out[pbase + i] = q;  // publish the leaf point and its index
            a.out_idx[pbase + i] = x;
          } else {
            q = __ldcs(a.out + pbase + i);
          }
          int64_t Pp[3];
          uint32_t s, own;
          w_point_pos(q, P.min, L, Pp, &s, &own);
          w_sample(grid, cnt, touched, &S.touched, Pp, s, own, (uint32_t)q.w, 1u);
        }
      } else {
        // inner child (octant k): its voxels, each one sample at its cell centre
        const uint32_t nch = __popc(c.child_mask);
        const uint64_t gfc = td.node_base + c.first_child;
        for (uint32_t rr = 0; rr < nch; ++rr) {
          const NodeAux& ca = v.aux[gfc + rr];
          const int4* rec = v.stage_in + ca.stage;
          int4* dst = v.dense + ca.dense;
          const bool fits = ca.dense + ca.occ <= v.dense_cap;  // else the build is redone with a larger array
          for (uint32_t i = threadIdx.x; i < ca.occ; i += blockDim.x) {
            const int4 vr = rec[i];
            if (fits) dst[i] = vr;  // publish the child's voxel
            int64_t Pp[3];
            uint32_t own;
            w_voxel_pos((uint32_t)vr.x, k, Pp, &own);
            w_sample(grid, cnt, touched, &S.touched, Pp, 1u, own, (uint32_t)vr.y, (uint32_t)vr.z);
          }
        }
      }
    }
    __syncthreads();
    // extraction: occupied cells (a count) grouped by child octant; cells
    // were updated by atomics in L2, so they are read past L1
    const uint32_t m = S.touched;
    for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) {
      const uint32_t cell = touched[i];
      if (__ldcg(cnt + cell)) {
        atomicAdd(&S.occ[cell_octant(cell)], 1u);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t tot = 0;
      for (uint32_t k = 0; k < 8; ++k) {
        S.base8[k] = tot;
        tot += S.occ[k];
      }
      S.base = atomicAdd(v.stage_used, (unsigned long long)tot);
      S.parent_ok = S.base + tot <= v.stage_cap;
      if (!S.parent_ok) atomicOr(&ctr->error, kErrStageCap);
      uint32_t rr = 0;
      for (uint32_t k = 0; k < 8; ++k) {
        if (!(P.child_mask & (1u << k))) {
          if (S.occ[k]) atomicOr(&ctr->error, kErrInternal);  // an occupied cell needs a sample of child k
          continue;
        }
        NodeAux& ca = v.aux[fc + rr++];
        ca.stage = S.base + S.base8[k];
        ca.occ = S.occ[k];
      }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) {
      const uint32_t cell = touched[i];
      unsigned long long* e = grid + 4ull * cell;
      const uint32_t n = __ldcg(cnt + cell);
      if (n && S.parent_ok) {
        const ulonglong2 rg = __ldcg(reinterpret_cast<const ulonglong2*>(e));
        const ulonglong2 bw = __ldcg(reinterpret_cast<const ulonglong2*>(e) + 1);
        const unsigned long long w = bw.y;
        const uint32_t k = cell_octant(cell);
        const uint32_t o = atomicAdd(&S.cur[k], 1u);
        int4 rec;
        rec.x = (int)cell;
        rec.y = (int)(w_round(rg.x, w) | (w_round(rg.y, w) << 8) | (w_round(bw.x, w) << 16) | 0xFF000000u);
        rec.z = (int)n;
        rec.w = (int)kNone;
        v.stage_out[S.base + S.base8[k] + o] = rec;
      }
      // leave the cell empty for the next parent (the grids stay all zero
      // between launches, so they are cleared only when first allocated)
      __stcg(reinterpret_cast<ulonglong2*>(e), make_ulonglong2(0ull, 0ull));
      __stcg(reinterpret_cast<ulonglong2*>(e) + 1, make_ulonglong2(0ull, 0ull));
      __stcg(cnt + cell, 0u);
    }
    __syncthreads();
  }
}

size_t wgrid_bytes_per_cta() { return (size_t)kGridCells * (32 + 4 + 4); }

cudaError_t launch_wvox(const BuildArgs& a, const VoxLevel& v, DevCounters* ctr, int ctas, cudaStream_t st) {
  if (!v.n_parents) return cudaSuccess;
  k_wvox<<<ctas, kBlock, 0, st>>>(a, v, ctr);
  note_launch();
  return cudaGetLastError();
}

}  // namespace lodk
