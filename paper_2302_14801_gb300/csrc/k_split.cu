// Split of the input into octree leaves (Section 4.1 of the paper):
// bounding box, hierarchical counting sort with recursive refinement of
// overflowing cells, and the breadth-first node table.
//
// GB300 design: every pass streams the 16-byte AoS points with coalesced
// 128-bit loads in 4096-point chunks; each CTA owns a contiguous run of
// chunks so that per-source state (a shared-memory histogram, a reduction)
// is flushed only when the source changes.  Counting grids of up to 8^4
// cells use a dense shared-memory histogram; larger grids (first grids up
// to 256^3 cells, deep refinement grids) count through a per-CTA
// shared-memory hash table of the cells the CTA's chunks touch.  Every
// counted cell is published with one global atomic and listed as (cell,
// count), so that the scatter claims one block of positions per listed
// cell; cells that miss the table or the list use warp-aggregated global
// atomics on their cursor.  Grid pyramids (per-level sums and
// exclusive-scan starts) are built in 4-level blocks in shared memory.
// With kept input indices the scatter writes one full 32-byte sector per
// point.  The root cubes are computed on the device (no host round trip
// after the bounding box).  No kernel ever waits on another CTA.
#include <climits>

#include "common.cuh"
#include "kernels.h"

namespace lodk {

namespace {

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

// Spread the low 8 bits of v to every third bit (bit i to bit 3i).
__device__ __forceinline__ uint32_t spread3_8(uint32_t v) {
  v = (v | (v << 8)) & 0x0000F00Fu;
  v = (v | (v << 4)) & 0x000C30C3u;
  v = (v | (v << 2)) & 0x00249249u;
  return v;
}

// Morton cell of point p inside a source grid (8^d cells under a cube of
// edge 2^log2size with min corner (mx, my, mz)): within every bit triple x
// is the most significant, so the low triple is the octant index
// k = 4*bx + 2*by + bz.  Grids have d <= 8, so each coordinate has at most
// 8 bits and the shift log2size - d is at most 31.
__device__ __forceinline__ uint32_t src_bin(const int4& p, int32_t mx, int32_t my, int32_t mz, uint32_t log2size,
                                            uint32_t d) {
  if (d == 0) return 0;
  const uint32_t sh = log2size - d;
  const uint32_t ux = ((uint32_t)p.x - (uint32_t)mx) >> sh;
  const uint32_t uy = ((uint32_t)p.y - (uint32_t)my) >> sh;
  const uint32_t uz = ((uint32_t)p.z - (uint32_t)mz) >> sh;
  return (spread3_8(ux) << 2) | (spread3_8(uy) << 1) | spread3_8(uz);
}

// Compact every third bit (inverse of spread3) for 8 output bits.
__device__ __forceinline__ uint32_t compact3(uint32_t v) {
  v &= 0x09249249u;
  v = (v | (v >> 2)) & 0x030C30C3u;
  v = (v | (v >> 4)) & 0x0300F00Fu;
  v = (v | (v >> 8)) & 0x030000FFu;
  v = (v | (v >> 16)) & 0x000003FFu;
  return v;
}

// Pointer to the points of a source and the tile-absolute base of its range.
__device__ __forceinline__ const int4* src_points(const BuildArgs& a, const SrcDesc& s, const TileDesc& t) {
  if (s.buf == 0) return t.in;  // round 0 reads the caller's input, index = input index
  return (s.buf == 1 ? a.tmp[0] : a.tmp[1]) + t.pt_base + s.pt_off;
}

// L2 policies: the streamed input is evicted first, so that the partly
// written sectors of the scatter's output runs stay in L2 until they are
// complete (a sector evicted half written costs a DRAM read-modify-write).
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint64_t l2_evict_last() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void st_keep(int4* p, const int4& q, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v4.s32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "r"(q.x), "r"(q.y), "r"(q.z),
               "r"(q.w), "l"(pol)
               : "memory");
}

// Asks the bulk-copy unit to bring [p, p + bytes) into L2 ahead of the loads
// that will read it (p 16-byte aligned, bytes a multiple of 16; nothing waits
// on it).  The counting pass fetches one chunk ahead with it (measured: 7 %
// faster on a 50M-point terrain cloud); the scatter gained nothing from it.
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// The next chunk of the same source, prefetched by one thread: its points
// are [first + kChunk, min(first + 2 kChunk, n)) of the same array.
__device__ __forceinline__ void prefetch_next_chunk(const int4* pts, uint64_t first, uint64_t n, bool same_src) {
  if (threadIdx.x != 0 || !same_src) return;
  const uint64_t nf = first + kChunk, ne = min(nf + kChunk, n);
  if (nf < ne) prefetch_l2(pts + nf, (uint32_t)((ne - nf) * sizeof(int4)));
}

// 16-byte streaming load with an L2 policy.
__device__ __forceinline__ int4 ld_policy(const int4* p, uint64_t pol) {
  int4 q;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s32 {%0, %1, %2, %3}, [%4], %5;"
               : "=r"(q.x), "=r"(q.y), "=r"(q.z), "=r"(q.w)
               : "l"(p), "l"(pol));
  return q;
}

// Depth of a refinement grid for a cell of n points: the levels that reach
// T if every level spreads the points over four children (surfaces), plus
// one level of slack for clustered data, so that one more round resolves
// most cells; capped at 8 and at 8^d <= 1.25 n cells (the grid's pyramids
// then take about as many bytes as its points).
__device__ __forceinline__ uint32_t choose_seg_depth(uint64_t n, uint32_t T, uint32_t level,
                                                     uint32_t log2size, uint32_t max_depth) {
  uint32_t need = 1;
  while (need < kRootMaxD && (n >> (2 * need)) > T) ++need;
  uint32_t dmem = 1;
  while (dmem < kRootMaxD && (1ull << (3 * (dmem + 1))) <= n + n / 4) ++dmem;
  uint32_t d = min(need + 1, dmem);
  d = min(d, max_depth - level);
  d = min(d, log2size);
  return max(d, 1u);
}

}  // namespace

// --------------------------------------------------------------- bounding box

__global__ void __launch_bounds__(kBlock) k_bbox(const TileDesc* __restrict__ tiles,
                                                 const uint32_t* __restrict__ chunk_tile, uint64_t n_chunks,
                                                 const uint64_t* __restrict__ tile_chunk0,
                                                 int* __restrict__ bbox) {
  __shared__ int red[32][6];
  const uint64_t per = (n_chunks + gridDim.x - 1) / gridDim.x;
  const uint64_t c0 = (uint64_t)blockIdx.x * per;
  const uint64_t c1 = min(c0 + per, n_chunks);
  uint32_t cur = kNone;
  int mn[3] = {INT_MAX, INT_MAX, INT_MAX}, mx[3] = {INT_MIN, INT_MIN, INT_MIN};

  auto flush = [&](uint32_t t) {
    const uint32_t w = threadIdx.x >> 5;
    int v[6] = {mn[0], mn[1], mn[2], mx[0], mx[1], mx[2]};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      v[i] = __reduce_min_sync(0xFFFFFFFFu, v[i]);
      v[i + 3] = __reduce_max_sync(0xFFFFFFFFu, v[i + 3]);
    }
    if (lane_id() == 0)
#pragma unroll
      for (int i = 0; i < 6; ++i) red[w][i] = v[i];
    __syncthreads();
    if (w == 0) {
      const bool ok = lane_id() < (blockDim.x >> 5);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        int a = ok ? red[lane_id()][i] : INT_MAX;
        int b = ok ? red[lane_id()][i + 3] : INT_MIN;
        a = __reduce_min_sync(0xFFFFFFFFu, a);
        b = __reduce_max_sync(0xFFFFFFFFu, b);
        if (lane_id() == 0) {
          atomicMin(&bbox[6 * t + i], a);
          atomicMax(&bbox[6 * t + 3 + i], b);
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      mn[i] = INT_MAX;
      mx[i] = INT_MIN;
    }
  };

  for (uint64_t c = c0; c < c1; ++c) {
    const uint32_t t = chunk_tile[c];
    if (t != cur) {
      if (cur != kNone) flush(cur);
      cur = t;
    }
    const TileDesc& td = tiles[t];
    const uint64_t first = (c - tile_chunk0[t]) << kChunkLog2;
    const uint64_t end = min(first + kChunk, (uint64_t)td.n);
    int4 p[kChunk / kBlock];
#pragma unroll
    for (int k = 0; k < (int)(kChunk / kBlock); ++k) {
      const uint64_t i = first + threadIdx.x + (uint64_t)k * kBlock;
      if (i < end) p[k] = ldg_stream(td.in + i);
    }
#pragma unroll
    for (int k = 0; k < (int)(kChunk / kBlock); ++k) {
      const uint64_t i = first + threadIdx.x + (uint64_t)k * kBlock;
      if (i < end) {
        mn[0] = min(mn[0], p[k].x);
        mn[1] = min(mn[1], p[k].y);
        mn[2] = min(mn[2], p[k].z);
        mx[0] = max(mx[0], p[k].x);
        mx[1] = max(mx[1], p[k].y);
        mx[2] = max(mx[2], p[k].z);
      }
    }
  }
  if (cur != kNone) flush(cur);
}

// Root cubes from the bounding boxes (see the reading of Section 4 in the
// oracle): min corner = bbox min, edge = the smallest power of two above the
// largest extent.  Written into each tile's first counting grid on the
// device, so the host need not wait for the boxes; a grid depth the host
// chose before knowing the cube that exceeds it raises *abort.
__global__ void k_roots(const TileDesc* __restrict__ tiles, const int* __restrict__ bbox, SrcDesc* srcs,
                        uint32_t n_tiles, uint32_t T, uint32_t max_depth, unsigned int* abort) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tiles) return;
  const uint32_t n = tiles[t].n;
  int32_t mn[3] = {0, 0, 0};
  uint32_t L = 0;
  if (n) {
    int64_t ext = 0;
    for (int k = 0; k < 3; ++k) {
      mn[k] = bbox[6 * t + k];
      const int64_t e = (int64_t)bbox[6 * t + 3 + k] - (int64_t)bbox[6 * t + k];
      ext = e > ext ? e : ext;
    }
    while (L < 33 && (int64_t(1) << L) <= ext) ++L;
  }
  SrcDesc& s = srcs[t];
  s.min[0] = mn[0];
  s.min[1] = mn[1];
  s.min[2] = mn[2];
  s.log2size = L;
  const uint32_t want = (n <= T || L == 0 || max_depth == 0) ? 0u : min(s.d, L);
  if (want != s.d) atomicOr(abort, 1u);
}

cudaError_t launch_roots(const TileDesc* tiles, const int* bbox, SrcDesc* srcs, uint32_t n_tiles, uint32_t T,
                         uint32_t max_depth, unsigned int* abort, cudaStream_t st) {
  if (!n_tiles) return cudaSuccess;
  k_roots<<<(n_tiles + 255) / 256, 256, 0, st>>>(tiles, bbox, srcs, n_tiles, T, max_depth, abort);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bbox(const TileDesc* tiles, const uint32_t* chunk_tile, uint64_t n_chunks,
                        const uint64_t* tile_chunk0, int* bbox, int grid, cudaStream_t st) {
  if (n_chunks == 0) return cudaSuccess;
  grid = (int)umin64((uint64_t)grid, n_chunks);
  k_bbox<<<grid, kBlock, 0, st>>>(tiles, chunk_tile, n_chunks, tile_chunk0, bbox);
  note_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------- counting
// Section 4.1.1 (count per cell of the grid) and 4.1.5 (count again inside
// the extended grids of overflowing cells): one histogram per source.
//
// Grids of up to 8^4 cells are counted in a dense shared-memory histogram.
// Larger first grids are counted through a per-CTA shared-memory hash table
// keyed by the cell's counter index: a CTA's contiguous run of chunks only
// touches the occupied cells of the cloud, each of which then costs one
// global add per CTA instead of one per point.  The table's (cell, count)
// list is kept for the scatter, which claims one block per cell.  Cells that
// arrive after the table is full are counted with per-point global atomics.

namespace {

__device__ __forceinline__ uint32_t priv_home(uint32_t key1) { return __umulhi(key1 * 0x9E3779B1u, kPrivSlots); }

// Slot of key1 (= counter index + 1) in a per-CTA table, inserting it if
// absent; -1 when kPrivProbe consecutive slots hold other cells (the table
// is then treated as full for this cell).  No shared fill counter is
// touched: every insert stays independent of the other warps.
__device__ __forceinline__ int priv_insert(uint32_t* keys, uint32_t key1) {
  uint32_t slot = priv_home(key1);
  for (uint32_t probe = 0; probe < kPrivProbe; ++probe) {
    const uint32_t k = ((volatile uint32_t*)keys)[slot];
    if (k == key1) return (int)slot;
    if (k == 0u) {
      const uint32_t old = atomicCAS(&keys[slot], 0u, key1);
      if (old == 0u || old == key1) return (int)slot;
    }
    slot = (slot + 1 == kPrivSlots) ? 0u : slot + 1;
  }
  return -1;
}

// Slot of key1 if present, -1 otherwise (the table is read-only here; keys
// are placed within kPrivProbe slots of their home, so the search ends
// there or at an empty slot).
__device__ __forceinline__ int priv_find(const uint32_t* keys, uint32_t key1) {
  uint32_t slot = priv_home(key1);
  for (uint32_t probe = 0; probe < kPrivProbe; ++probe) {
    const uint32_t k = keys[slot];
    if (k == key1) return (int)slot;
    if (k == 0u) return -1;
    slot = (slot + 1 == kPrivSlots) ? 0u : slot + 1;
  }
  return -1;
}

}  // namespace

__global__ void __launch_bounds__(kBlock, 1) k_count(BuildArgs a, const uint32_t* __restrict__ chunk_src,
                                                  const unsigned long long* __restrict__ n_chunks_p) {
  if (a.abort && *a.abort) return;
  __shared__ uint32_t hist[kSmemBins];
  __shared__ SrcDesc s;
  __shared__ uint32_t s_list;
  extern __shared__ __align__(16) uint32_t ptab[];  // kPrivSlots keys, then kPrivSlots counts
  uint32_t* pkeys = ptab;
  uint32_t* pcnt = ptab + kPrivSlots;
  const uint64_t n_chunks = *n_chunks_p;
  const uint64_t per = (n_chunks + gridDim.x - 1) / gridDim.x;
  const uint64_t c0 = (uint64_t)blockIdx.x * per;
  const uint64_t c1 = min(c0 + per, n_chunks);
  for (uint32_t i = threadIdx.x; i < kPrivSlots; i += blockDim.x) {
    pkeys[i] = 0u;
    pcnt[i] = 0u;
  }
  if (threadIdx.x == 0) {
    s_list = 0;
  }
  uint32_t cur = kNone;
  bool smem = false;
  uint32_t nbins = 0;

  uint2* list = a.lists + (uint64_t)blockIdx.x * kPrivSlots;
  auto flush = [&]() {
    __syncthreads();  // every thread's shared-memory increments are done
    if (smem) {
      // one global add per non-empty cell, and the (cell, count) pair into
      // the CTA's list while it has room, so that the scatter can claim the
      // cell's block at once
      uint32_t* dst = s.cnt + pyr_off(s.d);
      const uint32_t kbase = (uint32_t)(dst - a.cnt_base);
      const uint32_t lane = lane_id();
      for (uint32_t b0 = 0; b0 < nbins; b0 += blockDim.x) {
        const uint32_t b = b0 + threadIdx.x;
        const uint32_t h = b < nbins ? hist[b] : 0u;
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, h != 0u);
        uint32_t wbase = 0;
        if (lane == 0 && bal) wbase = atomicAdd(&s_list, (uint32_t)__popc(bal));
        wbase = __shfl_sync(0xFFFFFFFFu, wbase, 0);
        if (!h) continue;
        atomicAdd(dst + b, h);
        const uint32_t at = wbase + __popc(bal & ((1u << lane) - 1u));
        if (at < kListCap) list[at] = make_uint2(kbase + b, h);
      }
    }
    __syncthreads();
  };

  constexpr int kPer = (int)(kChunk / kBlock);
  const uint64_t pol_in = l2_evict_first();
  for (uint64_t c = c0; c < c1; ++c) {
    const uint32_t sid = chunk_src[c];
    if (sid != cur) {
      if (cur != kNone) flush();
      if (threadIdx.x == 0) s = a.srcs[sid];
      __syncthreads();
      cur = sid;
      nbins = 1u << (3 * s.d);
      smem = !s.priv;  // a dense grid (then nbins <= kSmemBins)
      if (smem)
        for (uint32_t b = threadIdx.x; b < nbins; b += blockDim.x) hist[b] = 0;
      __syncthreads();
    }
    const uint64_t first = (c - s.chunk0) << kChunkLog2;
    const uint64_t end = min(first + kChunk, (uint64_t)s.n);
    const int32_t mx = s.min[0], my = s.min[1], mz = s.min[2];
    const uint32_t lg = s.log2size, d = s.d;
    const int4* pts = src_points(a, s, a.tiles[s.tile]);
    prefetch_next_chunk(pts, first, s.n, c + 1 < c1 && chunk_src[c + 1] == sid);
    int4 p[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const uint64_t i = first + threadIdx.x + (uint64_t)k * kBlock;
      if (i < end) p[k] = ld_policy(pts + i, pol_in);
    }
    uint32_t bin[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const uint64_t i = first + threadIdx.x + (uint64_t)k * kBlock;
      bin[k] = i < end ? src_bin(p[k], mx, my, mz, lg, d) : 0u;
    }
    if (smem) {
#pragma unroll
      for (int k = 0; k < kPer; ++k) {
        const uint64_t i = first + threadIdx.x + (uint64_t)k * kBlock;
        if (i < end) atomicAdd(&hist[bin[k]], 1u);
      }
      continue;
    }
    const uint32_t kbase = (uint32_t)(s.cnt + pyr_off(d) - a.cnt_base);
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const uint64_t i = first + threadIdx.x + (uint64_t)k * kBlock;
      const unsigned m = __ballot_sync(0xFFFFFFFFu, i < end);
      if (i >= end) continue;
      const uint32_t key = kbase + bin[k];
      const int slot = priv_insert(pkeys, key + 1u);
      // a warp whose points all share one cell (scan-ordered input) adds once
      const int leader = __ffs(m) - 1;
      const int s0 = __shfl_sync(m, slot, leader);
      const bool same = __all_sync(m, slot == s0);
      if (same && s0 >= 0) {
        if ((int)lane_id() == leader) atomicAdd(&pcnt[s0], (uint32_t)__popc(m));
      } else if (slot >= 0) {
        atomicAdd(&pcnt[slot], 1u);
      } else {
        atomicAdd(a.cnt_base + key, 1u);  // table full: count globally
        if (a.diag) atomicAdd(&a.diag[0], 1ull);
      }
    }
  }
  if (cur != kNone) flush();
  // publish the table: one global add per distinct cell, and the CTA's list
  // (cells beyond its capacity are found by the scatter through the global
  // cursors instead)
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u;
  for (uint32_t i0 = 0; i0 < kPrivSlots; i0 += blockDim.x) {
    const uint32_t i = i0 + threadIdx.x;
    const uint32_t key1 = pkeys[i];
    const bool occ = key1 != 0u;
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, occ);
    uint32_t wbase = 0;
    if (lane == 0 && bal) wbase = atomicAdd(&s_list, (uint32_t)__popc(bal));
    wbase = __shfl_sync(0xFFFFFFFFu, wbase, 0);
    if (!occ) continue;
    atomicAdd(a.cnt_base + key1 - 1u, pcnt[i]);
    const uint32_t at = wbase + __popc(bal & ((1u << lane) - 1u));
    if (at < kListCap) list[at] = make_uint2(key1 - 1u, pcnt[i]);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    a.list_len[blockIdx.x] = min(s_list, kListCap);
    if (a.diag) atomicAdd(&a.diag[1], (unsigned long long)s_list);
  }
}

cudaError_t launch_count(const BuildArgs& a, const uint32_t* chunk_src, const unsigned long long* n_chunks,
                         int grid, cudaStream_t st) {
  static bool once = [] {
    cudaFuncSetAttribute(k_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(8 * kPrivSlots));
    return true;
  }();
  (void)once;
  k_count<<<grid, kBlock, 8 * kPrivSlots, st>>>(a, chunk_src, n_chunks);
  note_launch();
  return cudaGetLastError();
}


// ------------------------------------------------------------ pyramid: up-sweep
// Per-level counts (the counting-grid pyramid of Section 4.1.2) from the
// bottom histogram, 4 levels per CTA in shared memory.

__global__ void __launch_bounds__(512) k_pyr_up(BuildArgs a, const PyrJob* __restrict__ jobs) {
  if (a.abort && *a.abort) return;
  __shared__ uint32_t sm[4096 + 512 + 64 + 8];
  const PyrJob job = jobs[blockIdx.x];
  const SrcDesc& s = a.srcs[job.src];
  const uint32_t jb = job.lvl;
  const uint32_t k = min(4u, jb);
  const uint32_t nb = 1u << (3 * k);
  const uint32_t* bottom = s.cnt + pyr_off(jb) + (uint64_t)job.block * nb;
  for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) sm[i] = bottom[i];
  __syncthreads();
  uint32_t in_off = 0, n_in = nb, out_off = nb;
  for (uint32_t l = 1; l <= k; ++l) {
    const uint32_t n_out = n_in >> 3;
    uint32_t* dst = s.cnt + pyr_off(jb - l) + (uint64_t)job.block * n_out;
    for (uint32_t q = threadIdx.x; q < n_out; q += blockDim.x) {
      uint32_t sum = 0;
#pragma unroll
      for (int c = 0; c < 8; ++c) sum += sm[in_off + 8 * q + c];
      sm[out_off + q] = sum;
      dst[q] = sum;
    }
    __syncthreads();
    in_off = out_off;
    out_off += n_out;
    n_in = n_out;
  }
}

cudaError_t launch_pyr_up(const BuildArgs& a, const PyrJob* jobs, uint32_t n_jobs, cudaStream_t st) {
  if (!n_jobs) return cudaSuccess;
  k_pyr_up<<<n_jobs, 512, 0, st>>>(a, jobs);
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------- pyramid: down-sweep
// Exclusive-scan starts of every cell (the "target pointers" of Section
// 4.1.3: where each node's points go), top-down 4 levels per CTA.  At the
// bottom level the starts become the scatter cursors, and every cell with
// more than T points that can still be split becomes a refinement grid
// for the next round (Section 4.1.5, extended to any depth).

__global__ void __launch_bounds__(512) k_pyr_down(BuildArgs a, const PyrJob* __restrict__ jobs,
                                                  uint32_t next_base, uint32_t next_cap, uint32_t next_buf,
                                                  DevCounters* __restrict__ ctr) {
  if (a.abort && *a.abort) return;
  __shared__ uint32_t cnt[8 + 64 + 512 + 4096];
  __shared__ uint32_t sta[1 + 8 + 64 + 512 + 4096];
  const PyrJob job = jobs[blockIdx.x];
  const uint32_t sid = job.src;
  const SrcDesc s = a.srcs[sid];
  const uint32_t jt = job.lvl;
  const uint32_t k = min(4u, s.d - jt);
  // shared layout: level i (1..k) of the block subtree at offset (8^i - 8)/7
  uint32_t lo[5], lsz[5];
  lo[0] = 0;
  lsz[0] = 1;
  for (uint32_t i = 1; i <= 4; ++i) {
    lsz[i] = 1u << (3 * i);
    lo[i] = (uint32_t)((lsz[i] - 8) / 7);
  }
  for (uint32_t i = 1; i <= k; ++i) {
    const uint32_t* src = s.cnt + pyr_off(jt + i) + (uint64_t)job.block * lsz[i];
    for (uint32_t q = threadIdx.x; q < lsz[i]; q += blockDim.x) cnt[lo[i] + q] = src[q];
  }
  if (threadIdx.x == 0) {
    uint32_t top;
    if (jt == 0) {
      top = s.pt_off;
      s.start[0] = top;
    } else {
      top = s.start[pyr_off(jt) + job.block];
    }
    sta[0] = top;
  }
  __syncthreads();
  if (k == 0) return;  // a one-cell grid (d == 0) never overflows: its start is set above
  // sta layout: level 0 at [0], level i at 1 + lo[i]
  for (uint32_t i = 1; i <= k; ++i) {
    const uint32_t n_par = lsz[i - 1];
    const uint32_t par_off = (i == 1) ? 0 : 1 + lo[i - 1];
    uint32_t* gdst = s.start + pyr_off(jt + i) + (uint64_t)job.block * lsz[i];
    for (uint32_t q = threadIdx.x; q < n_par; q += blockDim.x) {
      uint32_t acc = sta[par_off + q];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        sta[1 + lo[i] + 8 * q + c] = acc;
        gdst[8 * q + c] = acc;
        acc += cnt[lo[i] + 8 * q + c];
      }
    }
    __syncthreads();
  }
  if (jt + k != s.d) return;
  // bottom level of the source: detect cells to refine
  const uint32_t level_b = s.level + s.d;
  const uint32_t log2_b = s.log2size - s.d;
  if (!(level_b < a.max_depth && log2_b > 0)) return;
  const uint32_t nbot = lsz[k];
  for (uint32_t q = threadIdx.x; q < nbot; q += blockDim.x) {
    const uint32_t n = cnt[lo[k] + q];
    if (n <= a.T) continue;
    const uint32_t c = job.block * nbot + q;  // Morton cell at the bottom level
    const unsigned long long id = atomicAdd(&ctr->new_srcs, 1ull);
    if (id >= next_cap) {
      atomicOr(&ctr->error, kErrSrcCap);
      continue;
    }
    atomicAdd(&ctr->new_points, (unsigned long long)n);
    const uint32_t g = next_base + (uint32_t)id;
    SrcDesc ns;
    ns.cnt = ns.start = ns.map = ns.ovf = nullptr;
    const uint32_t cx = compact3(c >> 2), cy = compact3(c >> 1), cz = compact3(c);
    ns.min[0] = (int32_t)((uint32_t)s.min[0] + (cx << log2_b));
    ns.min[1] = (int32_t)((uint32_t)s.min[1] + (cy << log2_b));
    ns.min[2] = (int32_t)((uint32_t)s.min[2] + (cz << log2_b));
    ns.tile = s.tile;
    ns.level = level_b;
    ns.log2size = log2_b;
    ns.d = choose_seg_depth(n, a.T, level_b, log2_b, a.max_depth);
    ns.buf = next_buf;
    ns.pt_off = sta[1 + lo[k] + q];
    ns.n = n;
    ns.chunk0 = 0;
    ns.priv = (1u << (3 * ns.d)) > a.dense_max ? 1u : 0u;  // counted through the per-CTA hash tables
    ns.pad = 0;
    a.srcs[g] = ns;
    s.map[c] = g;
    atomicOr(&s.ovf[c >> 5], 1u << (c & 31));
  }
}

cudaError_t launch_pyr_down(const BuildArgs& a, const PyrJob* jobs, uint32_t n_jobs, uint32_t next_base,
                            uint32_t next_cap, uint32_t next_buf, DevCounters* ctr, cudaStream_t st) {
  if (!n_jobs) return cudaSuccess;
  k_pyr_down<<<n_jobs, 512, 0, st>>>(a, jobs, next_base, next_cap, next_buf, ctr);
  note_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------- scatter
// Section 4.1.4 (insert): every point goes to its cell's cursor; points of
// cells that will be refined go to the ping-pong buffer of the next round,
// all others to their final place in the leaf-point array.  For large grids
// the CTA re-creates its counting table from its list, claims one block of
// positions per cell with one global atomic, and hands out positions inside
// the block with shared-memory atomics (the CTA processes the same chunks as
// in the counting pass).  Dense small grids claim cursors per point (one
// atomic per warp when all its points share a cell).

__global__ void __launch_bounds__(kBlock) k_scatter(BuildArgs a, const uint32_t* __restrict__ chunk_src,
                                                    const unsigned long long* __restrict__ n_chunks_p,
                                                    uint32_t round) {
  if (a.abort && *a.abort) return;
  __shared__ SrcDesc s;
  __shared__ uint32_t s_ovf[kSmemBins / 32];  // overflow mask of a dense grid
  // kPrivSlots keys, kPrivSlots cursors, kPrivSlots overflow flags
  extern __shared__ __align__(16) uint32_t ptab[];
  uint32_t* pkeys = ptab;
  uint32_t* pcur = ptab + kPrivSlots;
  uint8_t* pflag = reinterpret_cast<uint8_t*>(ptab + 2 * kPrivSlots);
  const uint64_t n_chunks = *n_chunks_p;
  const uint64_t per = (n_chunks + gridDim.x - 1) / gridDim.x;
  const uint64_t c0 = (uint64_t)blockIdx.x * per;
  const uint64_t c1 = min(c0 + per, n_chunks);
  int4* ovf_dst = (round & 1) ? a.tmp[1] : a.tmp[0];
  uint32_t* ovf_idx = (round & 1) ? a.tmp_idx[1] : a.tmp_idx[0];
  const uint32_t lane = lane_id();
  // claim this CTA's block of every cell it counted
  for (uint32_t i = threadIdx.x; i < kPrivSlots; i += blockDim.x) pkeys[i] = 0u;
  __syncthreads();
  {
    const uint32_t len = a.list_len[blockIdx.x];
    const uint2* list = a.lists + (uint64_t)blockIdx.x * kPrivSlots;
    // the listed cells belong to the CTA's sources, whose count regions are
    // laid out in source order: a binary search finds each cell's source,
    // whose overflow bit is kept beside the cursor
    const uint32_t sid_lo = c0 < c1 ? chunk_src[c0] : 0u, sid_hi = c0 < c1 ? chunk_src[c1 - 1] : 0u;
    for (uint32_t j = threadIdx.x; j < len; j += blockDim.x) {
      const uint2 e = list[j];
      // bounded probing, as in the counting pass: a cell that does not find
      // a slot near its home claims nothing here, and its points take
      // positions from the cell's global cursor instead
      uint32_t slot = priv_home(e.x + 1u);
      bool placed = false;
      for (uint32_t probe = 0; probe < kPrivProbe; ++probe) {
        if (atomicCAS(&pkeys[slot], 0u, e.x + 1u) == 0u) {
          placed = true;
          break;
        }
        slot = (slot + 1 == kPrivSlots) ? 0u : slot + 1;
      }
      if (!placed) continue;
      pcur[slot] = atomicAdd(a.cnt_base + e.x + a.cursor_delta, e.y);
      uint32_t lo = sid_lo, hi = sid_hi;  // last source whose count region starts at or before e.x
      while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if ((uint64_t)(a.srcs[mid].cnt - a.cnt_base) <= e.x) lo = mid;
        else hi = mid - 1;
      }
      const SrcDesc& es = a.srcs[lo];
      const uint32_t cell = e.x - (uint32_t)(es.cnt + pyr_off(es.d) - a.cnt_base);
      pflag[slot] = (uint8_t)((es.ovf[cell >> 5] >> (cell & 31u)) & 1u);
    }
  }
  __syncthreads();
  uint32_t cur = kNone;

  constexpr int kPer = (int)(kChunk / kBlock);
  const uint64_t pol_in = l2_evict_first(), pol_out = l2_evict_last();
  for (uint64_t c = c0; c < c1; ++c) {
    const uint32_t sid = chunk_src[c];
    if (sid != cur) {
      __syncthreads();
      if (threadIdx.x == 0) s = a.srcs[sid];
      __syncthreads();
      if (!s.priv)
        for (uint32_t w = threadIdx.x; w < ((1u << (3 * s.d)) + 31u) / 32u; w += blockDim.x) s_ovf[w] = s.ovf[w];
      __syncthreads();
      cur = sid;
    }
    const TileDesc& td = a.tiles[s.tile];
    const uint32_t* src_idx =
        s.buf == 0 ? td.in_idx : (s.buf == 1 ? a.tmp_idx[0] : a.tmp_idx[1]) + td.pt_base + s.pt_off;
    const uint64_t first = (c - s.chunk0) << kChunkLog2;
    const uint64_t end = min(first + kChunk, (uint64_t)s.n);
    uint32_t* cursor = s.start + pyr_off(s.d);
    const int32_t mx = s.min[0], my = s.min[1], mz = s.min[2];
    const uint32_t lg = s.log2size, d = s.d;
    const bool priv = s.priv != 0;
    const uint32_t kbase = (uint32_t)(s.cnt + pyr_off(d) - a.cnt_base);
    const int4* pts = src_points(a, s, td);
    int4 p[kPer];
    uint32_t bins[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const uint64_t i = first + threadIdx.x + (uint64_t)k * kBlock;
      p[k] = make_int4(0, 0, 0, 0);
      if (i < end) p[k] = ld_policy(pts + i, pol_in);
    }
#pragma unroll
    for (int k = 0; k < kPer; ++k) bins[k] = src_bin(p[k], mx, my, mz, lg, d);
    // claim every position before the first store that needs one
    uint32_t pb[kPer], ovf_bits = 0, agg = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const uint64_t i = first + threadIdx.x + (uint64_t)k * kBlock;
      const bool v = i < end;
      const unsigned m = __ballot_sync(0xFFFFFFFFu, v);
      pb[k] = 0;
      if (!v) continue;
      const uint32_t bin = bins[k];
      // the CTA's block of the cell (claimed from its list), else the
      // cell's global cursor (cells the list had no room for)
      const int slot = priv_find(pkeys, kbase + bin + 1u);
      const int leader = __ffs(m) - 1;
      const int s0 = __shfl_sync(m, slot, leader);
      const uint32_t b0 = __shfl_sync(m, bin, leader);
      if (__all_sync(m, slot == s0 && bin == b0)) {
        agg |= 1u << k;  // the whole warp's points share one cell: one claim
        if ((int)lane == leader)
          pb[k] = s0 >= 0 ? atomicAdd(&pcur[s0], (uint32_t)__popc(m)) : atomicAdd(cursor + bin, (uint32_t)__popc(m));
      } else {
        pb[k] = slot >= 0 ? atomicAdd(&pcur[slot], 1u) : atomicAdd(cursor + bin, 1u);
      }
      const uint32_t* om = priv ? s.ovf : s_ovf;
      const uint32_t f = slot >= 0 ? (uint32_t)pflag[slot] : (om[bin >> 5] >> (bin & 31u)) & 1u;
      ovf_bits |= f << k;
    }
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const uint64_t i = first + threadIdx.x + (uint64_t)k * kBlock;
      const unsigned m = __ballot_sync(0xFFFFFFFFu, i < end);
      if (i >= end) continue;
      uint32_t pos = pb[k];
      if (agg >> k & 1u) pos = __shfl_sync(m, pos, __ffs(m) - 1) + __popc(m & ((1u << lane) - 1u));
      const bool ovf = (ovf_bits >> k) & 1u;
      const uint64_t dst = td.pt_base + pos;
      const uint32_t idx = a.out_idx ? (src_idx ? src_idx[i] : (uint32_t)i) : 0u;
      if (ovf) {
        st_keep(ovf_dst + dst, p[k], pol_out);
        if (a.out_idx) ovf_idx[dst] = idx;
      } else if (a.wide) {
        // one full 32-byte sector per point and no separate 4-byte index
        // write (isolated sub-sector writes are the costliest kind)
        st_wide(a.wide + 2 * dst, p[k], idx);
      } else {
        st_keep(a.out + dst, p[k], pol_out);
        if (a.out_idx) a.out_idx[dst] = idx;
      }
    }
  }
}

cudaError_t launch_scatter(const BuildArgs& a, const uint32_t* chunk_src, const unsigned long long* n_chunks,
                           uint32_t round, int grid, cudaStream_t st) {
  static bool once = [] {
    cudaFuncSetAttribute(k_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(9 * kPrivSlots));
    return true;
  }();
  (void)once;
  k_scatter<<<grid, kBlock, 9 * kPrivSlots, st>>>(a, chunk_src, n_chunks, round);
  note_launch();
  return cudaGetLastError();
}


// ---------------------------------------------------------------- node table
// Breadth-first node list (Section 4.1.3 creates the node list from the
// count pyramid): one CTA per tile walks the levels; a node is split iff it
// holds more than T points, is above max_depth and larger than a unit cube.
// Children are the non-empty octants in octant order, their counts read
// from the pyramid of the grid that covers them (switching to the
// refinement grid of a cell at the bottom of a grid).  `refined` (the
// first round's count of refinement grids, or null): when the pass runs
// right after the first round and that round created refinement grids, the
// table would have to follow later rounds anyway, so the pass stands down
// at once (the host builds the table after the last round).

__global__ void __launch_bounds__(kBlock) k_nodes(BuildArgs a, lod_node_t* __restrict__ nodes,
                                                  NodeAux* __restrict__ aux, uint32_t* __restrict__ lvl_start,
                                                  uint32_t* __restrict__ n_nodes,
                                                  unsigned long long* __restrict__ leaf_cap,
                                                  DevCounters* __restrict__ ctr,
                                                  const unsigned long long* __restrict__ refined) {
  if (a.abort && *a.abort) return;
  if (refined && *refined) {
    if (threadIdx.x == 0) n_nodes[blockIdx.x] = kNone;
    return;
  }
  __shared__ uint32_t warp_sum[32];
  __shared__ uint32_t s_total;
  __shared__ int s_fail;
  const uint32_t t = blockIdx.x;
  const TileDesc td = a.tiles[t];
  lod_node_t* nd = nodes + td.node_base;
  NodeAux* ax = aux + td.node_base;
  uint32_t* ls = lvl_start + (uint64_t)t * (kMaxLevels + 1);
  if (threadIdx.x == 0) {
    lod_node_t r;
    const SrcDesc& rs = a.srcs[t];  // the tile's first counting grid covers the root cube
    r.min[0] = rs.min[0];
    r.min[1] = rs.min[1];
    r.min[2] = rs.min[2];
    r.level = 0;
    r.log2_size = (uint8_t)rs.log2size;
    r.child_mask = 0;
    r.flags = 0;
    r.parent = kNone;
    r.first_child = kNone;
    r.point_offset = 0;
    r.point_count = td.n;
    r.voxel_offset = 0;
    r.voxel_count = 0;
    r.reserved = 0;
    nd[0] = r;
    ax[0].src = t;
    ax[0].j = 0;
    ax[0].c = 0;
    s_fail = 0;
  }
  __syncthreads();
  uint32_t begin = 0, end = 1, level = 0;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  while (begin < end) {
    if (threadIdx.x == 0) ls[level] = begin;
    uint32_t next = end;
    for (uint32_t chunk = begin; chunk < end; chunk += blockDim.x) {
      const uint32_t i = chunk + threadIdx.x;
      const bool valid = i < end;
      uint32_t mask = 0, cc[8];
      uint32_t sid = 0, j = 0, c = 0;
      uint64_t cnt = 0;
      uint32_t lvl = 0, lg = 0;
      bool split = false;
      if (valid) {
        cnt = nd[i].point_count;
        lvl = nd[i].level;
        lg = nd[i].log2_size;
        sid = ax[i].src;
        j = ax[i].j;
        c = ax[i].c;
        split = cnt > a.T && lvl < a.max_depth && lg > 0;
        if (split && j == a.srcs[sid].d) {
          // bottom cell of its grid: continue in the cell's refinement grid
          // (not counted yet when this pass runs before the next round; the
          // host then discards the table and builds it after the rounds)
          const uint32_t child = a.srcs[sid].map[c];
          if (a.srcs[child].cnt == nullptr) {
            split = false;
            s_fail = 2;
          } else {
            sid = child;
            j = 0;
            c = 0;
            ax[i].src = sid;
            ax[i].j = 0;
            ax[i].c = 0;
          }
        }
        if (split) {
          const uint32_t* ch = a.srcs[sid].cnt + pyr_off(j + 1) + 8ull * c;
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            cc[k] = ch[k];
            mask |= (cc[k] ? 1u : 0u) << k;
          }
        }
      }
      const uint32_t nch = __popc(mask);
      // block exclusive scan of nch
      uint32_t incl = nch;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if ((int)lane >= o) incl += y;
      }
      if (lane == 31) warp_sum[warp] = incl;
      __syncthreads();
      if (warp == 0) {
        const uint32_t nw = blockDim.x >> 5;
        uint32_t w = lane < nw ? warp_sum[lane] : 0;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
          if ((int)lane >= o) wi += y;
        }
        if (lane < nw) warp_sum[lane] = wi - w;
        if (lane == nw - 1) s_total = wi;
      }
      __syncthreads();
      const uint32_t pos = warp_sum[warp] + incl - nch;
      const uint32_t total = s_total;
      const bool fits = (uint64_t)next + total <= td.node_cap;
      if (valid && fits) {
        const SrcDesc& sd = a.srcs[sid];
        const uint32_t st = sd.start[pyr_off(j) + c];
        // bottom cells: the start array was advanced by the scatter (cursor)
        nd[i].point_offset = (j < sd.d) ? st : st - (uint32_t)cnt;
        nd[i].child_mask = (uint8_t)mask;
        nd[i].flags = split ? 0 : (LOD_NODE_LEAF | (cnt > a.T ? LOD_NODE_OVERFULL : 0));
        nd[i].first_child = split ? next + pos : kNone;
        // per level: bound on the voxel records the node's octant can
        // contribute to its parent (all nodes), and the exact leaf points
        atomicAdd(&leaf_cap[lvl], (unsigned long long)umin64(cnt, kOctCells));
        if (!split) atomicAdd(&leaf_cap[kMaxLevels + 1 + lvl], (unsigned long long)cnt);
        if (split) {
          const uint32_t half = lg - 1;
          uint32_t r = 0;
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            if (!(mask >> k & 1u)) continue;
            const uint32_t id = next + pos + r++;
            lod_node_t q;
            q.min[0] = (int32_t)((uint32_t)nd[i].min[0] + ((uint32_t)((k >> 2) & 1) << half));
            q.min[1] = (int32_t)((uint32_t)nd[i].min[1] + ((uint32_t)((k >> 1) & 1) << half));
            q.min[2] = (int32_t)((uint32_t)nd[i].min[2] + ((uint32_t)(k & 1) << half));
            q.level = (uint8_t)(lvl + 1);
            q.log2_size = (uint8_t)half;
            q.child_mask = 0;
            q.flags = 0;
            q.parent = i;
            q.first_child = kNone;
            q.point_offset = 0;
            q.point_count = cc[k];
            q.voxel_offset = 0;
            q.voxel_count = 0;
            q.reserved = 0;
            nd[id] = q;
            ax[id].src = sid;
            ax[id].j = j + 1;
            ax[id].c = 8 * c + k;
            ax[id].occ = 0;
          }
        }
      }
      if (!fits && threadIdx.x == 0) s_fail = 1;
      next += total;
      __syncthreads();
      if (s_fail) break;
    }
    if (s_fail) break;
    begin = end;
    end = next;
    ++level;
  }
  if (threadIdx.x == 0) {
    ls[level] = begin;
    for (uint32_t l = level + 1; l <= kMaxLevels; ++l) ls[l] = begin;
    n_nodes[t] = s_fail ? kNone : end;
    if (s_fail == 1) atomicOr(&ctr->error, kErrNodeCap);
  }
}

cudaError_t launch_nodes(const BuildArgs& a, lod_node_t* nodes, NodeAux* aux, uint32_t* lvl_start,
                         uint32_t* n_nodes, unsigned long long* leaf_cap, DevCounters* ctr,
                         const unsigned long long* refined, cudaStream_t st) {
  k_nodes<<<a.n_tiles, kBlock, 0, st>>>(a, nodes, aux, lvl_start, n_nodes, leaf_cap, ctr, refined);
  note_launch();
  return cudaGetLastError();
}

}  // namespace lodk
