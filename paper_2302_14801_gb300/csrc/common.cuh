// Internal definitions shared by the kernels and the host orchestrator of the
// GB300 LOD builder.  Nothing here is part of the public C ABI (include/lod.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lod.h"

namespace lodk {

// ----------------------------------------------------------------- constants
constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr uint32_t kChunk = 4096;      // points per work chunk of the streaming kernels
constexpr uint32_t kChunkLog2 = 12;
constexpr uint32_t kMaxLevels = 34;    // levels 0..32 plus one sentinel slot
constexpr uint32_t kRootMaxD = 8;      // depth of the largest first counting grid (256^3 cells)
constexpr uint32_t kSmemBins = 4096;   // grids up to 8^4 bins are counted in shared memory
constexpr uint32_t kOctCells = 1u << 18;  // 64^3 cells of one child octant (Section 4.2)
constexpr uint32_t kBlock = 1024;

// Offset of level j inside a count/start pyramid stored level by level
// (level j holds 8^j cells in Morton order), and the pyramid's total size.
__host__ __device__ __forceinline__ uint64_t pyr_off(uint32_t j) {
  return ((uint64_t(1) << (3 * j)) - 1) / 7;
}
__host__ __device__ __forceinline__ uint64_t pyr_size(uint32_t d) { return pyr_off(d + 1); }

// ------------------------------------------------------------- descriptors

// One independent problem (a whole cloud for lod_build, one tile for the
// batched and serving paths).  Positions are tile-relative unless noted.
struct TileDesc {
  const int4* in;      // caller's input points (16-byte records)
  uint32_t n;          // points
  uint32_t log2S;      // root cube edge 2^log2S
  int32_t min[3];      // root cube min corner (bounding-box minimum)
  uint32_t node_cap;   // capacity of this tile's node region
  uint64_t pt_base;    // absolute base of the tile in the shared point buffers
  uint64_t node_base;  // absolute first node of the tile in the node buffer
  const uint32_t* in_idx;  // input index of each input point, or null (the position)
  uint32_t idx_bound;      // input indices are below this
  uint32_t level0;         // octree level of the tile's root
};

// A counting grid ("source"): 8^d cells under one cube, the whole root for
// the first grid of a tile, or an overflowing cell for a refinement grid
// (Section 4.1.5).  Its points occupy [pt_off, pt_off + n) of the tile.
struct SrcDesc {
  uint32_t* cnt;       // count pyramid, levels 0..d (level j: 8^j cells)
  uint32_t* start;     // start pyramid (tile-relative positions); its
                       // bottom level is the scatter cursor
  uint32_t* map;       // bottom cells: child source id where overflowing
  uint32_t* ovf;       // bottom cells: overflow bit mask
  int32_t min[3];
  uint32_t tile;
  uint32_t level;      // octree level of the source's root cell
  uint32_t log2size;   // edge of the source's root cell
  uint32_t d;          // grid depth (0..8)
  uint32_t buf;        // where its points are: 0 tile input, 1 tmpA, 2 tmpB
  uint32_t pt_off;
  uint32_t n;
  uint64_t chunk0;     // first chunk of this source in its round's chunk space
  uint32_t priv;       // 1: counted through per-CTA shared-memory tables
                       // (grids too large for a dense shared histogram)
  uint32_t pad;
};

// Build-wide settings shared by every kernel of one build.
struct BuildArgs {
  const TileDesc* tiles;
  SrcDesc* srcs;
  uint32_t n_tiles;
  uint32_t T;
  uint32_t max_depth;
  uint32_t mode;
  int4* out;           // leaf points, all tiles, absolute positions
  uint32_t* out_idx;   // original input index per leaf point (or null)
  int4* tmp[2];        // refinement ping-pong buffers (absolute positions)
  uint32_t* tmp_idx[2];
  int4* wide;          // when input indices are kept: the scatter writes each
                       // leaf point as one full 32-byte sector {point},{index}
                       // here (two int4 per position), and the bottom voxel
                       // pass writes out / out_idx contiguously from it
  // privatised counting of large grids: counters are keyed by their index
  // relative to cnt_base; each CTA leaves its (key, count) list in lists
  uint32_t* cnt_base;      // count region of the round's pool
  uint64_t cursor_delta;   // start region - count region (u32 elements)
  uint2* lists;            // kPrivSlots entries per CTA
  uint32_t* list_len;      // per CTA
  unsigned long long* diag;  // [0] points counted outside the tables, [1] table inserts
  // nonzero: a root grid's depth chosen before the bounding box was known
  // exceeds its cube; the split kernels then do nothing and the host
  // restarts with the depths fixed
  const unsigned int* abort;
  uint32_t dense_max;  // grids of at most this many cells count in a dense shared histogram (<= kSmemBins)
  uint32_t pad_;
};

constexpr uint32_t kPrivSlots = 24576;  // per-CTA table of distinct cells (192 KB counting, 216 KB scatter)
constexpr uint32_t kListCap = kPrivSlots / 4 * 3;  // listed cells per CTA (the scatter's table stays <= 3/4 full)
constexpr uint32_t kPrivProbe = 32;     // longest probe sequence before a cell counts as not fitting

// Per-node internal bookkeeping of the voxel pass, indexed by absolute node.
struct NodeAux {
  uint32_t src, j, c;  // counting grid, local level, Morton cell (split pass)
  uint32_t occ;        // voxels this node contributes to its parent's grid
  uint64_t stage;      // first staging record of that contribution
  uint64_t dense;      // absolute position of that contribution in the voxel array
};

// Counters written by kernels and read back by the host.
struct DevCounters {
  unsigned long long new_srcs;        // refinement grids created this round
  unsigned long long new_points;      // points inside them
  unsigned long long stage_used[2];   // staging records bump allocators
  unsigned long long level_voxels;    // voxels of the level just scanned
  unsigned long long vox_retries;     // voxel items whose cells need several accumulate passes
  unsigned long long vox_passes;      // passes over samples (mark and accumulate) of all voxel items
  unsigned long long vox_samples;     // samples read by all table passes (re-reads included)
  unsigned long long vox_max_item;    // samples of the level's largest item (statistics)
  unsigned int error;                 // nonzero: a kernel detected a problem
  unsigned int units;                 // voxel partition units queued this level
  unsigned int unit_head;             // units taken by the partition kernel
  unsigned int item_head;             // items taken by the first-attempt kernel
};

enum : uint32_t {
  kErrNodeCap = 1u,      // node capacity of a tile exceeded
  kErrStageCap = 2u,     // staging capacity exceeded
  kErrSrcCap = 4u,       // source table capacity exceeded
  kErrInternal = 8u,
};

// ----------------------------------------------------------- device helpers

__host__ __device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }

// splitmix64 (Steele, Lea & Flood, OOPSLA 2014): first output of a generator
// whose state is x.
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// 128^3 grid coordinate of an offset d (0 <= d < 2^L) inside a cube of edge
// 2^L (Section 4.2: every node samples onto a 128^3 grid).
__device__ __forceinline__ uint32_t grid_coord(uint32_t d, uint32_t L) {
  return L >= 7 ? d >> (L - 7) : (d << (7 - L));  // L <= 32, so L - 7 < 32
}

__device__ __forceinline__ int4 ldg_stream(const int4* p) { return __ldcs(p); }

// One 32-byte staging record {point, index, 0, 0, 0} moved with a single
// 256-bit access (sm_100 and later), evict-first.  p is 32-byte aligned.
__device__ __forceinline__ void st_wide(int4* p, const int4& q, uint32_t idx) {
  asm volatile("st.global.cs.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %6, %6};" ::"l"(p), "r"(q.x), "r"(q.y),
               "r"(q.z), "r"(q.w), "r"(idx), "r"(0u)
               : "memory");
}
__device__ __forceinline__ void ld_wide(const int4* p, int4& q, uint32_t& idx) {
  uint32_t u0, u1, u2;
  asm("ld.global.cs.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(q.x), "=r"(q.y), "=r"(q.z), "=r"(q.w), "=r"(idx), "=r"(u0), "=r"(u1), "=r"(u2)
               : "l"(p));
  (void)u0;
  (void)u1;
  (void)u2;
}

// ---------------------------------------------------------- sampling rules

// floor((s + n/2) / n) for a channel sum s of n 8-bit samples, i.e. the
// mean rounded half up, which lies in [0, 255].  A single-precision
// quotient is within 1 of it (relative error ~1e-7 on a value <= 255.5),
// and one exact integer comparison each way settles it, avoiding a 64-bit
// integer division.
__device__ __forceinline__ uint32_t round_mean(uint64_t s, uint64_t n) {
  const uint64_t num = s + (n >> 1);
  // 64-bit integer to float conversions run on the FP64 pipe, which is
  // narrow on this GPU: convert 32-bit values where they fit
  const float fnum = (num >> 32) ? (float)num : __uint2float_rn((uint32_t)num);
  const float fn = (n >> 32) ? (float)n : __uint2float_rn((uint32_t)n);
  uint32_t q = (uint32_t)__fdividef(fnum, fn);
  q = q > 255u ? 255u : q;
  if ((uint64_t)q * n > num) --q;
  else if ((uint64_t)(q + 1) * n <= num) ++q;
  return q;
}

__device__ __forceinline__ uint32_t mean_rgba(uint64_t r, uint64_t g, uint64_t b, uint64_t n) {
  return round_mean(r, n) | (round_mean(g, n) << 8) | (round_mean(b, n) << 16) | 0xFF000000u;
}

// Key of a sample in the single-sample modes; every cell keeps the sample
// of smallest key, and every key is below the empty entry's ~0 (the
// splitmix64 preimage of ~0 is not a 32-bit index).  `level` is the level
// of the node being filled.
//  - LOD_PICK: splitmix64(input index) (replaces Listing 1 with an exact,
//    order-independent rule).
//  - LOD_FIRST: the input index itself: the first sample in input order
//    (Section 4.2.1); a child's voxel carries its own first point, so the
//    bottom-up merge keeps the cell's first point.
//  - LOD_RANDOM: Listing 1 of Section 4.2.2: a 32-bit key holding the top
//    12 bits of a random number drawn for the sample at this level above
//    the low 20 bits of the sample's index, the largest key winning; equal
//    keys go to the larger index.  The random number is the high half of
//    splitmix64(level << 32 | index).  Minimising 2^64 - 2 - (key << 32 |
//    index) maximises (key, index).
template <int MODE>
__device__ __forceinline__ uint64_t pick_key(uint32_t ix, uint32_t level) {
  if (MODE == LOD_FIRST) return ix;
  if (MODE == LOD_RANDOM) {
    const uint32_t r = (uint32_t)(splitmix64(((uint64_t)level << 32) | ix) >> 32);
    const uint64_t key = (r & 0xFFF00000u) | (ix & 0x000FFFFFu);
    return 0xFFFFFFFFFFFFFFFEull - ((key << 32) | ix);
  }
  return splitmix64(ix);
}

}  // namespace lodk
