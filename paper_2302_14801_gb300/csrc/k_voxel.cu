// Bottom-up voxel sampling (Section 4.2 of the paper).
//
// The paper processes one node per workgroup with one 128^3 grid per SM in
// global memory (8 MB / 33 MB per workgroup, Sections 4.2.2-4.2.3).  Here a
// CTA handles one (parent, child octant) pair, an "item": the child's
// samples (its leaf points, or the voxels the child itself received one
// level below) all fall into one 64^3 octant of the parent's 128^3 grid
// (the observation of Section 4.2).  Sampling an item takes two passes over
// its samples, both in shared memory:
//
//  1. mark: every sample sets its cell's bit in a 32 KB occupancy bitmap of
//     the octant (the item's samples were asked into L2 when it started); a
//     block scan of the bitmap's population counts then stores, beside
//     every 32-cell word of the bitmap, the rank of its first occupied
//     cell, which numbers the item's D occupied cells 0..D-1 in cell order;
//  2. accumulate: every sample finds its cell's rank (one 8-byte read and
//     one population count) and updates the dense entry of that rank.
//
// No hashing and no probing: every lookup costs the same, D is exact before
// anything is accumulated (so the item's staging block is reserved to the
// record), and the voxels come out sorted by cell.  The dense entries of
// one pass hold 5120 to 10240 cells, depending on the mode; an item with
// more occupied cells takes its ranks in consecutive ranges, one accumulate
// pass each, and may hand ranges to other SMs.  Colour sums are exact
// integers (packed 24- or 32-bit fields while they provably cannot
// overflow, 64-bit otherwise); the single-sample modes (minimal-hash pick,
// first come of Section 4.2.1, random with the key of Listing 1) keep, per
// cell, the entry {key, rgba | index << 32} of minimal key, updated by a
// 128-bit compare-and-swap, so the picked colour travels with the winning
// key and is never gathered from the input.
//
// Every octant's voxels go to a staging area; a level scan then assigns
// each parent one contiguous voxel range (children are consecutive in node
// order), and the next level up copies the records to that range while it
// reads them (so each record is read once).
#include "common.cuh"
#include "kernels.h"

namespace lodk {

namespace {

constexpr int kSmemBytes = 224 * 1024;
// occupancy words: 32 cells of the bitmap and the rank of their first
// occupied cell, {word, rank} (8 bytes, one read and one population count
// per lookup)
constexpr uint32_t kWords = kOctCells / 32u;  // 8192
constexpr uint32_t kDenseOff = kWords * 8u;
constexpr uint32_t kDenseBytes = kSmemBytes - kDenseOff;
// cells one accumulate pass holds; every layout ends with the u32 cell of each rank
constexpr uint32_t kCapSmall = kDenseBytes / 16;   // filtered, <= 65535 points: u64 {R:24 G:24 n:16}, u32 B
constexpr uint32_t kCapNarrow = kDenseBytes / 20;  // filtered, 32-bit sums: u64 {R, G}, u64 {B, n}
constexpr uint32_t kCapWide = kDenseBytes / 32;    // filtered, 64-bit sums: 3 x u64, u32 n
constexpr uint32_t kCapPick = kDenseBytes / 24;    // single sample: {u64 key, u64 payload}, u32 n
constexpr uint64_t kNarrowMaxSamples = 0xFFFFFFFFull / 255;  // 32-bit channel sums cannot overflow
constexpr uint64_t kSmallMaxSamples = 0xFFFFu;               // 24-bit sums and a 16-bit count cannot
constexpr uint64_t kMask40 = (1ull << 40) - 1;
constexpr uint32_t kNoRank = 0xFFFFFFFFu;
// Filtered staging records of cells of fewer than kPackMaxCount points carry
// their exact sums in the record's last word (10 bits per channel), so that
// neither the extraction nor the next level up touches the 16-byte sums
// array for them; larger cells keep the last word kNone and their sums in
// that array.
constexpr uint64_t kPackMaxCount = 1024;

// A channel's exact sum s over n < 1024 points and its rounded mean
// m = floor((s + floor(n/2)) / n) determine the remainder
// s + floor(n/2) - m n, which lies in [0, n); the three remainders, 10 bits
// each, fit below bit 30 (so the word never equals kNone).
__device__ __forceinline__ uint32_t pack_remainders(uint64_t sr, uint64_t sg, uint64_t sb, uint64_t n, uint32_t m) {
  const uint32_t nn = (uint32_t)n, h = nn >> 1;
  const uint32_t rr = (uint32_t)sr + h - (m & 255u) * nn;
  const uint32_t rg = (uint32_t)sg + h - ((m >> 8) & 255u) * nn;
  const uint32_t rb = (uint32_t)sb + h - ((m >> 16) & 255u) * nn;
  return rr | (rg << 10) | (rb << 20);
}

// The sums of a packed record {cell, mean rgba, n, remainders} in the
// layout of the sums array: {R | G << 40, G >> 24 | B << 16}.
__device__ __forceinline__ ulonglong2 unpack_sums(const int4& rec) {
  const uint32_t m = (uint32_t)rec.y, nn = (uint32_t)rec.z, w = (uint32_t)rec.w, h = nn >> 1;
  const uint64_t sr = (m & 255u) * nn + (w & 1023u) - h;
  const uint64_t sg = ((m >> 8) & 255u) * nn + ((w >> 10) & 1023u) - h;
  const uint64_t sb = ((m >> 16) & 255u) * nn + ((w >> 20) & 1023u) - h;
  return make_ulonglong2(sr | (sg << 40), (sg >> 24) | (sb << 16));
}

// an item's samples prefetched into L2 when it starts: at most this many
// bytes (152 SMs x 256 KB stays well inside the 126 MB L2)
constexpr uint64_t kPrefetchBytes = 256u * 1024u;

// Ask the bulk-copy unit to bring [p, p + bytes) into L2 (p 16-byte
// aligned, bytes a multiple of 16; nothing waits on it).
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Set the occupancy bits of a thread's four samples (cells with ok[k]).
// The four bitmap words are read first, back to back, so the thread waits
// for shared memory once; only bits found clear are then set (most samples
// find theirs set already).  A read that misses a concurrent update only
// costs a redundant atomic.
__device__ __forceinline__ void mark_cells4(uint2* W, const uint32_t (&cell)[4], const bool (&ok)[4]) {
  uint32_t* w[4];
  uint32_t bit[4], cur[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    w[k] = &W[cell[k] >> 5].x;  // local cell x | y << 6 | z << 12: word cell / 32
    bit[k] = 1u << (cell[k] & 31u);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) cur[k] = ok[k] ? *((volatile uint32_t*)w[k]) : ~0u;
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (!(cur[k] & bit[k])) atomicOr(w[k], bit[k]);
}

// Ranks, among the item's occupied cells (cell order), of a thread's four
// samples' cells, minus lo; kNoRank for samples without ok[k] or outside
// [lo, lo + span).  The bitmap is read-only during an accumulate pass, so
// the four 8-byte word reads are issued together.
__device__ __forceinline__ void cell_ranks4(const uint2* W, const uint32_t (&cell)[4], const bool (&ok)[4],
                                            uint32_t lo, uint32_t span, uint32_t (&rk)[4]) {
  uint2 e[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) e[k] = ok[k] ? W[cell[k] >> 5] : make_uint2(0u, 0u);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t below = (1u << (cell[k] & 31u)) - 1u;
    const uint32_t r = e[k].y + __popc(e[k].x & below) - lo;
    rk[k] = (ok[k] && r < span) ? r : kNoRank;
  }
}

// Single-sample modes: the keys of the pick entries of a thread's four
// ranks, read together before any of them is updated (kNoRank: a key no
// sample beats).
template <bool PICKLIKE>
__device__ __forceinline__ void pre_keys4(const ulonglong2* E, const uint32_t (&rk)[4], uint64_t (&pre)[4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    pre[k] = 0ull;
    if (PICKLIKE && rk[k] != kNoRank) {
      asm volatile("ld.volatile.shared.u64 %0, [%1];"
                   : "=l"(pre[k])
                   : "r"((uint32_t)__cvta_generic_to_shared(E + rk[k])));
    }
  }
}

// Keep the sample of smaller key in a pick entry {key, rgba | index << 32}
// (keys of distinct samples differ).  `seen` is the entry's key as read
// earlier: keys only decrease while a pass runs, so a sample whose key is
// not below that read loses for sure and writes nothing.  Otherwise the
// entry is read again and the improvement installed with a 128-bit
// compare-and-swap, retried while others lower the entry meanwhile (each
// retry sees a strictly smaller key, so the loop ends; the bound only
// guards against a broken invariant).
__device__ __forceinline__ bool pick_update(ulonglong2* e, uint64_t h, uint64_t pay, uint64_t seen) {
  if (h >= seen) return true;
  const uint32_t addr = (uint32_t)__cvta_generic_to_shared(e);
  uint64_t c0, c1;
  asm volatile("ld.volatile.shared.v2.u64 {%0, %1}, [%2];" : "=l"(c0), "=l"(c1) : "r"(addr) : "memory");
  for (uint32_t tries = 0; h < c0; ++tries) {
    if (tries == (1u << 20)) return false;
    uint64_t p0, p1;
    asm volatile(
        "{\n .reg .b128 d, c, s;\n mov.b128 c, {%2, %3};\n mov.b128 s, {%4, %5};\n"
        " atom.shared.cas.b128 d, [%6], c, s;\n mov.b128 {%0, %1}, d;\n}"
        : "=l"(p0), "=l"(p1)
        : "l"(c0), "l"(c1), "l"(h), "l"(pay), "r"(addr)
        : "memory");
    if (p0 == c0 && p1 == c1) return true;
    c0 = p0;
    c1 = p1;
  }
  return true;
}

struct ItemInfo {
  uint32_t tile;
  uint64_t g;        // absolute node id of the item (the child)
  uint32_t kx, ky, kz;
  uint32_t Lp;       // parent log2 edge
  int32_t pmin[3];
  bool leaf;
  uint64_t n;        // samples
  uint64_t npts;     // original points in the child's cube
};

__device__ __forceinline__ uint32_t find_tile(const uint32_t* prefix, uint32_t n_tiles, uint32_t it) {
  uint32_t lo = 0, hi = n_tiles;  // largest t with prefix[t] <= it
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (prefix[mid] <= it) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Local cell (x | y << 6 | z << 12) of a point in the item's octant.
__device__ __forceinline__ uint32_t point_cell(const int4& q, const ItemInfo& I) {
  const uint32_t qx = grid_coord((uint32_t)q.x - (uint32_t)I.pmin[0], I.Lp) & 63u;
  const uint32_t qy = grid_coord((uint32_t)q.y - (uint32_t)I.pmin[1], I.Lp) & 63u;
  const uint32_t qz = grid_coord((uint32_t)q.z - (uint32_t)I.pmin[2], I.Lp) & 63u;
  return qx | (qy << 6) | (qz << 12);
}

// Local cell of a child's voxel (its cell in the child's 128^3 grid).
__device__ __forceinline__ uint32_t voxel_cell(uint32_t cell) {
  const uint32_t x = (cell & 127u) >> 1, y = ((cell >> 7) & 127u) >> 1, z = ((cell >> 14) & 127u) >> 1;
  return x | (y << 6) | (z << 12);
}

// Cell of the parent's 128^3 grid of a local cell.
__device__ __forceinline__ uint32_t parent_cell(uint32_t l, const ItemInfo& I) {
  return ((I.kx << 6) | (l & 63u)) | (((I.ky << 6) | ((l >> 6) & 63u)) << 7) | (((I.kz << 6) | (l >> 12)) << 14);
}

// One 32-byte {point, index} record, kept in L2 (it is read again).
__device__ __forceinline__ void ld_wide_keep(const int4* p, int4& q, uint32_t& idx) {
  uint32_t u0, u1, u2;
  asm("ld.global.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(q.x), "=r"(q.y), "=r"(q.z), "=r"(q.w), "=r"(idx), "=r"(u0), "=r"(u1), "=r"(u2)
      : "l"(p));
  (void)u0;
  (void)u1;
  (void)u2;
}

}  // namespace

int vox_smem_bytes() { return kSmemBytes; }

// Cells per accumulate pass of the four entry layouts (statistics and tests).
void vox_capacities(uint32_t* small, uint32_t* narrow, uint32_t* wide, uint32_t* pick) {
  *small = kCapSmall;
  *narrow = kCapNarrow;
  *wide = kCapWide;
  *pick = kCapPick;
}

// Shared state of one voxel CTA.
struct VoxShared {
  uint32_t D;                  // occupied cells of the item
  uint32_t r0, r1;             // rank interval this CTA accumulates
  uint32_t samples;            // samples read by the item's passes (statistics)
  unsigned long long stage;    // first staging record of the item (rank 0)
  uint32_t nch;                // inner items: children
  int32_t cmin[3];             // header: the child's min corner
  unsigned long long cparent, cfirst;  // header: parent node, first child (absolute)
  unsigned long long pbase;    // header: the child's first leaf point (absolute)
  uint32_t cpre[9];            // inner items: prefix of the children's record counts
  unsigned long long cstage[8];  // ... their first staging records
  unsigned long long cdense[8];  // ... their places in the voxel array
  uint32_t wsum[32];
  ItemInfo I;
};

// Reserve `n` consecutive slots of the unit queue; false when it is full
// (the reservation is all or nothing, so no slot is left unwritten).
__device__ __forceinline__ bool reserve_units(unsigned int* count, uint32_t cap, uint32_t n, uint32_t* first) {
  uint32_t old = *((volatile unsigned int*)count);
  for (int tries = 0; tries < 4096; ++tries) {
    if (old + n > cap) return false;
    const uint32_t prev = atomicCAS(count, old, old + n);
    if (prev == old) {
      *first = old;
      return true;
    }
    old = prev;
  }
  return false;
}

// Empty dense entries: all zero bytes in filtered mode (whatever the
// layout), {~0, 0} and a zero count in the single-sample modes.
template <int MODE>
__device__ __forceinline__ void vox_clear_dense(unsigned char* smem) {
  if (MODE == LOD_FILTER) {
    uint4* z = reinterpret_cast<uint4*>(smem + kDenseOff);
    for (uint32_t i = threadIdx.x; i < kDenseBytes / 16u; i += blockDim.x) z[i] = make_uint4(0, 0, 0, 0);
  } else {
    ulonglong2* E = reinterpret_cast<ulonglong2*>(smem + kDenseOff);
    uint32_t* cnt = reinterpret_cast<uint32_t*>(E + kCapPick);
    for (uint32_t i = threadIdx.x; i < kCapPick; i += blockDim.x) {
      E[i] = make_ulonglong2(~0ull, 0ull);
      cnt[i] = 0u;
    }
  }
}

static_assert(8u * kBlock == kWords, "the rank scan gives every warp 256 words");

// Voxelize one item (a child node c of an inner node p at level v.level):
// all of its ranks, or, for a queued unit (r_unit, p_unit), the ranks
// [D r / P, D (r + 1) / P) of its D occupied cells.  `first`: the item's
// first attempt, which reserves the item's staging block (D records) and,
// when its cells need several accumulate passes, may queue the ranges after
// the first for the partition kernel.  The CTA that holds range 0 also
// publishes what it reads (the leaf's points, the children's voxels).
// `next_item` (first attempts): where thread 0 leaves the item the CTA
// takes next, fetched while this one is marked.  `split_unit`: a range of an
// item split up front, whose leaf may not be published yet (the units of one
// item run side by side).
template <int MODE>
__device__ __forceinline__ void vox_item(const BuildArgs& a, const VoxLevel& v, DevCounters* __restrict__ ctr,
                                         unsigned char* smem, VoxShared& S, uint32_t it, uint32_t r_unit,
                                         uint32_t p_unit, bool first, uint32_t* next_item, bool split_unit = false) {
  uint2* const W = reinterpret_cast<uint2*>(smem);    // {word, rank} per 32 cells
  uint4* const W4 = reinterpret_cast<uint4*>(smem);   // two of them
  // The item's header, read by warp 0 in two dependent steps: lane 0 reads
  // the child node; then lane 8 reads the parent node while lanes 0..7 read
  // the children's records (inner items), all at once.
  if (threadIdx.x < 32) {
    const uint32_t ln = threadIdx.x;
    if (ln == 0) {
      const uint32_t t = find_tile(v.item_prefix, a.n_tiles, it);
      const uint32_t* ls = v.lvl_start + (uint64_t)t * (kMaxLevels + 1);
      const TileDesc& td = a.tiles[t];
      const uint64_t g = td.node_base + ls[v.level + 1] + (it - v.item_prefix[t]);
      const lod_node_t c = v.nodes[g];
      S.I.tile = t;
      S.I.g = g;
      S.cmin[0] = c.min[0];
      S.cmin[1] = c.min[1];
      S.cmin[2] = c.min[2];
      S.I.leaf = (c.flags & LOD_NODE_LEAF) != 0;
      S.I.n = S.I.leaf ? c.point_count : c.voxel_count;
      S.I.npts = c.point_count;
      S.cparent = td.node_base + c.parent;
      S.cfirst = td.node_base + c.first_child;
      S.pbase = td.pt_base + c.point_offset;
      S.nch = S.I.leaf ? 0u : (uint32_t)__popc(c.child_mask);
      S.samples = 0;
    }
    __syncwarp();
    const uint32_t nch = S.nch;
    if (S.I.leaf) {
      // the leaf's points (32-byte records where indices are kept), in
      // 64 KB pieces, one per lane
      const bool wsrc = a.wide != nullptr;
      const char* base = wsrc ? (const char*)(a.wide + 2 * S.pbase) : (const char*)(a.out + S.pbase);
      const uint64_t bytes = umin64(S.I.n * (wsrc ? 32u : 16u), kPrefetchBytes);
      const uint64_t off = (uint64_t)ln << 16;
      if (off < bytes) prefetch_l2(base + off, (uint32_t)umin64(bytes - off, 1u << 16));
    }
    if (ln == 8) {
      const lod_node_t p = v.nodes[S.cparent];
      S.I.Lp = p.log2_size;
      S.I.pmin[0] = p.min[0];
      S.I.pmin[1] = p.min[1];
      S.I.pmin[2] = p.min[2];
      S.I.kx = S.cmin[0] != p.min[0];
      S.I.ky = S.cmin[1] != p.min[1];
      S.I.kz = S.cmin[2] != p.min[2];
    }
    // the children's staged records, one flat sample sequence
    uint32_t occ = 0;
    if (ln < nch) {
      const NodeAux ca = v.aux[S.cfirst + ln];
      S.cstage[ln] = ca.stage;
      S.cdense[ln] = ca.dense;
      occ = ca.occ;
      if (occ) prefetch_l2(v.stage_in + ca.stage, (uint32_t)umin64((uint64_t)occ * 16u, 1u << 16));
    }
    if (ln < 8) {
      uint32_t incl = occ;  // prefix over lanes 0..7
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFu, incl, o);
        if ((int)ln >= o) incl += y;
      }
      if (ln == 0) S.cpre[0] = 0;
      S.cpre[ln + 1] = incl;
    }
  }
  for (uint32_t i = threadIdx.x; i < kWords / 2u; i += blockDim.x) W4[i] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  const ItemInfo& I = S.I;
  const TileDesc& td = a.tiles[I.tile];
  const lod_node_t& c = v.nodes[I.g];
  constexpr bool PICKLIKE = MODE != LOD_FILTER;  // one sample kept per cell
  // the narrowest sums that provably cannot overflow for the points of this cube
  const bool small = MODE == LOD_FILTER && I.npts <= kSmallMaxSamples;
  const bool narrow = MODE == LOD_FILTER && !small && I.npts <= kNarrowMaxSamples;
  const bool wide = MODE == LOD_FILTER && !small && !narrow;
  const uint32_t cap = PICKLIKE ? kCapPick : (small ? kCapSmall : (narrow ? kCapNarrow : kCapWide));
  const uint32_t C = (v.range_cells && v.range_cells < cap) ? v.range_cells : cap;  // ranks per pass
  // dense entries, one array per field (64-bit arrays first), then the cell of each rank
  unsigned char* const dn = smem + kDenseOff;
  unsigned long long* const A0 = reinterpret_cast<unsigned long long*>(dn);
  ulonglong2* const E = reinterpret_cast<ulonglong2*>(dn);
  unsigned long long* A1 = nullptr;
  unsigned long long* A2 = nullptr;
  uint32_t* B32 = nullptr;
  uint32_t* cnt = nullptr;
  uint32_t* K;
  if (PICKLIKE) {
    cnt = reinterpret_cast<uint32_t*>(E + kCapPick);
    K = cnt + kCapPick;
  } else if (small) {
    B32 = reinterpret_cast<uint32_t*>(A0 + kCapSmall);
    K = B32 + kCapSmall;
  } else if (narrow) {
    A1 = A0 + kCapNarrow;
    K = reinterpret_cast<uint32_t*>(A1 + kCapNarrow);
  } else {
    A1 = A0 + kCapWide;
    A2 = A1 + kCapWide;
    cnt = reinterpret_cast<uint32_t*>(A2 + kCapWide);
    K = cnt + kCapWide;
  }

  const uint64_t pbase = td.pt_base + c.point_offset;
  const int4* pts = a.out + pbase;
  const uint32_t* pidx = PICKLIKE ? a.out_idx + pbase : nullptr;
  // with kept indices the leaf is read from the 32-byte staging records and
  // published to the point / index arrays here, contiguously
  const int4* wsrc = a.wide ? a.wide + 2 * pbase : nullptr;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint32_t level = td.level0 + v.level;
  const bool lead = r_unit == 0;  // the one CTA of the item that publishes
  uint32_t seen = 0;              // samples this thread read (statistics)
  uint32_t passes = 1;
  // the next item's counter value; its latency hides behind the mark pass
  uint32_t next_k = 0;
  if (next_item && threadIdx.x == 0) next_k = atomicAdd(&ctr->item_head, 1u);

  // ---- pass 1: mark the occupied cells
  if (I.leaf) {
    const uint64_t n = I.n;
    const bool publish = wsrc != nullptr && lead;  // idempotent: a retried build writes the same values
    for (uint64_t base = 0; base < n; base += 4ull * blockDim.x) {
      int4 q[4];
      uint32_t x[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint64_t i = base + threadIdx.x + (uint64_t)k * blockDim.x;
        x[k] = 0u;
        q[k] = make_int4(0, 0, 0, 0);
        if (i < n) {
          if (wsrc) ld_wide_keep(wsrc + 2 * i, q[k], x[k]);
          else q[k] = __ldcg(pts + i);
        }
      }
      uint32_t cell[4];
      bool ok[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint64_t i = base + threadIdx.x + (uint64_t)k * blockDim.x;
        ok[k] = i < n;
        cell[k] = point_cell(q[k], I);
        if (ok[k]) {
          ++seen;
          if (publish) {
            a.out[pbase + i] = q[k];
            a.out_idx[pbase + i] = x[k];
          }
        }
      }
      mark_cells4(W, cell, ok);
    }
  } else {
    const uint32_t total = S.cpre[S.nch];
    uint32_t ci = 0;  // child of this thread's current sample (samples only move forward)
    for (uint32_t f0 = 0; f0 < total; f0 += 4u * blockDim.x) {
      int4 vr[4];
      uint64_t dst[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t f = f0 + threadIdx.x + (uint32_t)k * blockDim.x;
        vr[k] = make_int4(0, 0, 0, 0);
        dst[k] = 0;
        if (f < total) {
          while (f >= S.cpre[ci + 1]) ++ci;
          vr[k] = __ldcg(v.stage_in + S.cstage[ci] + (f - S.cpre[ci]));
          dst[k] = S.cdense[ci] + (f - S.cpre[ci]);
        }
      }
      uint32_t cell[4];
      bool ok[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t f = f0 + threadIdx.x + (uint32_t)k * blockDim.x;
        ok[k] = f < total;
        cell[k] = voxel_cell((uint32_t)vr[k].x);
        if (ok[k]) {
          ++seen;
          // publish the child's voxel (idempotent); an array found too
          // small makes the build rerun with the exact size
          // (filtered: without the packed sums, pick_index none)
          if (lead && dst[k] < v.dense_cap)
            v.dense[dst[k]] = PICKLIKE ? vr[k] : make_int4(vr[k].x, vr[k].y, vr[k].z, (int)kNone);
        }
      }
      mark_cells4(W, cell, ok);
    }
  }
  __syncthreads();

  // ---- rank the occupied cells: exclusive scan of the words' counts.  Warp
  // w ranks words [256 w, 256 w + 256), read as pairs {word, rank, word,
  // rank} by coalesced 16-byte loads: lane l holds pairs l, l + 32, l + 64
  // and l + 96 of the warp's 128.
  uint32_t next_it = next_k;
  if (next_item && threadIdx.x == 0 && v.order && next_k < v.n_items) next_it = v.order[next_k];
  {
    const uint32_t wbase = warp * 128u;
    uint4 e[4];
    uint32_t pre[4], tot = 0;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      e[m] = W4[wbase + lane + 32u * (uint32_t)m];
      const uint32_t c = __popc(e[m].x) + __popc(e[m].z);
      uint32_t incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if ((int)lane >= o) incl += y;
      }
      pre[m] = tot + incl - c;
      tot += __shfl_sync(0xFFFFFFFFu, incl, 31);
    }
    if (lane == 0) S.wsum[warp] = tot;
    __syncthreads();
    if (warp == 0) {
      const uint32_t w = S.wsum[lane];
      uint32_t wi = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
        if ((int)lane >= o) wi += y;
      }
      S.wsum[lane] = wi - w;
      if (lane == 31) S.D = wi;
    }
    __syncthreads();
    const uint32_t base = S.wsum[warp];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      e[m].y = base + pre[m];
      e[m].w = e[m].y + __popc(e[m].x);
      W4[wbase + lane + 32u * (uint32_t)m] = e[m];
    }
  }
  // thread 0: the item's first staging record.  The reservation (or, for
  // a unit, the read of the first attempt's) is issued here and its value
  // first used before the first extraction, so its latency overlaps the
  // accumulate pass.
  unsigned long long stg = 0;
  if (threadIdx.x == 0) {
    const uint32_t D = S.D;
    if (first) {
      stg = atomicAdd(v.stage_used, (unsigned long long)D);
      v.aux[I.g].occ = D;
      S.r0 = 0;
      S.r1 = D;
      const uint32_t P = (D + C - 1) / C;
      if (P > 1) atomicAdd(&ctr->vox_retries, 1ull);
      uint32_t q0 = 0;
      if (P > 1 && v.units && P >= v.queue_ranges && reserve_units(&ctr->units, v.unit_cap, P - 1, &q0)) {
        for (uint32_t r = 1; r < P; ++r) v.units[q0 + r - 1] = make_uint4(it, r, P, 0u);
        S.r1 = D / P;
      }
    } else {
      stg = v.aux[I.g].stage;  // reserved by the first attempt, or by the up-front split
      S.r0 = (uint32_t)((uint64_t)D * r_unit / p_unit);
      S.r1 = (uint32_t)((uint64_t)D * (r_unit + 1) / p_unit);
      if (r_unit == 0) v.aux[I.g].occ = D;
    }
  }
  __syncthreads();
  const uint32_t r1 = S.r1;
  const bool merge = !PICKLIKE && !wide && !v.no_merge;

  // Filtered, 32-bit sums (merge): runs of consecutive lanes whose k-th
  // samples share a rank (points in scan order often do) add their sums
  // first, so that only the run's first lane updates the entry (at most 32
  // samples of 8-bit channels or the sums of one cell, which the layout
  // bounds).  The four samples of a thread are reduced side by side
  // (segmented suffix sums by doubling, only as many steps as the longest
  // run needs); a warp without runs pays four shuffles and four votes.
  // dt[k] is cleared for the lanes whose sums went to another lane.
  auto merge4 = [&](const uint32_t (&rk)[4], uint32_t (&vr)[4], uint32_t (&vg)[4], uint32_t (&vb)[4],
                    uint32_t (&vn)[4], bool (&dt)[4]) {
    unsigned dm[4];  // bit i: lane i + 1 continues lane i's run
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t nxt = __shfl_down_sync(0xFFFFFFFFu, rk[k], 1);
      dm[k] = __ballot_sync(0xFFFFFFFFu, lane < 31u && dt[k] && nxt == rk[k]);
    }
    uint32_t x = dm[0] | dm[1] | dm[2] | dm[3];
    if (!x) return;
    uint32_t longest = 0;  // longest run of set bits (an upper bound over the four masks)
    while (x) {
      x &= x >> 1;
      ++longest;
    }
    uint32_t end[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) end[k] = (uint32_t)__ffs(~dm[k] & (0xFFFFFFFFu << lane)) - 1u;  // last lane of the run
    for (uint32_t o = 1; o <= longest; o <<= 1) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (!dm[k]) continue;  // warp-uniform
        const uint32_t tr = __shfl_down_sync(0xFFFFFFFFu, vr[k], o), tg = __shfl_down_sync(0xFFFFFFFFu, vg[k], o);
        const uint32_t tb = __shfl_down_sync(0xFFFFFFFFu, vb[k], o), tn = __shfl_down_sync(0xFFFFFFFFu, vn[k], o);
        if (lane + o <= end[k]) {
          vr[k] += tr;
          vg[k] += tg;
          vb[k] += tb;
          vn[k] += tn;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) dt[k] = dt[k] && (lane == 0 || !((dm[k] >> (lane - 1)) & 1u));
  };

  // update the dense entry of rank rk with one sample (or a run's sums).
  // Single-sample modes: pre is the entry's key as read before (see pick_update).
  auto update = [&](uint32_t rk, uint32_t cell, uint64_t r, uint64_t g, uint64_t b, uint32_t n, uint32_t ix,
                    uint32_t rgba, uint64_t pre) {
    K[rk] = cell;
    if (PICKLIKE) {
      if (!pick_update(&E[rk], pick_key<MODE>(ix, level), (uint64_t)rgba | ((uint64_t)ix << 32), pre))
        atomicOr(&ctr->error, kErrInternal);
      atomicAdd(&cnt[rk], n);
    } else if (small) {
      atomicAdd(&A0[rk], r | (g << 24) | ((uint64_t)n << 48));
      atomicAdd(&B32[rk], (uint32_t)b);
    } else if (narrow) {
      atomicAdd(&A0[rk], r | (g << 32));
      atomicAdd(&A1[rk], b | ((uint64_t)n << 32));
    } else {
      atomicAdd(&A0[rk], r);
      atomicAdd(&A1[rk], g);
      atomicAdd(&A2[rk], b);
      atomicAdd(&cnt[rk], n);
    }
  };

  // ---- pass 2: accumulate the ranks [lo, lo + span), one pass per range
  // a leaf read from 32-byte staging records is published (points and
  // indices, 20 bytes) by the mark pass of its first attempt: later passes
  // read the published copy
  const bool from_wide = wsrc != nullptr && split_unit;
  for (uint32_t lo = S.r0; lo < r1; lo += C) {
    const uint32_t span = r1 - lo < C ? r1 - lo : C;
    const bool last = r1 - lo <= C;  // the item's last read: let it leave L2 first
    ++passes;
    if (I.leaf) {
      const uint64_t n = I.n;
      for (uint64_t base = 0; base < n; base += 4ull * blockDim.x) {
        int4 q[4];
        uint32_t x[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint64_t i = base + threadIdx.x + (uint64_t)k * blockDim.x;
          x[k] = 0u;
          q[k] = make_int4(0, 0, 0, 0);
          if (i < n) {
            if (from_wide) {
              if (last) ld_wide(wsrc + 2 * i, q[k], x[k]);
              else ld_wide_keep(wsrc + 2 * i, q[k], x[k]);
            } else {
              q[k] = last ? __ldcs(pts + i) : __ldcg(pts + i);
              if (PICKLIKE) x[k] = last ? __ldcs(pidx + i) : __ldcg(pidx + i);
            }
          }
        }
        uint32_t cell[4], rk[4];
        bool ok[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint64_t i = base + threadIdx.x + (uint64_t)k * blockDim.x;
          ok[k] = i < n;
          seen += ok[k] ? 1u : 0u;
          cell[k] = point_cell(q[k], I);
        }
        cell_ranks4(W, cell, ok, lo, span, rk);
        uint64_t pre[4];
        pre_keys4<PICKLIKE>(E, rk, pre);
        uint32_t vr[4], vg[4], vb[4], vn[4];
        bool dt[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint32_t rgba = (uint32_t)q[k].w;
          vr[k] = rgba & 255u;
          vg[k] = (rgba >> 8) & 255u;
          vb[k] = (rgba >> 16) & 255u;
          vn[k] = 1u;
          dt[k] = rk[k] != kNoRank;
        }
        if (merge) merge4(rk, vr, vg, vb, vn, dt);
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (dt[k]) update(rk[k], cell[k], vr[k], vg[k], vb[k], vn[k], x[k], (uint32_t)q[k].w, pre[k]);
      }
    } else {
      const uint32_t total = S.cpre[S.nch];
      uint32_t ci = 0;
      for (uint32_t f0 = 0; f0 < total; f0 += 4u * blockDim.x) {
        int4 vr[4];
        ulonglong2 sm[4];
        uint64_t src[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint32_t f = f0 + threadIdx.x + (uint32_t)k * blockDim.x;
          vr[k] = make_int4(0, 0, 0, 0);
          sm[k] = make_ulonglong2(0ull, 0ull);
          src[k] = 0;
          if (f < total) {
            while (f >= S.cpre[ci + 1]) ++ci;
            src[k] = S.cstage[ci] + (f - S.cpre[ci]);
            vr[k] = last ? __ldcs(v.stage_in + src[k]) : __ldcg(v.stage_in + src[k]);
          }
        }
        if (!PICKLIKE) {
          // exact sums: in the record (cells of fewer than 1024 points), else
          // in the sums array
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint32_t f = f0 + threadIdx.x + (uint32_t)k * blockDim.x;
            if (f >= total) continue;
            if ((uint32_t)vr[k].w != kNone) sm[k] = unpack_sums(vr[k]);
            else sm[k] = last ? __ldcs(v.stage_in_sum + src[k]) : __ldcg(v.stage_in_sum + src[k]);
          }
        }
        uint32_t cell[4], rk[4];
        bool ok[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint32_t f = f0 + threadIdx.x + (uint32_t)k * blockDim.x;
          ok[k] = f < total;
          seen += ok[k] ? 1u : 0u;
          cell[k] = voxel_cell((uint32_t)vr[k].x);
        }
        cell_ranks4(W, cell, ok, lo, span, rk);
        uint64_t pre[4];
        pre_keys4<PICKLIKE>(E, rk, pre);
        // a child's voxel: {cell, rgba, count, picked index} and packed exact sums
        bool dt[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) dt[k] = rk[k] != kNoRank;
        if (merge) {
          uint32_t mr[4], mg[4], mb[4], mn[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            mr[k] = (uint32_t)(sm[k].x & kMask40);
            mg[k] = (uint32_t)((sm[k].x >> 40) | ((sm[k].y & 0xFFFFull) << 24));
            mb[k] = (uint32_t)(sm[k].y >> 16);
            mn[k] = (uint32_t)vr[k].z;
          }
          merge4(rk, mr, mg, mb, mn, dt);
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (dt[k]) update(rk[k], cell[k], mr[k], mg[k], mb[k], mn[k], 0u, 0u, 0ull);
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint64_t sr = sm[k].x & kMask40, sg = (sm[k].x >> 40) | ((sm[k].y & 0xFFFFull) << 24),
                           sb = sm[k].y >> 16;
            if (dt[k]) update(rk[k], cell[k], sr, sg, sb, (uint32_t)vr[k].z, (uint32_t)vr[k].w, (uint32_t)vr[k].y, pre[k]);
          }
        }
      }
    }
    if (threadIdx.x == 0) S.stage = stg;
    __syncthreads();  // every update of the pass is done
    const unsigned long long stage = S.stage;

    // ---- extract: rank lo + i goes to staging record stage + lo + i (cell
    // order), and the entry is left empty for the next pass or item
    for (uint32_t i = threadIdx.x; i < span; i += blockDim.x) {
      const uint32_t cell = K[i];
      const uint64_t o = stage + lo + i;
      int4 rec;
      rec.x = (int)parent_cell(cell, I);
      ulonglong2 sums = make_ulonglong2(0ull, 0ull);
      bool packed = false;  // filtered: the sums travel in the record itself
      if (PICKLIKE) {
        const ulonglong2 e = E[i];
        const uint32_t c32 = cnt[i];
        E[i] = make_ulonglong2(~0ull, 0ull);
        cnt[i] = 0u;
        const uint32_t best = (uint32_t)(e.y >> 32);
        if (best >= td.idx_bound || pick_key<MODE>(best, level) != e.x) {
          atomicOr(&ctr->error, kErrInternal);  // cannot happen for a cell that received a sample
          continue;
        }
        rec.y = (int)(uint32_t)e.y;
        rec.z = (int)c32;
        rec.w = (int)best;
      } else {
        uint64_t sr, sg, sb, n;
        if (small) {
          const uint64_t a0 = A0[i];
          sr = a0 & 0xFFFFFFull;
          sg = (a0 >> 24) & 0xFFFFFFull;
          n = a0 >> 48;
          sb = B32[i];
          A0[i] = 0ull;
          B32[i] = 0u;
        } else if (narrow) {
          const uint64_t a0 = A0[i], a1 = A1[i];
          sr = a0 & 0xFFFFFFFFull;
          sg = a0 >> 32;
          sb = a1 & 0xFFFFFFFFull;
          n = a1 >> 32;
          A0[i] = 0ull;
          A1[i] = 0ull;
        } else {
          sr = A0[i];
          sg = A1[i];
          sb = A2[i];
          n = cnt[i];
          A0[i] = 0ull;
          A1[i] = 0ull;
          A2[i] = 0ull;
          cnt[i] = 0u;
        }
        K[i] = 0u;  // the next item's layout may put an accumulator here
        const uint32_t m = mean_rgba(sr, sg, sb, n);
        rec.y = (int)m;
        rec.z = (int)n;
        rec.w = (int)kNone;
        if (n < kPackMaxCount) {
          rec.w = (int)pack_remainders(sr, sg, sb, n, m);
          packed = true;
        } else {
          sums.x = sr | (sg << 40);
          sums.y = (sg >> 24) | (sb << 16);
        }
      }
      if (o < v.stage_cap) {  // else the reservation reported kErrStageCap
        v.stage_out[o] = rec;
        if (!PICKLIKE && !packed) v.stage_out_sum[o] = sums;
      }
    }
    __syncthreads();
  }
  seen = __reduce_add_sync(0xFFFFFFFFu, seen);
  if (lane == 0 && seen) atomicAdd(&S.samples, seen);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (first) {
      v.aux[I.g].stage = stg;
      if (stg + S.D > v.stage_cap) atomicOr(&ctr->error, kErrStageCap);
    }
    if (next_item) *next_item = next_it;  // read after this item's last barrier
    atomicAdd(&ctr->vox_passes, (unsigned long long)passes);
    atomicAdd(&ctr->vox_samples, (unsigned long long)S.samples);
    if (first) atomicMax(&ctr->vox_max_item, (unsigned long long)I.n);
  }
  __syncthreads();
}

// First attempt of every item, taken by persistent CTAs (one per SM: the
// bitmap and the dense entries fill the shared memory) in the level's item
// order.  While an item is marked, its CTA already takes the next one.
template <int MODE>
__global__ void __launch_bounds__(kBlock, 1) k_vox(BuildArgs a, VoxLevel v, DevCounters* __restrict__ ctr) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ VoxShared S;
  __shared__ uint32_t s_item;
  vox_clear_dense<MODE>(smem);
  if (threadIdx.x == 0) {
    const uint32_t k = atomicAdd(&ctr->item_head, 1u);
    s_item = (v.order && k < v.n_items) ? v.order[k] : k;
  }
  __syncthreads();
  for (;;) {
    const uint32_t it = s_item;  // every thread reads it before the item's first barrier
    if (it >= v.n_items) break;
    vox_item<MODE>(a, v, ctr, smem, S, it, 0u, 1u, true, &s_item);
  }
}

// Rank ranges of items with many occupied cells, taken from the queue by
// persistent CTAs (the queue is complete when this starts).
template <int MODE>
__global__ void __launch_bounds__(kBlock, 1) k_vox_units(BuildArgs a, VoxLevel v, DevCounters* __restrict__ ctr) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ VoxShared S;
  __shared__ uint32_t s_unit;
  const uint32_t n_units = min(ctr->units, v.unit_cap);
  vox_clear_dense<MODE>(smem);
  for (;;) {
    if (threadIdx.x == 0) s_unit = atomicAdd(&ctr->unit_head, 1u);
    __syncthreads();
    const uint32_t u = s_unit;
    __syncthreads();
    if (u >= n_units) break;
    const uint4 w = v.units[u];
    vox_item<MODE>(a, v, ctr, smem, S, w.x, w.y, w.z, false, nullptr, w.w != 0u);
  }
}

// Levels with few items (the top of the tree) would leave most SMs idle
// with one CTA per item: every item is split up front into 2^m rank ranges
// (its staging block reserved here, for as many cells as it can occupy)
// and the partition kernel spreads them over the SMs.
__global__ void k_vox_split(BuildArgs a, VoxLevel v, DevCounters* __restrict__ ctr, uint32_t m) {
  const uint32_t it = blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= v.n_items) return;
  const uint32_t t = find_tile(v.item_prefix, a.n_tiles, it);
  const uint32_t* ls = v.lvl_start + (uint64_t)t * (kMaxLevels + 1);
  const uint64_t g = a.tiles[t].node_base + ls[v.level + 1] + (it - v.item_prefix[t]);
  const lod_node_t& c = v.nodes[g];
  const uint64_t n = (c.flags & LOD_NODE_LEAF) ? c.point_count : c.voxel_count;
  const uint64_t bound = umin64(n, kOctCells);
  const unsigned long long base = atomicAdd(v.stage_used, (unsigned long long)bound);
  if (base + bound > v.stage_cap) atomicOr(&ctr->error, kErrStageCap);
  v.aux[g].stage = base;
  v.aux[g].occ = 0u;
  const uint32_t q = atomicAdd(&ctr->units, 1u << m);
  if (q + (1u << m) > v.unit_cap) {
    atomicOr(&ctr->error, kErrInternal);
    return;
  }
  for (uint32_t j = 0; j < (1u << m); ++j) v.units[q + j] = make_uint4(it, j, 1u << m, 1u);
}

template <int MODE>
static void vox_attrs() {
  cudaFuncSetAttribute(k_vox<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  cudaFuncSetAttribute(k_vox_units<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
}

// One-time kernel attributes of the voxel pass (called before any launch,
// and before a stream capture of the voxel levels); returns the SM count.
int vox_init() {
  static int sms = [] {
    vox_attrs<LOD_FILTER>();
    vox_attrs<LOD_PICK>();
    vox_attrs<LOD_FIRST>();
    vox_attrs<LOD_RANDOM>();
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
  }();
  return sms;
}

template <int MODE>
static cudaError_t launch_vox_mode(const BuildArgs& a, const VoxLevel& v, DevCounters* ctr, cudaStream_t st) {
  const int sms = vox_init();
  if (v.units && v.n_items * 4u <= (uint32_t)sms) {
    uint32_t m = 0;
    while (m < 3 && (v.n_items << (m + 1)) <= (uint32_t)sms) ++m;
    k_vox_split<<<(v.n_items + 127) / 128, 128, 0, st>>>(a, v, ctr, m);
    note_launch();
    k_vox_units<MODE><<<sms, kBlock, kSmemBytes, st>>>(a, v, ctr);
    note_launch();
    return cudaGetLastError();
  }
  k_vox<MODE><<<v.n_items < (uint32_t)sms ? v.n_items : (uint32_t)sms, kBlock, kSmemBytes, st>>>(a, v, ctr);
  note_launch();
  if (v.units) k_vox_units<MODE><<<sms, kBlock, kSmemBytes, st>>>(a, v, ctr);
  if (v.units) note_launch();
  return cudaGetLastError();
}

cudaError_t launch_vox(const BuildArgs& a, const VoxLevel& v, DevCounters* ctr, cudaStream_t st) {
  if (!v.n_items) return cudaSuccess;
  switch (a.mode) {
    case LOD_PICK: return launch_vox_mode<LOD_PICK>(a, v, ctr, st);
    case LOD_FIRST: return launch_vox_mode<LOD_FIRST>(a, v, ctr, st);
    case LOD_RANDOM: return launch_vox_mode<LOD_RANDOM>(a, v, ctr, st);
    default: return launch_vox_mode<LOD_FILTER>(a, v, ctr, st);
  }
}

// Assign every item its place in the level's contiguous voxel block
// (exclusive scan of the occupied counts in node order), then give every
// parent the range of its children's items.
__global__ void __launch_bounds__(kBlock) k_level_scan(BuildArgs a, VoxLevel v, const uint32_t* __restrict__ parent_prefix,
                                                       uint32_t n_parents,
                                                       unsigned long long* __restrict__ tile_voxels,
                                                       DevCounters* __restrict__ ctr) {
  __shared__ unsigned long long warp_sum[32];
  __shared__ unsigned long long s_carry;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // this level's voxels follow those of the levels below in the voxel array
  const uint64_t level_base = v.vstate[0];
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (uint32_t chunk = 0; chunk < v.n_items; chunk += blockDim.x) {
    const uint32_t it = chunk + threadIdx.x;
    uint64_t g = 0;
    unsigned long long x = 0;
    if (it < v.n_items) {
      const uint32_t t = find_tile(v.item_prefix, a.n_tiles, it);
      g = a.tiles[t].node_base + v.lvl_start[(uint64_t)t * (kMaxLevels + 1) + v.level + 1] + (it - v.item_prefix[t]);
      x = v.aux[g].occ;
    }
    unsigned long long incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if ((int)lane >= o) incl += y;
    }
    if (lane == 31) warp_sum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const uint32_t nw = blockDim.x >> 5;
      unsigned long long w = lane < nw ? warp_sum[lane] : 0ull;
      unsigned long long wi = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
        if ((int)lane >= o) wi += y;
      }
      if (lane < nw) warp_sum[lane] = wi - w;
    }
    __syncthreads();
    const unsigned long long excl = s_carry + warp_sum[warp] + incl - x;
    if (it < v.n_items) v.aux[g].dense = level_base + excl;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) s_carry = excl + x;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    ctr->level_voxels = s_carry;
    if (level_base + s_carry > v.dense_cap) v.vstate[1] = 1ull;
  }
  __syncthreads();
  for (uint32_t ip = threadIdx.x; ip < n_parents; ip += blockDim.x) {
    const uint32_t t = find_tile(parent_prefix, a.n_tiles, ip);
    const TileDesc& td = a.tiles[t];
    const uint64_t pg = td.node_base + v.lvl_start[(uint64_t)t * (kMaxLevels + 1) + v.level] + (ip - parent_prefix[t]);
    lod_node_t& p = v.nodes[pg];
    if (p.flags & LOD_NODE_LEAF) continue;
    const uint64_t f = td.node_base + p.first_child;
    const uint64_t l = f + __popc(p.child_mask) - 1;
    const uint64_t off = v.aux[f].dense;
    const uint64_t cnt = v.aux[l].dense + v.aux[l].occ - off;
    p.voxel_offset = off;
    p.voxel_count = (uint32_t)cnt;
    atomicAdd(&tile_voxels[t], (unsigned long long)cnt);
  }
  __syncthreads();  // every thread has read vstate[0]
  if (threadIdx.x == 0) v.vstate[0] = level_base + s_carry;
  if (!v.next_order) return;
  // The order in which the next level up takes its items (the nodes of this
  // level): classes of equal bit length of the sample count, largest first,
  // so that the big items start early and every SM ends the level on small
  // ones.  Order within a class is immaterial (results do not depend on it).
  __shared__ uint32_t cls[33];
  if (threadIdx.x < 33) cls[threadIdx.x] = 0;
  __syncthreads();
  auto samples_class = [&](uint32_t ip) -> uint32_t {
    const uint32_t t = find_tile(parent_prefix, a.n_tiles, ip);
    const TileDesc& td = a.tiles[t];
    const lod_node_t& p = v.nodes[td.node_base + v.lvl_start[(uint64_t)t * (kMaxLevels + 1) + v.level] +
                                  (ip - parent_prefix[t])];
    const uint32_t n = (p.flags & LOD_NODE_LEAF) ? p.point_count : p.voxel_count;
    return 32u - (uint32_t)__clz(n);  // 0 for n = 0
  };
  for (uint32_t ip = threadIdx.x; ip < n_parents; ip += blockDim.x) atomicAdd(&cls[samples_class(ip)], 1u);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int c = 32; c >= 0; --c) {
      const uint32_t k = cls[c];
      cls[c] = run;
      run += k;
    }
  }
  __syncthreads();
  for (uint32_t ip = threadIdx.x; ip < n_parents; ip += blockDim.x)
    v.next_order[atomicAdd(&cls[samples_class(ip)], 1u)] = ip;
}

cudaError_t launch_level_scan(const BuildArgs& a, const VoxLevel& v, const uint32_t* parent_prefix,
                              uint32_t n_parents, unsigned long long* tile_voxels, DevCounters* ctr,
                              cudaStream_t st) {
  k_level_scan<<<1, kBlock, 0, st>>>(a, v, parent_prefix, n_parents, tile_voxels, ctr);
  note_launch();
  return cudaGetLastError();
}

// Publish the staged voxels of the items of the topmost processed level
// (their parents, the roots, have no parent pass that would copy them).
__global__ void __launch_bounds__(256) k_copy_items(BuildArgs a, VoxLevel v) {
  const uint32_t it = blockIdx.x;
  const uint32_t t = find_tile(v.item_prefix, a.n_tiles, it);
  const uint64_t g = a.tiles[t].node_base + v.lvl_start[(uint64_t)t * (kMaxLevels + 1) + v.level + 1] +
                     (it - v.item_prefix[t]);
  const NodeAux ca = v.aux[g];
  if (ca.dense + ca.occ > v.dense_cap) return;  // the build is redone with a larger array
  const bool filt = a.mode == LOD_FILTER;  // records may carry their sums packed
  for (uint32_t i = threadIdx.x; i < ca.occ; i += blockDim.x) {
    int4 rec = v.stage_out[ca.stage + i];
    const bool packed = filt && (uint32_t)rec.w != kNone;
    if (v.root_sums) v.root_sums[ca.dense + i] = packed ? unpack_sums(rec) : v.stage_out_sum[ca.stage + i];
    if (filt) rec.w = (int)kNone;
    v.dense[ca.dense + i] = rec;
  }
}

cudaError_t launch_copy_items(const BuildArgs& a, const VoxLevel& v, cudaStream_t st) {
  if (!v.n_items) return cudaSuccess;
  k_copy_items<<<v.n_items, 256, 0, st>>>(a, v);
  note_launch();
  return cudaGetLastError();
}

// Publish the leaf points and indices of tiles whose root is a leaf (no
// voxel pass reads those points): blockIdx.y selects the tile.
__global__ void __launch_bounds__(256) k_unwide(BuildArgs a, const uint32_t* __restrict__ tiles) {
  const TileDesc& td = a.tiles[tiles[blockIdx.y]];
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < td.n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t p = td.pt_base + i;
    int4 q;
    uint32_t x;
    ld_wide(a.wide + 2 * p, q, x);
    a.out[p] = q;
    a.out_idx[p] = x;
  }
}

cudaError_t launch_unwide(const BuildArgs& a, const uint32_t* tiles, uint32_t n_tiles, uint32_t max_points,
                          cudaStream_t st) {
  if (!n_tiles) return cudaSuccess;
  const uint32_t gx = (uint32_t)umin64(((uint64_t)max_points + 255) / 256, 1024);
  for (uint32_t t0 = 0; t0 < n_tiles; t0 += 65535) {
    const uint32_t m = n_tiles - t0 < 65535 ? n_tiles - t0 : 65535;
    k_unwide<<<dim3(gx ? gx : 1, m), 256, 0, st>>>(a, tiles + t0);
    note_launch();
  }
  return cudaGetLastError();
}

// Full-precision variant (Section 7): the input point each voxel of a
// single-sample mode picked, gathered from the caller's input into an
// array parallel to the voxel array.  blockIdx.y selects the tile.
__global__ void __launch_bounds__(256) k_voxel_points(const TileDesc* __restrict__ tiles,
                                                      const lod_node_t* __restrict__ nodes,
                                                      const uint32_t* __restrict__ n_nodes,
                                                      const int4* __restrict__ dense, int4* __restrict__ out) {
  const TileDesc& td = tiles[blockIdx.y];
  const uint32_t nn = n_nodes[blockIdx.y];
  for (uint32_t i = blockIdx.x; i < nn; i += gridDim.x) {
    const lod_node_t& nd = nodes[td.node_base + i];
    for (uint32_t j = threadIdx.x; j < nd.voxel_count; j += blockDim.x) {
      const uint32_t pick = (uint32_t)dense[nd.voxel_offset + j].w;
      out[nd.voxel_offset + j] = pick < td.n ? td.in[pick] : make_int4(0, 0, 0, 0);
    }
  }
}

cudaError_t launch_voxel_points(const TileDesc* tiles, uint32_t n_tiles, const lod_node_t* nodes,
                                const uint32_t* n_nodes, uint32_t max_nodes, const int4* dense, int4* out,
                                cudaStream_t st) {
  if (!n_tiles || !max_nodes) return cudaSuccess;
  const uint32_t gx = max_nodes < 4096 ? max_nodes : 4096;
  for (uint32_t t0 = 0; t0 < n_tiles; t0 += 65535) {
    const uint32_t m = n_tiles - t0 < 65535 ? n_tiles - t0 : 65535;
    k_voxel_points<<<dim3(gx, m), 256, 0, st>>>(tiles + t0, nodes, n_nodes + t0, dense, out);
    note_launch();
  }
  return cudaGetLastError();
}

// Gather each node's voxels to a new offset (compact per-result copies).
__global__ void __launch_bounds__(256) k_gather_voxels(const lod_node_t* __restrict__ nodes,
                                                       const uint64_t* __restrict__ new_off,
                                                       const int4* __restrict__ src, int4* __restrict__ dst) {
  const lod_node_t nd = nodes[blockIdx.x];
  const int4* s = src + nd.voxel_offset;
  int4* d = dst + new_off[blockIdx.x];
  for (uint32_t i = threadIdx.x; i < nd.voxel_count; i += blockDim.x) d[i] = s[i];
}

cudaError_t launch_gather_voxels(const lod_node_t* nodes, uint32_t n_nodes, const uint64_t* new_off,
                                 const int4* src, int4* dst, cudaStream_t st) {
  if (!n_nodes) return cudaSuccess;
  k_gather_voxels<<<n_nodes, 256, 0, st>>>(nodes, new_off, src, dst);
  note_launch();
  return cudaGetLastError();
}

}  // namespace lodk
