// Bottom-up voxel sampling (Section 4.2 of the paper).
//
// The paper processes one node per workgroup with one 128^3 grid per SM in
// global memory (8 MB / 33 MB per workgroup, Sections 4.2.2-4.2.3).  Here a
// CTA handles one (parent, child octant) pair: the child's samples (its
// leaf points, or the voxels the child itself received one level below)
// all fall into one 64^3 octant of the parent's 128^3 grid (the observation
// of Section 4.2), and their cells are accumulated in a 224 KB
// shared-memory open-addressing hash table instead of a dense grid.  An
// octant whose occupied cells exceed the table is processed in several
// hash-partitioned passes.  Colour sums are exact integers (32-bit lanes
// while they provably cannot overflow, 64-bit otherwise); the single-sample
// modes (minimal-hash pick, first come of Section 4.2.1, random with the
// key of Listing 1) keep, per cell, the entry {key, rgba | index << 32} of
// minimal key, updated by a 128-bit compare-and-swap, so the picked colour
// travels with the winning key and is never gathered from the input.
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
constexpr uint32_t kHn = kSmemBytes / 20;  // filtered, 32-bit sums: key + 2 x u64
constexpr uint32_t kHw = kSmemBytes / 32;  // filtered, 64-bit sums: key + 3 x u64 + count
constexpr uint32_t kHp = kSmemBytes / 24;  // pick: key + {u64 hash, u64 payload} + count
constexpr uint64_t kNarrowMaxSamples = 0xFFFFFFFFull / 255;  // 32-bit channel sums cannot overflow
constexpr uint64_t kMask40 = (1ull << 40) - 1;

constexpr uint32_t kProbe = 48;       // longest probe sequence before the table counts as full
constexpr uint32_t kProbeSpill = 8;   // ... in passes that spill: cells that find no slot this close to
                                      // home go to the spill list, so the table stays at a load where
                                      // every lookup is short

// Cells one table pass can be expected to hold (linear probing stays short
// up to about three quarters full); sizes the partitioning after an overflow.
__device__ __forceinline__ uint32_t table_capacity(uint32_t H) { return H / 4 * 3; }

__device__ __forceinline__ uint32_t part_of(uint32_t key1, uint32_t mlog) {
  return mlog ? (key1 * 0x85EBCA6Bu) >> (32 - mlog) : 0u;
}

__device__ __forceinline__ uint32_t home_slot(uint32_t key1, uint32_t H) { return __umulhi(key1 * 0x9E3779B1u, H); }

// Keep the sample of smaller hash in a pick entry {hash, rgba | index << 32}
// (hashes of distinct indices differ: splitmix64 is a bijection).  Most
// samples lose against the value read first and never write; an improvement
// is installed with a 128-bit compare-and-swap, retried while others lower
// the entry meanwhile (each retry sees a strictly smaller hash, so the loop
// ends; the bound only guards against a broken invariant).
__device__ __forceinline__ bool pick_update(ulonglong2* e, uint64_t h, uint64_t pay) {
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

// Linear probing from `slot`, whose content was observed as k: the slot of
// key1 (= local cell + 1), inserting it if absent.  Returns -1 when kProbe
// consecutive slots hold other cells: the table is too full and the item
// is redone in more partitions.  No shared fill counter is updated, so
// inserts of different warps never serialise on one address.
__device__ __forceinline__ int resolve_slot(uint32_t* keys, uint32_t H, uint32_t key1, uint32_t slot, uint32_t k,
                                            uint32_t limit = kProbe) {
  for (uint32_t probe = 0; probe < limit; ++probe) {
    if (k == key1) return (int)slot;
    if (k == 0u) {
      const uint32_t old = atomicCAS(&keys[slot], 0u, key1);
      if (old == 0u || old == key1) return (int)slot;
    }
    slot = (slot + 1 == H) ? 0u : slot + 1;
    k = ((volatile uint32_t*)keys)[slot];
  }
  return -1;
}

__device__ __forceinline__ int find_or_insert(uint32_t* keys, uint32_t H, uint32_t key1, uint32_t limit = kProbe) {
  const uint32_t slot = home_slot(key1, H);
  return resolve_slot(keys, H, key1, slot, ((volatile uint32_t*)keys)[slot], limit);
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

__device__ __forceinline__ uint32_t point_key1(const int4& q, const ItemInfo& I) {
  const uint32_t qx = grid_coord((uint32_t)q.x - (uint32_t)I.pmin[0], I.Lp) & 63u;
  const uint32_t qy = grid_coord((uint32_t)q.y - (uint32_t)I.pmin[1], I.Lp) & 63u;
  const uint32_t qz = grid_coord((uint32_t)q.z - (uint32_t)I.pmin[2], I.Lp) & 63u;
  return (qx | (qy << 6) | (qz << 12)) + 1u;
}

__device__ __forceinline__ uint32_t voxel_key1(uint32_t cell) {
  const uint32_t x = (cell & 127u) >> 1, y = ((cell >> 7) & 127u) >> 1, z = (cell >> 14) >> 1;
  return (x | (y << 6) | (z << 12)) + 1u;
}

__device__ __forceinline__ uint32_t key_to_cell(uint32_t key1, const ItemInfo& I) {
  const uint32_t l = key1 - 1u;
  return ((I.kx << 6) | (l & 63u)) | (((I.ky << 6) | ((l >> 6) & 63u)) << 7) |
         (((I.kz << 6) | (l >> 12)) << 14);
}

}  // namespace

int vox_smem_bytes() { return kSmemBytes; }

// Shared state of one voxel CTA.
struct VoxShared {
  uint32_t used, out, fail, sp, seen, queued;
  uint32_t clean;  // the table holds no entry (set by a complete extraction)
  uint32_t spill_n[2];  // records in the CTA's two spill lists
  uint32_t spill_in;    // records the current spill pass reads
  uint32_t spilling;    // the item spilled: its staging block is reserved whole
  unsigned long long base;  // first staging record of the current pass's output
  ItemInfo I;
  uint2 stack[48];          // pending {partition, log2 partitions} of the item
};

constexpr uint32_t kMaxQueuedLog = 6;  // an overflowing item is queued as at most 64 units
constexpr uint32_t kSpillMark = 0xFFu;  // stack entry {list, kSpillMark}: a pass over a spill list
constexpr uint32_t kMaxPartLog = 16;   // deeper partitions cannot overflow (a few cells each)

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

// Voxelize one item (a child node c of an inner node p at level v.level):
// its samples are hashed into the shared table, one pass per partition of
// its cells.  `first`: the item's first attempt, all cells in one pass; if
// the table overflows, the item is split into 2^m hash partitions that the
// partition kernel processes in parallel (or, when the queue is full, this
// CTA processes them itself).  A partition that still overflows is split in
// two, depth first, by the CTA that holds it.
template <int MODE>
__device__ __forceinline__ void vox_item(const BuildArgs& a, const VoxLevel& v, DevCounters* __restrict__ ctr,
                                         unsigned char* smem, VoxShared& S, uint32_t it, uint32_t p_first,
                                         uint32_t m_first, bool first) {
  if (threadIdx.x == 0) {
    const uint32_t t = find_tile(v.item_prefix, a.n_tiles, it);
    const uint32_t* ls = v.lvl_start + (uint64_t)t * (kMaxLevels + 1);
    const TileDesc& td = a.tiles[t];
    const uint64_t g = td.node_base + ls[v.level + 1] + (it - v.item_prefix[t]);
    const lod_node_t c = v.nodes[g];
    const lod_node_t p = v.nodes[td.node_base + c.parent];
    S.I.tile = t;
    S.I.g = g;
    S.I.Lp = p.log2_size;
    S.I.pmin[0] = p.min[0];
    S.I.pmin[1] = p.min[1];
    S.I.pmin[2] = p.min[2];
    S.I.kx = c.min[0] != p.min[0];
    S.I.ky = c.min[1] != p.min[1];
    S.I.kz = c.min[2] != p.min[2];
    S.I.leaf = (c.flags & LOD_NODE_LEAF) != 0;
    S.I.n = S.I.leaf ? c.point_count : c.voxel_count;
    S.I.npts = c.point_count;
    S.stack[0] = make_uint2(p_first, m_first);
    S.sp = 1;
    S.queued = 0;
    S.spilling = 0;
    S.spill_n[0] = S.spill_n[1] = 0;
  }
  __syncthreads();
  const ItemInfo& I = S.I;
  const TileDesc& td = a.tiles[I.tile];
  const lod_node_t& c = v.nodes[I.g];
  constexpr bool PICKLIKE = MODE != LOD_FILTER;  // one sample kept per cell
  // 32-bit channel sums cannot overflow when the cube holds few enough points
  const bool narrow = MODE == LOD_FILTER && I.npts <= kNarrowMaxSamples;
  const uint32_t H = PICKLIKE ? kHp : (narrow ? kHn : kHw);
  // shared-memory carve-up (u64 arrays first)
  unsigned long long* A0 = reinterpret_cast<unsigned long long*>(smem);
  unsigned long long* A1 = A0 + H;
  unsigned long long* A2 = A1 + H;  // wide only
  ulonglong2* E = reinterpret_cast<ulonglong2*>(smem);  // pick entries
  uint32_t* keys;
  uint32_t* cnt32;
  if (PICKLIKE) {
    keys = reinterpret_cast<uint32_t*>(E + H);
    cnt32 = keys + H;
  } else if (narrow) {
    keys = reinterpret_cast<uint32_t*>(A0 + 2 * H);
    cnt32 = nullptr;
  } else {
    keys = reinterpret_cast<uint32_t*>(A0 + 3 * H);
    cnt32 = keys + H;
  }

  const uint64_t bound = umin64(I.n, kOctCells);  // cells the item can occupy
  const uint64_t pbase = td.pt_base + c.point_offset;
  const int4* pts = a.out + pbase;
  const uint32_t* pidx = PICKLIKE ? a.out_idx + pbase : nullptr;
  // with kept indices the leaf is read from the 32-byte staging records and
  // published to the point / index arrays here, contiguously
  const int4* wsrc = a.wide ? a.wide + 2 * pbase : nullptr;
  const uint32_t nch = __popc(c.child_mask);
  const uint64_t fc = td.node_base + (c.first_child == kNone ? 0 : c.first_child);
  const uint32_t lane = threadIdx.x & 31u;
  uint32_t passes = 0;
  bool split = false;

  for (;;) {
    __syncthreads();
    if (S.sp == 0) break;
    const uint2 pm = S.stack[S.sp - 1];
    const uint32_t part = pm.x, mlog = pm.y;
    // Spill lists: in the item's first pass and in the passes over its
    // spill lists, a sample whose cell finds no slot is appended (its cell
    // key and its position) to a list in global memory instead of failing
    // the pass; the cells in the table are then complete and are extracted,
    // and the list is processed by another pass over an empty table.  Only
    // a list that outgrows its space fails the item (which is then redone
    // in hash partitions).
    const bool spill_pass = mlog == kSpillMark;
    const bool can_spill = v.spill != nullptr && first && (spill_pass || mlog == 0);
    const uint32_t sp_out_id = spill_pass ? 1u - part : 0u;
    uint2* const sp_out = can_spill ? v.spill + ((uint64_t)blockIdx.x * 2 + sp_out_id) * v.spill_cap : nullptr;
    const uint2* const sp_in = spill_pass ? v.spill + ((uint64_t)blockIdx.x * 2 + part) * v.spill_cap : nullptr;
    const uint32_t probe_limit = can_spill ? kProbeSpill : kProbe;
    if (!S.clean) {
      // an empty entry is all zero bytes in filtered mode whatever the
      // table's layout, so a clean table serves every item
      if (PICKLIKE) {
        for (uint32_t i = threadIdx.x; i < H; i += blockDim.x) {
          keys[i] = 0u;
          E[i] = make_ulonglong2(~0ull, 0ull);
          cnt32[i] = 0u;
        }
      } else {
        uint4* z = reinterpret_cast<uint4*>(smem);
        for (uint32_t i = threadIdx.x; i < (uint32_t)kSmemBytes / 16u; i += blockDim.x) z[i] = make_uint4(0, 0, 0, 0);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      S.sp -= 1;
      S.used = 0;
      S.fail = 0;
      S.seen = 0;
      S.clean = 0;
      S.spill_in = spill_pass ? S.spill_n[part] : 0u;
      if (can_spill) S.spill_n[sp_out_id] = 0;
    }
    __syncthreads();
    ++passes;
    // append this lane's sample (cell key, position) to the output list when
    // `want`; warp-aggregated, called by every lane of the warp
    auto spill_warp = [&](bool want, uint32_t key1, uint32_t src) {
      const unsigned m = __ballot_sync(0xFFFFFFFFu, want);
      if (!m) return;
      const int leader = __ffs(m) - 1;
      uint32_t base = 0;
      if ((int)lane == leader) base = atomicAdd(&S.spill_n[sp_out_id], (uint32_t)__popc(m));
      base = __shfl_sync(0xFFFFFFFFu, base, leader);
      if (!want) return;
      const uint32_t pos = base + __popc(m & ((1u << lane) - 1u));
      if (pos < v.spill_cap) sp_out[pos] = make_uint2(key1, src);
      else S.fail = 1;
    };
    auto spill_one = [&](uint32_t key1, uint32_t src) {
      const uint32_t pos = atomicAdd(&S.spill_n[sp_out_id], 1u);
      if (pos < v.spill_cap) sp_out[pos] = make_uint2(key1, src);
      else S.fail = 1;
    };
    uint32_t seen = 0;  // samples this thread went through (for the overflow estimate)

    if (spill_pass) {
      // a spill list: every record names its cell and where its sample is
      for (uint32_t i = threadIdx.x; i < S.spill_in; i += blockDim.x) {
        const uint2 sr = sp_in[i];
        const uint32_t key1 = sr.x, src = sr.y;
        ++seen;
        const int slot = find_or_insert(keys, H, key1, probe_limit);
        if (slot < 0) {
          spill_one(key1, src);
          continue;
        }
        if (I.leaf) {
          int4 q;
          uint32_t ix = 0;
          if (wsrc) {
            ld_wide(wsrc + 2 * (uint64_t)src, q, ix);
          } else {
            q = pts[src];
            if (PICKLIKE) ix = pidx[src];
          }
          const uint32_t rgba = (uint32_t)q.w;
          if (PICKLIKE) {
            if (!pick_update(&E[slot], pick_key<MODE>(ix, td.level0 + v.level), (uint64_t)rgba | ((uint64_t)ix << 32)))
              atomicOr(&ctr->error, kErrInternal);
            atomicAdd(&cnt32[slot], 1u);
          } else if (narrow) {
            atomicAdd(&A0[slot], (uint64_t)(rgba & 255u) | ((uint64_t)((rgba >> 8) & 255u) << 32));
            atomicAdd(&A1[slot], (uint64_t)((rgba >> 16) & 255u) | (1ull << 32));
          } else {
            atomicAdd(&A0[slot], (uint64_t)(rgba & 255u));
            atomicAdd(&A1[slot], (uint64_t)((rgba >> 8) & 255u));
            atomicAdd(&A2[slot], (uint64_t)((rgba >> 16) & 255u));
            atomicAdd(&cnt32[slot], 1u);
          }
        } else {
          const int4 vr = v.stage_in[src];
          if (PICKLIKE) {
            const uint32_t idx = (uint32_t)vr.w;
            if (!pick_update(&E[slot], pick_key<MODE>(idx, td.level0 + v.level),
                             (uint64_t)(uint32_t)vr.y | ((uint64_t)idx << 32)))
              atomicOr(&ctr->error, kErrInternal);
            atomicAdd(&cnt32[slot], (uint32_t)vr.z);
          } else {
            const ulonglong2 sm = v.stage_in_sum[src];
            const uint64_t sr = sm.x & kMask40, sg = (sm.x >> 40) | ((sm.y & 0xFFFFull) << 24), sb = sm.y >> 16;
            if (narrow) {
              atomicAdd(&A0[slot], sr | (sg << 32));
              atomicAdd(&A1[slot], sb | ((uint64_t)(uint32_t)vr.z << 32));
            } else {
              atomicAdd(&A0[slot], sr);
              atomicAdd(&A1[slot], sg);
              atomicAdd(&A2[slot], sb);
              atomicAdd(&cnt32[slot], (uint32_t)vr.z);
            }
          }
        }
      }
    } else if (I.leaf) {
      const uint64_t n = I.n;
      const uint64_t step = 2ull * blockDim.x;
      // Lanes of a warp whose points share a cell are merged first (point
      // order follows the scan in real data, so whole warps often hit one
      // cell); one leader per distinct cell then probes and updates the
      // table.  All sums stay exact: at most 32 samples are merged.
      // merge(): lanes of a warp whose points share a cell add up their
      // colours; returns whether this lane carries the update (a leader, or
      // any lane with a sample in pick mode).
      auto merge = [&](uint32_t key1, const int4& q, uint32_t& r, uint32_t& g, uint32_t& b,
                       uint32_t& n_same, unsigned& peers) -> bool {
        const unsigned act = __ballot_sync(0xFFFFFFFFu, key1 != 0u);
        const uint32_t rgba = (uint32_t)q.w;
        r = rgba & 255u;
        g = (rgba >> 8) & 255u;
        b = (rgba >> 16) & 255u;
        n_same = 1;
        peers = 1u << lane;
        if (key1 == 0u) return false;
        // most pick updates lose the comparison against the entry they
        // read, so the single-sample modes skip the merge (and so does the
        // filtered mode when tuned to)
        if (PICKLIKE || v.no_merge) return true;
        peers = __match_any_sync(act, key1);
        n_same = __popc(peers);
        if (n_same > 1) {
          r = __reduce_add_sync(peers, r);
          g = __reduce_add_sync(peers, g);
          b = __reduce_add_sync(peers, b);
        }
        return (int)lane == __ffs(peers) - 1;
      };
      auto update = [&](int slot, uint32_t key1, const int4& q, uint32_t ix, uint32_t r, uint32_t g, uint32_t b,
                        uint32_t n_same) {
        if (slot < 0) {
          if (!can_spill) S.fail = 1;  // else every lane of the group spills its own sample
          return;
        }
        if (PICKLIKE) {
          if (!pick_update(&E[slot], pick_key<MODE>(ix, td.level0 + v.level),
                           (uint64_t)(uint32_t)q.w | ((uint64_t)ix << 32)))
            atomicOr(&ctr->error, kErrInternal);
          atomicAdd(&cnt32[slot], n_same);
        } else if (narrow) {
          atomicAdd(&A0[slot], (uint64_t)r | ((uint64_t)g << 32));
          atomicAdd(&A1[slot], (uint64_t)b | ((uint64_t)n_same << 32));
        } else {
          atomicAdd(&A0[slot], (uint64_t)r);
          atomicAdd(&A1[slot], (uint64_t)g);
          atomicAdd(&A2[slot], (uint64_t)b);
          atomicAdd(&cnt32[slot], n_same);
        }
      };
      // both samples of a pair are merged, then both home slots are read
      // before either probe is resolved, so their shared-memory latencies
      // overlap
      auto accumulate2 = [&](uint32_t k0, const int4& q0, uint32_t x0, uint32_t i0, uint32_t k1, const int4& q1,
                             uint32_t x1, uint32_t i1) {
        uint32_t r0, g0, b0, n0, r1, g1, b1, n1;
        unsigned p0, p1;
        const bool l0 = merge(k0, q0, r0, g0, b0, n0, p0);
        const bool l1 = merge(k1, q1, r1, g1, b1, n1, p1);
        uint32_t h0 = 0, h1 = 0, e0 = 0, e1 = 0;
        if (l0) {
          h0 = home_slot(k0, H);
          e0 = ((volatile uint32_t*)keys)[h0];
        }
        if (l1) {
          h1 = home_slot(k1, H);
          e1 = ((volatile uint32_t*)keys)[h1];
        }
        int s0 = 0, s1 = 0;
        if (l0) update(s0 = resolve_slot(keys, H, k0, h0, e0, probe_limit), k0, q0, x0, r0, g0, b0, n0);
        if (l1) update(s1 = resolve_slot(keys, H, k1, h1, e1, probe_limit), k1, q1, x1, r1, g1, b1, n1);
        // a group whose leader found no slot spills all its samples (one
        // vote when no lane of the warp failed)
        if (can_spill && __any_sync(0xFFFFFFFFu, (l0 && s0 < 0) || (l1 && s1 < 0))) {
          const unsigned f0 = __ballot_sync(0xFFFFFFFFu, l0 && s0 < 0);
          const unsigned f1 = __ballot_sync(0xFFFFFFFFu, l1 && s1 < 0);
          spill_warp(k0 != 0u && ((f0 >> (__ffs(p0) - 1)) & 1u), k0, i0);
          spill_warp(k1 != 0u && ((f1 >> (__ffs(p1) - 1)) & 1u), k1, i1);
        }
      };
      // Software pipeline over pairs of points: the loads of the next pair
      // are in flight while the current pair is hashed and accumulated.
      auto load = [&](uint64_t i, int4& q, uint32_t& x) {
        if (wsrc) {
          ld_wide(wsrc + 2 * i, q, x);
        } else {
          q = __ldcs(pts + i);
          if (PICKLIKE) x = __ldcs(pidx + i);
        }
      };
      const bool publish = wsrc != nullptr && part == 0;
      int4 q0 = make_int4(0, 0, 0, 0), q1 = q0;
      uint32_t x0 = 0, x1 = 0;
      {
        const uint64_t a0 = threadIdx.x, a1 = a0 + blockDim.x;
        if (a0 < n) load(a0, q0, x0);
        if (a1 < n) load(a1, q1, x1);
      }
      for (uint64_t base = 0; base < n; base += step) {
        const uint64_t a0 = base + threadIdx.x, a1 = a0 + blockDim.x;
        const uint64_t b0 = a0 + step, b1 = a1 + step;
        int4 r0 = q0, r1 = q1;
        uint32_t y0 = 0, y1 = 0;
        if (b0 < n) load(b0, r0, y0);
        if (b1 < n) load(b1, r1, y1);
        // the whole warp leaves together: accumulate() uses full-warp
        // collectives, so no lane may stop while its neighbours go on
        if (__any_sync(0xFFFFFFFFu, *((volatile uint32_t*)&S.fail) != 0u)) break;
        if (publish) {  // idempotent: a retried item writes the same values
          if (a0 < n) {
            a.out[pbase + a0] = q0;
            a.out_idx[pbase + a0] = x0;
          }
          if (a1 < n) {
            a.out[pbase + a1] = q1;
            a.out_idx[pbase + a1] = x1;
          }
        }
        uint32_t k0 = 0u, k1 = 0u;
        if (a0 < n) {
          ++seen;
          k0 = point_key1(q0, I);
          if (part_of(k0, mlog) != part) k0 = 0u;
        }
        if (a1 < n) {
          ++seen;
          k1 = point_key1(q1, I);
          if (part_of(k1, mlog) != part) k1 = 0u;
        }
        accumulate2(k0, q0, x0, (uint32_t)a0, k1, q1, x1, (uint32_t)a1);
        q0 = r0;
        q1 = r1;
        x0 = y0;
        x1 = y1;
      }
    } else {
      // inner child: its voxels are the staged records of its own children
      for (uint32_t r = 0; r < nch; ++r) {
        const NodeAux& ca = v.aux[fc + r];
        const int4* rec = v.stage_in + ca.stage;
        const ulonglong2* sums = (MODE == LOD_FILTER) ? v.stage_in_sum + ca.stage : nullptr;
        int4* dst = v.dense + ca.dense;
        const uint32_t m = ca.occ;
        const bool fits = ca.dense + m <= v.dense_cap;  // else the build is redone with a larger array
        for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) {
          if (*((volatile uint32_t*)&S.fail)) break;
          const int4 vr = rec[i];
          ++seen;
          if (part == 0 && fits) dst[i] = vr;  // publish the child's voxel (idempotent)
          const uint32_t key1 = voxel_key1((uint32_t)vr.x);
          if (part_of(key1, mlog) != part) continue;
          const int slot = find_or_insert(keys, H, key1, probe_limit);
          if (slot < 0) {
            if (can_spill) spill_one(key1, (uint32_t)(ca.stage + i));
            else S.fail = 1;
            continue;
          }
          if (PICKLIKE) {
            const uint32_t idx = (uint32_t)vr.w;
            if (!pick_update(&E[slot], pick_key<MODE>(idx, td.level0 + v.level),
                             (uint64_t)(uint32_t)vr.y | ((uint64_t)idx << 32)))
              atomicOr(&ctr->error, kErrInternal);
            atomicAdd(&cnt32[slot], (uint32_t)vr.z);
          } else {
            const ulonglong2 sm = sums[i];
            const uint64_t sr = sm.x & kMask40, sg = (sm.x >> 40) | ((sm.y & 0xFFFFull) << 24), sb = sm.y >> 16;
            if (narrow) {
              atomicAdd(&A0[slot], sr | (sg << 32));
              atomicAdd(&A1[slot], sb | ((uint64_t)(uint32_t)vr.z << 32));
            } else {
              atomicAdd(&A0[slot], sr);
              atomicAdd(&A1[slot], sg);
              atomicAdd(&A2[slot], sb);
              atomicAdd(&cnt32[slot], (uint32_t)vr.z);
            }
          }
        }
      }
    }
    __syncthreads();  // every insert of the pass is done
    if (S.fail) {
      // occupied cells of this pass, and how far the pass got
      {
        uint32_t mine = 0;
        for (uint32_t i = threadIdx.x; i < H; i += blockDim.x) mine += keys[i] != 0u ? 1u : 0u;
        mine = __reduce_add_sync(0xFFFFFFFFu, mine);
        seen = __reduce_add_sync(0xFFFFFFFFu, seen);
        if (lane == 0) {
          if (mine) atomicAdd(&S.used, mine);
          if (seen) atomicAdd(&S.seen, seen);
        }
      }
      __syncthreads();
      const uint32_t used = S.used;
      split = true;
      if (threadIdx.x == 0) {
        if (spill_pass || S.spilling) atomicOr(&ctr->error, kErrInternal);  // spill lists only shrink
        bool handed = false;
        if (first && mlog == 0) {
          // the cells of the whole item get one staging block, filled by
          // the passes over its partitions in any order
          S.base = atomicAdd(v.stage_used, (unsigned long long)bound);
          if (S.base + bound > v.stage_cap) atomicOr(&ctr->error, kErrStageCap);
          v.aux[I.g].stage = S.base;
          v.aux[I.g].occ = 0u;
          if (v.units) {
            // occupied cells projected from the part seen so far
            const uint64_t sn = S.seen ? S.seen : 1u;
            const uint64_t est = umin64(bound, (uint64_t)used * I.n / sn + (uint64_t)used / 4 + 1);
            const uint64_t per = table_capacity(H);
            uint32_t m = 1;
            while (m < kMaxQueuedLog && (est >> m) > per) ++m;
            uint32_t q0 = 0;
            if (reserve_units(&ctr->units, v.unit_cap, 1u << m, &q0)) {
              for (uint32_t j = 0; j < (1u << m); ++j) v.units[q0 + j] = make_uint4(it, j, m, 0u);
              handed = true;
              S.queued = 1;
            }
          }
        }
        if (!handed) {
          if (mlog >= kMaxPartLog) {
            atomicOr(&ctr->error, kErrInternal);
          } else {  // split this partition in two, depth first
            S.stack[S.sp] = make_uint2(2 * part + 1, mlog + 1);
            S.stack[S.sp + 1] = make_uint2(2 * part, mlog + 1);
            S.sp += 2;
          }
        }
      }
      continue;
    }

    // extract this pass's occupied cells into the item's staging block: the
    // item's first pass reserves its whole block (at most min(samples,
    // 64^3) cells, what the level's staging is sized for), and every warp
    // appends its cells through the item's counter
    if (threadIdx.x == 0) {
      const bool spilled = can_spill && S.spill_n[sp_out_id] > 0;
      if (first && mlog == 0) {
        const unsigned long long blk = atomicAdd(v.stage_used, (unsigned long long)bound);
        if (blk + bound > v.stage_cap) atomicOr(&ctr->error, kErrStageCap);
        v.aux[I.g].stage = blk;
        v.aux[I.g].occ = 0u;
        if (spilled) S.spilling = 1;
      }
      S.base = v.aux[I.g].stage;
      if (spilled) {  // next: a pass over the samples this one spilled
        S.stack[S.sp] = make_uint2(sp_out_id, kSpillMark);
        S.sp += 1;
      }
    }
    __syncthreads();
    {
      unsigned int* const occ_ctr = &v.aux[I.g].occ;
      const uint64_t base = S.base;
      // four slots per thread (16-byte key loads), a warp scan of their
      // occupied counts, one append per warp
      for (uint32_t q0 = 0; q0 < H; q0 += 4u * blockDim.x) {
        const uint32_t i = q0 + 4u * threadIdx.x;
        uint32_t kk[4];
        if (i + 3u < H) {
          const uint4 k4 = *reinterpret_cast<const uint4*>(keys + i);
          kk[0] = k4.x;
          kk[1] = k4.y;
          kk[2] = k4.z;
          kk[3] = k4.w;
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j) kk[j] = i + j < H ? keys[i + j] : 0u;
        }
        const uint32_t c = (kk[0] != 0u) + (kk[1] != 0u) + (kk[2] != 0u) + (kk[3] != 0u);
        uint32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
          if ((int)lane >= o) incl += t;
        }
        const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
        if (!total) continue;
        uint32_t wb = 0;
        if (lane == 31) wb = atomicAdd(occ_ctr, total);
        wb = __shfl_sync(0xFFFFFFFFu, wb, 31);
        const bool room = (uint64_t)wb + total <= bound && base + wb + total <= v.stage_cap;
        if (lane == 31 && !room) atomicOr(&ctr->error, kErrStageCap);
        uint32_t pos = wb + incl - c;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint32_t key1 = kk[j];
          if (!key1) continue;
          const uint32_t slot = i + j;
          const uint64_t o = base + pos++;
          // read the entry and leave it empty for the next pass or item
          keys[slot] = 0u;
          ulonglong2 e = make_ulonglong2(0ull, 0ull);
          uint32_t c32 = 0;
          uint64_t sr = 0, sg = 0, sb = 0, n = 0;
          if (PICKLIKE) {
            e = E[slot];
            c32 = cnt32[slot];
            E[slot] = make_ulonglong2(~0ull, 0ull);
            cnt32[slot] = 0u;
          } else if (narrow) {
            sr = A0[slot] & 0xFFFFFFFFull;
            sg = A0[slot] >> 32;
            sb = A1[slot] & 0xFFFFFFFFull;
            n = A1[slot] >> 32;
            A0[slot] = 0ull;
            A1[slot] = 0ull;
          } else {
            sr = A0[slot];
            sg = A1[slot];
            sb = A2[slot];
            n = cnt32[slot];
            A0[slot] = 0ull;
            A1[slot] = 0ull;
            A2[slot] = 0ull;
            cnt32[slot] = 0u;
          }
          if (!room) continue;
          const uint32_t cell = key_to_cell(key1, I);
          int4 rec;
          rec.x = (int)cell;
          if (PICKLIKE) {
            const uint32_t best = (uint32_t)(e.y >> 32);
            if (best >= td.idx_bound || pick_key<MODE>(best, td.level0 + v.level) != e.x) {
              atomicOr(&ctr->error, kErrInternal);  // cannot happen for a cell that received a sample
              continue;
            }
            rec.y = (int)(uint32_t)e.y;
            rec.z = (int)c32;
            rec.w = (int)best;
          } else {
            rec.y = (int)mean_rgba(sr, sg, sb, n);
            rec.z = (int)n;
            rec.w = (int)kNone;
            ulonglong2 sm;
            sm.x = sr | (sg << 40);
            sm.y = (sg >> 24) | (sb << 16);
            v.stage_out_sum[o] = sm;
          }
          v.stage_out[o] = rec;
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) S.clean = 1;
  }
  if (threadIdx.x == 0) {
    atomicAdd(&ctr->vox_passes, (unsigned long long)passes);
    if (split && first) atomicAdd(&ctr->vox_retries, 1ull);
  }
  __syncthreads();
}

// First attempt of every item, taken in order by persistent CTAs (one per
// SM: the table fills the shared memory).  A table left empty by the last
// extraction is not cleared again.
template <int MODE>
__global__ void __launch_bounds__(kBlock, 1) k_vox(BuildArgs a, VoxLevel v, DevCounters* __restrict__ ctr) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ VoxShared S;
  __shared__ uint32_t s_item;
  if (threadIdx.x == 0) S.clean = 0;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(&ctr->item_head, 1u);
    __syncthreads();
    const uint32_t it = s_item;
    __syncthreads();
    if (it >= v.n_items) break;
    vox_item<MODE>(a, v, ctr, smem, S, it, 0u, 0u, true);
  }
}

// Partitions of the items that overflowed their first attempt, taken from
// the queue by persistent CTAs (the queue is complete when this starts).
template <int MODE>
__global__ void __launch_bounds__(kBlock, 1) k_vox_units(BuildArgs a, VoxLevel v, DevCounters* __restrict__ ctr) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ VoxShared S;
  __shared__ uint32_t s_unit;
  const uint32_t n_units = min(ctr->units, v.unit_cap);
  if (threadIdx.x == 0) S.clean = 0;
  for (;;) {
    if (threadIdx.x == 0) s_unit = atomicAdd(&ctr->unit_head, 1u);
    __syncthreads();
    const uint32_t u = s_unit;
    __syncthreads();
    if (u >= n_units) break;
    const uint4 w = v.units[u];
    vox_item<MODE>(a, v, ctr, smem, S, w.x, w.y, w.z, false);
  }
}

// Levels with few items (the top of the tree) would leave most SMs idle
// with one CTA per item: every item is split up front into 2^m hash
// partitions (its staging block reserved here) and the partition kernel
// spreads them over the SMs.
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
  for (uint32_t j = 0; j < (1u << m); ++j) v.units[q + j] = make_uint4(it, j, m, 0u);
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
  for (uint32_t i = threadIdx.x; i < ca.occ; i += blockDim.x) {
    v.dense[ca.dense + i] = v.stage_out[ca.stage + i];
    if (v.root_sums) v.root_sums[ca.dense + i] = v.stage_out_sum[ca.stage + i];
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
