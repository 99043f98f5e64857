// CPU oracle for the LOD construction — TEST INFRASTRUCTURE ONLY.
//
// Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may
// load this library.  The product path never links or calls it, and it
// shares no code, header, table or helper with the CUDA library.
//
// It is a plain, single-threaded restatement of what the method computes,
// written from the definitions with no blocking or fusion; the average and
// pick modes are computed top-down per node, without bottom-up merging:
//
//  * Root cube (Section 4 with the reading that the paper's float coordinates
//    become int32): the bounding box minimum is the cube's min corner and
//    its edge S is the smallest power of two strictly greater than the
//    largest per-axis extent.  N = 0 gives an empty root leaf at the origin.
//  * Split into leaves (Section 4.1): a node holding more than T points is
//    subdivided into its non-empty octants; a node with at most T points is
//    a leaf.  The fixed 8-level grid plus one 4-level extension of Section
//    4.1.5 becomes "recurse until it fits", capped by max_depth and by unit
//    cubes (such capped leaves may exceed T and are flagged overfull).
//    Merging 2x2x2 groups whose sum stays below T (Section 4.1.2) yields the
//    same tree apart from the T boundary, which follows "at most T points".
//  * Octant index k = (bx << 2) | (by << 1) | bz, b = the half a point falls
//    into along each axis; children are listed in ascending k.
//  * Node order: breadth first by level, within a level by the parent's
//    order and then ascending octant (ascending path key).
//  * Leaf point layout (Section 4.1.3 allocates each leaf's points; the
//    layout is free there): leaves are laid out depth first in octant
//    order, so every subtree owns one contiguous point range.
//  * Voxel sampling (Section 4.2): every inner node gets the occupied cells
//    of a 128^3 grid over its cube.  Cell-wise average (Section 4.2.3) with
//    exact u64 sums over all original points of the cube and a rounded-half-
//    up integer mean, alpha 255; sample pick (replacing the random pick of
//    Section 4.2.2, Listing 1) keeps the point of minimal splitmix64(index);
//    first come (Section 4.2.1; mode 3) keeps the first point of the cell in
//    input order.
//  * Random (Section 4.2.2 with the key of Listing 1; mode 4) also follows
//    the paper's bottom-up order: an inner node samples its children's
//    samples (points of leaf children, voxels of inner children), each with
//    a 32-bit key of 12 random bits above the low 20 bits of its index,
//    and every cell keeps the sample of largest key.  The random number of
//    a sample is drawn afresh for each node from a counter-based generator
//    (the high half of splitmix64(level << 32 | index)), and equal keys go
//    to the larger index.
//  * Neighbourhood-weighted average (Section 4.2.4; mode 2) follows the
//    paper's own order instead, since its result depends on it: inner nodes
//    deepest level first, each sampling its children's samples (the points
//    of leaf children, the voxels of inner children at their cell centres).
//    A sample adds weight max(0, 1 - distance to the cell centre, in cells)
//    times its colour to the cells of the 2x2x2 block around it and marks
//    the cell it lies in as occupied; an occupied cell's colour is its
//    weighted sum over its weight sum, rounded half up.  The paper fixes no
//    precision; the weights are taken in the kernel's (single precision,
//    rounded to multiples of 2^-24), since the rounding of the mean is an
//    integer decision both sides must take alike.
//
// Function-level citations are beside each function.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <utility>
#include <vector>

namespace {

struct OPoint {
  int32_t x, y, z;
  uint32_t rgba;
};

struct ONode {
  int32_t min[3] = {0, 0, 0};
  uint32_t level = 0;
  uint32_t log2_size = 0;
  uint32_t child_mask = 0;
  uint32_t flags = 0;  // bit0 leaf, bit1 overfull
  uint32_t parent = UINT32_MAX;
  uint32_t first_child = UINT32_MAX;
  uint64_t point_offset = 0;
  uint64_t point_count = 0;
  uint64_t voxel_offset = 0;
  uint32_t voxel_count = 0;
};

struct OVoxel {
  uint32_t cell, rgba, count, pick_index;
};

constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr uint32_t kModeWeighted = 2u;
constexpr uint32_t kModeFirst = 3u;
constexpr uint32_t kModeRandom = 4u;
constexpr uint32_t kLeaf = 1u;
constexpr uint32_t kOverfull = 2u;

// splitmix64: the first output of a splitmix64 generator whose state is x
// (Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
// OOPSLA 2014): advance the state by the golden-ratio increment, then two
// xor-shift-multiply rounds and a final xor-shift, all modulo 2^64.
uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Section 4.2.2, Listing 1: the 32-bit key of a sample with index i drawn
// while filling a node at `level`: the top 12 bits of a 32-bit random number
// above the low 20 bits of i.  The random number is the high half of
// splitmix64(level << 32 | i).  Returned with i appended below it, so that
// comparing the 64-bit values compares the keys and breaks ties by index.
uint64_t random_key(uint32_t i, uint32_t level) {
  const uint32_t r = (uint32_t)(splitmix64(((uint64_t)level << 32) | i) >> 32);
  const uint32_t key = (r & 0xFFF00000u) | (i & 0x000FFFFFu);
  return ((uint64_t)key << 32) | i;
}

// Offset of point p from the cube min c along one axis, as a non-negative
// 64-bit integer (the cube contains p, so 0 <= d < 2^log2_size <= 2^32).
inline int64_t rel(int32_t p, int32_t c) { return (int64_t)p - (int64_t)c; }

// 128^3 grid coordinate of an offset d inside a cube of edge 2^L
// (Section 4.2: samples are projected onto a 128^3 grid per node).
inline uint32_t grid_coord(int64_t d, uint32_t L) {
  if (L >= 7) return (uint32_t)(d >> (L - 7));
  return (uint32_t)(d << (7 - L));
}

struct Builder {
  const OPoint* pts;
  const uint32_t* input_index = nullptr;  // input index of pts[i] when pts is a subset, else i
  uint64_t n;
  uint32_t T, mode, max_depth;
  std::vector<ONode> nodes;
  std::vector<std::vector<uint32_t>> leaf_lists;  // per node id; only leaves
  std::vector<OVoxel> voxels;
  std::vector<OPoint> leaf_points;
  std::vector<uint32_t> leaf_index;

  uint32_t in_index(uint32_t i) const { return input_index ? input_index[i] : i; }

  // Section 4.2 + 4.2.3 / replacement of 4.2.2: the voxels of one inner node
  // computed directly from every original point inside its cube.
  void voxelize(ONode& nd, const std::vector<uint32_t>& idx) {
    std::vector<std::pair<uint32_t, uint32_t>> keyed;  // (cell, point index)
    keyed.reserve(idx.size());
    for (uint32_t i : idx) {
      const OPoint& p = pts[i];
      uint32_t qx = grid_coord(rel(p.x, nd.min[0]), nd.log2_size);
      uint32_t qy = grid_coord(rel(p.y, nd.min[1]), nd.log2_size);
      uint32_t qz = grid_coord(rel(p.z, nd.min[2]), nd.log2_size);
      keyed.emplace_back(qx | (qy << 7) | (qz << 14), i);
    }
    std::sort(keyed.begin(), keyed.end());
    nd.voxel_offset = voxels.size();
    size_t a = 0;
    while (a < keyed.size()) {
      size_t b = a;
      while (b < keyed.size() && keyed[b].first == keyed[a].first) ++b;
      OVoxel v;
      v.cell = keyed[a].first;
      v.count = (uint32_t)(b - a);
      if (mode == 0) {
        // Cell-wise average (Section 4.2.3): sum each channel over all
        // samples of the cell, then the arithmetic mean, rounded half up.
        uint64_t sr = 0, sg = 0, sb = 0;
        for (size_t j = a; j < b; ++j) {
          uint32_t c = pts[keyed[j].second].rgba;
          sr += c & 0xFFu;
          sg += (c >> 8) & 0xFFu;
          sb += (c >> 16) & 0xFFu;
        }
        uint64_t cnt = b - a;
        uint32_t r = (uint32_t)((sr + cnt / 2) / cnt);
        uint32_t g = (uint32_t)((sg + cnt / 2) / cnt);
        uint32_t bl = (uint32_t)((sb + cnt / 2) / cnt);
        v.rgba = r | (g << 8) | (bl << 16) | (255u << 24);
        v.pick_index = kNone;
      } else {
        // Sample pick: the one point of the cell whose splitmix64(index) is
        // smallest (splitmix64 is a bijection, so the minimum is unique).
        // First come (Section 4.2.1, mode 3): the first sample of the cell
        // in input order, i.e. the smallest input index; a child voxel
        // carries its own first point, so bottom up gives the same point.
        auto key = [&](uint32_t i) -> uint64_t { return mode == kModeFirst ? in_index(i) : splitmix64(in_index(i)); };
        uint32_t best = keyed[a].second;
        uint64_t best_h = key(best);
        for (size_t j = a + 1; j < b; ++j) {
          uint64_t h = key(keyed[j].second);
          if (h < best_h) {
            best_h = h;
            best = keyed[j].second;
          }
        }
        v.rgba = pts[best].rgba;
        v.pick_index = in_index(best);
      }
      voxels.push_back(v);
      a = b;
    }
    nd.voxel_count = (uint32_t)(voxels.size() - nd.voxel_offset);
  }

  // Section 4.2.2: one inner node's voxels under the random strategy, from
  // its children's samples (their voxels must exist already).  Each sample
  // falls into one cell of this node's grid; the cell keeps the sample of
  // largest random_key at this node's level and counts the original points.
  void voxelize_random(uint32_t id) {
    ONode& nd = nodes[id];
    struct RCell {
      uint64_t key = 0;
      uint32_t index = 0, rgba = 0;
      uint64_t count = 0;
    };
    std::map<uint32_t, RCell> cells;
    auto sample = [&](uint32_t cell, uint32_t index, uint32_t rgba, uint64_t count) {
      RCell& c = cells[cell];
      const uint64_t k = random_key(index, nd.level);
      if (c.count == 0 || k > c.key) {
        c.key = k;
        c.index = index;
        c.rgba = rgba;
      }
      c.count += count;
    };
    uint32_t c = nd.first_child;
    for (uint32_t k = 0; k < 8; ++k) {
      if (!(nd.child_mask & (1u << k))) continue;
      const ONode& ch = nodes[c];
      if (ch.flags & kLeaf) {
        for (uint32_t i : leaf_lists[c]) {
          const OPoint& p = pts[i];
          const uint32_t qx = grid_coord(rel(p.x, nd.min[0]), nd.log2_size);
          const uint32_t qy = grid_coord(rel(p.y, nd.min[1]), nd.log2_size);
          const uint32_t qz = grid_coord(rel(p.z, nd.min[2]), nd.log2_size);
          sample(qx | (qy << 7) | (qz << 14), in_index(i), p.rgba, 1);
        }
      } else {
        // a child cell q lies in the cell 64 b + q / 2 of this node (the
        // child is octant b, half the edge)
        const uint32_t b[3] = {(k >> 2) & 1u, (k >> 1) & 1u, k & 1u};
        for (uint32_t v = 0; v < ch.voxel_count; ++v) {
          const OVoxel& vx = voxels[ch.voxel_offset + v];
          const uint32_t q[3] = {vx.cell & 127u, (vx.cell >> 7) & 127u, (vx.cell >> 14) & 127u};
          uint32_t own[3];
          for (int a = 0; a < 3; ++a) own[a] = 64u * b[a] + (q[a] >> 1);
          sample(own[0] | (own[1] << 7) | (own[2] << 14), vx.pick_index, vx.rgba, vx.count);
        }
      }
      ++c;
    }
    nd.voxel_offset = voxels.size();
    for (const auto& kv : cells) {
      OVoxel v;
      v.cell = kv.first;
      v.rgba = kv.second.rgba;
      v.count = (uint32_t)kv.second.count;
      v.pick_index = kv.second.index;
      voxels.push_back(v);
    }
    nd.voxel_count = (uint32_t)(voxels.size() - nd.voxel_offset);
  }

  // Section 4.2.4: one inner node's voxels under the neighbourhood-weighted
  // average, from its children's samples (their voxels must exist already).
  // Positions are in units of the node's grid cells, so the node's cube is
  // [0, 128)^3 and cell j has its centre at j + 1/2.  The paper fixes no
  // precision, and the rounding of the mean is an integer decision, so the
  // weights are taken in the precision the kernel uses: single precision
  // with every operation rounded on its own, then rounded to a multiple of
  // 2^-24 (ties to even); the weighted sums are exact integers and the mean
  // is rounded half up exactly.
  struct WCell {
    uint64_t r = 0, g = 0, b = 0, w = 0;  // weighted colour sums, weight sum (units of 2^-24)
    uint64_t count = 0;                   // original points in the cell
    bool occupied = false;
  };
  static void add_weighted(std::map<uint32_t, WCell>& cells, const double pos[3], const uint32_t own[3],
                           uint32_t rgba, uint64_t count) {
    WCell& home = cells[own[0] | (own[1] << 7) | (own[2] << 14)];
    home.occupied = true;
    home.count += count;
    // the cells whose centres lie within one cell width along every axis:
    // floor(pos - 1/2) and the next one, inside the grid; the offset to the
    // first is exact in double and rounded once to single precision, the
    // offset to the second is that minus one in single precision
    int64_t lo[3];
    float e0[3];
    for (int a = 0; a < 3; ++a) {
      lo[a] = (int64_t)std::floor(pos[a] - 0.5);
      e0[a] = (float)(pos[a] - ((double)lo[a] + 0.5));
    }
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          const int64_t j[3] = {lo[0] + dx, lo[1] + dy, lo[2] + dz};
          const int dd[3] = {dx, dy, dz};
          bool inside = true;
          float e[3];
          for (int a = 0; a < 3; ++a) {
            if (j[a] < 0 || j[a] > 127) inside = false;
            e[a] = dd[a] ? e0[a] - 1.0f : e0[a];
          }
          if (!inside) continue;
          const float d2 = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
          if (!(d2 < 1.0f)) continue;  // linear weight, zero from one cell on
          const float w = 1.0f - std::sqrt(d2);
          const uint64_t wq = (uint64_t)std::nearbyint(w * 16777216.0f);
          if (wq == 0) continue;
          WCell& c = cells[(uint32_t)j[0] | ((uint32_t)j[1] << 7) | ((uint32_t)j[2] << 14)];
          c.r += wq * (rgba & 0xFFu);
          c.g += wq * ((rgba >> 8) & 0xFFu);
          c.b += wq * ((rgba >> 16) & 0xFFu);
          c.w += wq;
        }
  }

  // A point sample of node nd: its position in grid cells and its cell.
  static void weighted_point(std::map<uint32_t, WCell>& cells, const ONode& nd, const OPoint& p) {
    const double scale = std::ldexp(1.0, 7 - (int)nd.log2_size);  // grid cells per unit of length
    const int64_t d[3] = {rel(p.x, nd.min[0]), rel(p.y, nd.min[1]), rel(p.z, nd.min[2])};
    double pos[3];
    uint32_t own[3];
    for (int a = 0; a < 3; ++a) {
      pos[a] = (double)d[a] * scale;
      own[a] = grid_coord(d[a], nd.log2_size);
    }
    add_weighted(cells, pos, own, p.rgba, 1);
  }

  // A voxel of the inner child in octant k, taken as one sample at the
  // centre of its cell; the child is one octant (half the edge) of the node.
  static void weighted_voxel(std::map<uint32_t, WCell>& cells, uint32_t k, const OVoxel& vx) {
    const uint32_t b[3] = {(k >> 2) & 1u, (k >> 1) & 1u, k & 1u};
    const uint32_t q[3] = {vx.cell & 127u, (vx.cell >> 7) & 127u, (vx.cell >> 14) & 127u};
    double pos[3];
    uint32_t own[3];
    for (int a = 0; a < 3; ++a) {
      pos[a] = 64.0 * b[a] + ((double)q[a] + 0.5) / 2.0;
      own[a] = 64u * b[a] + (q[a] >> 1);
    }
    add_weighted(cells, pos, own, vx.rgba, vx.count);
  }

  // Occupied cells only, in cell order; colour = weighted mean rounded half
  // up (exact integer division), alpha 255.
  static void weighted_emit(const std::map<uint32_t, WCell>& cells, std::vector<OVoxel>& out) {
    for (const auto& kv : cells) {
      const WCell& wc = kv.second;
      if (!wc.occupied) continue;
      auto channel = [&](uint64_t sum) {
        const uint64_t q = sum / wc.w, rem = sum - q * wc.w;
        const uint64_t m = q + (2 * rem >= wc.w ? 1u : 0u);
        return (uint32_t)std::min<uint64_t>(m, 255);
      };
      OVoxel v;
      v.cell = kv.first;
      v.rgba = channel(wc.r) | (channel(wc.g) << 8) | (channel(wc.b) << 16) | (255u << 24);
      v.count = (uint32_t)wc.count;
      v.pick_index = kNone;
      out.push_back(v);
    }
  }

  void voxelize_weighted(uint32_t id) {
    ONode& nd = nodes[id];
    std::map<uint32_t, WCell> cells;
    uint32_t c = nd.first_child;
    for (uint32_t k = 0; k < 8; ++k) {
      if (!(nd.child_mask & (1u << k))) continue;
      const ONode& ch = nodes[c];
      if (ch.flags & kLeaf) {
        // a leaf child's samples are its points
        for (uint32_t i : leaf_lists[c]) weighted_point(cells, nd, pts[i]);
      } else {
        // an inner child's samples are its voxels
        for (uint32_t v = 0; v < ch.voxel_count; ++v) weighted_voxel(cells, k, voxels[ch.voxel_offset + v]);
      }
      ++c;
    }
    nd.voxel_offset = voxels.size();
    weighted_emit(cells, voxels);
    nd.voxel_count = (uint32_t)(voxels.size() - nd.voxel_offset);
  }

  // Depth-first leaf layout: each node's point_offset is where its subtree
  // starts; a leaf copies its points there in input order.
  uint64_t layout(uint32_t id, uint64_t offset) {
    ONode& nd = nodes[id];
    nd.point_offset = offset;
    if (nd.flags & kLeaf) {
      const std::vector<uint32_t>& l = leaf_lists[id];
      for (size_t j = 0; j < l.size(); ++j) {
        leaf_points[offset + j] = pts[l[j]];
        leaf_index[offset + j] = l[j];
      }
      return offset + l.size();
    }
    uint32_t c = nd.first_child;
    for (uint32_t k = 0; k < 8; ++k)
      if (nd.child_mask & (1u << k)) offset = layout(c++, offset);
    return offset;
  }

  void run() {
    // Root cube.
    ONode root;
    if (n > 0) {
      int32_t lo[3] = {pts[0].x, pts[0].y, pts[0].z};
      int32_t hi[3] = {pts[0].x, pts[0].y, pts[0].z};
      for (uint64_t i = 1; i < n; ++i) {
        const int32_t c[3] = {pts[i].x, pts[i].y, pts[i].z};
        for (int a = 0; a < 3; ++a) {
          lo[a] = std::min(lo[a], c[a]);
          hi[a] = std::max(hi[a], c[a]);
        }
      }
      int64_t extent = 0;
      for (int a = 0; a < 3; ++a) extent = std::max(extent, (int64_t)hi[a] - (int64_t)lo[a]);
      uint32_t L = 0;
      while ((int64_t(1) << L) <= extent) ++L;  // smallest 2^L > extent
      for (int a = 0; a < 3; ++a) root.min[a] = lo[a];
      root.log2_size = L;
    }
    nodes.push_back(root);
    leaf_lists.emplace_back();

    // Breadth-first split, one level at a time (Section 4.1).
    std::vector<std::pair<uint32_t, std::vector<uint32_t>>> cur, next;
    {
      std::vector<uint32_t> all(n);
      for (uint64_t i = 0; i < n; ++i) all[i] = (uint32_t)i;
      cur.emplace_back(0u, std::move(all));
    }
    while (!cur.empty()) {
      next.clear();
      for (auto& item : cur) {
        uint32_t id = item.first;
        std::vector<uint32_t>& idx = item.second;
        nodes[id].point_count = idx.size();
        const bool split = idx.size() > T && nodes[id].level < max_depth && nodes[id].log2_size > 0;
        if (!split) {
          nodes[id].flags = kLeaf | (idx.size() > T ? kOverfull : 0u);
          leaf_lists[id] = std::move(idx);
          continue;
        }
        // Inner node: partition into octants.
        const ONode parent = nodes[id];
        const uint32_t half = parent.log2_size - 1;
        std::vector<uint32_t> part[8];
        for (uint32_t i : idx) {
          const OPoint& p = pts[i];
          uint32_t bx = (uint32_t)((rel(p.x, parent.min[0]) >> half) & 1);
          uint32_t by = (uint32_t)((rel(p.y, parent.min[1]) >> half) & 1);
          uint32_t bz = (uint32_t)((rel(p.z, parent.min[2]) >> half) & 1);
          part[(bx << 2) | (by << 1) | bz].push_back(i);
        }
        nodes[id].first_child = (uint32_t)nodes.size();
        for (uint32_t k = 0; k < 8; ++k) {
          if (part[k].empty()) continue;
          nodes[id].child_mask |= 1u << k;
          ONode ch;
          const int64_t step = int64_t(1) << half;
          ch.min[0] = (int32_t)(parent.min[0] + ((k >> 2) & 1) * step);
          ch.min[1] = (int32_t)(parent.min[1] + ((k >> 1) & 1) * step);
          ch.min[2] = (int32_t)(parent.min[2] + (k & 1) * step);
          ch.level = parent.level + 1;
          ch.log2_size = half;
          ch.parent = id;
          nodes.push_back(ch);
          leaf_lists.emplace_back();
          next.emplace_back((uint32_t)(nodes.size() - 1), std::move(part[k]));
        }
        if (mode != kModeWeighted && mode != kModeRandom) voxelize(nodes[id], idx);
      }
      std::swap(cur, next);
    }
    if (mode == kModeWeighted || mode == kModeRandom) {
      // bottom up: breadth-first ids put every child after its parent
      for (size_t id = nodes.size(); id-- > 0;) {
        if (nodes[id].flags & kLeaf) continue;
        if (mode == kModeWeighted) voxelize_weighted((uint32_t)id);
        else voxelize_random((uint32_t)id);
      }
    }
    leaf_points.resize(n);
    leaf_index.resize(n);
    layout(0, 0);
  }
};

}  // namespace

struct oracle_result {
  Builder b;
};

extern "C" {

// mode 0: cell-wise average, 1: sample pick, 2: neighbourhood-weighted
// average, 3: first come, 4: random (Listing 1 key).  Returns 0 on success,
// 1 on invalid arguments, 2 on allocation failure.
int oracle_build(const void* points, uint64_t n, uint32_t leaf_threshold, uint32_t mode,
                 uint32_t max_depth, oracle_result** out) {
  if (!out || (n > 0 && !points) || leaf_threshold == 0 || mode > kModeRandom || max_depth > 32 ||
      n > 0xFFFFFFFFull)
    return 1;
  oracle_result* r = new (std::nothrow) oracle_result();
  if (!r) return 2;
  r->b.pts = static_cast<const OPoint*>(points);
  r->b.n = n;
  r->b.T = leaf_threshold;
  r->b.mode = mode;
  r->b.max_depth = max_depth;
  try {
    r->b.run();
  } catch (const std::bad_alloc&) {
    delete r;
    return 2;
  }
  *out = r;
  return 0;
}

uint64_t oracle_n_nodes(const oracle_result* r) { return r->b.nodes.size(); }
uint64_t oracle_n_voxels(const oracle_result* r) { return r->b.voxels.size(); }

// Node fields as separate arrays, each sized oracle_n_nodes().
void oracle_get_nodes(const oracle_result* r, int32_t* min3, uint8_t* level, uint8_t* log2_size,
                      uint8_t* child_mask, uint8_t* flags, uint32_t* parent, uint32_t* first_child,
                      uint64_t* point_offset, uint64_t* point_count, uint64_t* voxel_offset,
                      uint32_t* voxel_count) {
  const std::vector<ONode>& v = r->b.nodes;
  for (size_t i = 0; i < v.size(); ++i) {
    for (int a = 0; a < 3; ++a) min3[3 * i + a] = v[i].min[a];
    level[i] = (uint8_t)v[i].level;
    log2_size[i] = (uint8_t)v[i].log2_size;
    child_mask[i] = (uint8_t)v[i].child_mask;
    flags[i] = (uint8_t)v[i].flags;
    parent[i] = v[i].parent;
    first_child[i] = v[i].first_child;
    point_offset[i] = v[i].point_offset;
    point_count[i] = v[i].point_count;
    voxel_offset[i] = v[i].voxel_offset;
    voxel_count[i] = v[i].voxel_count;
  }
}

// Voxels as rows of (cell, rgba, count, pick_index).
void oracle_get_voxels(const oracle_result* r, uint32_t* out4) {
  const std::vector<OVoxel>& v = r->b.voxels;
  for (size_t i = 0; i < v.size(); ++i) {
    out4[4 * i + 0] = v[i].cell;
    out4[4 * i + 1] = v[i].rgba;
    out4[4 * i + 2] = v[i].count;
    out4[4 * i + 3] = v[i].pick_index;
  }
}

// Leaf points in layout order (rows x, y, z, rgba) and their input indices.
void oracle_get_points(const oracle_result* r, int32_t* out4, uint32_t* index) {
  const Builder& b = r->b;
  for (uint64_t i = 0; i < b.n; ++i) {
    out4[4 * i + 0] = b.leaf_points[i].x;
    out4[4 * i + 1] = b.leaf_points[i].y;
    out4[4 * i + 2] = b.leaf_points[i].z;
    out4[4 * i + 3] = (int32_t)b.leaf_points[i].rgba;
    index[i] = b.leaf_index[i];
  }
}

void oracle_free(oracle_result* r) { delete r; }

// The voxels of one cube (min corner min3, edge 2^log2_size) computed from
// the n points given, which must be every input point inside that cube;
// index[i] is the input index of points[i] (the pick's argument).  Rows of
// (cell, rgba, count, pick_index) sorted by cell go to out4, which holds
// at least n rows; returns the number of rows, or -1 on invalid arguments
// (a point outside the cube, log2_size > 32).
int64_t oracle_cube_voxels(const void* points, const uint32_t* index, uint64_t n, const int32_t* min3,
                           uint32_t log2_size, uint32_t mode, uint32_t* out4) {
  // the weighted average and the random strategy depend on the children's
  // voxels: not defined per cube
  if ((n > 0 && (!points || !index || !out4)) || !min3 || log2_size > 32 || mode == kModeWeighted ||
      mode == kModeRandom || mode > kModeRandom)
    return -1;
  const OPoint* p = static_cast<const OPoint*>(points);
  for (uint64_t i = 0; i < n; ++i) {
    const int64_t d[3] = {rel(p[i].x, min3[0]), rel(p[i].y, min3[1]), rel(p[i].z, min3[2])};
    for (int a = 0; a < 3; ++a)
      if (d[a] < 0 || d[a] >= (int64_t(1) << log2_size)) return -1;
  }
  Builder b;
  b.pts = p;
  b.input_index = index;
  b.n = n;
  b.mode = mode;
  ONode nd{};
  for (int a = 0; a < 3; ++a) nd.min[a] = min3[a];
  nd.log2_size = log2_size;
  std::vector<uint32_t> all(n);
  for (uint64_t i = 0; i < n; ++i) all[i] = (uint32_t)i;
  b.voxelize(nd, all);
  for (size_t i = 0; i < b.voxels.size(); ++i) {
    out4[4 * i + 0] = b.voxels[i].cell;
    out4[4 * i + 1] = b.voxels[i].rgba;
    out4[4 * i + 2] = b.voxels[i].count;
    out4[4 * i + 3] = b.voxels[i].pick_index;
  }
  return (int64_t)b.voxels.size();
}

// The neighbourhood-weighted voxels (Section 4.2.4) of one inner node (min
// corner min3, edge 2^log2_size) from the samples its children give: the
// n_points points of its leaf children (any order) and the n_voxels voxels
// (rows of cell, rgba, count, pick_index) of its inner children, octant[j]
// being the child octant of voxel j.  Rows of (cell, rgba, count,
// 0xFFFFFFFF) sorted by cell go to out4 (at least n_points + n_voxels rows);
// returns their number, or -1 on invalid arguments.
int64_t oracle_weighted_node(const void* points, uint64_t n_points, const uint32_t* voxels4, const uint8_t* octant,
                             uint64_t n_voxels, const int32_t* min3, uint32_t log2_size, uint32_t* out4) {
  if ((n_points && !points) || (n_voxels && (!voxels4 || !octant)) || !min3 || !out4 || log2_size > 32 ||
      log2_size == 0)
    return -1;
  ONode nd{};
  for (int a = 0; a < 3; ++a) nd.min[a] = min3[a];
  nd.log2_size = log2_size;
  std::map<uint32_t, Builder::WCell> cells;
  const OPoint* p = static_cast<const OPoint*>(points);
  for (uint64_t i = 0; i < n_points; ++i) {
    const int64_t d[3] = {rel(p[i].x, min3[0]), rel(p[i].y, min3[1]), rel(p[i].z, min3[2])};
    for (int a = 0; a < 3; ++a)
      if (d[a] < 0 || d[a] >= (int64_t(1) << log2_size)) return -1;
    Builder::weighted_point(cells, nd, p[i]);
  }
  for (uint64_t j = 0; j < n_voxels; ++j) {
    if (octant[j] > 7) return -1;
    const OVoxel vx{voxels4[4 * j], voxels4[4 * j + 1], voxels4[4 * j + 2], voxels4[4 * j + 3]};
    Builder::weighted_voxel(cells, octant[j], vx);
  }
  std::vector<OVoxel> out;
  Builder::weighted_emit(cells, out);
  for (size_t i = 0; i < out.size(); ++i) {
    out4[4 * i + 0] = out[i].cell;
    out4[4 * i + 1] = out[i].rgba;
    out4[4 * i + 2] = out[i].count;
    out4[4 * i + 3] = out[i].pick_index;
  }
  return (int64_t)out.size();
}

uint64_t oracle_splitmix64(uint64_t x) { return splitmix64(x); }

uint64_t oracle_random_key(uint32_t i, uint32_t level) { return random_key(i, level); }

}  // extern "C"
