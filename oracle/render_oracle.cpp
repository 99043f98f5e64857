// CPU oracle of the LOD rasteriser — TEST INFRASTRUCTURE ONLY.
//
// Only tests/ and bench.py's CPU legs may load this library; the product
// path never links or calls it, and it shares no code with the CUDA path.
//
// A plain restatement of the rendering of Section 5 for a finished LOD
// octree, written into a headless framebuffer instead of a graphics API:
//  * a node is drawn when it lies (at least partly) in the view frustum and
//    every ancestor is refined; a node is refined when it is drawn and its
//    projected bounding box is larger than a pixel threshold (the paper
//    uses about 100 pixels, matching the 128^3 voxel grid);
//  * a drawn inner node draws its voxels (each at the centre of its cell)
//    except those lying in an octant whose child node is drawn, because the
//    child replaces them; a drawn leaf draws all its points;
//  * every sample is projected with a row-major 4x4 matrix applied to its
//    position relative to an integer origin; samples behind the camera or
//    outside the normalised device cube are dropped; a pixel keeps the
//    sample of smallest (depth, colour), depth being z/w * 1/2 + 1/2 (the
//    usual depth-buffer value, in [0, 1]).
// All arithmetic is single precision, each operation rounded on its own
// (the library is compiled without floating-point contraction), in the
// order written here, so that every pixel decision is reproducible.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

struct Cam {
  float m[16];
  int64_t origin[3];
  uint32_t width, height;
  float threshold;
};

struct Clip {
  float x, y, z, w;
};

// clip = M (p, 1), each row summed left to right
Clip project(const Cam& c, const float p[3]) {
  float r[4];
  for (int i = 0; i < 4; ++i) {
    float s = c.m[4 * i + 0] * p[0];
    s = s + c.m[4 * i + 1] * p[1];
    s = s + c.m[4 * i + 2] * p[2];
    s = s + c.m[4 * i + 3];
    r[i] = s;
  }
  return {r[0], r[1], r[2], r[3]};
}

// The eight corners of the cube [min, min + 2^L)^3, relative to the origin.
void corners(const Cam& c, const int32_t mn[3], uint32_t L, Clip out[8]) {
  float lo[3], hi[3];
  const float edge = std::ldexp(1.0f, (int)L);
  for (int a = 0; a < 3; ++a) {
    lo[a] = (float)((int64_t)mn[a] - c.origin[a]);
    hi[a] = lo[a] + edge;
  }
  for (int k = 0; k < 8; ++k) {
    const float p[3] = {(k & 4) ? hi[0] : lo[0], (k & 2) ? hi[1] : lo[1], (k & 1) ? hi[2] : lo[2]};
    out[k] = project(c, p);
  }
}

// Outside the frustum when all corners lie beyond one of its six planes.
bool in_frustum(const Clip k[8]) {
  bool all[6] = {true, true, true, true, true, true};
  for (int i = 0; i < 8; ++i) {
    all[0] = all[0] && (k[i].x < -k[i].w);
    all[1] = all[1] && (k[i].x > k[i].w);
    all[2] = all[2] && (k[i].y < -k[i].w);
    all[3] = all[3] && (k[i].y > k[i].w);
    all[4] = all[4] && (k[i].z < -k[i].w);
    all[5] = all[5] && (k[i].z > k[i].w);
  }
  for (int j = 0; j < 6; ++j)
    if (all[j]) return false;
  return true;
}

// Width or height in pixels of the projected corners, whichever is larger;
// a box reaching behind the camera counts as infinitely large.
float projected_size(const Cam& c, const Clip k[8]) {
  float x0 = 0, x1 = 0, y0 = 0, y1 = 0;
  for (int i = 0; i < 8; ++i) {
    if (!(k[i].w > 0.0f)) return INFINITY;
    const float sx = (k[i].x / k[i].w * 0.5f + 0.5f) * (float)c.width;
    const float sy = (k[i].y / k[i].w * 0.5f + 0.5f) * (float)c.height;
    if (i == 0 || sx < x0) x0 = sx;
    if (i == 0 || sx > x1) x1 = sx;
    if (i == 0 || sy < y0) y0 = sy;
    if (i == 0 || sy > y1) y1 = sy;
  }
  const float w = x1 - x0, h = y1 - y0;
  return w > h ? w : h;
}

void splat(const Cam& c, const float p[3], uint32_t rgba, uint64_t* fb, uint64_t* drawn) {
  const Clip q = project(c, p);
  if (!(q.w > 0.0f)) return;
  const float nx = q.x / q.w, ny = q.y / q.w, nz = q.z / q.w;
  if (nx < -1.0f || nx > 1.0f || ny < -1.0f || ny > 1.0f || nz < -1.0f || nz > 1.0f) return;
  uint32_t px = (uint32_t)std::floor((nx * 0.5f + 0.5f) * (float)c.width);
  uint32_t py = (uint32_t)std::floor((ny * 0.5f + 0.5f) * (float)c.height);
  if (px >= c.width) px = c.width - 1;
  if (py >= c.height) py = c.height - 1;
  const float depth = nz * 0.5f + 0.5f;
  uint32_t dbits;
  std::memcpy(&dbits, &depth, 4);
  const uint64_t key = ((uint64_t)dbits << 32) | rgba;
  uint64_t& f = fb[(uint64_t)py * c.width + px];
  if (key < f) f = key;
  ++*drawn;
}

}  // namespace

extern "C" {

// Render an LOD octree (node fields as separate arrays, n_nodes of each;
// voxels as rows of cell, rgba, count, pick_index; leaf points as rows of
// x, y, z, rgba) into fb (width * height keys, overwritten).  m: row-major
// 4x4 matrix; origin: integer origin the positions are taken relative to;
// threshold: refinement size in pixels.  visible (n_nodes bytes) receives
// which nodes were drawn.  Returns the number of samples drawn, or -1 on
// invalid arguments.
int64_t oracle_render(uint32_t n_nodes, const int32_t* min3, const uint8_t* log2_size, const uint8_t* child_mask,
                      const uint8_t* flags, const uint32_t* parent, const uint32_t* first_child,
                      const uint64_t* point_offset, const uint64_t* point_count, const uint64_t* voxel_offset,
                      const uint32_t* voxel_count, const uint32_t* voxels4, const int32_t* points4, const float* m,
                      const int32_t* origin, uint32_t width, uint32_t height, float threshold, uint64_t* fb,
                      uint8_t* visible) {
  if (!n_nodes || !min3 || !m || !origin || !fb || !visible || width == 0 || height == 0) return -1;
  Cam c;
  for (int i = 0; i < 16; ++i) c.m[i] = m[i];
  for (int a = 0; a < 3; ++a) c.origin[a] = origin[a];
  c.width = width;
  c.height = height;
  c.threshold = threshold;
  for (uint64_t i = 0; i < (uint64_t)width * height; ++i) fb[i] = ~0ull;
  // breadth-first node order: a parent comes before its children
  std::vector<uint8_t> refined(n_nodes, 0);
  for (uint32_t i = 0; i < n_nodes; ++i) {
    Clip k[8];
    corners(c, &min3[3 * i], log2_size[i], k);
    const bool parent_ok = parent[i] == 0xFFFFFFFFu || refined[parent[i]];
    visible[i] = parent_ok && in_frustum(k);
    refined[i] = visible[i] && !(flags[i] & 1u) && projected_size(c, k) > threshold;
  }
  uint64_t drawn = 0;
  for (uint32_t i = 0; i < n_nodes; ++i) {
    if (!visible[i]) continue;
    const uint32_t L = log2_size[i];
    if (flags[i] & 1u) {
      for (uint64_t j = 0; j < point_count[i]; ++j) {
        const int32_t* q = &points4[4 * (point_offset[i] + j)];
        const float p[3] = {(float)((int64_t)q[0] - c.origin[0]), (float)((int64_t)q[1] - c.origin[1]),
                            (float)((int64_t)q[2] - c.origin[2])};
        splat(c, p, (uint32_t)q[3], fb, &drawn);
      }
      continue;
    }
    // the drawn children of this node, by octant
    bool child_drawn[8] = {false, false, false, false, false, false, false, false};
    uint32_t ch = first_child[i];
    for (uint32_t k = 0; k < 8; ++k)
      if (child_mask[i] & (1u << k)) child_drawn[k] = visible[ch++] != 0;
    for (uint32_t j = 0; j < voxel_count[i]; ++j) {
      const uint32_t* v = &voxels4[4 * (voxel_offset[i] + j)];
      const uint32_t q[3] = {v[0] & 127u, (v[0] >> 7) & 127u, v[0] >> 14};
      const uint32_t oct = ((q[0] >> 6) << 2) | ((q[1] >> 6) << 1) | (q[2] >> 6);
      if (child_drawn[oct]) continue;  // the child replaces this voxel
      float p[3];
      for (int a = 0; a < 3; ++a) {
        const float lo = (float)((int64_t)min3[3 * i + a] - c.origin[a]);
        p[a] = lo + std::ldexp((float)(2 * q[a] + 1), (int)L - 8);  // cell centre
      }
      splat(c, p, v[1], fb, &drawn);
    }
  }
  return (int64_t)drawn;
}

}  // extern "C"
