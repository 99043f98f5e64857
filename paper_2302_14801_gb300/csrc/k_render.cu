// Rendering of an LOD octree (Section 5 of the paper) into a headless
// framebuffer, as CUDA kernels instead of draw calls.
//
// Node selection: a node is drawn when it lies at least partly inside the
// view frustum and every ancestor is refined; a node is refined when it is
// drawn and its projected bounding box is larger than a pixel threshold
// (about 100 pixels in the paper, matching the 128^3 voxel grid).  The
// paper's layered structure replaces, not adds: a drawn inner node skips
// its voxels that lie in an octant whose child is drawn (the child draws
// finer samples there), and a drawn leaf draws all its points.
//
// Every drawn sample is projected with a row-major 4x4 matrix applied to
// its position relative to an integer origin (so that large int32
// coordinates keep their precision), and a pixel keeps the sample of
// smallest (depth, colour) through a 64-bit atomicMin on
// (float bits of depth) << 32 | rgba, depth = z/w * 1/2 + 1/2 in [0, 1]
// (non-negative floats order like their bits).
// All arithmetic is single precision with every operation rounded on its
// own (explicit _rn intrinsics, no fused multiply-add), so each pixel
// decision is reproducible bit for bit.
#include <cmath>

#include "common.cuh"
#include "kernels.h"

namespace lodk {

namespace {

struct RClip {
  float x, y, z, w;
};

__device__ __forceinline__ RClip r_project(const lod_camera_t& c, float px, float py, float pz) {
  float r[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float s = __fmul_rn(c.view_proj[4 * i + 0], px);
    s = __fadd_rn(s, __fmul_rn(c.view_proj[4 * i + 1], py));
    s = __fadd_rn(s, __fmul_rn(c.view_proj[4 * i + 2], pz));
    s = __fadd_rn(s, c.view_proj[4 * i + 3]);
    r[i] = s;
  }
  return {r[0], r[1], r[2], r[3]};
}

__device__ __forceinline__ float r_rel(int32_t v, int32_t o) { return __ll2float_rn((long long)v - (long long)o); }

// Frustum test and projected size (pixels) of the cube [min, min + 2^L)^3;
// a cube reaching behind the camera has infinite size.
__device__ void r_box(const lod_camera_t& c, const lod_node_t& nd, bool* inside, float* size) {
  const float edge = __int_as_float((int)(127u + nd.log2_size) << 23);  // 2^L, L <= 32
  float lo[3], hi[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lo[a] = r_rel(nd.min[a], c.origin[a]);
    hi[a] = __fadd_rn(lo[a], edge);
  }
  bool all[6] = {true, true, true, true, true, true};
  bool behind = false;
  float x0 = 0.f, x1 = 0.f, y0 = 0.f, y1 = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const RClip q = r_project(c, (k & 4) ? hi[0] : lo[0], (k & 2) ? hi[1] : lo[1], (k & 1) ? hi[2] : lo[2]);
    all[0] = all[0] && (q.x < -q.w);
    all[1] = all[1] && (q.x > q.w);
    all[2] = all[2] && (q.y < -q.w);
    all[3] = all[3] && (q.y > q.w);
    all[4] = all[4] && (q.z < -q.w);
    all[5] = all[5] && (q.z > q.w);
    if (!(q.w > 0.0f)) {
      behind = true;
      continue;
    }
    const float sx = __fmul_rn(__fadd_rn(__fmul_rn(__fdiv_rn(q.x, q.w), 0.5f), 0.5f), (float)c.width);
    const float sy = __fmul_rn(__fadd_rn(__fmul_rn(__fdiv_rn(q.y, q.w), 0.5f), 0.5f), (float)c.height);
    if (k == 0 || sx < x0) x0 = sx;
    if (k == 0 || sx > x1) x1 = sx;
    if (k == 0 || sy < y0) y0 = sy;
    if (k == 0 || sy > y1) y1 = sy;
  }
  *inside = !(all[0] || all[1] || all[2] || all[3] || all[4] || all[5]);
  const float w = __fsub_rn(x1, x0), h = __fsub_rn(y1, y0);
  *size = behind ? INFINITY : (w > h ? w : h);
}

__device__ __forceinline__ void r_splat(const lod_camera_t& c, float px, float py, float pz, uint32_t rgba,
                                        unsigned long long* fb, unsigned long long* drawn) {
  const RClip q = r_project(c, px, py, pz);
  if (!(q.w > 0.0f)) return;
  const float nx = __fdiv_rn(q.x, q.w), ny = __fdiv_rn(q.y, q.w), nz = __fdiv_rn(q.z, q.w);
  if (nx < -1.0f || nx > 1.0f || ny < -1.0f || ny > 1.0f || nz < -1.0f || nz > 1.0f) return;
  uint32_t ix = (uint32_t)floorf(__fmul_rn(__fadd_rn(__fmul_rn(nx, 0.5f), 0.5f), (float)c.width));
  uint32_t iy = (uint32_t)floorf(__fmul_rn(__fadd_rn(__fmul_rn(ny, 0.5f), 0.5f), (float)c.height));
  ix = ix < c.width ? ix : c.width - 1;
  iy = iy < c.height ? iy : c.height - 1;
  const float depth = __fadd_rn(__fmul_rn(nz, 0.5f), 0.5f);
  const unsigned long long key = ((unsigned long long)__float_as_uint(depth) << 32) | rgba;
  atomicMin(fb + (uint64_t)iy * c.width + ix, key);
  atomicAdd(drawn, 1ull);
}

}  // namespace

// One thread per node: drawn iff the node and every ancestor are in the
// frustum and every ancestor projects larger than the threshold.
__global__ void k_render_select(const lod_node_t* __restrict__ nodes, uint32_t n_nodes, lod_camera_t c,
                                uint8_t* __restrict__ visible, unsigned int* __restrict__ n_visible) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_nodes) return;
  bool inside;
  float size;
  r_box(c, nodes[i], &inside, &size);
  bool vis = inside;
  for (uint32_t p = nodes[i].parent, depth = 0; vis && p != kNone && depth < 64; p = nodes[p].parent, ++depth) {
    r_box(c, nodes[p], &inside, &size);
    vis = inside && size > c.lod_pixels;
  }
  visible[i] = vis ? 1 : 0;
  if (vis) atomicAdd(n_visible, 1u);
}

// Persistent CTAs walk the drawn nodes: leaves splat their points, inner
// nodes their voxels outside the octants of drawn children.
__global__ void __launch_bounds__(256) k_render_draw(const lod_node_t* __restrict__ nodes, uint32_t n_nodes,
                                                     const int4* __restrict__ points, const int4* __restrict__ voxels,
                                                     lod_camera_t c, const uint8_t* __restrict__ visible,
                                                     unsigned long long* __restrict__ fb,
                                                     unsigned long long* __restrict__ drawn) {
  for (uint32_t i = blockIdx.x; i < n_nodes; i += gridDim.x) {
    if (!visible[i]) continue;
    const lod_node_t nd = nodes[i];
    if (nd.flags & LOD_NODE_LEAF) {
      for (uint64_t j = threadIdx.x; j < nd.point_count; j += blockDim.x) {
        const int4 q = points[nd.point_offset + j];
        r_splat(c, r_rel(q.x, c.origin[0]), r_rel(q.y, c.origin[1]), r_rel(q.z, c.origin[2]), (uint32_t)q.w, fb,
                drawn);
      }
      continue;
    }
    uint32_t child_drawn = 0;  // bit k: the child in octant k is drawn
    for (uint32_t k = 0, ch = nd.first_child; k < 8; ++k)
      if (nd.child_mask & (1u << k)) child_drawn |= (uint32_t)visible[ch++] << k;
    float lo[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) lo[a] = r_rel(nd.min[a], c.origin[a]);
    // cell centre (2 q + 1) 2^(L - 8): an exact power-of-two scaling
    const float scale = __int_as_float((int)(127 + (int)nd.log2_size - 8) << 23);
    for (uint32_t j = threadIdx.x; j < nd.voxel_count; j += blockDim.x) {
      const int4 v = voxels[nd.voxel_offset + j];
      const uint32_t cell = (uint32_t)v.x;
      const uint32_t q[3] = {cell & 127u, (cell >> 7) & 127u, cell >> 14};
      const uint32_t oct = ((q[0] >> 6) << 2) | ((q[1] >> 6) << 1) | (q[2] >> 6);
      if (child_drawn & (1u << oct)) continue;  // the child replaces this voxel
      float p[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) p[a] = __fadd_rn(lo[a], __fmul_rn((float)(2u * q[a] + 1u), scale));
      r_splat(c, p[0], p[1], p[2], (uint32_t)v.y, fb, drawn);
    }
  }
}

cudaError_t launch_render(const lod_node_t* nodes, uint32_t n_nodes, const int4* points, const int4* voxels,
                          const lod_camera_t& cam, uint8_t* visible, unsigned int* n_visible,
                          unsigned long long* fb, unsigned long long* drawn, int sms, cudaStream_t st) {
  if (!n_nodes) return cudaSuccess;
  k_render_select<<<(n_nodes + 255) / 256, 256, 0, st>>>(nodes, n_nodes, cam, visible, n_visible);
  note_launch();
  const uint32_t grid = n_nodes < (uint32_t)(8 * sms) ? n_nodes : (uint32_t)(8 * sms);
  k_render_draw<<<grid, 256, 0, st>>>(nodes, n_nodes, points, voxels, cam, visible, fb, drawn);
  note_launch();
  return cudaGetLastError();
}

}  // namespace lodk
