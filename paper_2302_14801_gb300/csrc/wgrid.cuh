// Dense-grid accumulation shared by the neighbourhood-weighted voxel pass
// (Section 4.2.4) and the merge of out-of-core chunks: per grid cell one
// 32-byte sector of four 64-bit sums, a 32-bit count, and a list of the
// cells touched since the grid was last emptied.  Internal.
#pragma once

#include "common.cuh"

namespace lodk {

constexpr uint32_t kGridCells = 1u << 21;  // 128^3
constexpr float kWScale = 16777216.0f;     // 2^24: fixed-point weight unit

// One weighted contribution to grid cell `cell`: the first toucher (the
// weight sum was zero before) lists the cell for extraction.
__device__ __forceinline__ void w_add(unsigned long long* grid, uint32_t* touched, uint32_t* n_touched,
                                      uint32_t cell, uint32_t wq, uint32_t rgba) {
  unsigned long long* e = grid + 4ull * cell;
  const unsigned long long old = atomicAdd(e + 3, (unsigned long long)wq);
  if (old == 0ull) touched[atomicAdd(n_touched, 1u)] = cell;
  atomicAdd(e + 0, (unsigned long long)wq * (rgba & 255u));
  atomicAdd(e + 1, (unsigned long long)wq * ((rgba >> 8) & 255u));
  atomicAdd(e + 2, (unsigned long long)wq * ((rgba >> 16) & 255u));
}

// One sample whose position along axis a is P_a / 2^(s+1) cells (P_a an
// integer), colour rgba, `count` original points, lying in cell own:
// weights max(0, 1 - distance) to the cells floor(pos - 1/2) and the next
// one per axis, inside the grid.  The offset of the sample from the centre
// of cell j is (P - (2j + 1) 2^s) / 2^(s+1), rounded to single precision;
// the squared distance, its square root and 1 minus it are single-precision
// operations each rounded on its own (no fused multiply-add), and the
// weight is rounded to the nearest multiple of 2^-24 (ties to even).
__device__ __forceinline__ void w_sample(unsigned long long* grid, uint32_t* cnt, uint32_t* touched,
                                         uint32_t* n_touched, const int64_t P[3], uint32_t s, uint32_t own,
                                         uint32_t rgba, uint32_t count) {
  const float inv = __int_as_float((int)(127u - (s + 1u)) << 23);  // 2^-(s+1), s + 1 <= 33
  int32_t j0[3];
  float e0[3], e1[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int64_t h = int64_t(1) << s;
    j0[a] = (int32_t)((P[a] - h) >> (s + 1));  // floor(pos - 1/2)
    e0[a] = __fmul_rn(__ll2float_rn(P[a] - (2 * (int64_t)j0[a] + 1) * h), inv);
    e1[a] = __fsub_rn(e0[a], 1.0f);  // offset to the centre of j0 + 1
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int32_t jx = j0[0] + ((k >> 2) & 1), jy = j0[1] + ((k >> 1) & 1), jz = j0[2] + (k & 1);
    if ((uint32_t)jx > 127u || (uint32_t)jy > 127u || (uint32_t)jz > 127u) continue;
    const float ex = (k & 4) ? e1[0] : e0[0];
    const float ey = (k & 2) ? e1[1] : e0[1];
    const float ez = (k & 1) ? e1[2] : e0[2];
    const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)), __fmul_rn(ez, ez));
    if (d2 >= 1.0f) continue;
    const uint32_t wq = __float2uint_rn(__fmul_rn(__fsub_rn(1.0f, __fsqrt_rn(d2)), kWScale));
    if (!wq) continue;
    w_add(grid, touched, n_touched, (uint32_t)jx | ((uint32_t)jy << 7) | ((uint32_t)jz << 14), wq, rgba);
  }
  atomicAdd(&cnt[own], count);
}

// A point sample of a node with min corner mn and edge 2^L: its position
// 2 (p - mn) / 2^(s+1) cells with s = L - 7 (cubes of edge >= 128), or
// 2 (p - mn) 2^(7-L) / 2 (smaller cubes: s = 0), and its cell.
__device__ __forceinline__ void w_point_pos(const int4& q, const int32_t mn[3], uint32_t L, int64_t P[3],
                                            uint32_t* s, uint32_t* own) {
  *s = L >= 7 ? L - 7 : 0u;
  const uint32_t up = L >= 7 ? 0u : 7u - L;
  const uint32_t d[3] = {(uint32_t)q.x - (uint32_t)mn[0], (uint32_t)q.y - (uint32_t)mn[1],
                         (uint32_t)q.z - (uint32_t)mn[2]};
  uint32_t o = 0;
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    P[ax] = (int64_t)((uint64_t)d[ax] << (1 + up));
    o |= grid_coord(d[ax], L) << (7 * ax);
  }
  *own = o;
}

// A voxel of the child in octant k taken as one sample at the centre of its
// cell q: position 64 b + (q + 1/2) / 2 = (256 b + 2 q + 1) / 4 cells
// (s = 1), lying in cell 64 b + q / 2.
__device__ __forceinline__ void w_voxel_pos(uint32_t cell, uint32_t k, int64_t P[3], uint32_t* own) {
  const uint32_t b[3] = {(k >> 2) & 1u, (k >> 1) & 1u, k & 1u};
  const uint32_t q[3] = {cell & 127u, (cell >> 7) & 127u, cell >> 14};
  uint32_t o = 0;
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    P[ax] = (int64_t)(256u * b[ax] + 2u * q[ax] + 1u);
    o |= (64u * b[ax] + (q[ax] >> 1)) << (7 * ax);
  }
  *own = o;
}

// Weighted mean of one channel, rounded half up: floor(s / w + 1/2).
__device__ __forceinline__ uint32_t w_round(unsigned long long s, unsigned long long w) {
  const unsigned long long q = s / w, r = s - q * w;
  const unsigned long long m = q + (2 * r >= w ? 1ull : 0ull);
  return m > 255ull ? 255u : (uint32_t)m;
}

// Octant of a parent-grid cell x | y << 7 | z << 14: k = 4 bx + 2 by + bz.
__device__ __forceinline__ uint32_t cell_octant(uint32_t cell) {
  return (((cell >> 6) & 1u) << 2) | (((cell >> 13) & 1u) << 1) | ((cell >> 20) & 1u);
}

}  // namespace lodk
