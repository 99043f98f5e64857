// Root cubes of a batch of point clouds without any device allocation.
//
// Some callers cannot call cudaMalloc at all: a plug-in living inside a host
// application whose own allocator owns every byte of device memory, a
// real-time renderer that must not let an allocation synchronise the device
// in the middle of a frame, or code that runs under a fixed memory budget
// decided up front.  This entry point serves them: it computes the same
// bounding box and power-of-two root cube that lod_build starts from, but
// every piece of scratch memory it needs (the table of tiles and the per-tile
// min/max accumulators) lives in one statically sized device array that the
// library carries with it, so the only device memory it touches is the
// caller's input and output.
//
// The static array is created once per device that loads the library and
// stays until the process exits.  Every call reuses it and leaves its own
// contents behind; the call clears what must start from a known value.
// Because all calls share the one array, two calls whose work overlaps on
// the GPU (different streams, or different host threads) race with each
// other and may return wrong results: serialise them on one stream.
#include <climits>
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace lodk {
namespace {

constexpr uint32_t kNaMaxTiles = 4096;  // largest batch one call accepts

struct NaTile {
  const int4* in;
  uint64_t n;
};

struct NaScratch {
  NaTile tiles[kNaMaxTiles];  // 64 KB
  int box[kNaMaxTiles][6];    // 96 KB: min x, y, z, max x, y, z
};

// 160 KB of scratch per device, the whole working memory of the call.
static __device__ __align__(256) NaScratch g_na_scratch;

// Device address of g_na_scratch for each device, looked up once with that
// device current (in host code the symbol is only a stand-in, not an address).
std::mutex g_na_mu;
NaScratch* g_na_ptr[64] = {};

cudaError_t na_scratch(NaScratch** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_na_scratch);
    if (e != cudaSuccess) return e;
    g_na_ptr[dev] = static_cast<NaScratch*>(p);
  }
  *out = g_na_ptr[dev];
  return cudaSuccess;
}

__global__ void k_na_clear(NaScratch* s, uint32_t nt) {
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
    s->box[t][0] = s->box[t][1] = s->box[t][2] = INT_MAX;
    s->box[t][3] = s->box[t][4] = s->box[t][5] = INT_MIN;
  }
}

// Per-tile min/max: blockIdx.y selects the tile, the x dimension strides
// over its points with 16-byte loads; one block reduction and six atomics
// per CTA into the tile's accumulators.
__global__ void __launch_bounds__(256) k_na_bbox(NaScratch* s) {
  __shared__ int red[8][6];
  const uint32_t t = blockIdx.y;
  const int4* in = s->tiles[t].in;
  const uint64_t n = s->tiles[t].n;
  int v[6] = {INT_MAX, INT_MAX, INT_MAX, INT_MIN, INT_MIN, INT_MIN};
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const int4 p = __ldcs(in + i);
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
  const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < 6; ++k) red[w][k] = v[k];
  __syncthreads();
  if (threadIdx.x < 6) {
    int r = red[0][threadIdx.x];
    for (uint32_t j = 1; j < (blockDim.x >> 5); ++j)
      r = threadIdx.x < 3 ? min(r, red[j][threadIdx.x]) : max(r, red[j][threadIdx.x]);
    if (threadIdx.x < 3) atomicMin(&s->box[t][threadIdx.x], r);
    else atomicMax(&s->box[t][threadIdx.x], r);
  }
}

// Root cube of each tile: min corner = bounding-box minimum, edge = the
// smallest power of two strictly greater than the largest extent; an empty
// tile gets the origin and edge 1.  Output: 4 int32 per tile.
__global__ void k_na_cube(const NaScratch* s, uint32_t nt, int32_t* out) {
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
    int32_t* o = out + 4 * (uint64_t)t;
    if (s->tiles[t].n == 0) {
      o[0] = o[1] = o[2] = o[3] = 0;
      continue;
    }
    int64_t ext = 0;
    for (int a = 0; a < 3; ++a) {
      o[a] = s->box[t][a];
      const int64_t e = (int64_t)s->box[t][3 + a] - (int64_t)s->box[t][a];
      ext = e > ext ? e : ext;
    }
    int32_t L = 0;
    while ((int64_t(1) << L) <= ext) ++L;
    o[3] = L;
  }
}

}  // namespace
}  // namespace lodk

extern "C" int lod_root_cubes_noalloc(const lod_point_t* const* d_tiles, const uint64_t* n, uint32_t n_tiles,
                                      int32_t* d_cubes, void* stream) {
  using namespace lodk;
  if (!d_tiles || !n || !d_cubes || n_tiles == 0) return LOD_ERR_INVALID_ARG;
  if (n_tiles > kNaMaxTiles) return LOD_ERR_INVALID_ARG;  // more tiles than the scratch holds
  if (reinterpret_cast<uintptr_t>(d_cubes) & 3u) return LOD_ERR_INVALID_ARG;
  uint64_t max_n = 0;
  for (uint32_t t = 0; t < n_tiles; ++t) {
    if (n[t] > 0xFFFFFFFFull) return LOD_ERR_INVALID_ARG;
    if (n[t] && (!d_tiles[t] || (reinterpret_cast<uintptr_t>(d_tiles[t]) & 15u))) return LOD_ERR_INVALID_ARG;
    max_n = n[t] > max_n ? n[t] : max_n;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  NaScratch* s = nullptr;
  cudaError_t e = na_scratch(&s);
  if (e != cudaSuccess) return LOD_ERR_CUDA;
  // upload the tile table in slices from a small stack buffer (no heap use)
  NaTile slice[256];
  for (uint32_t t0 = 0; t0 < n_tiles; t0 += 256) {
    const uint32_t m = n_tiles - t0 < 256 ? n_tiles - t0 : 256;
    for (uint32_t i = 0; i < m; ++i) slice[i] = {reinterpret_cast<const int4*>(d_tiles[t0 + i]), n[t0 + i]};
    e = cudaMemcpyAsync(&s->tiles[t0], slice, m * sizeof(NaTile), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return LOD_ERR_CUDA;
  }
  k_na_clear<<<(n_tiles + 255) / 256, 256, 0, st>>>(s, n_tiles);
  lodk::note_launch();
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint64_t gx = (max_n + 256 * 16 - 1) / (256 * 16);
  gx = gx < 1 ? 1 : (gx > (uint64_t)(4 * sms) ? (uint64_t)(4 * sms) : gx);
  k_na_bbox<<<dim3((unsigned)gx, n_tiles), 256, 0, st>>>(s);
  lodk::note_launch();
  k_na_cube<<<(n_tiles + 255) / 256, 256, 0, st>>>(s, n_tiles, d_cubes);
  lodk::note_launch();
  e = cudaGetLastError();
  return e == cudaSuccess ? LOD_OK : LOD_ERR_CUDA;
}
