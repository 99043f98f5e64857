// Root cubes of a batch of point clouds without any device allocation.
//
// Some callers cannot call cudaMalloc at all: a plug-in living inside a host
// application whose own allocator owns every byte of device memory, a
// real-time renderer that must not let an allocation synchronise the device
// in the middle of a frame, or code that runs under a fixed memory budget
// decided up front.  This entry point serves them: it computes the same
// bounding box and power-of-two root cube that lod_build starts from, but
// every piece of scratch memory it needs (the table of tiles, its work-item
// prefix and the per-tile min/max accumulators) lives in one statically
// sized device array that the library carries with it, so the only device
// memory it touches is the caller's input and output.
//
// The static array is created once per device that loads the library and
// stays until the process exits.  Every call reuses it and leaves its own
// contents behind; the call clears what must start from a known value.
// Because all calls share the one array, two calls whose work overlaps on
// the GPU (different streams, or different host threads) race with each
// other and may return wrong results: serialise them on one stream.  The
// array's device address is looked up once per device and kept, so the
// call is not supported after cudaDeviceReset in the same process.
#include <climits>
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace lodk {
namespace {

constexpr uint32_t kNaMaxTiles = 4096;  // largest batch one call accepts
constexpr uint32_t kNaSlice = 128;      // tiles handed to the device per table-writing launch
constexpr uint32_t kNaChunk = 4096;     // points per work item of the bounding-box pass

struct NaTile {
  const int4* in;
  uint64_t n;
};

struct NaScratch {
  NaTile tiles[kNaMaxTiles];           // 64 KB
  uint64_t chunk0[kNaMaxTiles + 1];    // 32 KB: first work item of each tile (prefix)
  int box[kNaMaxTiles][6];             // 96 KB: min x, y, z, max x, y, z
};

// 192 KB of scratch per device, the whole working memory of the call.
static __device__ __align__(256) NaScratch g_na_scratch;

// Device address of g_na_scratch for each device, looked up once with that
// device current (in host code the symbol is only a stand-in, not an
// address).  The cached address is not renewed after cudaDeviceReset.
std::mutex g_na_mu;
NaScratch* g_na_ptr[64] = {};

cudaError_t na_scratch(int dev, NaScratch** out) {
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
    if (e != cudaSuccess) return e;
    g_na_ptr[dev] = static_cast<NaScratch*>(p);
  }
  *out = g_na_ptr[dev];
  return cudaSuccess;
}

// One slice of the tile table, passed by value as a kernel parameter (about
// 3 KB, under the 4 KB parameter limit), so that no host buffer has to stay
// alive after the call returns.
struct NaSlice {
  uint32_t t0, m;
  NaTile t[kNaSlice];
  uint64_t chunk0[kNaSlice];
};

// Install one slice of the table and reset its tiles' accumulators.
__global__ void k_na_set(NaScratch* s, NaSlice sl) {
  const uint32_t i = threadIdx.x;
  if (i >= sl.m) return;
  const uint32_t t = sl.t0 + i;
  s->tiles[t] = sl.t[i];
  s->chunk0[t] = sl.chunk0[i];
  s->box[t][0] = s->box[t][1] = s->box[t][2] = INT_MAX;
  s->box[t][3] = s->box[t][4] = s->box[t][5] = INT_MIN;
}

// Per-tile min/max over one flat list of work items: item c is the c-th
// run of kNaChunk points counted over all tiles in order, so a batch of
// very uneven tiles gives every CTA the same amount of work.  Each warp
// reduces its item's points and publishes six atomics; a tile holds
// c0 = chunk0[t] <= c < chunk0[t + 1].
__global__ void __launch_bounds__(256) k_na_bbox(NaScratch* s, uint32_t nt, uint64_t n_items) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t c = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < n_items; c += warps) {
    uint32_t lo = 0, hi = nt;  // largest t with chunk0[t] <= c (that tile is not empty)
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (s->chunk0[mid] <= c) lo = mid;
      else hi = mid;
    }
    const uint32_t t = lo;
    const int4* in = s->tiles[t].in;
    const uint64_t n = s->tiles[t].n;
    const uint64_t b = (c - s->chunk0[t]) * kNaChunk;
    const uint64_t e = b + kNaChunk < n ? b + kNaChunk : n;
    int v[6] = {INT_MAX, INT_MAX, INT_MAX, INT_MIN, INT_MIN, INT_MIN};
    for (uint64_t i = b + lane; i < e; i += 32) {
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
    if (lane < 3) atomicMin(&s->box[t][lane], v[lane]);
    else if (lane < 6) atomicMax(&s->box[t][lane], v[lane]);
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
  for (uint32_t t = 0; t < n_tiles; ++t) {
    if (n[t] > 0xFFFFFFFFull) return LOD_ERR_INVALID_ARG;
    if (n[t] && (!d_tiles[t] || (reinterpret_cast<uintptr_t>(d_tiles[t]) & 15u))) return LOD_ERR_INVALID_ARG;
  }
  (void)cudaGetLastError();  // an error left by an earlier, unrelated call is not this call's
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LOD_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    return LOD_ERR_CUDA;
  NaScratch* s = nullptr;
  if (na_scratch(dev, &s) != cudaSuccess) return LOD_ERR_CUDA;
  // the tile table goes to the device as kernel parameters, slice by slice
  NaSlice sl;
  uint64_t items = 0;
  for (uint32_t t0 = 0; t0 < n_tiles; t0 += kNaSlice) {
    sl.t0 = t0;
    sl.m = n_tiles - t0 < kNaSlice ? n_tiles - t0 : kNaSlice;
    for (uint32_t i = 0; i < sl.m; ++i) {
      sl.t[i] = {reinterpret_cast<const int4*>(d_tiles[t0 + i]), n[t0 + i]};
      sl.chunk0[i] = items;
      items += (n[t0 + i] + kNaChunk - 1) / kNaChunk;
    }
    k_na_set<<<1, kNaSlice, 0, st>>>(s, sl);
    lodk::note_launch();
  }
  if (items) {
    uint64_t grid = (items + 7) / 8;  // one work item per warp, 8 warps per CTA
    if (grid > (uint64_t)(4 * sms)) grid = (uint64_t)(4 * sms);
    k_na_bbox<<<(unsigned)grid, 256, 0, st>>>(s, n_tiles, items);
    lodk::note_launch();
  }
  k_na_cube<<<(n_tiles + 255) / 256, 256, 0, st>>>(s, n_tiles, d_cubes);
  lodk::note_launch();
  return cudaGetLastError() == cudaSuccess ? LOD_OK : LOD_ERR_CUDA;
}
