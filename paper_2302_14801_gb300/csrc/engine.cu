// Host orchestration of a (batched) LOD build.
//
// The device work of all tiles of a batch runs in the same launches: one
// bounding-box pass, then counting rounds (first grid per tile, then the
// refinement grids of overflowing cells), the node tables (one CTA per
// tile), and the bottom-up voxel levels.  The host reads back small
// counters between phases to size the next allocations: once per counting
// round (the root cubes are set on the device, so the bounding box needs no
// read-back unless a cube is too small for the first grid's depth), once
// more when refinement rounds make the node table follow them, and once
// after all voxel levels, which are enqueued together with no read-back
// between them.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "engine.h"
#include "kernels.h"

namespace lodk {

namespace {

#define LOD_CK(x)                                                           \
  do {                                                                      \
    cudaError_t e_ = (x);                                                   \
    if (e_ != cudaSuccess) {                                                \
      return e_ == cudaErrorMemoryAllocation ? LOD_ERR_OOM : LOD_ERR_CUDA;  \
    }                                                                       \
  } while (0)

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

// Device scratch kept between the builds of one stream.  Blocks are handed
// out best fit and given back when a buffer is released; the same stream
// enqueues every later use, so reuse is stream ordered.  Steady-state
// builds thus make no allocator calls for scratch (large stream-ordered
// allocations from a fragmented pool can take a fraction of a
// millisecond each).  A workspace serves one build at a time.
struct Workspace {
  struct Block {
    void* p;
    size_t bytes;
    bool used;
  };
  std::vector<Block> blocks;
  bool busy = false;
  // dense grids of the weighted mode (Section 4.2.4): zeroed when
  // allocated, and every launch leaves the cells it touched empty again
  void* wgrid = nullptr;
  size_t wgrid_bytes = 0;
  int take(size_t b) {
    int best = -1;
    for (size_t i = 0; i < blocks.size(); ++i)
      if (!blocks[i].used && blocks[i].bytes >= b && (best < 0 || blocks[i].bytes < blocks[best].bytes))
        best = (int)i;
    if (best < 0) {
      const size_t r = (b + (2u << 20) - 1) & ~size_t((2u << 20) - 1);
      void* p = nullptr;
      if (cudaMalloc(&p, r) != cudaSuccess) {
        (void)cudaGetLastError();
        // give the idle blocks back and retry once
        for (auto& k : blocks)
          if (!k.used && k.p) {
            cudaFree(k.p);
            k.p = nullptr;
            k.bytes = 0;
          }
        if (cudaMalloc(&p, r) != cudaSuccess) {
          (void)cudaGetLastError();
          return -1;
        }
      }
      for (size_t i = 0; i < blocks.size(); ++i)
        if (!blocks[i].p) {
          blocks[i] = {p, r, false};
          best = (int)i;
          break;
        }
      if (best < 0) {
        blocks.push_back({p, r, false});
        best = (int)blocks.size() - 1;
      }
    }
    blocks[best].used = true;
    return best;
  }
};

std::mutex g_ws_mu;
std::map<std::pair<int, cudaStream_t>, Workspace*> g_ws;

// Exclusive use of the calling stream's workspace for one build (none when
// another build on the same stream holds it, or when disabled).
struct WsLease {
  Workspace* ws = nullptr;
  WsLease(cudaStream_t st, bool enable) {
    if (!enable) return;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    std::lock_guard<std::mutex> lk(g_ws_mu);
    Workspace*& w = g_ws[{dev, st}];
    if (!w) w = new Workspace();
    if (w->busy) return;
    w->busy = true;
    ws = w;
  }
  ~WsLease() {
    if (!ws) return;
    std::lock_guard<std::mutex> lk(g_ws_mu);
    ws->busy = false;
  }
};

// Allocation-failure injection for tests of the error paths, on the host
// side (the failing allocation is never requested from CUDA, so no device
// state is involved): with LOD_INJECT_OOM_AT=k in the environment, the k-th
// device allocation of every build on this thread fails as out of memory.
thread_local int64_t tl_oom_countdown = -1;

void arm_oom_injection() {
  const char* e = std::getenv("LOD_INJECT_OOM_AT");
  tl_oom_countdown = (e && *e) ? std::atoll(e) : -1;
}

// Stream-ordered device buffer released on destruction; from the build's
// workspace when it has one (scratch), else from the stream-ordered pool
// (results, which outlive the build).
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t st;
  Workspace* ws = nullptr;
  int blk = -1;
  explicit DevBuf(cudaStream_t s, Workspace* w = nullptr) : st(s), ws(w) {}
  DevBuf(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  cudaError_t alloc(size_t b) {
    release();
    if (tl_oom_countdown > 0 && --tl_oom_countdown == 0) return cudaErrorMemoryAllocation;
    if (b == 0) b = 16;
    if (ws) {
      const int k = ws->take(b);
      if (k >= 0) {
        blk = k;
        p = ws->blocks[k].p;
        bytes = b;
        return cudaSuccess;
      }
    }
    bytes = b;
    return cudaMallocAsync(&p, b, st);
  }
  // grow keeping the first `keep` bytes
  cudaError_t grow(size_t b, size_t keep) {
    if (b <= bytes) return cudaSuccess;
    DevBuf q(st, ws);
    cudaError_t e = q.alloc(b);
    if (e != cudaSuccess) return e;
    if (p && keep) {
      e = cudaMemcpyAsync(q.p, p, std::min(keep, bytes), cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return e;
    }
    std::swap(p, q.p);
    std::swap(bytes, q.bytes);
    std::swap(blk, q.blk);
    return cudaSuccess;
  }
  void release() {
    if (p) {
      if (blk >= 0) ws->blocks[blk].used = false;
      else cudaFreeAsync(p, st);
    }
    p = nullptr;
    bytes = 0;
    blk = -1;
  }
  void* take() {  // only for pool buffers
    void* q = p;
    p = nullptr;
    bytes = 0;
    return q;
  }
  template <class T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

// Pinned host staging for read-backs, one per host thread.
struct HostStage {
  void* p = nullptr;
  size_t bytes = 0;
  ~HostStage() {
    if (p) cudaFreeHost(p);
  }
  void* get(size_t b) {
    if (b > bytes) {
      if (p) cudaFreeHost(p);
      bytes = std::max<size_t>(b, 1 << 16);
      if (cudaMallocHost(&p, bytes) != cudaSuccess) {
        p = nullptr;
        bytes = 0;
      }
    }
    return p;
  }
};
thread_local HostStage tl_stage;

// Pinned host arena for small uploads: cudaMemcpyAsync from pageable memory
// synchronises the stream, from pinned memory it does not.  The arena is
// recycled at every host synchronisation of the build (all earlier copies
// have completed by then).
struct Uploader {
  cudaStream_t st;
  char* base = nullptr;
  size_t cap = 0, used = 0;
  std::vector<char*> retired;
  explicit Uploader(cudaStream_t s) : st(s) {}
  ~Uploader() {
    cudaStreamSynchronize(st);
    for (char* r : retired) cudaFreeHost(r);
    if (base) cudaFreeHost(base);
  }
  cudaError_t put(void* dst, const void* src, size_t bytes) {
    if (!bytes) return cudaSuccess;
    const size_t need = (bytes + 255) & ~size_t(255);
    if (used + need > cap) {
      if (base) retired.push_back(base);
      cap = std::max<size_t>(need, std::max<size_t>(cap * 2, 1 << 20));
      void* q = nullptr;
      cudaError_t e = cudaMallocHost(&q, cap);
      if (e != cudaSuccess) {
        base = nullptr;
        cap = used = 0;
        return e;
      }
      base = static_cast<char*>(q);
      used = 0;
    }
    std::memcpy(base + used, src, bytes);
    cudaError_t e = cudaMemcpyAsync(dst, base + used, bytes, cudaMemcpyHostToDevice, st);
    used += need;
    return e;
  }
  // call right after a stream synchronisation
  void recycle() {
    used = 0;
    for (char* r : retired) cudaFreeHost(r);
    retired.clear();
  }
};

uint32_t ceil_log4(double x) {
  uint32_t d = 0;
  double v = 1.0;
  while (v < x && d < 32) {
    v *= 4.0;
    ++d;
  }
  return d;
}

// Depth of a tile's first counting grid: deep enough that surface-like
// clouds reach leaf size without refinement (about 4x fewer points per
// level), capped at 256^3 cells, the cube's own size and max_depth.
std::atomic<uint32_t> g_tune_root_depth{0};
std::atomic<uint32_t> g_tune_ctas_per_sm{0};
std::atomic<uint32_t> g_tune_queue_ranges{0};  // 0: default (4), 1: an item's ranges stay in its CTA
std::atomic<uint32_t> g_tune_range_cells{0};   // 0: what the shared memory holds
std::atomic<uint32_t> g_tune_dense_bins{0};  // 0: kSmemBins
std::atomic<uint32_t> g_tune_graph{0};       // 1: the voxel levels run as one CUDA graph
std::atomic<uint32_t> g_tune_no_merge{0};    // 1: no warp merge of same-cell samples in the voxel pass

// Stream capture of a build's voxel levels into a CUDA graph, launched as
// one unit on the build's stream.  The capture runs on a stream of the
// calling thread's own (the legacy default stream cannot be captured); a
// capture still open when the build returns early is ended and dropped.
struct GraphCapture {
  cudaStream_t st;   // the build's stream: the graph is launched here
  cudaStream_t cap = nullptr;
  bool active = false;
  explicit GraphCapture(cudaStream_t s) : st(s) {}
  GraphCapture(const GraphCapture&) = delete;
  cudaError_t begin() {
    thread_local cudaStream_t own = nullptr;
    if (!own) {
      const cudaError_t e = cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking);
      if (e != cudaSuccess) return e;
    }
    cap = own;
    const cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    active = e == cudaSuccess;
    return e;
  }
  cudaError_t launch() {
    active = false;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cap, &g);
    if (e != cudaSuccess) return e;
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(x, st);
    if (x) cudaGraphExecDestroy(x);  // an executable graph in flight is freed when it completes
    cudaGraphDestroy(g);
    return e;
  }
  ~GraphCapture() {
    if (!active) return;
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(cap, &g);
    if (g) cudaGraphDestroy(g);
    (void)cudaGetLastError();
  }
};

uint32_t choose_root_depth(uint64_t n, uint32_t T, uint32_t log2S, uint32_t max_depth) {
  if (n <= T || log2S == 0 || max_depth == 0) return 0;
  const uint32_t forced = g_tune_root_depth.load();
  uint32_t d = forced ? forced : ceil_log4((double)n / (double)T) + 1;
  d = std::min(d, kRootMaxD);
  d = std::min(d, log2S);
  d = std::min(d, max_depth);
  return std::max(d, 1u);
}

uint64_t ipow8(uint32_t d) { return uint64_t(1) << (3 * d); }

// Shared-memory pool layout of a set of sources (all ovf words, then all
// count pyramids, start pyramids and maps), so that the parts that must
// start at zero (ovf, counts) are one contiguous range.
struct PoolLayout {
  uint64_t ovf = 0, cnt = 0, start = 0, map = 0, total = 0, zero = 0;  // in u32 units
};

PoolLayout layout_pool(const std::vector<SrcDesc>& v, size_t first, size_t n, std::vector<uint64_t>* offs) {
  PoolLayout L;
  uint64_t o_ovf = 0, o_cnt = 0, o_map = 0;
  offs->assign(4 * n, 0);
  for (size_t i = 0; i < n; ++i) {
    const uint32_t d = v[first + i].d;
    (*offs)[4 * i + 0] = o_ovf;
    o_ovf += (ipow8(d) + 31) / 32;
    (*offs)[4 * i + 1] = o_cnt;
    (*offs)[4 * i + 2] = o_cnt;  // same offset inside the start region
    o_cnt += pyr_size(d);
    (*offs)[4 * i + 3] = o_map;
    o_map += ipow8(d);
  }
  L.ovf = 0;
  L.cnt = o_ovf;
  L.start = L.cnt + o_cnt;
  L.map = L.start + o_cnt;
  L.total = L.map + o_map;
  L.zero = L.start;  // ovf + cnt
  return L;
}

// ------------------------------------------------------------ profiling
struct KStat {
  uint64_t launches = 0;
  double ms = 0.0, bytes = 0.0;
};
std::mutex g_prof_mu;
std::map<std::string, KStat> g_prof;
std::vector<cudaEvent_t> g_event_pool;
std::atomic<bool> g_prof_on{false};
std::atomic<uint64_t> g_launches{0};

cudaEvent_t pool_event() {
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_event_pool.empty()) {
      cudaEvent_t e = g_event_pool.back();
      g_event_pool.pop_back();
      return e;
    }
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

bool debug_stats();

// Brackets every launch of one build with events on the build stream when
// profiling is on; resolves them after the build's host synchronisations.
// With LOD_DEBUG_STATS the launches' device timeline is printed as well.
struct Prof {
  struct Rec {
    const char* name;
    cudaEvent_t a, b;
    double bytes;
  };
  cudaStream_t st;
  bool on;
  cudaEvent_t a = nullptr;
  cudaEvent_t origin = nullptr;  // first event of the build (timeline printing)
  std::string timeline;
  std::vector<Rec> recs;
  explicit Prof(cudaStream_t s) : st(s), on(g_prof_on.load()) {}
  ~Prof() {
    // unresolved records (error paths): give the events back
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto& r : recs) {
      g_event_pool.push_back(r.a);
      g_event_pool.push_back(r.b);
    }
    if (origin) g_event_pool.push_back(origin);
    if (!timeline.empty()) std::fprintf(stderr, "[lod] device ms:%s\n", timeline.c_str());
  }
  void begin() {
    if (!on) return;
    if (!origin && debug_stats()) {
      origin = pool_event();
      if (origin) cudaEventRecord(origin, st);
    }
    a = pool_event();
    if (a) cudaEventRecord(a, st);
  }
  void end(const char* name, double bytes) {
    if (!on || !a) return;
    cudaEvent_t b = pool_event();
    if (!b) return;
    cudaEventRecord(b, st);
    recs.push_back({name, a, b, bytes});
    a = nullptr;
  }
  // call after the stream has been synchronised
  void resolve() {
    if (recs.empty()) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto& r : recs) {
      float ms = 0.f;
      if (origin) {
        float t0 = 0.f, t1 = 0.f;
        if (cudaEventElapsedTime(&t0, origin, r.a) == cudaSuccess &&
            cudaEventElapsedTime(&t1, origin, r.b) == cudaSuccess) {
          char buf[96];
          std::snprintf(buf, sizeof(buf), " %s@%.3f-%.3f", r.name, t0, t1);
          timeline += buf;
        }
      }
      if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
        KStat& k = g_prof[r.name];
        k.launches += 1;
        k.ms += ms;
        k.bytes += r.bytes;
      }
      g_event_pool.push_back(r.a);
      g_event_pool.push_back(r.b);
    }
    recs.clear();
  }
};

// LOD_DEBUG_STATS=1 prints per-level voxel statistics of every build to stderr.
bool debug_stats() {
  static const bool on = [] {
    const char* e = std::getenv("LOD_DEBUG_STATS");
    return e && e[0] == '1';
  }();
  return on;
}

}  // namespace

// Device bytes held by the workspace of (current device, st).
uint64_t workspace_bytes(cudaStream_t st) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  std::lock_guard<std::mutex> lk(g_ws_mu);
  auto it = g_ws.find({dev, st});
  if (it == g_ws.end() || !it->second) return 0;
  uint64_t b = it->second->wgrid_bytes;
  for (auto& k : it->second->blocks) b += k.p ? k.bytes : 0;
  return b;
}

// Free the workspace of (current device, st); the stream must be idle.
void release_workspace(cudaStream_t st) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  Workspace* w = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_ws_mu);
    auto it = g_ws.find({dev, st});
    if (it == g_ws.end() || !it->second || it->second->busy) return;
    w = it->second;
    g_ws.erase(it);
  }
  for (auto& k : w->blocks)
    if (k.p) cudaFree(k.p);
  if (w->wgrid) cudaFree(w->wgrid);
  delete w;
}


uint32_t default_root_depth(uint64_t n, uint32_t T, uint32_t max_depth) {
  if (n <= T || max_depth == 0 || T == 0) return 0;
  uint32_t d = ceil_log4((double)n / (double)T) + 1;
  d = std::min(d, kRootMaxD);
  d = std::min(d, max_depth);
  return std::max(d, 1u);
}

int set_tuning(const lod_tuning_t& t) {
  if (t.root_depth > kRootMaxD || t.stream_ctas_per_sm > 8) return LOD_ERR_INVALID_ARG;
  const uint32_t b = t.dense_bins_max;
  if (b && (b != 8 && b != 64 && b != 512 && b != 4096)) return LOD_ERR_INVALID_ARG;
  if (t.vox_queue_ranges > 4096 || t.graph_voxel_levels > 1 || t.vox_no_merge > 1) return LOD_ERR_INVALID_ARG;
  if (t.vox_range_cells > (1u << 18) || t.reserved[0]) return LOD_ERR_INVALID_ARG;
  g_tune_graph.store(t.graph_voxel_levels);
  g_tune_no_merge.store(t.vox_no_merge);
  g_tune_root_depth.store(t.root_depth);
  g_tune_ctas_per_sm.store(t.stream_ctas_per_sm);
  g_tune_dense_bins.store(b);
  g_tune_queue_ranges.store(t.vox_queue_ranges);
  g_tune_range_cells.store(t.vox_range_cells);
  return LOD_OK;
}

int get_tuning(lod_tuning_t* t) {
  std::memset(t, 0, sizeof(*t));
  t->root_depth = g_tune_root_depth.load();
  t->stream_ctas_per_sm = g_tune_ctas_per_sm.load();
  t->dense_bins_max = g_tune_dense_bins.load();
  t->vox_queue_ranges = g_tune_queue_ranges.load();
  t->vox_range_cells = g_tune_range_cells.load();
  t->graph_voxel_levels = g_tune_graph.load();
  t->vox_no_merge = g_tune_no_merge.load();
  return LOD_OK;
}

int profile_enable(bool on) {
  g_prof_on.store(on);
  return LOD_OK;
}

int profile_reset() {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof.clear();
  g_launches.store(0);
  return LOD_OK;
}

int profile_read(lod_kernel_stat_t* out, uint32_t cap, uint32_t* n) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  uint32_t i = 0;
  for (auto& kv : g_prof) {
    if (out && i < cap) {
      std::memset(&out[i], 0, sizeof(lod_kernel_stat_t));
      std::strncpy(out[i].name, kv.first.c_str(), sizeof(out[i].name) - 1);
      out[i].launches = kv.second.launches;
      out[i].total_ms = kv.second.ms;
      out[i].alg_bytes = kv.second.bytes;
    }
    ++i;
  }
  if (n) *n = i;
  return LOD_OK;
}

uint64_t launch_count() { return g_launches.load(); }
void note_launch() { g_launches.fetch_add(1); }

static std::mutex g_free_mu;
static cudaStream_t g_free_streams[64] = {};

cudaStream_t free_stream() {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_free_mu);
  if (dev < 0 || dev >= 64) return nullptr;
  if (!g_free_streams[dev]) cudaStreamCreateWithFlags(&g_free_streams[dev], cudaStreamNonBlocking);
  return g_free_streams[dev];
}

SharedBuffers::~SharedBuffers() {
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) return;
  cudaSetDevice(device);
  cudaStream_t fs = free_stream();
  for (void* q : {points, index, nodes, voxels, voxel_points, root_sums, input})
    if (q) cudaFreeAsync(q, fs);
  cudaSetDevice(prev);
}

bool valid_mode(uint32_t mode) {
  return mode == LOD_FILTER || mode == LOD_PICK || mode == LOD_WEIGHTED || mode == LOD_FIRST || mode == LOD_RANDOM;
}

bool valid_params(const lod_params_t& p) {
  const bool single = p.mode == LOD_PICK || p.mode == LOD_FIRST || p.mode == LOD_RANDOM;
  if (p.flags & ~(uint32_t)(LOD_FLAG_LEAF_INDEX | LOD_FLAG_FULL_PRECISION)) return false;
  if ((p.flags & LOD_FLAG_FULL_PRECISION) && !single) return false;
  return p.leaf_threshold != 0 && valid_mode(p.mode) && p.max_depth <= 32;
}

// The single-sample modes need every leaf point's input index.
bool keeps_index(const lod_params_t& p) {
  return p.mode == LOD_PICK || p.mode == LOD_FIRST || p.mode == LOD_RANDOM || (p.flags & LOD_FLAG_LEAF_INDEX);
}

uint64_t estimate_result_bytes(uint64_t n, const lod_params_t& p) {
  const bool idx = keeps_index(p);
  const uint64_t T = std::max<uint32_t>(p.leaf_threshold, 1);
  const uint64_t nodes = 64 + 16 * ((n + T - 1) / T);
  return n * 16 + (idx ? n * 4 : 0) + (n / 2 + 1024) * 16 + nodes * sizeof(lod_node_t);
}

uint64_t estimate_build_bytes(uint64_t n, const lod_params_t& p) {
  const uint64_t T = std::max<uint32_t>(p.leaf_threshold, 1);
  const uint32_t d = choose_root_depth(n, (uint32_t)T, 32, 32);
  const uint64_t pool = (2 * pyr_size(d) + ipow8(d) + ipow8(d) / 32 + 1) * 4;
  const uint64_t nodes = 64 + 16 * ((n + T - 1) / T);
  // result + one refinement buffer + two staging levels of one record per
  // point (plus exact sums when filtering) + the voxel array's first
  // estimate + node aux + pool, plus the 32-byte leaf staging of modes that
  // keep input indices
  const bool keep_idx = keeps_index(p);
  const uint64_t staging = n * (p.mode == LOD_FILTER ? 64 : 32);
  return estimate_result_bytes(n, p) + n * 20 + staging + n * 8 + (keep_idx ? n * 32 : 0) +
         nodes * sizeof(NodeAux) + pool + (16u << 20);
}

// Keep freed blocks of the device's stream-ordered pool instead of returning
// them to the driver at every synchronisation (the pool's default), so that
// repeated builds reuse their buffers without re-mapping memory.
static void retain_pool_memory() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  done[dev] = true;
}

// Host-side phase clock of one build (printed with LOD_DEBUG_STATS).
struct PhaseClock {
  bool on = debug_stats();
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now(), last = t0;
  std::string line;
  void tick(const char* what) {
    if (!on) return;
    const auto now = std::chrono::steady_clock::now();
    char buf[96];
    std::snprintf(buf, sizeof(buf), " %s +%.3f", what, std::chrono::duration<double, std::milli>(now - last).count());
    line += buf;
    last = now;
  }
  ~PhaseClock() {
    if (on)
      std::fprintf(stderr, "[lod] host ms:%s | total %.3f\n", line.c_str(),
                   std::chrono::duration<double, std::milli>(last - t0).count());
  }
};

namespace {
constexpr int kRetryWithRoots = -100;  // internal: redo the build with root cubes read back first
}

static int run_build_impl(const TileInput* tin, uint32_t nt, const lod_params_t& prm, cudaStream_t st,
                          std::shared_ptr<SharedBuffers>* shared_out, std::vector<TileResult>* tiles_out,
                          BuildStats* stats, bool use_workspace, bool sync_roots, const BuildOptions& opt);

// Builds normally go without a host round trip after the bounding box: the
// root cubes are set on the device and the first grids' depths chosen from
// the point counts alone.  When a cloud's cube turns out smaller than such
// a depth allows (a tiny spatial extent), the build is redone with the
// cubes read back first.
int run_build(const TileInput* tin, uint32_t nt, const lod_params_t& prm, cudaStream_t st,
              std::shared_ptr<SharedBuffers>* shared_out, std::vector<TileResult>* tiles_out, BuildStats* stats,
              bool use_workspace, const BuildOptions& opt) {
  // tiles with a prescribed cube take the path that sets the cubes on the host
  bool given = false;
  for (uint32_t t = 0; tin && t < nt; ++t) given = given || tin[t].cube != nullptr;
  const int rc = run_build_impl(tin, nt, prm, st, shared_out, tiles_out, stats, use_workspace, given, opt);
  if (rc != kRetryWithRoots) return rc;
  return run_build_impl(tin, nt, prm, st, shared_out, tiles_out, stats, use_workspace, true, opt);
}

static int run_build_impl(const TileInput* tin, uint32_t nt, const lod_params_t& prm, cudaStream_t st,
                          std::shared_ptr<SharedBuffers>* shared_out, std::vector<TileResult>* tiles_out,
                          BuildStats* stats, bool use_workspace, bool sync_roots, const BuildOptions& opt) {
  BuildStats S;
  PhaseClock clk;
  arm_oom_injection();
  WsLease lease(st, use_workspace);  // declared first: outlives every scratch buffer
  Workspace* const ws = lease.ws;
  if (nt == 0 || !tin) return LOD_ERR_INVALID_ARG;
  retain_pool_memory();
  if (!valid_params(prm)) return LOD_ERR_INVALID_ARG;
  const bool want_idx = keeps_index(prm);
  const uint32_t T = prm.leaf_threshold;
  const uint32_t dense_max = g_tune_dense_bins.load() ? g_tune_dense_bins.load() : kSmemBins;

  // ---- tile table and round-0 chunk space
  std::vector<TileDesc> td(nt);
  std::vector<uint64_t> chunk0(nt + 1, 0);
  uint64_t M = 0;
  for (uint32_t t = 0; t < nt; ++t) {
    const uint64_t n = tin[t].n;
    if (n > 0xFFFFFFFFull) return LOD_ERR_INVALID_ARG;
    if (n > 0 && (!tin[t].d_points || (reinterpret_cast<uintptr_t>(tin[t].d_points) & 15u)))
      return LOD_ERR_INVALID_ARG;
    std::memset(&td[t], 0, sizeof(TileDesc));
    td[t].in = reinterpret_cast<const int4*>(tin[t].d_points);
    td[t].n = (uint32_t)n;
    td[t].in_idx = tin[t].d_index;
    td[t].idx_bound = tin[t].index_bound ? tin[t].index_bound : (uint32_t)n;
    td[t].level0 = tin[t].level0;
    if (tin[t].d_index && (prm.flags & LOD_FLAG_FULL_PRECISION)) return LOD_ERR_INVALID_ARG;
    td[t].pt_base = M;
    M += n;
    chunk0[t + 1] = chunk0[t] + (n + kChunk - 1) / kChunk;
  }
  const uint64_t n_chunks0 = chunk0[nt];
  std::vector<uint32_t> chunk_tile(n_chunks0);
  for (uint32_t t = 0; t < nt; ++t)
    for (uint64_t c = chunk0[t]; c < chunk0[t + 1]; ++c) chunk_tile[c] = t;

  auto sh = std::make_shared<SharedBuffers>();
  LOD_CK(cudaGetDevice(&sh->device));
  // CTAs per SM of the streaming passes: by default 2, and 4 for builds of
  // at least 128 chunks per CTA of the 2-per-SM grid (about 160M points),
  // whose longer per-CTA chunk runs balance better in smaller pieces
  // (measured: 1B points 2.4 ms faster per build; 50M points 2 % slower
  // with 4)
  const uint32_t cps = g_tune_ctas_per_sm.load();
  const uint32_t cps_default = n_chunks0 >= 128ull * 2u * (uint64_t)sm_count() ? 4u : 2u;
  const int grid = (int)(cps ? cps : cps_default) * sm_count();
  Uploader up_(st);
  Prof prof(st);
#define LOD_LAUNCH(name, bytes, call) \
  do {                                \
    prof.begin();                     \
    LOD_CK(call);                     \
    prof.end(name, (double)(bytes));  \
    ++S.launches;                     \
  } while (0)

  DevBuf d_points(st), d_index(st);  // results
  DevBuf d_tiles(st, ws), d_chunk0(st, ws), d_chunk_src(st, ws), d_bbox(st, ws), d_ctr(st, ws), d_nchunks(st, ws);
  LOD_CK(d_points.alloc(M * 16));
  if (want_idx) LOD_CK(d_index.alloc(M * 4));
  LOD_CK(d_tiles.alloc(nt * sizeof(TileDesc)));
  LOD_CK(d_chunk0.alloc((nt + 1) * sizeof(uint64_t)));
  LOD_CK(d_chunk_src.alloc(std::max<uint64_t>(n_chunks0, 1) * 4));
  LOD_CK(d_bbox.alloc(nt * 6 * sizeof(int)));
  LOD_CK(d_ctr.alloc(sizeof(DevCounters)));
  LOD_CK(d_nchunks.alloc(sizeof(unsigned long long)));
  LOD_CK(cudaMemsetAsync(d_ctr.p, 0, sizeof(DevCounters), st));
  LOD_CK(up_.put(d_tiles.p, td.data(), nt * sizeof(TileDesc)));
  LOD_CK(up_.put(d_chunk0.p, chunk0.data(), (nt + 1) * sizeof(uint64_t)));
  if (n_chunks0)
    LOD_CK(up_.put(d_chunk_src.p, chunk_tile.data(), n_chunks0 * 4));
  {
    std::vector<int> init(6 * nt);
    for (uint32_t t = 0; t < nt; ++t)
      for (int i = 0; i < 3; ++i) {
        init[6 * t + i] = INT_MAX;
        init[6 * t + 3 + i] = INT_MIN;
      }
    LOD_CK(up_.put(d_bbox.p, init.data(), init.size() * sizeof(int)));
  }

  // ---- bounding box (root cube)
  LOD_LAUNCH("bbox", 16.0 * M,
             launch_bbox(d_tiles.as<TileDesc>(), d_chunk_src.as<uint32_t>(), n_chunks0, d_chunk0.as<uint64_t>(),
                         d_bbox.as<int>(), grid, st));
  std::vector<int> bbox(6 * nt);
  DevBuf d_abort(st, ws);
  if (sync_roots) {
    LOD_CK(cudaMemcpyAsync(bbox.data(), d_bbox.p, bbox.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
    LOD_CK(cudaStreamSynchronize(st));
    clk.tick("bbox");
    up_.recycle();
    prof.resolve();
    ++S.host_syncs;
  } else {
    LOD_CK(d_abort.alloc(sizeof(unsigned int)));
    LOD_CK(cudaMemsetAsync(d_abort.p, 0, sizeof(unsigned int), st));
  }

  std::vector<SrcDesc> srcs(nt);
  uint64_t src_bound0 = 0;
  for (uint32_t t = 0; t < nt; ++t) {
    if (!sync_roots) {
      // cube unknown yet (set on the device); depth from the counts alone
      SrcDesc& s = srcs[t];
      std::memset(&s, 0, sizeof(SrcDesc));
      s.tile = t;
      s.d = choose_root_depth(td[t].n, T, 32, prm.max_depth);
      s.n = td[t].n;
      s.chunk0 = chunk0[t];
      s.priv = ipow8(s.d) > dense_max ? 1u : 0u;
      src_bound0 += td[t].n / (T + 1ull);
      continue;
    }
    if (tin[t].cube) {
      for (int a = 0; a < 3; ++a) td[t].min[a] = tin[t].cube[a];
      td[t].log2S = (uint32_t)tin[t].cube[3];
      if (tin[t].cube[3] < 0 || tin[t].cube[3] > 32) return LOD_ERR_INVALID_ARG;
    } else if (td[t].n == 0) {
      td[t].min[0] = td[t].min[1] = td[t].min[2] = 0;
      td[t].log2S = 0;
    } else {
      int64_t ext = 0;
      for (int a = 0; a < 3; ++a) {
        td[t].min[a] = bbox[6 * t + a];
        ext = std::max<int64_t>(ext, (int64_t)bbox[6 * t + 3 + a] - (int64_t)bbox[6 * t + a]);
      }
      uint32_t L = 0;
      while ((int64_t(1) << L) <= ext) ++L;  // smallest power of two > extent
      td[t].log2S = L;
    }
    SrcDesc& s = srcs[t];
    std::memset(&s, 0, sizeof(SrcDesc));
    for (int a = 0; a < 3; ++a) s.min[a] = td[t].min[a];
    s.tile = t;
    s.level = 0;
    s.log2size = td[t].log2S;
    s.d = choose_root_depth(td[t].n, T, td[t].log2S, prm.max_depth);
    s.buf = 0;
    s.pt_off = 0;
    s.n = td[t].n;
    s.chunk0 = chunk0[t];
    s.priv = ipow8(s.d) > dense_max ? 1u : 0u;  // counted through the per-CTA hash tables
    src_bound0 += td[t].n / (T + 1ull);
  }

  // ---- counting rounds
  DevBuf d_srcs(st, ws), d_jobs(st, ws), d_tmp0(st, ws), d_tmp1(st, ws), d_tmpi0(st, ws), d_tmpi1(st, ws),
      d_lists(st, ws), d_llen(st, ws);
  LOD_CK(d_lists.alloc((size_t)grid * kPrivSlots * sizeof(uint2)));
  LOD_CK(d_llen.alloc((size_t)grid * sizeof(uint32_t)));
  std::vector<std::unique_ptr<DevBuf>> pools;
  uint64_t src_cap = nt + src_bound0 + 16;
  LOD_CK(d_srcs.alloc(src_cap * sizeof(SrcDesc)));

  BuildArgs A;
  std::memset(&A, 0, sizeof(A));
  A.n_tiles = nt;
  A.T = T;
  A.max_depth = prm.max_depth;
  A.mode = prm.mode;
  A.out = d_points.as<int4>();
  A.out_idx = want_idx ? d_index.as<uint32_t>() : nullptr;
  A.lists = d_lists.as<uint2>();
  A.list_len = d_llen.as<uint32_t>();
  A.abort = sync_roots ? nullptr : d_abort.as<unsigned int>();
  A.dense_max = dense_max;
  // modes that keep input indices stage each leaf point as one 32-byte record
  DevBuf d_wide(st, ws);
  if (want_idx) {
    LOD_CK(d_wide.alloc(M * 32));
    A.wide = d_wide.as<int4>();
  }
  DevBuf d_diag(st, ws);
  if (debug_stats()) {
    LOD_CK(d_diag.alloc(4 * sizeof(unsigned long long)));
    LOD_CK(cudaMemsetAsync(d_diag.p, 0, 4 * sizeof(unsigned long long), st));
    A.diag = d_diag.as<unsigned long long>();
  }

  // ---- node table (Section 4.1.3): enqueued right after the first round's
  // scatter, before its counters are read, so that a build without
  // refinement needs no extra round trip (the table is redone if rounds
  // follow)
  std::vector<uint32_t> node_cap(nt);
  for (uint32_t t = 0; t < nt; ++t) node_cap[t] = (uint32_t)std::min<uint64_t>(64 + 16 * ((td[t].n + T - 1) / T), 0x7FFFFFFFull);
  DevBuf d_nodes(st);  // result
  DevBuf d_aux(st, ws), d_lvl(st, ws), d_nn(st, ws), d_leafcap(st, ws), d_nctr(st, ws);
  std::vector<uint32_t> n_nodes(nt), lvl((size_t)nt * (kMaxLevels + 1));
  // [0, L): per level sum over all nodes of min(points, 64^3); [L, 2L): exact leaf points
  std::vector<unsigned long long> leaf_cap(2 * (kMaxLevels + 1));
  uint64_t total_cap = 0;
  // refined: the first round's count of refinement grids (the pass stands
  // down when it is nonzero), or null after the last round
  auto enqueue_nodes = [&](const unsigned long long* refined) -> int {
    total_cap = 0;
    for (uint32_t t = 0; t < nt; ++t) {
      td[t].node_base = total_cap;
      td[t].node_cap = node_cap[t];
      total_cap += node_cap[t];
    }
    LOD_CK(up_.put(d_tiles.p, td.data(), nt * sizeof(TileDesc)));
    LOD_CK(d_nodes.alloc(total_cap * sizeof(lod_node_t)));
    LOD_CK(d_aux.alloc(total_cap * sizeof(NodeAux)));
    LOD_CK(d_lvl.alloc(lvl.size() * 4));
    LOD_CK(d_nn.alloc(nt * 4));
    LOD_CK(d_leafcap.alloc(leaf_cap.size() * 8));
    LOD_CK(d_nctr.alloc(sizeof(DevCounters)));
    LOD_CK(cudaMemsetAsync(d_leafcap.p, 0, leaf_cap.size() * 8, st));
    LOD_CK(cudaMemsetAsync(d_nctr.p, 0, sizeof(DevCounters), st));
    LOD_LAUNCH("nodes", 0,
               launch_nodes(A, d_nodes.as<lod_node_t>(), d_aux.as<NodeAux>(), d_lvl.as<uint32_t>(),
                            d_nn.as<uint32_t>(), d_leafcap.as<unsigned long long>(), d_nctr.as<DevCounters>(),
                            refined, st));
    LOD_CK(cudaMemcpyAsync(n_nodes.data(), d_nn.p, nt * 4, cudaMemcpyDeviceToHost, st));
    LOD_CK(cudaMemcpyAsync(lvl.data(), d_lvl.p, lvl.size() * 4, cudaMemcpyDeviceToHost, st));
    LOD_CK(cudaMemcpyAsync(leaf_cap.data(), d_leafcap.p, leaf_cap.size() * 8, cudaMemcpyDeviceToHost, st));
    return LOD_OK;
  };
  bool nodes_enqueued = false;

  uint32_t round_first = 0, round_n = nt, n_src = nt;
  uint64_t round_chunks = n_chunks0;
  for (uint32_t round = 0;; ++round) {
    ++S.rounds;
    // pool for this round's grids
    std::vector<uint64_t> offs;
    const PoolLayout L = layout_pool(srcs, round_first, round_n, &offs);
    pools.emplace_back(new DevBuf(st, ws));
    DevBuf& pool = *pools.back();
    LOD_CK(pool.alloc(L.total * 4));
    LOD_CK(cudaMemsetAsync(pool.p, 0, L.zero * 4, st));
    uint32_t* pb = pool.as<uint32_t>();
    A.cnt_base = pb + L.cnt;
    A.cursor_delta = L.start - L.cnt;
    for (uint32_t i = 0; i < round_n; ++i) {
      SrcDesc& s = srcs[round_first + i];
      s.ovf = pb + L.ovf + offs[4 * i + 0];
      s.cnt = pb + L.cnt + offs[4 * i + 1];
      s.start = pb + L.start + offs[4 * i + 2];
      s.map = pb + L.map + offs[4 * i + 3];
    }
    LOD_CK(up_.put(d_srcs.as<SrcDesc>() + round_first, srcs.data() + round_first,
                           round_n * sizeof(SrcDesc)));
    if (round == 0 && !sync_roots)
      LOD_LAUNCH("roots", 0,
                 launch_roots(d_tiles.as<TileDesc>(), d_bbox.as<int>(), d_srcs.as<SrcDesc>(), nt, T,
                              prm.max_depth, d_abort.as<unsigned int>(), st));
    LOD_CK(up_.put(d_nchunks.p, &round_chunks, sizeof(round_chunks)));
    A.tiles = d_tiles.as<TileDesc>();
    A.srcs = d_srcs.as<SrcDesc>();
    A.tmp[0] = d_tmp0.as<int4>();
    A.tmp[1] = d_tmp1.as<int4>();
    A.tmp_idx[0] = d_tmpi0.as<uint32_t>();
    A.tmp_idx[1] = d_tmpi1.as<uint32_t>();

    const int cgrid = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)grid, round_chunks));
    uint64_t round_points = 0;
    for (uint32_t i = 0; i < round_n; ++i) round_points += srcs[round_first + i].n;
    LOD_LAUNCH("count", 16.0 * round_points,
               launch_count(A, d_chunk_src.as<uint32_t>(), d_nchunks.as<unsigned long long>(), cgrid, st));

    // pyramid jobs: up passes (bottom levels d, d-4, ...), down passes (tops 0, 4, ...)
    std::vector<std::vector<PyrJob>> up, down;
    for (uint32_t i = 0; i < round_n; ++i) {
      const uint32_t sid = round_first + i;
      const uint32_t d = srcs[sid].d;
      uint32_t pass = 0;
      for (int jb = (int)d; jb > 0; jb -= 4, ++pass) {
        if (up.size() <= pass) up.emplace_back();
        const uint32_t k = std::min<uint32_t>(4, jb);
        const uint64_t blocks = ipow8(jb - k);
        for (uint64_t b = 0; b < blocks; ++b) up[pass].push_back({sid, (uint32_t)jb, (uint32_t)b});
      }
      pass = 0;
      for (uint32_t jt = 0; jt < d || (d == 0 && jt == 0); jt += 4, ++pass) {
        if (down.size() <= pass) down.emplace_back();
        const uint64_t blocks = ipow8(jt);
        for (uint64_t b = 0; b < blocks; ++b) down[pass].push_back({sid, jt, (uint32_t)b});
        if (d == 0) break;
      }
    }
    size_t n_jobs = 0;
    for (auto& v : up) n_jobs += v.size();
    for (auto& v : down) n_jobs += v.size();
    std::vector<PyrJob> all;
    all.reserve(n_jobs);
    for (auto& v : up) all.insert(all.end(), v.begin(), v.end());
    for (auto& v : down) all.insert(all.end(), v.begin(), v.end());
    LOD_CK(d_jobs.alloc(std::max<size_t>(all.size(), 1) * sizeof(PyrJob)));
    LOD_CK(up_.put(d_jobs.p, all.data(), all.size() * sizeof(PyrJob)));
    size_t jo = 0;
    for (auto& v : up) {
      LOD_LAUNCH("pyramid_up", 0, launch_pyr_up(A, d_jobs.as<PyrJob>() + jo, (uint32_t)v.size(), st));
      jo += v.size();
    }
    // capacity of the source table for grids created by this round
    const uint64_t need = (uint64_t)n_src + round_points / (T + 1ull) + 16;
    if (need > src_cap) {
      LOD_CK(d_srcs.grow(need * sizeof(SrcDesc), (size_t)n_src * sizeof(SrcDesc)));
      src_cap = need;
      A.srcs = d_srcs.as<SrcDesc>();
    }
    LOD_CK(cudaMemsetAsync(d_ctr.p, 0, sizeof(DevCounters), st));
    const uint32_t next_buf = 1 + (round & 1);
    for (auto& v : down) {
      LOD_LAUNCH("pyramid_down", 0,
                 launch_pyr_down(A, d_jobs.as<PyrJob>() + jo, (uint32_t)v.size(), n_src,
                                 (uint32_t)(src_cap - n_src), next_buf, d_ctr.as<DevCounters>(), st));
      jo += v.size();
    }
    // the cells refined by this round (if any) go to a ping-pong buffer; it
    // is set up before the counters are known so that the scatter follows
    // the pyramid without a host round trip
    {
      DevBuf& tb = (round & 1) ? d_tmp1 : d_tmp0;
      DevBuf& ti = (round & 1) ? d_tmpi1 : d_tmpi0;
      if (!tb.p) {
        LOD_CK(tb.alloc(M * 16));
        if (want_idx) LOD_CK(ti.alloc(M * 4));
      }
      A.tmp[0] = d_tmp0.as<int4>();
      A.tmp[1] = d_tmp1.as<int4>();
      A.tmp_idx[0] = d_tmpi0.as<uint32_t>();
      A.tmp_idx[1] = d_tmpi1.as<uint32_t>();
    }
    LOD_LAUNCH("scatter", 32.0 * round_points,
               launch_scatter(A, d_chunk_src.as<uint32_t>(), d_nchunks.as<unsigned long long>(), round, cgrid, st));
    if (round == 0) {
      const int rc = enqueue_nodes(&d_ctr.as<DevCounters>()->new_srcs);
      if (rc != LOD_OK) return rc;
      nodes_enqueued = true;
    }
    DevCounters* hc = static_cast<DevCounters*>(tl_stage.get(sizeof(DevCounters) + sizeof(unsigned int)));
    if (!hc) return LOD_ERR_OOM;
    unsigned int* h_abort = reinterpret_cast<unsigned int*>(hc + 1);
    *h_abort = 0;
    LOD_CK(cudaMemcpyAsync(hc, d_ctr.p, sizeof(DevCounters), cudaMemcpyDeviceToHost, st));
    if (round == 0 && !sync_roots)
      LOD_CK(cudaMemcpyAsync(h_abort, d_abort.p, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
    LOD_CK(cudaStreamSynchronize(st));
    clk.tick("round");
    if (*h_abort) {
      prof.resolve();
      return kRetryWithRoots;
    }
    up_.recycle();
    prof.resolve();
    ++S.host_syncs;
    if (hc->error) return LOD_ERR_INTERNAL;
    if (A.diag) {
      unsigned long long dg[2] = {0, 0};
      LOD_CK(cudaMemcpy(dg, A.diag, sizeof(dg), cudaMemcpyDeviceToHost));
      std::fprintf(stderr, "[lod] round %u: %u grids, %llu points, root depth %u, %llu counted outside "
                   "the CTA tables, %llu table inserts\n", round, round_n, (unsigned long long)round_points,
                   srcs[round_first].d, dg[0], dg[1]);
    }
    const uint32_t new_srcs = (uint32_t)hc->new_srcs;
    const uint64_t new_points = hc->new_points;
    if (!new_srcs) break;
    nodes_enqueued = false;  // the table must follow the refinement rounds

    // next round: the new grids, their chunk space
    srcs.resize(n_src + new_srcs);
    LOD_CK(cudaMemcpyAsync(srcs.data() + n_src, d_srcs.as<SrcDesc>() + n_src, new_srcs * sizeof(SrcDesc),
                           cudaMemcpyDeviceToHost, st));
    LOD_CK(cudaStreamSynchronize(st));
    clk.tick("new_srcs");
    ++S.host_syncs;
    round_first = n_src;
    round_n = new_srcs;
    n_src += new_srcs;
    round_chunks = 0;
    for (uint32_t i = 0; i < round_n; ++i) {
      SrcDesc& s = srcs[round_first + i];
      s.chunk0 = round_chunks;
      round_chunks += (s.n + kChunk - 1) / kChunk;
    }
    std::vector<uint32_t> cs(round_chunks);
    for (uint32_t i = 0; i < round_n; ++i) {
      const SrcDesc& s = srcs[round_first + i];
      const uint64_t nc = (s.n + kChunk - 1) / kChunk;
      for (uint64_t c = 0; c < nc; ++c) cs[s.chunk0 + c] = round_first + i;
    }
    (void)new_points;
    LOD_CK(d_chunk_src.alloc(std::max<uint64_t>(round_chunks, 1) * 4));
    LOD_CK(up_.put(d_chunk_src.p, cs.data(), round_chunks * 4));
  }

  // ---- node tables: check the table enqueued with the first round (or
  // build it now), growing the capacity of tiles that overflowed
  for (int attempt = 0;; ++attempt) {
    if (!nodes_enqueued) {
      const int rc = enqueue_nodes(nullptr);
      if (rc != LOD_OK) return rc;
      LOD_CK(cudaStreamSynchronize(st));
      clk.tick("nodes");
      up_.recycle();
      prof.resolve();
      ++S.host_syncs;
    }
    nodes_enqueued = false;
    bool retry = false;
    for (uint32_t t = 0; t < nt; ++t)
      if (n_nodes[t] == kNone) {
        node_cap[t] = (uint32_t)std::min<uint64_t>(uint64_t(node_cap[t]) * 4, 0x7FFFFFFFull);
        retry = true;
      }
    if (!retry) break;
    if (attempt > 8) return LOD_ERR_INTERNAL;
  }
  std::vector<uint32_t> n_levels(nt);
  uint32_t max_levels = 0;
  for (uint32_t t = 0; t < nt; ++t) {
    uint32_t l = 0;
    while (l < kMaxLevels && lvl[(size_t)t * (kMaxLevels + 1) + l] < n_nodes[t]) ++l;
    n_levels[t] = l;
    max_levels = std::max(max_levels, l);
    S.nodes += n_nodes[t];
  }
  pools.clear();
  d_tmp0.release();
  d_tmp1.release();
  d_tmpi0.release();
  d_tmpi1.release();

  // ---- voxel levels, bottom-up (Section 4.2).  Every level is enqueued
  // without a host round trip: the staging of one level holds at most
  // min(points, 64^3) records per item (known from the node pass), each
  // level's place in the voxel array is kept on the device, and the voxel
  // array starts at an estimate; if the levels need more, the phase is run
  // once more with the exact size (every step of it is idempotent).
  DevBuf d_dense(st);  // result
  DevBuf d_stage0(st, ws), d_stage1(st, ws), d_sum0(st, ws), d_sum1(st, ws), d_pref(st, ws), d_tvox(st, ws);
  DevBuf d_units(st, ws), d_lctr(st, ws), d_vstate(st, ws), d_order(st, ws);
  const bool filt = prm.mode == LOD_FILTER;
  const int n_vlev = max_levels >= 2 ? (int)max_levels - 1 : 0;  // parent levels max_levels-2 .. 0
  const size_t pstride = 2 * (size_t)(nt + 1);
  std::vector<uint32_t> pref((size_t)std::max(n_vlev, 1) * pstride, 0u);
  uint32_t max_items = 1;
  for (int l = 0; l < n_vlev; ++l) {
    uint32_t* ip = &pref[(size_t)l * pstride];  // items (nodes at level l + 1) per tile, prefix
    uint32_t* pp = ip + (nt + 1);               // parents (nodes at level l) per tile, prefix
    for (uint32_t t = 0; t < nt; ++t) {
      const uint32_t* ls = &lvl[(size_t)t * (kMaxLevels + 1)];
      ip[t + 1] = ip[t] + (ls[l + 2] - ls[l + 1]);
      pp[t + 1] = pp[t] + (ls[l + 1] - ls[l]);
    }
    max_items = std::max(max_items, ip[nt]);
  }
  LOD_CK(d_pref.alloc(pref.size() * 4));
  LOD_CK(up_.put(d_pref.p, pref.data(), pref.size() * 4));
  // one level's staging holds at most min(points, 64^3) records per item
  uint64_t stage_cap = 1;
  for (int l = 0; l < n_vlev; ++l) stage_cap = std::max<uint64_t>(stage_cap, leaf_cap[l + 1] + 1);
  if (n_vlev > 0) {
    LOD_CK(d_stage0.alloc(stage_cap * 16));
    LOD_CK(d_stage1.alloc(stage_cap * 16));
    if (filt) {
      LOD_CK(d_sum0.alloc(stage_cap * 16));
      LOD_CK(d_sum1.alloc(stage_cap * 16));
    }
  }
  // weighted mode: one dense grid per persistent CTA
  const bool weighted = prm.mode == LOD_WEIGHTED;
  const int wctas = sm_count();
  const size_t cells = size_t(1) << 21;
  DevBuf d_wtmp(st);
  unsigned char* wbase = nullptr;
  if (weighted && n_vlev > 0) {
    const size_t wbytes = (size_t)wctas * wgrid_bytes_per_cta();
    const size_t wzero = (size_t)wctas * cells * 36;  // sums and counts start at zero; the lists need not
    if (ws) {
      if (ws->wgrid_bytes < wbytes) {
        if (ws->wgrid) {
          LOD_CK(cudaStreamSynchronize(st));
          cudaFree(ws->wgrid);
          ws->wgrid = nullptr;
          ws->wgrid_bytes = 0;
        }
        LOD_CK(cudaMalloc(&ws->wgrid, wbytes));
        ws->wgrid_bytes = wbytes;
        LOD_CK(cudaMemsetAsync(ws->wgrid, 0, wzero, st));
      }
      wbase = static_cast<unsigned char*>(ws->wgrid);
    } else {
      LOD_CK(d_wtmp.alloc(wbytes));
      LOD_CK(cudaMemsetAsync(d_wtmp.p, 0, wzero, st));
      wbase = d_wtmp.as<unsigned char>();
    }
  }
  const uint32_t units_cap = (uint32_t)std::min<uint64_t>((uint64_t)max_items * 64, 1u << 20);
  LOD_CK(d_units.alloc((size_t)units_cap * sizeof(uint4)));
  if (!weighted) LOD_CK(d_order.alloc((size_t)max_items * 4));
  const size_t lctr_bytes = (size_t)std::max(n_vlev, 1) * sizeof(DevCounters);
  LOD_CK(d_lctr.alloc(lctr_bytes));
  LOD_CK(d_vstate.alloc(2 * sizeof(unsigned long long)));
  LOD_CK(d_tvox.alloc(nt * 8));
  uint64_t dense_cap = std::max<uint64_t>(M / 2, 4096);
  std::vector<DevCounters> lctr(std::max(n_vlev, 1));
  unsigned long long vstate[2] = {0, 0};
  std::vector<unsigned long long> tvox(nt);
  std::vector<size_t> vox_rec(std::max(n_vlev, 1), 0);
  static const char* kVoxLevelNames[kMaxLevels] = {
      "voxelize_L00", "voxelize_L01", "voxelize_L02", "voxelize_L03", "voxelize_L04", "voxelize_L05",
      "voxelize_L06", "voxelize_L07", "voxelize_L08", "voxelize_L09", "voxelize_L10", "voxelize_L11",
      "voxelize_L12", "voxelize_L13", "voxelize_L14", "voxelize_L15", "voxelize_L16", "voxelize_L17",
      "voxelize_L18", "voxelize_L19", "voxelize_L20", "voxelize_L21", "voxelize_L22", "voxelize_L23",
      "voxelize_L24", "voxelize_L25", "voxelize_L26", "voxelize_L27", "voxelize_L28", "voxelize_L29",
      "voxelize_L30", "voxelize_L31", "voxelize_L32", "voxelize_L33"};
  A.tiles = d_tiles.as<TileDesc>();
  DevBuf d_rsums(st);  // result (out-of-core merges): exact sums of the roots' voxels
  for (int attempt = 0;; ++attempt) {
    LOD_CK(d_dense.alloc(dense_cap * 16));
    if (opt.keep_root_sums && filt) LOD_CK(d_rsums.alloc(dense_cap * 16));
    LOD_CK(cudaMemsetAsync(d_tvox.p, 0, nt * 8, st));
    LOD_CK(cudaMemsetAsync(d_lctr.p, 0, lctr_bytes, st));
    LOD_CK(cudaMemsetAsync(d_vstate.p, 0, 2 * sizeof(unsigned long long), st));
    // optionally, every level's launches go into one CUDA graph (the
    // levels need no host round trip, so they can be captured as a unit)
    GraphCapture cap(st);
    const bool use_graph = g_tune_graph.load() != 0 && !prof.on && n_vlev > 0;
    if (use_graph) {
      vox_init();  // kernel attributes are set outside the capture
      LOD_CK(cap.begin());
    }
    const cudaStream_t vst = use_graph ? cap.cap : st;  // where the levels are enqueued
    VoxLevel vl;
    std::memset(&vl, 0, sizeof(vl));
    for (int l = n_vlev - 1; l >= 0; --l) {
      const uint32_t* ip = &pref[(size_t)l * pstride];
      const uint32_t n_items = ip[nt], n_par = ip[nt + 1 + nt];
      DevCounters* lc = d_lctr.as<DevCounters>() + l;
      const int par = (l + 1) & 1;
      vl.level = (uint32_t)l;
      vl.n_items = n_items;
      vl.item_prefix = d_pref.as<uint32_t>() + (size_t)l * pstride;
      vl.lvl_start = d_lvl.as<uint32_t>();
      vl.nodes = d_nodes.as<lod_node_t>();
      vl.aux = d_aux.as<NodeAux>();
      vl.stage_out = (par ? d_stage1 : d_stage0).as<int4>();
      vl.stage_out_sum = filt ? (par ? d_sum1 : d_sum0).as<ulonglong2>() : nullptr;
      vl.stage_cap = stage_cap;
      vl.stage_in = (par ? d_stage0 : d_stage1).as<int4>();
      vl.stage_in_sum = filt ? (par ? d_sum0 : d_sum1).as<ulonglong2>() : nullptr;
      vl.dense = d_dense.as<int4>();
      vl.stage_used = &lc->stage_used[0];
      vl.units = d_units.as<uint4>();
      vl.unit_cap = units_cap;
      vl.dense_cap = dense_cap;
      vl.vstate = d_vstate.as<unsigned long long>();
      vl.parent_prefix = d_pref.as<uint32_t>() + (size_t)l * pstride + (nt + 1);
      vl.n_parents = n_par;
      // the deepest level takes its items in node order; every level scan
      // orders the items of the level above, larger ones first
      vl.order = (l == n_vlev - 1 || weighted) ? nullptr : d_order.as<uint32_t>();
      vl.next_order = (l == 0 || weighted) ? nullptr : d_order.as<uint32_t>();
      {
        const uint32_t q = g_tune_queue_ranges.load();
        vl.queue_ranges = q == 0 ? 4u : (q == 1 ? 0xFFFFFFFFu : q);
        vl.range_cells = g_tune_range_cells.load();
      }
      vl.no_merge = g_tune_no_merge.load();
      if (weighted) {
        vl.wgrid = reinterpret_cast<unsigned long long*>(wbase);
        vl.wcnt = reinterpret_cast<uint32_t*>(wbase + (size_t)wctas * cells * 32);
        vl.wtouch = reinterpret_cast<uint32_t*>(wbase + (size_t)wctas * cells * 36);
        LOD_LAUNCH(debug_stats() ? kVoxLevelNames[l] : "voxelize", 0,
                   launch_wvox(A, vl, lc, (int)std::min<uint32_t>((uint32_t)wctas, n_par), vst));
      } else {
        LOD_LAUNCH(debug_stats() ? kVoxLevelNames[l] : "voxelize", 0, launch_vox(A, vl, lc, vst));
      }
      vox_rec[l] = prof.recs.size();
      LOD_LAUNCH("level_scan", 0,
                 launch_level_scan(A, vl, d_pref.as<uint32_t>() + (size_t)l * pstride + (nt + 1), n_par,
                                   d_tvox.as<unsigned long long>(), lc, vst));
    }
    if (n_vlev > 0) {
      // the roots' voxels: the items of the top level have no parent pass
      // that would copy their staged records
      vl.root_sums = d_rsums.as<ulonglong2>();
      LOD_LAUNCH("publish_top", 0, launch_copy_items(A, vl, vst));
      vl.root_sums = nullptr;
    }
    if (use_graph) LOD_CK(cap.launch());
    LOD_CK(cudaMemcpyAsync(lctr.data(), d_lctr.p, lctr_bytes, cudaMemcpyDeviceToHost, st));
    LOD_CK(cudaMemcpyAsync(vstate, d_vstate.p, sizeof(vstate), cudaMemcpyDeviceToHost, st));
    LOD_CK(cudaMemcpyAsync(tvox.data(), d_tvox.p, nt * 8, cudaMemcpyDeviceToHost, st));
    LOD_CK(cudaStreamSynchronize(st));
    clk.tick("voxels");
    ++S.host_syncs;
    for (int l = 0; l < n_vlev; ++l)
      if (lctr[l].error) return LOD_ERR_INTERNAL;
    if (vstate[1] && attempt == 0) {
      dense_cap = std::max<uint64_t>(vstate[0], 1);  // exact: every level's count is known now
      prof.resolve();
      continue;
    }
    if (vstate[1]) return LOD_ERR_INTERNAL;
    break;
  }
  const uint64_t V = vstate[0];
  {
    // reads: leaf points and the children's voxels; writes: this level's voxels
    uint64_t V_child = 0;
    for (int l = n_vlev - 1; l >= 0; --l) {
      const uint64_t lv = lctr[l].level_voxels;
      if (prof.on && vox_rec[l] >= 1 && vox_rec[l] <= prof.recs.size())
        prof.recs[vox_rec[l] - 1].bytes = 16.0 * (double)(leaf_cap[kMaxLevels + 1 + l + 1] + V_child + lv);
      if (debug_stats())
        std::fprintf(stderr, "[lod] level %d: items %u (leaf points %llu, child voxels %llu) -> voxels %llu, "
                     "items with several rank ranges %llu, sample passes %llu, queued ranges %u, samples read %llu, largest item %llu\n", l,
                     pref[(size_t)l * pstride + nt], (unsigned long long)leaf_cap[kMaxLevels + 1 + l + 1],
                     (unsigned long long)V_child, (unsigned long long)lv,
                     (unsigned long long)lctr[l].vox_retries, (unsigned long long)lctr[l].vox_passes,
                     lctr[l].units, (unsigned long long)lctr[l].vox_samples,
                     (unsigned long long)lctr[l].vox_max_item);
      V_child = lv;
    }
    if (prof.on && n_vlev > 0 && !prof.recs.empty()) prof.recs.back().bytes = 32.0 * (double)V_child;
  }
  if (A.wide) {
    // a root that is a leaf is no voxel item: publish its points here
    std::vector<uint32_t> leaf_roots;
    uint32_t max_n = 0;
    uint64_t moved = 0;
    for (uint32_t t = 0; t < nt; ++t)
      if (n_levels[t] == 1 && td[t].n > 0) {
        leaf_roots.push_back(t);
        max_n = std::max(max_n, td[t].n);
        moved += td[t].n;
      }
    if (!leaf_roots.empty()) {
      LOD_CK(d_units.alloc(leaf_roots.size() * 4));
      LOD_CK(up_.put(d_units.p, leaf_roots.data(), leaf_roots.size() * 4));
      LOD_LAUNCH("publish_leaf_roots", 52.0 * moved,
                 launch_unwide(A, d_units.as<uint32_t>(), (uint32_t)leaf_roots.size(), max_n, st));
    }
  }
  // trim the voxel array when the estimate was more than three times too
  // generous (a copy of the voxels; smaller slack is cheaper to keep)
  if (dense_cap > 3 * V + 65536 && !d_rsums.p) {
    DevBuf exact(st);
    LOD_CK(exact.alloc(std::max<uint64_t>(V, 1) * 16));
    if (V) LOD_CK(cudaMemcpyAsync(exact.p, d_dense.p, V * 16, cudaMemcpyDeviceToDevice, st));
    std::swap(exact.p, d_dense.p);
    std::swap(exact.bytes, d_dense.bytes);
    dense_cap = std::max<uint64_t>(V, 1);
  }
  // full-precision variant: the picked input points, parallel to the voxels
  DevBuf d_vpts(st);  // result
  if ((prm.flags & LOD_FLAG_FULL_PRECISION) && V) {
    uint32_t max_nodes = 0;
    for (uint32_t t = 0; t < nt; ++t) max_nodes = std::max(max_nodes, n_nodes[t]);
    LOD_CK(d_vpts.alloc(dense_cap * 16));
    LOD_LAUNCH("voxel_points", 32.0 * V,
               launch_voxel_points(d_tiles.as<TileDesc>(), nt, d_nodes.as<lod_node_t>(), d_nn.as<uint32_t>(), max_nodes,
                                   d_dense.as<int4>(), d_vpts.as<int4>(), st));
  }
  up_.recycle();
  prof.resolve();

  // ---- results
  tiles_out->assign(nt, TileResult());
  for (uint32_t t = 0; t < nt; ++t) {
    TileResult& r = (*tiles_out)[t];
    r.pt_base = td[t].pt_base;
    r.n_points = td[t].n;
    r.node_base = td[t].node_base;
    r.n_nodes = n_nodes[t];
    r.n_levels = n_levels[t];
    r.n_voxels = tvox[t];
  }
  sh->bytes = M * 16 + (want_idx ? M * 4 : 0) + total_cap * sizeof(lod_node_t) + dense_cap * 16 +
              (d_vpts.p ? dense_cap * 16 : 0);
  sh->voxel_points = d_vpts.take();
  if (d_rsums.p) sh->bytes += dense_cap * 16;
  sh->root_sums = d_rsums.take();
  sh->points = d_points.take();
  sh->index = want_idx ? d_index.take() : nullptr;
  sh->nodes = d_nodes.take();
  sh->voxels = d_dense.take();
  *shared_out = sh;
  S.voxels = V;
  if (stats) *stats = S;
  clk.tick("end");
  return LOD_OK;
}

}  // namespace lodk
