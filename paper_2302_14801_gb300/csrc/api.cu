// C ABI of the LOD builder (declared in include/lod.h): argument checks,
// result objects, host copies and the serving loop.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "engine.h"
#include "kernels.h"
#include "result.h"

static_assert(sizeof(lod_point_t) == 16, "point record is 16 bytes");
static_assert(sizeof(lod_node_t) == 56, "node record is 56 bytes");
static_assert(sizeof(lod_voxel_t) == 16, "voxel record is 16 bytes");
static_assert(sizeof(lod_view_t) == 64, "view is 64 bytes");
static_assert(sizeof(lod_params_t) == 16, "params are 16 bytes");
static_assert(sizeof(lod_camera_t) == 96, "camera is 96 bytes");
static_assert(sizeof(lod_render_stats_t) == 16, "render stats are 16 bytes");

namespace {

int to_status(cudaError_t e) {
  if (e == cudaSuccess) return LOD_OK;
  return e == cudaErrorMemoryAllocation ? LOD_ERR_OOM : LOD_ERR_CUDA;
}

lod_params_t defaults() {
  lod_params_t p;
  p.leaf_threshold = 50000;
  p.mode = LOD_FILTER;
  p.max_depth = 21;
  p.flags = 0;
  return p;
}

}  // namespace

extern "C" {

int lod_params_init(lod_params_t* p) {
  if (!p) return LOD_ERR_INVALID_ARG;
  *p = defaults();
  return LOD_OK;
}

int lod_build(const lod_point_t* d_points, uint64_t n, const lod_params_t* params, void* stream,
              lod_result_t** out) {
  if (!out) return LOD_ERR_INVALID_ARG;
  const lod_params_t p = params ? *params : defaults();
  lodk::TileInput ti{d_points, n};
  std::shared_ptr<lodk::SharedBuffers> sh;
  std::vector<lodk::TileResult> tr;
  const int rc = lodk::run_build(&ti, 1, p, static_cast<cudaStream_t>(stream), &sh, &tr, nullptr);
  if (rc != LOD_OK) return rc;
  lod_result_t* r = make_result(sh, tr[0], p.mode, sh->bytes);
  if (!r) return LOD_ERR_OOM;
  *out = r;
  return LOD_OK;
}

int lod_build_from_host(const lod_point_t* h_points, uint64_t n, const lod_params_t* params, void* stream,
                        lod_result_t** out) {
  if (!out || (n && !h_points) || n > 0xFFFFFFFFull) return LOD_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  void* d = nullptr;
  if (n) {
    cudaError_t e = cudaMallocAsync(&d, n * sizeof(lod_point_t), st);
    if (e != cudaSuccess) return to_status(e);
    e = cudaMemcpyAsync(d, h_points, n * sizeof(lod_point_t), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
      cudaFreeAsync(d, st);
      return to_status(e);
    }
  }
  const int rc = lod_build(static_cast<const lod_point_t*>(d), n, params, stream, out);
  if (d) cudaFreeAsync(d, st);
  return rc;
}

int lod_build_batched(const lod_point_t* const* d_tiles, const uint64_t* n, uint32_t n_tiles,
                      const lod_params_t* params, void* stream, lod_result_t** out) {
  if (!d_tiles || !n || !out || n_tiles == 0) return LOD_ERR_INVALID_ARG;
  const lod_params_t p = params ? *params : defaults();
  std::vector<lodk::TileInput> ti(n_tiles);
  uint64_t total = 0;
  for (uint32_t t = 0; t < n_tiles; ++t) {
    ti[t] = {d_tiles[t], n[t]};
    total += n[t];
  }
  std::shared_ptr<lodk::SharedBuffers> sh;
  std::vector<lodk::TileResult> tr;
  const int rc = lodk::run_build(ti.data(), n_tiles, p, static_cast<cudaStream_t>(stream), &sh, &tr, nullptr);
  if (rc != LOD_OK) return rc;
  std::vector<lod_result_t*> rs(n_tiles, nullptr);
  for (uint32_t t = 0; t < n_tiles; ++t) {
    const uint64_t share = total ? (uint64_t)((double)sh->bytes * (double)n[t] / (double)total) : 0;
    rs[t] = make_result(sh, tr[t], p.mode, share);
    if (!rs[t]) {
      for (auto* q : rs) delete q;
      return LOD_ERR_OOM;
    }
  }
  for (uint32_t t = 0; t < n_tiles; ++t) out[t] = rs[t];
  return LOD_OK;
}

int lod_result_view(const lod_result_t* r, lod_view_t* v) {
  if (!r || !v) return LOD_ERR_INVALID_ARG;
  std::memset(v, 0, sizeof(*v));
  v->nodes = static_cast<const lod_node_t*>(r->sh->nodes) + r->tr.node_base;
  v->n_nodes = r->tr.n_nodes;
  v->n_levels = r->tr.n_levels;
  v->points = static_cast<const lod_point_t*>(r->sh->points) + r->tr.pt_base;
  v->point_index = r->sh->index ? static_cast<const uint32_t*>(r->sh->index) + r->tr.pt_base : nullptr;
  v->n_points = r->tr.n_points;
  v->voxels = static_cast<const lod_voxel_t*>(r->sh->voxels);
  v->n_voxels = r->tr.n_voxels;
  v->mode = r->mode;
  return LOD_OK;
}

int lod_result_copy_to_host(const lod_result_t* r, lod_node_t* nodes, lod_point_t* points, uint32_t* index,
                            lod_voxel_t* voxels, void* stream) {
  if (!r) return LOD_ERR_INVALID_ARG;
  if (index && !r->sh->index) return LOD_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  lod_view_t v;
  lod_result_view(r, &v);
  cudaError_t e = cudaSuccess;
  if (points && v.n_points)
    e = cudaMemcpyAsync(points, v.points, v.n_points * sizeof(lod_point_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && index && v.n_points)
    e = cudaMemcpyAsync(index, v.point_index, v.n_points * 4, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return to_status(e);
  if (!nodes && !voxels) return to_status(cudaStreamSynchronize(st));
  std::vector<lod_node_t> hn(v.n_nodes);
  e = cudaMemcpyAsync(hn.data(), v.nodes, v.n_nodes * sizeof(lod_node_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return to_status(e);
  std::vector<uint64_t> off(v.n_nodes);
  uint64_t acc = 0;
  for (uint32_t i = 0; i < v.n_nodes; ++i) {
    off[i] = acc;
    acc += hn[i].voxel_count;
  }
  if (voxels && acc) {
    void *d_off = nullptr, *d_tmp = nullptr;
    e = cudaMallocAsync(&d_off, v.n_nodes * 8, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_tmp, acc * 16, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_off, off.data(), v.n_nodes * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = lodk::launch_gather_voxels(v.nodes, v.n_nodes, static_cast<const uint64_t*>(d_off),
                                     reinterpret_cast<const int4*>(v.voxels), static_cast<int4*>(d_tmp), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(voxels, d_tmp, acc * 16, cudaMemcpyDeviceToHost, st);
    if (d_off) cudaFreeAsync(d_off, st);
    if (d_tmp) cudaFreeAsync(d_tmp, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return to_status(e);
  }
  if (nodes) {
    for (uint32_t i = 0; i < v.n_nodes; ++i) hn[i].voxel_offset = off[i];
    std::memcpy(nodes, hn.data(), hn.size() * sizeof(lod_node_t));
  }
  return LOD_OK;
}

int lod_result_voxel_points(const lod_result_t* r, const lod_point_t** d_points) {
  if (!r || !d_points || !r->sh->voxel_points) return LOD_ERR_INVALID_ARG;
  *d_points = static_cast<const lod_point_t*>(r->sh->voxel_points);
  return LOD_OK;
}

int lod_result_copy_voxel_points_to_host(const lod_result_t* r, lod_point_t* points, void* stream) {
  if (!r || !r->sh->voxel_points || (!points && r->tr.n_voxels)) return LOD_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  lod_view_t v;
  lod_result_view(r, &v);
  std::vector<lod_node_t> hn(v.n_nodes);
  cudaError_t e = cudaMemcpyAsync(hn.data(), v.nodes, v.n_nodes * sizeof(lod_node_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return to_status(e);
  std::vector<uint64_t> off(v.n_nodes);
  uint64_t acc = 0;
  for (uint32_t i = 0; i < v.n_nodes; ++i) {
    off[i] = acc;
    acc += hn[i].voxel_count;
  }
  if (!acc) return LOD_OK;
  void *d_off = nullptr, *d_tmp = nullptr;
  e = cudaMallocAsync(&d_off, v.n_nodes * 8, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&d_tmp, acc * 16, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_off, off.data(), v.n_nodes * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = lodk::launch_gather_voxels(v.nodes, v.n_nodes, static_cast<const uint64_t*>(d_off),
                                   static_cast<const int4*>(r->sh->voxel_points), static_cast<int4*>(d_tmp), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(points, d_tmp, acc * 16, cudaMemcpyDeviceToHost, st);
  if (d_off) cudaFreeAsync(d_off, st);
  if (d_tmp) cudaFreeAsync(d_tmp, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return to_status(e);
}

int lod_render(const lod_result_t* r, const lod_camera_t* cam, uint64_t* d_framebuffer, void* stream,
               lod_render_stats_t* stats) {
  if (!r || !cam || !d_framebuffer || (reinterpret_cast<uintptr_t>(d_framebuffer) & 7u)) return LOD_ERR_INVALID_ARG;
  if (cam->width == 0 || cam->height == 0 || (uint64_t)cam->width * cam->height > (1ull << 31) ||
      !(cam->lod_pixels >= 0.0f))
    return LOD_ERR_INVALID_ARG;
  for (float f : cam->view_proj)
    if (!std::isfinite(f)) return LOD_ERR_INVALID_ARG;
  lod_camera_t c = *cam;
  if (c.lod_pixels == 0.0f) c.lod_pixels = 100.0f;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  lod_view_t v;
  lod_result_view(r, &v);
  const uint64_t pixels = (uint64_t)c.width * c.height;
  cudaError_t e = cudaMemsetAsync(d_framebuffer, 0xFF, pixels * 8, st);
  if (e != cudaSuccess) return to_status(e);
  // scratch: drawn-node flags and two counters
  void* scratch = nullptr;
  const size_t cnt_off = ((size_t)v.n_nodes + 15) & ~size_t(15);
  e = cudaMallocAsync(&scratch, cnt_off + 16, st);
  if (e != cudaSuccess) return to_status(e);
  unsigned long long* drawn = reinterpret_cast<unsigned long long*>(static_cast<char*>(scratch) + cnt_off);
  unsigned int* n_vis = reinterpret_cast<unsigned int*>(drawn + 1);
  e = cudaMemsetAsync(drawn, 0, 16, st);
  int dev = 0, sms = 1;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = lodk::launch_render(v.nodes, v.n_nodes, reinterpret_cast<const int4*>(v.points),
                            reinterpret_cast<const int4*>(v.voxels), c, static_cast<uint8_t*>(scratch), n_vis,
                            reinterpret_cast<unsigned long long*>(d_framebuffer), drawn, sms, st);
  unsigned long long host[2] = {0, 0};
  if (e == cudaSuccess && stats) {
    e = cudaMemcpyAsync(host, drawn, 16, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  cudaFreeAsync(scratch, st);
  if (e != cudaSuccess) return to_status(e);
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->samples_drawn = host[0];
    stats->visible_nodes = (uint32_t)host[1];
  }
  return LOD_OK;
}

uint64_t lod_result_device_bytes(const lod_result_t* r) { return r ? r->bytes : 0; }

void lod_free(lod_result_t* r) {
  if (!r) return;
  if (r->budget) r->budget->release(r->bytes);
  delete r;
}

uint64_t lod_scratch_bytes(void* stream) { return lodk::workspace_bytes(static_cast<cudaStream_t>(stream)); }

int lod_trim(void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return to_status(e);
  lodk::release_workspace(st);
  int dev = 0;
  cudaMemPool_t pool;
  if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess)
    e = cudaMemPoolTrimTo(pool, 0);
  return to_status(e);
}

int lod_set_tuning(const lod_tuning_t* t) { return t ? lodk::set_tuning(*t) : LOD_ERR_INVALID_ARG; }
int lod_get_tuning(lod_tuning_t* t) { return t ? lodk::get_tuning(t) : LOD_ERR_INVALID_ARG; }

int lod_autotune(const lod_point_t* d_points, uint64_t n, const lod_params_t* params, void* stream,
                 lod_tuning_t* best, float* best_ms) {
  if (!d_points || n == 0 || !best) return LOD_ERR_INVALID_ARG;
  const lod_params_t p = params ? *params : defaults();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  lod_tuning_t before;
  lodk::get_tuning(&before);
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    return LOD_ERR_CUDA;
  }
  // one build to warm up, one timed
  auto time_with = [&](const lod_tuning_t& t, float* ms) -> int {
    int rc = lodk::set_tuning(t);
    for (int rep = 0; rep < 2 && rc == LOD_OK; ++rep) {
      lod_result_t* r = nullptr;
      if (rep == 1) cudaEventRecord(a, st);
      rc = lod_build(d_points, n, &p, st, &r);
      if (rep == 1) cudaEventRecord(b, st);
      if (rc == LOD_OK) {
        lod_free(r);
        if (rep == 1 && cudaEventSynchronize(b) == cudaSuccess) cudaEventElapsedTime(ms, a, b);
      }
    }
    return rc;
  };
  // coordinate descent: each knob in turn over its candidates, the others
  // held at the best found so far
  const uint32_t d0 = lodk::default_root_depth(n, p.leaf_threshold, p.max_depth);
  std::vector<uint32_t> depths = {0};
  if (d0 > 1) depths.push_back(d0 - 1);
  if (d0 >= 1 && d0 < 8) depths.push_back(d0 + 1);
  lod_tuning_t win;
  std::memset(&win, 0, sizeof(win));
  float win_ms = -1.f;
  int rc = time_with(win, &win_ms);
  for (int knob = 0; knob < 5 && rc == LOD_OK; ++knob) {
    std::vector<uint32_t> cand;
    if (knob == 0) cand = {2u, 3u, 4u};     // CTAs per SM of the streaming passes (default 2 or 4 by size)
    if (knob == 1) cand = std::vector<uint32_t>(depths.begin() + 1, depths.end());
    if (knob == 2) cand = {512u};           // dense shared histograms up to 512 cells (default 4096)
    if (knob == 3) cand = {1u, 2u};         // an item's rank ranges: never handed to other SMs, from 2 (default 4)
    if (knob == 4 && p.mode == LOD_FILTER) cand = {1u};  // no warp merge of same-cell samples
    for (uint32_t c : cand) {
      lod_tuning_t t = win;
      if (knob == 0) t.stream_ctas_per_sm = c;
      if (knob == 1) t.root_depth = c;
      if (knob == 2) t.dense_bins_max = c;
      if (knob == 3) t.vox_queue_ranges = c;
      if (knob == 4) t.vox_no_merge = c;
      float ms = 0.f;
      if ((rc = time_with(t, &ms)) != LOD_OK) break;
      if (ms < win_ms) {
        win_ms = ms;
        win = t;
      }
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc != LOD_OK) {
    lodk::set_tuning(before);
    return rc;
  }
  lodk::set_tuning(win);
  *best = win;
  if (best_ms) *best_ms = win_ms;
  return LOD_OK;
}

int lod_profile_enable(int on) { return lodk::profile_enable(on != 0); }
int lod_profile_reset(void) { return lodk::profile_reset(); }
int lod_profile_read(lod_kernel_stat_t* stats, uint32_t capacity, uint32_t* n_stats) {
  if (!n_stats) return LOD_ERR_INVALID_ARG;
  return lodk::profile_read(stats, capacity, n_stats);
}
uint64_t lod_launch_count(void) { return lodk::launch_count(); }

const char* lod_error_string(int status) {
  switch (status) {
    case LOD_OK: return "ok";
    case LOD_NOT_READY: return "not ready";
    case LOD_ERR_INVALID_ARG: return "invalid argument";
    case LOD_ERR_OOM: return "device out of memory";
    case LOD_ERR_BUDGET: return "request exceeds the HBM budget";
    case LOD_ERR_CUDA: return "CUDA error";
    case LOD_ERR_TIMEOUT: return "timed out";
    case LOD_ERR_INTERNAL: return "internal consistency check failed";
    default: return "unknown status";
  }
}

}  // extern "C"

// ------------------------------------------------------------------ serving

namespace {

struct Request {
  uint64_t ticket = 0;
  const lod_point_t* d_points = nullptr;
  uint64_t n = 0;
  lod_params_t params;
  uint64_t est = 0;
  bool done = false;
  int status = LOD_NOT_READY;
  lod_result_t* result = nullptr;
};

}  // namespace

struct lod_server {
  lod_server_config_t cfg;
  int device = 0;
  std::shared_ptr<Budget> budget = std::make_shared<Budget>();
  std::mutex mu;  // queue + table
  std::condition_variable cv_done;
  std::deque<std::shared_ptr<Request>> queue;
  std::unordered_map<uint64_t, std::shared_ptr<Request>> table;
  std::vector<std::thread> workers;
  uint64_t next_ticket = 1;
  bool stop = false;

  void worker_main() {
    cudaSetDevice(device);
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return;
    // Each worker builds on its own stream and keeps that stream's scratch
    // workspace between builds; the workspace's bytes stay counted against
    // the budget (ws_acc), so a request only needs what exceeds them.
    uint64_t ws_acc = 0, need = 0;
    int blocked = 0;
    for (;;) {
      std::shared_ptr<Request> rq;
      bool trim = false;
      {
        // admission: FIFO head, once it fits into what the budget has left
        std::unique_lock<std::mutex> lk(budget->mu);
        for (;;) {
          {
            std::lock_guard<std::mutex> qk(mu);
            if (!queue.empty()) {
              auto& h = queue.front();
              need = h->est > ws_acc ? h->est - ws_acc : 0;
              if (budget->in_use + need <= budget->limit) {
                rq = h;
                queue.pop_front();
                budget->in_use += need;
                blocked = 0;
              } else if (ws_acc && ++blocked >= 2) {
                // the budget is short and this worker's idle workspace holds
                // part of it: give the workspace back
                trim = true;
              } else if (stop) {
                // shutting down and the budget is held by resident results
                h->status = LOD_ERR_BUDGET;
                h->done = true;
                queue.pop_front();
                cv_done.notify_all();
                continue;
              }
            } else if (stop) {
              break;
            }
          }
          if (rq || trim) break;
          budget->cv.wait_for(lk, std::chrono::milliseconds(50));
        }
      }
      if (trim) {
        cudaStreamSynchronize(st);
        lodk::release_workspace(st);
        budget->release(ws_acc);
        ws_acc = 0;
        blocked = 0;
        continue;
      }
      if (!rq) break;
      lodk::TileInput ti{rq->d_points, rq->n};
      std::shared_ptr<lodk::SharedBuffers> sh;
      std::vector<lodk::TileResult> tr;
      int rc = lodk::run_build(&ti, 1, rq->params, st, &sh, &tr, nullptr);
      lod_result_t* res = nullptr;
      if (rc == LOD_OK) {
        res = make_result(sh, tr[0], rq->params.mode, sh->bytes);
        if (!res) rc = LOD_ERR_OOM;
      }
      // the build's transient footprint is returned; the result and the
      // worker's workspace stay counted
      const uint64_t ws_now = lodk::workspace_bytes(st);
      {
        std::lock_guard<std::mutex> lk(budget->mu);
        budget->in_use -= std::min(budget->in_use, need + ws_acc);
        budget->in_use += ws_now;
        ws_acc = ws_now;
        if (res) {
          budget->in_use += res->bytes;
          res->budget = budget;
        }
      }
      budget->cv.notify_all();
      {
        std::lock_guard<std::mutex> lk(mu);
        rq->status = rc;
        rq->result = res;
        rq->done = true;
      }
      cv_done.notify_all();
    }
    cudaStreamSynchronize(st);
    lodk::release_workspace(st);
    budget->release(ws_acc);
    cudaStreamDestroy(st);
  }
};

extern "C" {

int lod_server_create(const lod_server_config_t* cfg, lod_server_t** out) {
  if (!cfg || !out || cfg->max_inflight == 0 || cfg->hbm_budget_bytes == 0) return LOD_ERR_INVALID_ARG;
  lod_server_t* s = new (std::nothrow) lod_server_t();
  if (!s) return LOD_ERR_OOM;
  s->cfg = *cfg;
  cudaGetDevice(&s->device);
  s->budget->limit = cfg->hbm_budget_bytes;
  try {
    for (uint32_t i = 0; i < cfg->max_inflight; ++i) s->workers.emplace_back(&lod_server::worker_main, s);
  } catch (...) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stop = true;
    }
    for (auto& w : s->workers) w.join();
    delete s;
    return LOD_ERR_OOM;
  }
  *out = s;
  return LOD_OK;
}

int lod_submit(lod_server_t* s, const lod_point_t* d_points, uint64_t n, const lod_params_t* params,
               uint64_t* ticket) {
  if (!s || !ticket || (n && !d_points) || n > 0xFFFFFFFFull) return LOD_ERR_INVALID_ARG;
  auto rq = std::make_shared<Request>();
  rq->d_points = d_points;
  rq->n = n;
  rq->params = params ? *params : defaults();
  if (!lodk::valid_params(rq->params)) return LOD_ERR_INVALID_ARG;
  rq->est = lodk::estimate_build_bytes(n, rq->params);
  if (rq->est > s->budget->limit) return LOD_ERR_BUDGET;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return LOD_ERR_INVALID_ARG;
    rq->ticket = s->next_ticket++;
    s->table[rq->ticket] = rq;
    s->queue.push_back(rq);
  }
  s->budget->cv.notify_all();
  *ticket = rq->ticket;
  return LOD_OK;
}

static int take_if_done(lod_server_t* s, uint64_t ticket, lod_result_t** out, bool* found) {
  auto it = s->table.find(ticket);
  *found = it != s->table.end();
  if (!*found) return LOD_ERR_INVALID_ARG;
  if (!it->second->done) return LOD_NOT_READY;
  const int rc = it->second->status;
  if (rc == LOD_OK) *out = it->second->result;
  s->table.erase(it);
  return rc;
}

int lod_poll(lod_server_t* s, uint64_t ticket, lod_result_t** out) {
  if (!s || !out) return LOD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  bool found;
  return take_if_done(s, ticket, out, &found);
}

int lod_wait(lod_server_t* s, uint64_t ticket, uint32_t timeout_ms, lod_result_t** out) {
  if (!s || !out) return LOD_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
  for (;;) {
    bool found;
    const int rc = take_if_done(s, ticket, out, &found);
    if (rc != LOD_NOT_READY) return rc;
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
      const int rc2 = take_if_done(s, ticket, out, &found);
      return rc2 == LOD_NOT_READY ? LOD_ERR_TIMEOUT : rc2;
    }
  }
}

uint64_t lod_server_bytes_in_use(const lod_server_t* s) {
  if (!s) return 0;
  std::lock_guard<std::mutex> lk(s->budget->mu);
  return s->budget->in_use;
}

int lod_server_destroy(lod_server_t* s) {
  if (!s) return LOD_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->budget->cv.notify_all();
  for (auto& w : s->workers) w.join();
  // requests finished but never polled: release their results
  for (auto& kv : s->table)
    if (kv.second->done && kv.second->result) lod_free(kv.second->result);
  delete s;
  return LOD_OK;
}

}  // extern "C"
