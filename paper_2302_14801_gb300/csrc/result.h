// The result object behind the C ABI's lod_result_t, and the budget a
// server counts resident results against — internal.
#pragma once

#include <condition_variable>
#include <memory>
#include <mutex>
#include <new>

#include "engine.h"

// Budget accounting shared between a server and the results it returned
// (results may outlive the server).
struct Budget {
  std::mutex mu;
  std::condition_variable cv;
  uint64_t limit = 0;
  uint64_t in_use = 0;
  void release(uint64_t b) {
    {
      std::lock_guard<std::mutex> lk(mu);
      in_use = b > in_use ? 0 : in_use - b;
    }
    cv.notify_all();
  }
};

struct lod_result {
  std::shared_ptr<lodk::SharedBuffers> sh;
  lodk::TileResult tr;
  uint32_t mode = 0;
  uint64_t bytes = 0;
  std::shared_ptr<Budget> budget;  // set when a server accounts for this result
};

inline lod_result_t* make_result(const std::shared_ptr<lodk::SharedBuffers>& sh, const lodk::TileResult& tr,
                                 uint32_t mode, uint64_t share) {
  lod_result_t* r = new (std::nothrow) lod_result_t();
  if (!r) return nullptr;
  r->sh = sh;
  r->tr = tr;
  r->mode = mode;
  r->bytes = share;
  return r;
}

