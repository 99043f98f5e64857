// Host orchestration of one (batched) LOD build — internal.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <vector>

#include "lod.h"

namespace lodk {

// Device buffers produced by one build and shared by its results.
struct SharedBuffers {
  int device = 0;
  void* points = nullptr;   // leaf points of all tiles
  void* index = nullptr;    // original indices (or null)
  void* nodes = nullptr;    // node tables of all tiles
  void* voxels = nullptr;   // voxels of all tiles
  void* voxel_points = nullptr;  // full-precision picked points, parallel to voxels (or null)
  void* root_sums = nullptr;     // BuildOptions::keep_root_sums: packed exact sums parallel to voxels
  void* input = nullptr;    // owned copy of host input (lod_build_from_host), or null
  uint64_t bytes = 0;
  ~SharedBuffers();
};

struct TileResult {
  uint64_t pt_base = 0, n_points = 0;
  uint64_t node_base = 0;
  uint32_t n_nodes = 0, n_levels = 0;
  uint64_t n_voxels = 0;
};

struct BuildStats {
  uint32_t rounds = 0;       // counting rounds (1 + refinement rounds)
  uint32_t host_syncs = 0;
  uint32_t launches = 0;
  uint64_t voxels = 0;
  uint64_t nodes = 0;
};

struct TileInput {
  const lod_point_t* d_points;
  uint64_t n;
  // Optional, for builds of one part of a larger cloud (out-of-core chunks):
  const uint32_t* d_index = nullptr;  // input index of every point (device), used by the pick rules and
                                      // reported as pick_index / leaf index; null: the position in d_points
  uint32_t index_bound = 0;           // indices are < index_bound (0: n)
  const int32_t* cube = nullptr;      // host: min x, y, z and log2 edge of the root cube (null: bounding box)
  uint32_t level0 = 0;                // octree level of the root (the random pick draws per level)
};

struct BuildOptions {
  bool keep_root_sums = false;  // filtered mode: keep the exact sums of every root's voxels
};

// Runs the complete build of n_tiles independent tiles on stream st.
// On LOD_OK fills *shared and tiles_out (one entry per tile).  With
// use_workspace the build's scratch comes from device memory kept for the
// stream between builds (see workspace_bytes).
int run_build(const TileInput* tiles, uint32_t n_tiles, const lod_params_t& params, cudaStream_t st,
              std::shared_ptr<SharedBuffers>* shared, std::vector<TileResult>* tiles_out, BuildStats* stats,
              bool use_workspace = true, const BuildOptions& opt = BuildOptions());

// Device bytes kept for stream st's builds between builds, and their release
// (the stream must be idle).
uint64_t workspace_bytes(cudaStream_t st);
void release_workspace(cudaStream_t st);

// Parameter checks shared by every entry point, and whether a build keeps
// the input index of every leaf point.
bool valid_params(const lod_params_t& p);
bool keeps_index(const lod_params_t& p);

// Rough device footprint (bytes) of building n points (result + temporaries).
uint64_t estimate_build_bytes(uint64_t n, const lod_params_t& params);
// Rough device footprint of a finished result of n points.
uint64_t estimate_result_bytes(uint64_t n, const lod_params_t& params);

// Default depth of a tile's first counting grid (8^d cells) for n points,
// before the cap by the cube's size (a set root_depth is ignored here).
uint32_t default_root_depth(uint64_t n, uint32_t T, uint32_t max_depth);

// Process-wide tuning (see lod_set_tuning in lod.h).
int set_tuning(const lod_tuning_t& t);
int get_tuning(lod_tuning_t* t);

// Process-wide kernel profiling (see lod_profile_* in lod.h).
int profile_enable(bool on);
int profile_reset();
int profile_read(lod_kernel_stat_t* out, uint32_t cap, uint32_t* n);
uint64_t launch_count();

// The out-of-core build of lod_build_out_of_core (ooc.cu).
int build_out_of_core(const lod_point_t* h, uint64_t n, const lod_params_t& prm, const lod_ooc_config_t& cfg,
                      cudaStream_t st, std::shared_ptr<SharedBuffers>* sh_out, TileResult* tr_out);

// A library-owned non-blocking stream of the current device used to
// release buffers asynchronously.
cudaStream_t free_stream();

}  // namespace lodk
