// Host-side launch wrappers of the LOD kernels (internal).
#pragma once

#include "common.cuh"

namespace lodk {

// Counts kernel launches of the library (lod_launch_count); every launch
// site calls it once per kernel it launches.
void note_launch();

struct PyrJob {
  uint32_t src;    // source id
  uint32_t lvl;    // up: bottom level of the block; down: top level of the block
  uint32_t block;  // block index (cell index at the block's top level)
};

// ----- split (Section 4.1) -----
cudaError_t launch_bbox(const TileDesc* tiles, const uint32_t* chunk_tile, uint64_t n_chunks,
                        const uint64_t* tile_chunk0, int* bbox, int grid, cudaStream_t st);
cudaError_t launch_roots(const TileDesc* tiles, const int* bbox, SrcDesc* srcs, uint32_t n_tiles, uint32_t T,
                         uint32_t max_depth, unsigned int* abort, cudaStream_t st);
cudaError_t launch_count(const BuildArgs& a, const uint32_t* chunk_src, const unsigned long long* n_chunks,
                         int grid, cudaStream_t st);
cudaError_t launch_pyr_up(const BuildArgs& a, const PyrJob* jobs, uint32_t n_jobs, cudaStream_t st);
cudaError_t launch_pyr_down(const BuildArgs& a, const PyrJob* jobs, uint32_t n_jobs, uint32_t next_base,
                            uint32_t next_cap, uint32_t next_buf, DevCounters* ctr, cudaStream_t st);
cudaError_t launch_scatter(const BuildArgs& a, const uint32_t* chunk_src, const unsigned long long* n_chunks,
                           uint32_t round, int grid, cudaStream_t st);
cudaError_t launch_nodes(const BuildArgs& a, lod_node_t* nodes, NodeAux* aux, uint32_t* lvl_start,
                         uint32_t* n_nodes, unsigned long long* leaf_cap, DevCounters* ctr,
                         const unsigned long long* refined, cudaStream_t st);

// ----- voxel sampling (Section 4.2) -----
struct VoxLevel {
  uint32_t level;              // parent level l; items are the nodes at level l + 1
  uint32_t n_items;
  const uint32_t* item_prefix; // n_tiles + 1 prefix of items per tile
  const uint32_t* lvl_start;   // n_tiles x (kMaxLevels + 1)
  lod_node_t* nodes;
  NodeAux* aux;
  int4* stage_out;             // staging records written by this level
  ulonglong2* stage_out_sum;   // filtered mode: exact sums, parallel to stage_out
  uint64_t stage_cap;
  const int4* stage_in;        // staging of the level below (items at level l + 2)
  const ulonglong2* stage_in_sum;
  int4* dense;                 // public voxel array
  unsigned long long* stage_used;
  uint4* units;                // queue of {item, range r, ranges P} of items with many occupied cells
  uint32_t unit_cap;
  uint64_t dense_cap;          // records the public voxel array holds
  unsigned long long* vstate;  // [0] voxels of the levels done so far, [1] nonzero: dense_cap too small
  // weighted mode (Section 4.2.4): parents of this level and the per-CTA
  // dense grids (2^21 cells each: four u64 sums, a u32 count, a touched list)
  const uint32_t* parent_prefix;  // n_tiles + 1 prefix of parents (nodes at level l) per tile
  uint32_t n_parents;
  unsigned long long* wgrid;
  uint32_t* wcnt;
  uint32_t* wtouch;
  ulonglong2* root_sums;  // filtered: exact sums of the top level's voxels, parallel to dense (or null)
  // rank ranges: an item whose occupied cells need P >= queue_ranges
  // accumulate passes hands ranges 1..P-1 to the partition kernel (0xFFFFFFFF:
  // never); range_cells (nonzero) caps the cells of one pass below what the
  // shared memory holds
  uint32_t queue_ranges;
  uint32_t range_cells;
  const uint32_t* order;  // the order in which the first-attempt kernel takes the items (null: node order)
  uint32_t* next_order;   // written by the level scan: the order of the next level's items (or null)
  uint32_t no_merge;  // 1: filtered samples of a warp that share a cell are not merged before the table
};
cudaError_t launch_vox(const BuildArgs& a, const VoxLevel& v, DevCounters* ctr, cudaStream_t st);
// Section 4.2.4: one persistent CTA per grid over the parents of a level.
cudaError_t launch_wvox(const BuildArgs& a, const VoxLevel& v, DevCounters* ctr, int ctas, cudaStream_t st);
size_t wgrid_bytes_per_cta();
cudaError_t launch_level_scan(const BuildArgs& a, const VoxLevel& v, const uint32_t* parent_prefix,
                              uint32_t n_parents, unsigned long long* tile_voxels, DevCounters* ctr,
                              cudaStream_t st);
cudaError_t launch_copy_items(const BuildArgs& a, const VoxLevel& v, cudaStream_t st);
cudaError_t launch_unwide(const BuildArgs& a, const uint32_t* tiles, uint32_t n_tiles, uint32_t max_points,
                          cudaStream_t st);
cudaError_t launch_voxel_points(const TileDesc* tiles, uint32_t n_tiles, const lod_node_t* nodes,
                                const uint32_t* n_nodes, uint32_t max_nodes, const int4* dense, int4* out,
                                cudaStream_t st);
cudaError_t launch_gather_voxels(const lod_node_t* nodes, uint32_t n_nodes, const uint64_t* new_off,
                                 const int4* src, int4* dst, cudaStream_t st);

int vox_smem_bytes();
void vox_capacities(uint32_t* small, uint32_t* narrow, uint32_t* wide, uint32_t* pick);
int vox_init();

// ----- out-of-core build (Section 7) -----
struct OocGrid {  // top grid: 8^D cells at depth D below the root cube [min, min + 2^L)^3
  int32_t min[3];
  uint32_t L, D;
};
struct MergeSeg {  // the samples one child gives its parent
  const int4* recs;         // points (x, y, z, rgba) or voxels (cell, rgba, count, pick_index)
  const ulonglong2* sums;   // voxels, filtered mode: packed exact sums
  const uint32_t* idx;      // points, single-sample modes: input indices
  uint32_t n;
  uint32_t kind;            // 0 points, 1 voxels
  uint32_t octant;          // voxels: the child's octant in the parent
  uint32_t pad;
};
struct MergeJob {  // one root-side node
  int32_t min[3];
  uint32_t log2, level, seg0, nseg, pad;
};
struct MergeOut {
  unsigned long long* grid;  // per CTA: kGridCells x 4 u64
  uint32_t* cnt;             // per CTA: kGridCells
  uint32_t* touched;         // per CTA: kGridCells
  unsigned int* job_head;
  int4* recs;                // voxels of every job, bump-allocated
  ulonglong2* sums;          // filtered: their packed exact sums
  unsigned long long* used;
  uint64_t cap;
  ulonglong2* result;        // per job: {first voxel, count}
  unsigned int* error;
};
cudaError_t launch_ooc_bbox(const int4* pts, uint64_t n, int* box, int sms, cudaStream_t st);
cudaError_t launch_ooc_count(const int4* pts, uint64_t n, const OocGrid& g, unsigned int* counts, int sms,
                             cudaStream_t st);
cudaError_t launch_ooc_chunk_of(const int4* pts, uint64_t n, const OocGrid& g, const uint32_t* cell_chunk,
                                uint32_t n_chunks, uint32_t* chunk_of, unsigned int* hist, unsigned int* err, int sms,
                                cudaStream_t st);
cudaError_t launch_ooc_partition(const int4* pts, uint64_t n, uint32_t first, const uint32_t* chunk_of,
                                 uint32_t n_chunks, unsigned int* cursor, int4* out, uint32_t* out_idx, int sms,
                                 cudaStream_t st);
cudaError_t launch_merge(uint32_t mode, const MergeJob* jobs, uint32_t n_jobs, const MergeSeg* segs,
                         const MergeOut& o, int ctas, cudaStream_t st);

// ----- rendering (Section 5) -----
cudaError_t launch_render(const lod_node_t* nodes, uint32_t n_nodes, const int4* points, const int4* voxels,
                          const lod_camera_t& cam, uint8_t* visible, unsigned int* n_visible,
                          unsigned long long* fb, unsigned long long* drawn, int sms, cudaStream_t st);

}  // namespace lodk
