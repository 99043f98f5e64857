/*
 * lod.h — C ABI of the GB300 (sm_103a) LOD builder for point clouds.
 *
 * The library builds the hybrid voxel-point octree of "GPU-Accelerated LOD
 * Generation for Point Clouds" (Schuetz, Kerbl, Klaus, Wimmer 2023):
 *   - Section 4.1: the input points are split top-down into an octree whose
 *     leaves hold at most T original points (hierarchical counting sort);
 *   - Section 4.2: every inner node is then filled bottom-up with the
 *     occupied cells ("voxels") of a 128^3 grid laid over its cube.
 * Sampling modes:
 *   - LOD_FILTER: the cell-wise average of Section 4.2.3, made exact — each
 *     voxel carries the integer mean (rounded half up) of the RGB of all
 *     original points inside its cell, accumulated as unsigned 64-bit sums;
 *     alpha is 255.
 *   - LOD_PICK: replaces the random pick of Section 4.2.2 (Listing 1) by an
 *     order-independent rule — each voxel keeps the original point of
 *     minimal splitmix64(input index); pick_index is that index.
 *   - LOD_WEIGHTED: the neighbourhood-weighted average of Section 4.2.4 —
 *     an inner node samples its children's samples (points of leaf
 *     children; voxels of inner children at their cell centres with their
 *     8-bit colours); each sample adds weight max(0, 1 - distance to the
 *     cell centre in cells) times its colour to the cells of the 2x2x2
 *     block around it and occupies the cell it lies in; an occupied cell's
 *     colour is its weighted sum over its weight sum, rounded half up,
 *     alpha 255.  Weights are fp32, rounded to 24 fractional bits and
 *     summed exactly, so results are deterministic; they agree with an
 *     exact-arithmetic evaluation except where a mean lies within about
 *     1e-5 of a rounding boundary.
 *   - LOD_FIRST: first come (Section 4.2.1), with input order defining
 *     "first" — each voxel keeps its cell's point of smallest input index.
 *   - LOD_RANDOM: the random pick of Section 4.2.2 with Listing 1's 32-bit
 *     key (12 random bits above the low 20 bits of the sample index, the
 *     largest key kept), drawn afresh at every level from the children's
 *     samples; the random bits are the top 12 of the high half of
 *     splitmix64(level << 32 | input index), equal keys go to the larger
 *     index.
 *
 * Every entry point is extern "C", takes plain pointers and sizes, and
 * returns an int status (LOD_OK on success).  Pointers documented as
 * "device" must be CUDA device memory of the current device; "host" means
 * ordinary (optionally pinned) host memory.  A stream argument is a
 * cudaStream_t passed as void* (NULL = the legacy default stream).
 *
 * Ownership.  Inputs stay owned by the caller and must remain valid and
 * unmodified until the call that consumes them has completed (for
 * lod_build: until it returns; for lod_submit: until lod_poll/lod_wait
 * returns the result).  Every output buffer is owned by an lod_result_t and
 * released by lod_free().  Nothing is retained after lod_free().
 *
 * Thread safety.  lod_build / lod_build_batched / lod_build_from_host may be
 * called from several host threads on different streams.  A server object
 * (lod_server_t) is internally synchronised.
 */
#ifndef LOD_H_
#define LOD_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
enum {
  LOD_OK = 0,
  LOD_NOT_READY = 1,       /* lod_poll: the request has not finished yet      */
  LOD_ERR_INVALID_ARG = 2, /* bad pointer, size, alignment or parameter       */
  LOD_ERR_OOM = 3,         /* device allocation failed                        */
  LOD_ERR_BUDGET = 4,      /* request can never fit the server's HBM budget   */
  LOD_ERR_CUDA = 5,        /* a CUDA call or kernel launch failed             */
  LOD_ERR_TIMEOUT = 6,     /* lod_wait: timed out                             */
  LOD_ERR_INTERNAL = 7     /* internal consistency check failed               */
};

/* ------------------------------------------------------------------ data */

/* Input point, 16 bytes, array-of-structs.  rgba is RGBA8 with R in the low
 * byte and A in the high byte.  Arrays of points must be 16-byte aligned
 * (cudaMalloc and torch allocations are). */
typedef struct lod_point {
  int32_t x, y, z;
  uint32_t rgba;
} lod_point_t;

enum { LOD_FILTER = 0, LOD_PICK = 1, LOD_WEIGHTED = 2, LOD_FIRST = 3, LOD_RANDOM = 4 };

/* LOD_FLAG_LEAF_INDEX: keep the original input index of every leaf point
 * (always kept in the single-sample modes LOD_PICK, LOD_FIRST and
 * LOD_RANDOM, whose sampling rules need it).
 * LOD_FLAG_FULL_PRECISION: the full-precision variant of Section 7 for the
 * single-sample modes — every voxel also carries the input point it picked,
 * unquantised (see lod_result_voxel_points); other modes reject the flag. */
enum { LOD_FLAG_LEAF_INDEX = 1u, LOD_FLAG_FULL_PRECISION = 2u };

/* Build parameters.
 *   leaf_threshold  T >= 1: a node with more than T points is split into its
 *                   non-empty octants (Section 3; the paper uses T = 50k).
 *   mode            LOD_FILTER, LOD_PICK, LOD_WEIGHTED, LOD_FIRST or
 *                   LOD_RANDOM.
 *   max_depth       <= 32: nodes at this level are leaves even above T.
 *                   Unit cubes (edge 1) are leaves too; such leaves may hold
 *                   more than T points and are flagged LOD_NODE_OVERFULL.
 *   flags           LOD_FLAG_* bits (unknown bits are rejected). */
typedef struct lod_params {
  uint32_t leaf_threshold;
  uint32_t mode;
  uint32_t max_depth;
  uint32_t flags;
} lod_params_t;

enum { LOD_NODE_LEAF = 1u, LOD_NODE_OVERFULL = 2u };

/* One octree node, 56 bytes.
 *   min, log2_size  the node's cube [min, min + 2^log2_size)^3.  The root's
 *                   min is the bounding-box minimum and its edge the smallest
 *                   power of two strictly greater than the largest extent
 *                   (N = 0: one empty leaf at the origin with edge 1).
 *   level           0 for the root.
 *   child_mask      bit k set if octant k has a child; octant
 *                   k = 4*bx + 2*by + bz, b = upper half along x, y, z.
 *   flags           LOD_NODE_LEAF / LOD_NODE_OVERFULL.
 *   parent          node index, 0xFFFFFFFF for the root.
 *   first_child     index of the child of the lowest set octant; the
 *                   children follow contiguously in octant order;
 *                   0xFFFFFFFF for leaves.
 *   point_offset,   the node's subtree owns the contiguous leaf-point range
 *   point_count     [point_offset, point_offset + point_count).
 *   voxel_offset,   inner nodes: their voxels (index into the view's voxel
 *   voxel_count     array); leaves: 0, 0.
 * Nodes are ordered breadth first; within a level by parent, then octant. */
typedef struct lod_node {
  int32_t min[3];
  uint8_t level, log2_size, child_mask, flags;
  uint32_t parent, first_child;
  uint64_t point_offset, point_count;
  uint64_t voxel_offset;
  uint32_t voxel_count, reserved;
} lod_node_t;

/* One voxel of an inner node, 16 bytes (Section 4.2).
 *   cell        x | y << 7 | z << 14, the 128^3 grid cell relative to the
 *               node's cube (cell edge 2^log2_size / 128).
 *   rgba        LOD_FILTER: rounded-half-up mean RGB, A = 255;
 *               LOD_WEIGHTED: rounded-half-up weighted mean RGB, A = 255;
 *               single-sample modes: colour of the picked input point.
 *   count       number of original points inside the cell.
 *   pick_index  single-sample modes: input index of the picked point;
 *               LOD_FILTER, LOD_WEIGHTED: 0xFFFFFFFF.
 * Voxel order within a node is unspecified. */
typedef struct lod_voxel {
  uint32_t cell, rgba, count, pick_index;
} lod_voxel_t;

/* Read-only view of a result.  All pointers are device pointers owned by
 * the result.
 *   points      n_points leaf points in layout order: leaves are laid out
 *               depth first in octant order (every subtree is contiguous);
 *               order inside a leaf is unspecified.
 *   point_index original input index of each leaf point, or NULL if not kept.
 *   voxels      base of the voxel array that nodes[i].voxel_offset indexes;
 *               n_voxels is the number of voxels of this result.  Results of
 *               one lod_build_batched call share one voxel array. */
typedef struct lod_view {
  const lod_node_t* nodes;
  uint32_t n_nodes;
  uint32_t n_levels;
  const lod_point_t* points;
  const uint32_t* point_index;
  uint64_t n_points;
  const lod_voxel_t* voxels;
  uint64_t n_voxels;
  uint32_t mode;
  uint32_t reserved;
} lod_view_t;

typedef struct lod_result lod_result_t;

/* ------------------------------------------------------------------- API */

/* Fill *p with the defaults: T = 50000, LOD_FILTER, max_depth 21, flags 0. */
int lod_params_init(lod_params_t* p);

/* Build the LOD octree of n device points (Sections 4.1 and 4.2).
 *   d_points  device, 16-byte aligned, n records; read only.  n < 2^32.
 *   params    host; NULL selects the defaults.
 *   stream    cudaStream_t as void*; all device work is ordered on it.
 *   out       host; receives a new result on LOD_OK (untouched otherwise).
 * Blocks the calling host thread until the build has completed on the
 * stream.  Errors: LOD_ERR_INVALID_ARG, LOD_ERR_OOM, LOD_ERR_CUDA. */
int lod_build(const lod_point_t* d_points, uint64_t n, const lod_params_t* params, void* stream,
              lod_result_t** out);

/* Same, with the points in host memory: they are copied to the device on
 * the stream first (pinned memory makes the copy asynchronous). */
int lod_build_from_host(const lod_point_t* h_points, uint64_t n, const lod_params_t* params,
                        void* stream, lod_result_t** out);

/* Build n_tiles independent octrees in one batched pass: every stage runs
 * as one launch over the work of all tiles (one device work list).  No
 * passage of the paper defines this call (the paper builds one cloud at a
 * time); it serves workloads of many independent scan tiles, and each
 * tile's octree is the one Sections 4.1 and 4.2 define for that tile.
 *   d_tiles   host array of n_tiles device pointers (each 16-byte aligned).
 *   n         host array of n_tiles point counts (each < 2^32).
 *   out       host array of n_tiles result pointers, filled on LOD_OK.
 * Each result is freed separately; they share device buffers internally,
 * which are released when the last of them is freed.  Results are
 * identical to n_tiles separate lod_build calls. */
int lod_build_batched(const lod_point_t* const* d_tiles, const uint64_t* n, uint32_t n_tiles,
                      const lod_params_t* params, void* stream, lod_result_t** out);

/* Fill *view (host) with the device pointers and sizes of result r. */
int lod_result_view(const lod_result_t* r, lod_view_t* view);

/* Copy a result to host memory (stream-ordered; synchronises before
 * returning).  Any output pointer may be NULL to skip that part.
 *   nodes   n_nodes records; voxel_offset is rewritten to index `voxels`.
 *   points  n_points leaf points;  index  n_points indices (needs a kept
 *           index, else LOD_ERR_INVALID_ARG);
 *   voxels  n_voxels records, grouped per node in node order. */
int lod_result_copy_to_host(const lod_result_t* r, lod_node_t* nodes, lod_point_t* points,
                            uint32_t* index, lod_voxel_t* voxels, void* stream);

/* Full-precision variant (Section 7; built with LOD_FLAG_FULL_PRECISION):
 * *d_points (device, owned by the result) receives an array parallel to
 * the view's voxel array — element voxel_offset + j of a node is the input
 * point (x, y, z, rgba) that voxel j of that node picked, i.e. the input
 * record at its pick_index.  Returns LOD_ERR_INVALID_ARG when the result
 * was built without the flag. */
int lod_result_voxel_points(const lod_result_t* r, const lod_point_t** d_points);

/* Copy those points to host memory in the order lod_result_copy_to_host
 * gives the voxels (grouped per node in node order); `points` holds the
 * result's n_voxels records.  Synchronises `stream` before returning. */
int lod_result_copy_voxel_points_to_host(const lod_result_t* r, lod_point_t* points, void* stream);

/* Device bytes held by a result (its share of shared buffers included). */
uint64_t lod_result_device_bytes(const lod_result_t* r);

/* Release a result; NULL is a no-op. */
void lod_free(lod_result_t* r);

/* Static description of a status code. */
const char* lod_error_string(int status);

/* ------------------------------------------------------ device memory */

/* Every build keeps its scratch buffers (counting pools, ping-pong and
 * staging arrays: up to about 100 bytes per input point) in a workspace
 * tied to (current device, stream), reused by the next build on that stream
 * without allocator calls; results come from the device's stream-ordered
 * pool, which the library sets to keep freed memory for reuse.  The paper
 * has no counterpart (its buffers are allocated once, Section 4.1.6).
 * lod_scratch_bytes: device bytes the workspace of `stream` holds now.
 * lod_trim: waits for `stream` to finish its work, frees its workspace and
 *   returns the pool's unused memory to the device.  Results stay valid;
 *   the next build on the stream allocates its scratch again.  A workspace
 *   that a build on another thread is using at that moment is left alone.
 *   Returns LOD_ERR_CUDA if the synchronisation reports an error. */
uint64_t lod_scratch_bytes(void* stream);
int lod_trim(void* stream);

/* --------------------------------------------------------- out of core */

/* Out-of-core build (Section 7: a cloud too large to build in device memory
 * at once is split into chunks that are built one batch at a time, and the
 * coarsest nodes above the chunks are filled afterwards).
 *   chunk_points   the largest chunk (subtree) built at once; >= T; 0: 10M.
 *                  A chunk root is a node of at most chunk_points points, a
 *                  leaf of the octree, or a node 8 levels below the root
 *                  (such chunks may be larger).
 *   stream_points  points moved host -> device per transfer (0: 16M).
 *   batch_points   points of the chunks built together (0: 256M). */
typedef struct lod_ooc_config {
  uint64_t chunk_points;
  uint64_t stream_points;
  uint64_t batch_points;
} lod_ooc_config_t;

/* Build the LOD octree of n points in host memory (h_points, read three
 * times: bounding box, top-level counts, partition into chunks) holding
 * only the output and one batch of chunks under construction in device
 * memory.  The result is identical to lod_build of the same points
 * (pick_index and leaf indices are input indices of the whole cloud) and
 * is used like any other result.  Uses page-locked host memory of 20 bytes
 * per point for the partitioned chunks.  LOD_FLAG_FULL_PRECISION is not
 * supported here (LOD_ERR_INVALID_ARG).  Blocks until done.
 * Errors: LOD_ERR_INVALID_ARG, LOD_ERR_OOM, LOD_ERR_CUDA, LOD_ERR_INTERNAL. */
int lod_build_out_of_core(const lod_point_t* h_points, uint64_t n, const lod_params_t* params,
                          const lod_ooc_config_t* cfg, void* stream, lod_result_t** out);

/* ------------------------------------------------------- no allocation */

/* Root cube of each of n_tiles point clouds, computed without allocating
 * any device memory.  The paper has no counterpart to this call; it exists
 * for callers that cannot call cudaMalloc (a plug-in whose host application
 * owns all device memory, a render loop that must not let an allocation
 * synchronise the device, code held to a fixed memory budget).
 *   d_tiles  host array of n_tiles device pointers (16-byte aligned; may be
 *            NULL where n[t] == 0).
 *   n        host array of n_tiles point counts (each < 2^32).
 *   n_tiles  1 .. 4096; larger batches return LOD_ERR_INVALID_ARG.
 *   d_cubes  device, caller-owned, 4 int32 per tile: min x, y, z of the
 *            root cube (the bounding-box minimum) and log2 of its edge (the
 *            smallest power of two strictly greater than the largest
 *            extent) — the root node lod_build produces; an empty tile
 *            gives 0, 0, 0, 0.
 *   stream   cudaStream_t as void*; the call is asynchronous on it.
 * Scratch: a 192 KB array in static device memory, one per device that
 * loads the library, held until the process exits.  The first call on a
 * device looks up that array's device address and keeps it; make that
 * first call before any stream capture, and do not use the call after
 * cudaDeviceReset in the same process.  All calls share the array, so
 * calls whose work overlaps on the GPU race with one another: issue them
 * on one stream. */
int lod_root_cubes_noalloc(const lod_point_t* const* d_tiles, const uint64_t* n, uint32_t n_tiles,
                           int32_t* d_cubes, void* stream);

/* --------------------------------------------------------------- tuning */

/* Launch and tiling parameters that change speed, never results.  They are
 * process-wide; set them while no build is running.  Zero means "default".
 *   root_depth      depth d of each tile's first counting grid (8^d cells,
 *                   1..8, still capped by the cube and max_depth); default:
 *                   one more level than a surface-like cloud needs to reach
 *                   the leaf threshold.
 *   stream_ctas_per_sm  CTAs per SM of the streaming passes (default: 4
 *                   for builds of at least 128 chunks of 4096 points per
 *                   CTA of a 2-per-SM grid, about 160M points on 152 SMs;
 *                   2 below).
 *   dense_bins_max  counting grids of at most this many cells are counted
 *                   in a dense shared-memory histogram, larger ones through
 *                   per-CTA shared-memory hash tables (8..4096, a power of
 *                   8; default 4096).
 *   vox_queue_ranges  the voxel pass numbers an item's occupied cells in
 *                   cell order and accumulates them in ranges of what one
 *                   CTA's shared memory holds (5120 to 10240 cells); an
 *                   item needing P >= vox_queue_ranges ranges hands ranges
 *                   2..P to other SMs (default 4; 1: every range stays with
 *                   the item's CTA; at most 4096).
 *   graph_voxel_levels  1: every build captures the launches of all its
 *                   voxel levels (which need no host round trip between
 *                   them) into one CUDA graph and launches that (0: plain
 *                   launches, the default).  Ignored while profiling.
 *   vox_no_merge    1: in filtered mode the lanes of a warp whose points share
 *                   a cell do not add their colours together before updating
 *                   the table (0: they do, the default).
 *   vox_range_cells  at most this many cells per accumulate range of the
 *                   voxel pass (1..262144; default: what shared memory
 *                   holds); smaller values only add passes. */
typedef struct lod_tuning {
  uint32_t root_depth;
  uint32_t stream_ctas_per_sm;
  uint32_t dense_bins_max;
  uint32_t vox_queue_ranges;
  uint32_t graph_voxel_levels;
  uint32_t vox_no_merge;
  uint32_t vox_range_cells;
  uint32_t reserved[1];  /* must be 0 */
} lod_tuning_t;

int lod_set_tuning(const lod_tuning_t* t);
int lod_get_tuning(lod_tuning_t* t);

/* Autotuner: times lod_build of the caller's cloud (device pointer, n points,
 * params; on `stream`) under candidate tunings, two builds each (the first
 * untimed), by coordinate descent from the defaults: stream_ctas_per_sm 2,
 * 3 and 4; root_depth one less and one more than the default; dense_bins_max
 * 512; vox_queue_ranges 1 (never) and 2; in filtered mode
 * vox_no_merge 1 — each knob in turn, the others held at the best so far.  Keeps the fastest with lod_set_tuning and
 * returns it in *best (and its build time in *best_ms when not NULL).
 * Results are freed; nothing else is kept.  Costs about 18 builds; like
 * lod_set_tuning it changes process-wide state, so call it while no other
 * build runs.  Returns LOD_ERR_INVALID_ARG for n == 0 or a missing pointer,
 * or the first build error (the previous tuning is then restored).  The
 * paper has no counterpart (it uses one fixed configuration, Section
 * 4.1.6). */
int lod_autotune(const lod_point_t* d_points, uint64_t n, const lod_params_t* params, void* stream,
                 lod_tuning_t* best, float* best_ms);

/* ------------------------------------------------------------ rendering */

/* Camera of lod_render.  A sample at integer position p is projected as
 * clip = view_proj * (p - origin, 1) with view_proj row-major (clip.x is
 * row 0 . (p - origin, 1)); it is drawn when clip.w > 0 and x/w, y/w, z/w
 * all lie in [-1, 1], at pixel floor((x/w * 0.5 + 0.5) * width),
 * floor((y/w * 0.5 + 0.5) * height) (clamped to the last row / column).
 * lod_pixels is the refinement threshold of Section 5 (a node's children
 * are considered when its projected bounding box spans more than this many
 * pixels; 0 selects 100, the paper's value for a 128^3 grid). */
typedef struct lod_camera {
  float view_proj[16];
  int32_t origin[3];
  uint32_t width, height;
  float lod_pixels;
  uint32_t reserved[2];
} lod_camera_t;

typedef struct lod_render_stats {
  uint32_t visible_nodes;  /* nodes drawn */
  uint32_t reserved;
  uint64_t samples_drawn;  /* voxels and points that reached a pixel */
} lod_render_stats_t;

/* Render result r into a headless framebuffer (Section 5, restated as CUDA
 * kernels instead of draw calls).  A node is drawn when it is at least
 * partly inside the view frustum and every ancestor is drawn and projects
 * larger than lod_pixels; a drawn inner node draws its voxels (at their
 * cell centres) except those in an octant whose child is drawn, a drawn
 * leaf draws its points.  Each pixel of d_framebuffer (device,
 * width * height uint64, row-major, 8-byte aligned, caller-owned) receives
 * the smallest key (float bits of depth) << 32 | rgba over the samples
 * landing there, depth = z/w * 0.5 + 0.5 in [0, 1], or 0xFFFFFFFFFFFFFFFF
 * where none does; the call overwrites every pixel.  Single-precision arithmetic with every operation rounded on
 * its own, so images are reproducible bit for bit.  Asynchronous on
 * `stream` unless stats is not NULL (it then waits for the counts).
 * Errors: LOD_ERR_INVALID_ARG, LOD_ERR_OOM, LOD_ERR_CUDA. */
int lod_render(const lod_result_t* r, const lod_camera_t* cam, uint64_t* d_framebuffer, void* stream,
               lod_render_stats_t* stats);

/* ------------------------------------------------------------ profiling */

/* Per-kernel statistics accumulated by the library while profiling is on:
 * every kernel launch is bracketed by CUDA events recorded on the stream it
 * is launched on, and its elapsed time and algorithmic bytes (the bytes the
 * method itself has to move for that launch: 16 B per point read, 16 B per
 * point or voxel record written or read) are added to its entry. */
typedef struct lod_kernel_stat {
  char name[32];
  uint64_t launches;
  double total_ms;
  double alg_bytes;
} lod_kernel_stat_t;

/* Switch event timing on (1) or off (0); process-wide, off by default. */
int lod_profile_enable(int on);
/* Clear the accumulated statistics and the launch counter. */
int lod_profile_reset(void);
/* Copy up to `capacity` entries into stats (host); *n_stats receives the
 * number of distinct kernels recorded. */
int lod_profile_read(lod_kernel_stat_t* stats, uint32_t capacity, uint32_t* n_stats);
/* Number of kernels this library has launched since the last reset
 * (counted whether or not profiling is on). */
uint64_t lod_launch_count(void);

/* -------------------------------------------------------------- serving */

/* A server admits tile-build requests as they arrive and runs them
 * concurrently on the device (continuous batching): a request is started as
 * soon as a slot is free and its estimated device footprint fits in what
 * the HBM budget has left after the resident results of earlier requests;
 * results stay resident (counted against the budget) until lod_free().
 *   hbm_budget_bytes  device bytes for in-flight builds + resident results.
 *   max_inflight      concurrent builds (streams), >= 1.
 * Results are bit-identical to lod_build of the same request alone. */
typedef struct lod_server_config {
  uint64_t hbm_budget_bytes;
  uint32_t max_inflight;
  uint32_t reserved;
} lod_server_config_t;

typedef struct lod_server lod_server_t;

int lod_server_create(const lod_server_config_t* cfg, lod_server_t** out);

/* No passage of the paper defines the serving calls below (lod_submit,
 * lod_poll, lod_wait); they add request admission around lod_build, whose
 * result each request receives unchanged.
 *
 * Enqueue a build of n device points (kept valid by the caller until the
 * result is returned).  *ticket identifies the request.  Returns
 * LOD_ERR_BUDGET if the request alone exceeds the budget. */
int lod_submit(lod_server_t* s, const lod_point_t* d_points, uint64_t n, const lod_params_t* params,
               uint64_t* ticket);

/* Non-blocking (no paper counterpart, see lod_submit): LOD_OK and *out set
 * when the request has finished (the ticket is then consumed),
 * LOD_NOT_READY otherwise, or the build's error. */
int lod_poll(lod_server_t* s, uint64_t ticket, lod_result_t** out);

/* Blocking variant of lod_poll with a timeout in milliseconds. */
int lod_wait(lod_server_t* s, uint64_t ticket, uint32_t timeout_ms, lod_result_t** out);

/* Device bytes currently counted against the budget. */
uint64_t lod_server_bytes_in_use(const lod_server_t* s);

/* Finish all queued requests, release the worker threads and the server.
 * Results already returned stay valid. */
int lod_server_destroy(lod_server_t* s);

#ifdef __cplusplus
}
#endif

#endif /* LOD_H_ */
