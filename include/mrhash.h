/*
 * mrhash.h - C ABI of libmrhash, a B300 (sm_103a) implementation of the per-frame hot path of the variance-adaptive,
 * hash-based multi-resolution TSDF map of "Resolution Where It Counts" (MrHash, arXiv 2511.21459).
 *
 * Per frame the library
 *   - allocates the voxel blocks that the rays' truncation bands cross, in one flat GPU spatial hash whose entries
 *     point into one block heap per resolution level                                  (Sec. 3.2, Eq. 4, Fig. 3)
 *   - fuses every observation into a per-voxel truncated signed distance D, weight W, colour and Welford sum of
 *     squared deviations S2 (sigma^2 = S2 / W)                       (Sec. 3.1, Eq. 1 LiDAR, Eq. 2 camera, Eq. 3-6)
 *   - averages the voxel variances of every touched block and re-levels it: below the level's threshold the block
 *     is resampled at the next coarser level (merge); above h times the finer level's threshold it is resampled at
 *     the next finer level (split, the inverse extension)                               (Sec. 3.2.1, Fig. 2, Fig. 4)
 *   - raycasts the adaptive grid into a depth image                                       (Fig. 2, "render")
 *
 * Conventions
 *   - Units are metres. Poses are 4x4 row-major double matrices mapping sensor coordinates to world coordinates.
 *     Camera frames follow OpenCV (x right, y down, z forward); depth images hold z-depth (float32, 0 or NaN =
 *     invalid); pixel centres sit at integer (u, v); colour is interleaved uint8 RGB.
 *   - Levels: 0 is the finest. A block has a constant metric edge E = 8 v_0; level l stores (8 >> l)^3 voxels of
 *     edge v_l = v_0 2^l. Voxel i of a block of side n sits at x + n (y + n z).
 *   - Ownership: the caller owns every input and output buffer and the CUDA stream. Buffers marked "_dev" are device
 *     pointers on the map's device; "_host" are host pointers. The library owns the map's device memory and retains
 *     no caller pointer after a call returns. All device work is ordered on the stream passed in (NULL = legacy
 *     default stream).
 *   - Errors: no call aborts or throws. Argument errors are found on the host before any launch and return
 *     MRH_ERR_INVALID_ARG. Capacity errors found on the device (hash probe limit, empty block heap, full touched
 *     list) set a sticky device status word; the map stays usable (the failing blocks are skipped) and the next
 *     synchronising call (mrh_get_stats, mrh_count_blocks, mrh_extract_blocks, mrh_sync) returns the first error.
 *   - Thread safety: calls on one map must not run concurrently from several host threads.
 */
#ifndef MRHASH_H
#define MRHASH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mrh_map mrh_map; /* opaque, owned by the library */

typedef enum {
  MRH_OK = 0,
  MRH_ERR_INVALID_ARG = 1,   /* bad argument; nothing was launched */
  MRH_ERR_OUT_OF_MEMORY = 2, /* device allocation failed in mrh_map_create */
  MRH_ERR_HASH_FULL = 3,     /* a key found no free slot within the probe limit; that key was dropped */
  MRH_ERR_POOL_EMPTY = 4,    /* a level's block heap ran out; that allocation or re-level was skipped */
  MRH_ERR_LIST_FULL = 5,     /* a per-frame list overflowed (touched blocks > max_touched, or LiDAR observations >
                                max_observations); the excess was not fused */
  MRH_ERR_CUDA = 6,          /* a CUDA runtime call failed (see mrh_last_cuda_error) */
  MRH_ERR_CAPACITY = 7,      /* caller-provided output buffers are too small */
  MRH_ERR_STATIC_LIMIT = 8   /* more blocks than mrh_extract_blocks_noalloc's fixed scratch holds */
} mrh_status;

enum { MRH_STORAGE_FP32 = 0, MRH_STORAGE_FP16 = 1 };

/* Pinhole camera (Eq. 2): projection u = fx x/z + cx, v = fy y/z + cy. Depth outside [min_depth, max_depth] is
 * treated as invalid. */
typedef struct {
  float fx, fy, cx, cy;
  int32_t width, height;
  float min_depth, max_depth;
} mrh_pinhole;

/* Map parameters (Sec. 3.2 grid, Sec. 3.2.1 merging criterion, Sec. 4.1.4 implementation details). */
typedef struct {
  float base_voxel_size;     /* voxel edge of the coarsest level v_{L-1} [m]; v_0 = base / 2^(L-1) */
  int32_t n_levels;          /* L, 1..3 */
  float truncation;          /* tau [m] (Sec. 3.1); 2 tau must not exceed 8 block edges */
  double var_threshold[2];   /* theta_l [m^2]: a block at level l merges to l+1 when its mean voxel variance < theta_l */
  double split_hysteresis;   /* h >= 1: a block at level l > 0 splits when its mean variance > h theta_{l-1}; 0 = off */
  int32_t min_obs;           /* k_min: re-levelling needs mean weight >= k_min over the block's observed voxels */
  uint32_t hash_slots_log2;  /* hash table size 2^k slots of 16 bytes, k in [10, 28] */
  uint32_t max_blocks[3];    /* block heap capacity per level */
  uint32_t max_touched;      /* capacity of the per-frame touched-block list */
  uint32_t max_observations; /* LiDAR: capacity of the per-frame (point, voxel) observation buffer; 0 for camera-only */
  int32_t storage;           /* MRH_STORAGE_FP32 (D, colour float) or MRH_STORAGE_FP16 (D, colour half) */
  int32_t has_color;         /* 1: fuse colour (running mean of uint8 RGB, stored 0..255) */
  float min_range, max_range;/* LiDAR: points with |x_s| outside [min_range, max_range] are skipped */
} mrh_map_params;

/* Per-frame counters of the last integrated frame and map totals. */
typedef struct {
  uint64_t frame;            /* frames integrated so far */
  uint64_t valid_rays;       /* rays that allocated blocks in the last frame */
  uint64_t touched;          /* blocks fused in the last frame */
  uint64_t new_blocks;       /* blocks created in the last frame */
  uint64_t merged, split;    /* re-level events in the last frame */
  uint64_t fp64_rechecks;    /* block variances within the decision band recomputed in double */
  uint64_t live_blocks[3];   /* blocks currently held per level */
  uint64_t touched_level[3]; /* blocks fused in the last frame, per level */
  uint64_t observations;     /* voxel updates applied in the last frame */
  uint32_t status;           /* sticky device status bits (see mrh_status) */
} mrh_stats;

/* Kernel groups for mrh_get_profile. */
enum {
  MRH_K_BEGIN = 0,     /* per-frame counter reset */
  MRH_K_ALLOC = 1,     /* ray -> block allocation */
  MRH_K_BIN = 2,       /* heap assignment of new blocks, level binning */
  MRH_K_LIDAR_OBS = 3, /* LiDAR observation count / scan / fill */
  MRH_K_FUSE = 4,      /* fusion + block variance + re-levelling */
  MRH_K_RELEASE = 5,   /* freed heap blocks back to their free stacks */
  MRH_K_RAYCAST = 6,   /* raycast */
  MRH_K_COUNT = 7
};

/* Create a map on CUDA device `device`. Allocates the hash table, one block heap per level and per-frame lists.
 * Returns MRH_ERR_INVALID_ARG for out-of-range parameters, MRH_ERR_OUT_OF_MEMORY if allocation fails. */
mrh_status mrh_map_create(const mrh_map_params* params, int device, mrh_map** out);

/* Release all device memory of the map (after synchronising its device). NULL is accepted. */
mrh_status mrh_map_destroy(mrh_map* map);

/* Integrate one pinhole depth frame (Sec. 3.1 "Cameras", Eq. 2, Eq. 3, Welford S2 of Sec. 3.2.1, merging of
 * Sec. 3.2.1). depth_dev: height x width float32 z-depth; rgb_dev: height x width x 3 uint8 or NULL. T_wc_host:
 * 16 doubles, world <- camera. Asynchronous on `stream`. */
mrh_status mrh_integrate_depth(mrh_map* map, const mrh_pinhole* K, const double* T_wc_host, const float* depth_dev,
                               const uint8_t* rgb_dev, void* stream);

/* Integrate one LiDAR scan (Sec. 3.1 "3D Point Cloud", Eq. 1): xyz_dev holds n points (n x 3 float32, sensor
 * frame; NaN = no return). Observations of one voxel are applied in ascending point index. T_ws_host: world <- sensor.
 * Asynchronous on `stream`. */
mrh_status mrh_integrate_points(mrh_map* map, const double* T_ws_host, const float* xyz_dev, uint64_t n,
                                void* stream);

/* ---- batched multi-scene integration (not in the paper: many maps fused per step, one launch per phase) ---- */

typedef struct mrh_batch mrh_batch; /* opaque; refers to maps it does not own */

enum { MRH_BATCH_GRAPH = 1, MRH_BATCH_AUTOTUNE = 2 };

/* One map's input for one batched step. */
typedef struct {
  mrh_pinhole K;            /* intrinsics; width/height must equal the camera given to mrh_batch_create */
  double T_wc[16];          /* world <- camera, row-major */
  const float* depth_dev;   /* height x width float32 z-depth */
  const uint8_t* rgb_dev;   /* height x width x 3 uint8, or NULL */
  float* raycast_dev;       /* height x width float32: raycast of the same view after integration, or NULL */
} mrh_batch_frame;

/* Group n (1..64) maps of one device and one storage layout (same storage and has_color) whose frames have the
 * fixed sizes of cams[i]. flags: MRH_BATCH_AUTOTUNE runs the first steps after the first as timed trials of
 * alternative launch shapes (allocation CTA tile and probe width, fusion warps per CTA and grid, raycast warp tile)
 * and keeps the fastest (every shape computes the same result); MRH_BATCH_GRAPH captures the step into a CUDA graph
 * once tuning is done and replays it (needs a non-default stream). The batch owns per-map image buffers; the maps
 * must outlive it. */
mrh_status mrh_batch_create(mrh_map* const* maps, const mrh_pinhole* cams, int n, int flags, mrh_batch** out);

/* Integrate frames[i] into map i for every map of the batch (the per-map semantics of mrh_integrate_depth followed by
 * mrh_raycast into raycast_dev when given), as one launch per phase over all maps. Asynchronous on `stream`; the
 * frames array may be reused when the call returns. */
mrh_status mrh_batch_integrate(mrh_batch* batch, const mrh_batch_frame* frames, void* stream);

/* The launch shapes in use: {alloc tile width, alloc tile height, probe width, fusion warps per CTA, fusion CTAs per
 * SM, raycast warp tile (0: 8x4, 1: 16x2), tuned (0/1), graph captured (0/1)}. */
mrh_status mrh_batch_config(const mrh_batch* batch, int* config_out8);

/* Release the batch (not its maps). NULL is accepted. */
mrh_status mrh_batch_destroy(mrh_batch* batch);

/* Raycast the map from a pinhole view (the rendering branch of Fig. 2): depth_out_dev receives height x width
 * float32 z-depth of the first observed zero crossing, 0 where none. Empty blocks are skipped whole.
 * Asynchronous on `stream`. */
mrh_status mrh_raycast(mrh_map* map, const mrh_pinhole* K, const double* T_wc_host, float* depth_out_dev,
                       void* stream);

/* Number of allocated blocks and voxels (synchronises `stream`). */
mrh_status mrh_count_blocks(mrh_map* map, uint64_t* n_blocks, uint64_t* n_voxels, void* stream);

/* Copy every allocated block out, sorted by key (x, then y, then z). Outputs (device): keys_dev n x 3 int32,
 * levels_dev n uint8, voxel_offset_dev n + 1 uint64 (voxels of block b are [off[b], off[b+1])), tsdf_dev, weight_dev,
 * s2_dev V float32 each (FP16 storage is widened exactly), color_dev V x 3 float32 or NULL. Capacities are in blocks
 * and voxels; MRH_ERR_CAPACITY if too small. Synchronises `stream`. */
mrh_status mrh_extract_blocks(mrh_map* map, int32_t* keys_dev, uint8_t* levels_dev, uint64_t* voxel_offset_dev,
                              float* tsdf_dev, float* weight_dev, float* s2_dev, float* color_dev,
                              uint64_t capacity_blocks, uint64_t capacity_voxels, uint64_t* n_blocks_out,
                              uint64_t* n_voxels_out, void* stream);

/* Same output as mrh_extract_blocks, but it allocates no device memory: no cudaMalloc, cudaMallocAsync or cudaFree.
 * (The paper has no counterpart; this exists for callers of the library.) Meant for callers that cannot allocate
 * at read-out time: a process that has handed all device memory to a fixed arena or to a framework's caching
 * allocator, so a fresh allocation would fail, or a latency-bounded loop in which an allocation (which can
 * synchronise the device) is not acceptable. Its sort and offset scratch is one file-scope device array of
 * MRH_NOALLOC_MAX_BLOCKS blocks (about 5 MiB) that every GPU loading the library holds until the process exits;
 * maps holding more blocks return MRH_ERR_STATIC_LIMIT before any work is queued.
 * The first call on a device looks up that array's device address (once per device, with the map's device
 * current); make that first call before any stream capture. Every call shares the one array per device and keeps
 * the last call's contents (the call clears what must start at zero itself), so calls whose GPU work overlaps in
 * time, on any stream or map of the same device, race: order them on one stream or synchronise between them.
 * Arguments, outputs, ordering and the synchronisation of `stream` are those of mrh_extract_blocks. */
#define MRH_NOALLOC_MAX_BLOCKS (1u << 18)
mrh_status mrh_extract_blocks_noalloc(mrh_map* map, int32_t* keys_dev, uint8_t* levels_dev,
                                      uint64_t* voxel_offset_dev, float* tsdf_dev, float* weight_dev, float* s2_dev,
                                      float* color_dev, uint64_t capacity_blocks, uint64_t capacity_voxels,
                                      uint64_t* n_blocks_out, uint64_t* n_voxels_out, void* stream);

/* Counters of the last frame and map totals (synchronises `stream`); returns the sticky device status. */
mrh_status mrh_get_stats(mrh_map* map, mrh_stats* out, void* stream);

/* Wait for `stream` and return the sticky device status. */
mrh_status mrh_sync(mrh_map* map, void* stream);

/* Clear the sticky device status (stream-ordered). */
mrh_status mrh_clear_status(mrh_map* map, void* stream);

/* Per-kernel device time: when enabled, every kernel group of later calls is bracketed by CUDA events on the
 * caller's stream (profiling adds two event records per group; off by default; do not enable it while capturing a
 * CUDA graph). */
mrh_status mrh_set_profiling(mrh_map* map, int enable);

/* Accumulated device milliseconds and launch counts per kernel group (MRH_K_*) since the last reset; n entries are
 * written (n <= MRH_K_COUNT). Launch counts are kept whether or not profiling is on. Synchronises `stream`. If
 * `reset` is non-zero the accumulators are cleared after reading. */
mrh_status mrh_get_profile(mrh_map* map, double* ms_out, uint64_t* launches_out, int n, int reset, void* stream);

/* Hash slot of block key (x, y, z) in a table of 2^log2_slots slots: Eq. 4, H = (x p1 xor y p2 xor z p3) mod n_hash
 * with p1 = 73856093, p2 = 19349669, p3 = 83492791 in 32-bit unsigned arithmetic. Host-only helper. */
uint32_t mrh_hash_slot(int32_t x, int32_t y, int32_t z, uint32_t log2_slots);

/* Human-readable name of a status code. */
const char* mrh_status_string(mrh_status status);

/* Text of the last CUDA error seen by the calling thread's last failing call (empty if none). */
const char* mrh_last_cuda_error(void);

/* Library version string. */
const char* mrh_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MRHASH_H */
