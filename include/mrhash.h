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
  MRH_ERR_STATIC_LIMIT = 8,  /* more blocks than mrh_extract_blocks_noalloc's fixed scratch holds */
  MRH_ERR_INCONSISTENT = 9   /* the hash table's committed blocks disagree with the heaps' live-block count (a
                                read-out would drop or invent blocks); the outputs are not valid */
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
  double var_threshold[2];   /* theta_l [m^2]: a block at level l merges to l + 1 when its mean voxel variance is
                                below theta_l */
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
  uint64_t updated_voxels;   /* distinct voxels updated in the last frame (a voxel with several observations counts
                                once) */
  uint64_t lidar_restaged;   /* LiDAR: points of the last scan whose observations exceeded the per-point stage and
                                were written by a second walk (correct either way; a cost diagnostic) */
  uint64_t evicted;          /* streaming: blocks moved to the archive before the last frame */
  uint64_t restored;         /* streaming: archived blocks the last frame allocated again (brought back) */
  uint64_t archived;         /* streaming: blocks in the archive now */
  uint64_t lidar_max_voxel_obs; /* LiDAR: the most observations one voxel received in the last scan (a coarse voxel
                                   near the sensor collects hundreds; they are applied in point order) */
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
  MRH_K_MESH = 7,      /* Marching Cubes mesh extraction */
  MRH_K_STREAM = 8,    /* streaming: eviction before a frame, restore after binning */
  MRH_K_COUNT = 9
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
 * frame; NaN = no return; n <= 2^23). Observations of one voxel are applied in ascending point index. T_ws_host:
 * world <- sensor. The map keeps per-point buffers (the ray and its staged observations, 840 bytes per point) grown to
 * the largest n seen.
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

/* Device time of the phases of the last mrh_batch_integrate call, in ms (waits for it): ms_out4[0] allocation,
 * [1] binning, [2] fusion (the fusion kernel alone), [3] re-level release + raycast. The step records its phase
 * boundaries with CUDA events on its stream (inside the captured graph as well). MRH_ERR_INVALID_ARG before the
 * first step. */
mrh_status mrh_batch_last_step_ms(const mrh_batch* batch, float* ms_out4);

/* Release the batch (not its maps). NULL is accepted. */
mrh_status mrh_batch_destroy(mrh_batch* batch);

/* ---- Learned level predictor (an addition to the paper's method; the paper has no counterpart).
 * A 16 -> 64 -> 64 -> 3 multilayer perceptron with GELU activations reads 16 features of a NEW block taken from the
 * current depth frame or LiDAR scan and predicts the level the variance rule of Sec. 3.2.1 would give that block after
 * fusing the sequence. With a predictor set, mrh_integrate_depth and mrh_integrate_points allocate each new block at
 * the predicted level instead of the finest one (Sec. 3.2.1 starts every block fine), so a block predicted coarse is
 * never fused at the fine level. The variance rule still runs on every touched block afterwards and re-levels any
 * block the network got wrong. Batched integration always uses the plain rule.
 *
 * LiDAR features (float32, in this order; rounded to BF16): every valid point's end point p = T x (double) in fixed
 * point gives its block and its position q in the block in units of E / 1024 (integers in [0, 1024)); a new block
 * takes the moments of the q of its end points (count n, centroid m, covariance C, block units; none for a block that
 * holds only the truncation band). With c the block centre relative to the sensor, r = |c|, u = c / r and o = m - 1/2
 * the centroid's offset from the centre:
 *   f0 r;  f1 S(o.u E / tau);  f2 S(sqrt(u^T C u) E / tau);  f3 sqrt(tr C - u^T C u);  f4 S(n / 16);  f5 E / r;
 *   f6 sqrt(C_zz);  f7 |o - (o.u) u|;  f8 1 if n > 0 else 0;  f9 |u_z|;  f10 u_z;  f11 sqrt(tr C);  f12 1 / r;
 *   f13 1 (LiDAR);  f14 tau / E;  f15 1;  all zero statistics when n = 0. c is formed in double and converted to
 *   float; the rest is float arithmetic.
 *
 * Camera features (float32, in this order; computed on the device from the frame's range image rho = z |(q_x, q_y, 1)|,
 * q = ((u - cx)/fx, (v - cy)/fy), and rounded to BF16): with c the block centre in camera coordinates, r = |c|,
 * (u0, v0) its projection rounded to the nearest pixel, s = clamp(floor(fx E / (4 c_z)), 1, 16) pixels and a 5 x 5
 * grid of range samples p_ij at (u0 + (i-2) s, v0 + (j-2) s) (invalid or outside = missing):
 *   f0 r;  f1 S((mean p - r) / tau);  f2 S(std p / tau);  f3 S((max p - min p) / E);  f4 fraction of the 25
 *   samples present;  f5 E / r;  f6, f7 S(|central difference of p| along u and v per metre of lateral offset, r s /
 *   fx metres per step);  f8 S(mean |second difference of p along u| / E);  f9, f10 |2 (u / width - 1/2)|,
 *   |2 (v / height - 1/2)|;  f11 c_z / r;  f12 1 / r;  f13 0 (camera);  f14 tau / E;  f15 1;
 *   with S(x) = x / (1 + |x|).
 * A block whose centre projects outside the image (or behind the camera) gets the finest level and no record.
 *
 * Network: x = BF16(f); h1 = BF16(GELU(W1^T x + b1)); h2 = BF16(GELU(W2^T h1 + b2)); logits = W3^T h2 + b3; the
 * level is the first argmax, clamped to n_levels - 1. Sums are float32 in index order; GELU(x) = x (1 + erf(x /
 * sqrt 2)) / 2 with erf from Abramowitz & Stegun 7.1.26 and exp by Cody-Waite reduction and a degree-6 Taylor
 * polynomial, so every decision is reproducible on a CPU. Parameters are packed as W1 [16][64] (input-major), b1
 * [64], W2 [64][64], b2 [64], W3 [64][3], b3 [3]: MRH_MLP_PARAMS values. */
#define MRH_MLP_IN 16
#define MRH_MLP_HIDDEN 64
#define MRH_MLP_LEVELS 3
#define MRH_MLP_PARAMS (MRH_MLP_IN * MRH_MLP_HIDDEN + MRH_MLP_HIDDEN + MRH_MLP_HIDDEN * MRH_MLP_HIDDEN + \
                        MRH_MLP_HIDDEN + MRH_MLP_HIDDEN * MRH_MLP_LEVELS + MRH_MLP_LEVELS)

/* Set the map's predictor from MRH_MLP_PARAMS BF16 bit patterns (host; copied, so the caller keeps ownership), or
 * turn it off with NULL. n_params must equal MRH_MLP_PARAMS; an inf or NaN weight is rejected. Waits for all work on
 * the map's device first (frames in flight read the previous weights). */
mrh_status mrh_set_predictor(mrh_map* map, const uint16_t* bf16_weights_host, uint64_t n_params);

/* Record the features of every new block of later depth frames and LiDAR scans (training data for the predictor):
 * up to `capacity` records of (key x, y, z; 16 features), in no particular order; later ones are counted but dropped.
 * 0 turns recording off and frees its buffers. Waits for all work on the map's device first. */
mrh_status mrh_set_feature_capture(mrh_map* map, uint32_t capacity);

/* Copy the recorded features out: keys_dev n x 3 int32, features_dev n x 16 float32 (device), n_out = n records
 * stored, n_seen_out (nullable) = records offered since the last reset (> n when some were dropped). MRH_ERR_CAPACITY
 * (nothing copied) if capacity < n. With `reset` non-zero the record is emptied afterwards. Synchronises `stream`.
 * MRH_ERR_INVALID_ARG if recording is off. */
mrh_status mrh_get_features(mrh_map* map, int32_t* keys_dev, float* features_dev, uint32_t capacity, uint32_t* n_out,
                            uint64_t* n_seen_out, int reset, void* stream);

/* Trainer of the predictor on the GPU: FP32 master weights, a BF16 copy used by the forward and backward passes (the
 * same network as above, with the derivative of each BF16 rounding taken as 1), softmax cross-entropy loss averaged
 * over the batch, and Adam (beta1 0.9, beta2 0.999, epsilon 1e-8, bias-corrected). */
typedef struct mrh_mlp mrh_mlp; /* opaque, owned by the library */

/* Create a trainer on `device` from MRH_MLP_PARAMS float32 initial weights (host, packed as above, finite). */
mrh_status mrh_mlp_create(const float* init_host, int device, mrh_mlp** out);

/* Release the trainer. NULL is accepted. */
mrh_status mrh_mlp_destroy(mrh_mlp* mlp);

/* One Adam step on a batch: x_dev n x 16 float32 features, labels_dev n int32 levels in [0, 3), lr > 0; loss_dev
 * (one float32, device) receives the batch's mean loss before the step. Asynchronous on `stream`. */
mrh_status mrh_mlp_train_step(mrh_mlp* mlp, const float* x_dev, const int32_t* labels_dev, uint32_t n, float lr,
                              float* loss_dev, void* stream);

/* Mean loss and its gradient with respect to the BF16 weights (grad_dev MRH_MLP_PARAMS float32, device), without
 * updating anything. Asynchronous on `stream`. */
mrh_status mrh_mlp_loss_grad(const mrh_mlp* mlp, const float* x_dev, const int32_t* labels_dev, uint32_t n,
                             float* loss_dev, float* grad_dev, void* stream);

/* Logits of n samples (logits_dev n x 3 float32, device) with the BF16 weights. Asynchronous on `stream`. */
mrh_status mrh_mlp_predict(const mrh_mlp* mlp, const float* x_dev, uint32_t n, float* logits_dev, void* stream);

/* Copy the FP32 master weights and/or the BF16 weights (bit patterns) to the host; either may be NULL, not both.
 * Synchronises `stream`. */
mrh_status mrh_mlp_get_weights(const mrh_mlp* mlp, float* master_host, uint16_t* bf16_host, void* stream);

/* Raycast the map from a pinhole view (the rendering branch of Fig. 2; the paper renders through splats and gives no
 * raycaster, so the march is this library's reading): depth_out_dev receives height x width float32 z-depth of the
 * first observed + -> - zero crossing of the trilinear TSDF, 0 where none. Empty bricks and blocks are skipped whole.
 * Optional outputs (device, NULL to skip), at the hit point and from the same 8 trilinear corners:
 *   normal_out_dev  height x width x 3 float32, world frame: the normalised gradient of the trilinear interpolant
 *                   (pointing towards positive distance, i.e. out of the surface);
 *   rgb_out_dev     height x width x 3 uint8: the trilinear mean of the stored colour, rounded half up and clamped
 *                   (maps created with has_color only, else MRH_ERR_INVALID_ARG).
 * Both are 0 where there is no hit, or where the hit's block or one of the corners is unallocated or unobserved.
 * Asynchronous on `stream`. */
mrh_status mrh_raycast(mrh_map* map, const mrh_pinhole* K, const double* T_wc_host, float* depth_out_dev,
                       float* normal_out_dev, uint8_t* rgb_out_dev, void* stream);

/* Multi-resolution Marching Cubes over every allocated block (Sec. 3.4, Figs. 5 and 6). Output: triangles as 9
 * float32 each (three vertices x, y, z in metres, counter-clockwise seen from the side of positive distance), in no
 * particular order, written to tris_dev (device; NULL with capacity 0 only counts); n_tris_out receives the number of
 * triangles. MRH_ERR_CAPACITY when that number exceeds capacity (the first `capacity` triangles written are then
 * some subset). Cells: every voxel is the low corner of one cell reaching the next voxel centres along +x, +y, +z; the
 * cells of a block's last voxels reach the first centre of the neighbouring block (so coarse cells next to finer
 * blocks are shortened and the levels tile space), and there is none where that neighbour is missing. Cell corners take
 * the trilinear field on the grid of the block containing them (reading voxels of any level); cells with an
 * unallocated or unobserved corner read emit nothing. The case table is Marching Cubes' (inside = value below zero),
 * with the two inside corners of an ambiguous face kept apart. Synchronises `stream`. */
mrh_status mrh_extract_mesh(mrh_map* map, float* tris_dev, uint64_t capacity, uint64_t* n_tris_out, void* stream);

/* Vertex collapse of a triangle soup (the final step of Sec. 3.4; the paper gives only the idea, this is the
 * library's reading): every vertex falls in the cell floor(p * (1 / delta)) (float, per axis) of a grid of spacing
 * delta (metres, > 0); each occupied cell becomes one vertex, the lexicographically smallest (x, then y, then z) of
 * its members, numbered in ascending cell order (x, then y, then z); triangles take their vertices' cells and those
 * with two equal indices are dropped, the rest keep their soup order. Inputs: tris_dev n_tris x 9 float32 (device;
 * e.g. from mrh_extract_mesh). Outputs (device): verts_dev n_verts x 3 float32, faces_dev n_faces x 3 int32;
 * n_verts_out, n_faces_out receive the counts (MRH_ERR_CAPACITY when either exceeds its capacity; nothing beyond a
 * capacity is written). MRH_ERR_INVALID_ARG for delta <= 0, n_tris > 2^28, or a vertex whose cell index exceeds
 * 2^20 in magnitude. Uses temporary device memory (up to about 450 bytes per input triangle) on the map's device;
 * synchronises `stream`. */
mrh_status mrh_weld_mesh(mrh_map* map, const float* tris_dev, uint64_t n_tris, float delta, float* verts_dev,
                         uint64_t cap_verts, int32_t* faces_dev, uint64_t cap_faces, uint64_t* n_verts_out,
                         uint64_t* n_faces_out, void* stream);

/* Contrast quadtree of an RGB image (the rendering branch, Sec. 3.5, Eq. 10, Algorithm 1; no map needed). rgb_dev:
 * height x width x 3 uint8 (device, interleaved). A node's contrast is the Rec. 601 luma weights (0.2989, 0.5870,
 * 0.1140) applied to the per-channel mean squared deviation of its pixels from their mean, in byte units, computed from
 * exact integer sums ((n S2 - S1^2) / n^2 per channel). A node splits when its larger side exceeds `min_size` (>= 1)
 * pixels and n^2 times its contrast, l0 N0 + l1 N1 + l2 N2 in double with N = n S2 - S1^2, exceeds threshold n n
 * (double); it splits at its midpoints (x0 + w / 2, y0 + h / 2, rounded down) into its non-empty quarters; the
 * others are leaves. Output: leaves_dev n x 4 int32
 * (x, y, w, h) in no particular order; n_leaves_out receives n (MRH_ERR_CAPACITY when n > capacity; at most capacity
 * are written). Uses temporary device memory (about 80 bytes per pixel) on `device`; synchronises `stream`. */
mrh_status mrh_quadtree(const uint8_t* rgb_dev, int width, int height, double threshold, int min_size,
                        int32_t* leaves_dev, uint64_t capacity, uint64_t* n_leaves_out, int device, void* stream);

/* The case table used by mrh_extract_mesh (host, no device work): ntri[256] triangles per case, tri[256 * 15] edge
 * triples (-1 unused), edge_end[12 * 2] corner pairs. Corner c lies at (c & 1, c >> 1 & 1, c >> 2 & 1) of the cell;
 * edge 4a + r joins the r-th corner (ascending) with bit a clear to its neighbour along axis a. */
void mrh_mesh_case_table(uint8_t* ntri, int8_t* tri, int8_t* edge_end);

/* Capacity-driven streaming (Sec. 3.3; the selection rule is this library's reading). Before each integration call,
 * when some level holds more than `fraction` (0 < fraction <= 1) of its max_blocks (float comparison of the counts),
 * every resident block outside the frame's view moves to the archive with its level and payload: for a depth frame, a
 * block whose circumscribed sphere misses the pinhole's view cone between min_depth and max_depth; for a point scan, a
 * block whose centre lies farther than `radius` metres from the scan origin. Its hash slot becomes a tombstone (not
 * reused: size hash_slots_log2 for every block the map will ever hold) and its heap block is freed. A later frame that
 * allocates the key again gets the block back at its archived level before fusion. The archive holds archive_blocks
 * blocks in pinned host memory (archive_blocks x the level-0 block size), mapped into the device's address space, so
 * neither direction needs a host round trip; a key keeps its archive slot. Extraction, meshing and raycasting see the
 * resident blocks only. fraction = 0 switches streaming off (archived blocks stay archived; it cannot be switched on
 * again). MRH_ERR_INVALID_ARG with a predictor or feature capture set (they are not combined), for a new capacity while
 * the archive holds blocks, or for arguments out of range; MRH_ERR_OUT_OF_MEMORY if the archive cannot be allocated.
 * A full archive leaves the remaining blocks resident and reports MRH_ERR_CAPACITY through the status. Maps with
 * streaming are not accepted by mrh_batch_create. Synchronises the device. */
mrh_status mrh_set_streaming(mrh_map* map, float fraction, float radius, uint32_t archive_blocks);

/* Tile-based Gaussian-splat rendering (the rendering branch, Sec. 3.5, Eqs. 7-9; no map needed). Inputs (device,
 * float32): means_dev n x 3 (world), covs_dev n x 6 (world covariance Sigma_W as xx, xy, xz, yy, yz, zz), opacity_dev n
 * (alpha, expected in [0, 1]), colors_dev n x 3 (any units); n < 2^32. K: pinhole (fx, fy > 0, 0 < min_depth <=
 * max_depth); T_wc_host: camera-to-world pose, 4 x 4 row-major double.
 * Each Gaussian is projected (Eq. 7): camera-frame mean R^T (mu - t), image mean by the pinhole, image covariance
 * Sigma_I = J R^T Sigma_W R J^T with J the projection's Jacobian at the camera-frame mean; it is not drawn when its
 * camera z lies outside [min_depth, max_depth] or Sigma_I is not positive definite. Gaussian m reaches pixel (u, v)
 * (image coordinates u, v) when its squared Mahalanobis distance q <= 9 and |u - mu_u| <= 3 sqrt(Sigma_uu),
 * |v - mu_v| <= 3 sqrt(Sigma_vv) (all float, fixed operation order). Pixel colour (Eq. 8) = sum over the Gaussians
 * that reach it, in increasing camera z (ties by index), of C_m a_m exp(-q_m / 2) times the product of
 * (1 - a_l exp(-q_l / 2)) over those in front (Eq. 9); a pixel stops once that product (its transmittance) is below
 * 1e-4, which changes its colour by less than 1e-4 times the largest colour.
 * Outputs (device): rgb_out_dev height x width x 3 float32; trans_out_dev height x width float32 (the remaining
 * transmittance; nullable). n_pairs_out (nullable) receives the number of (16 x 16 tile, Gaussian) pairs; more than
 * 2^31 - 1 gives MRH_ERR_CAPACITY and nothing is rendered. Uses temporary device memory (about 88 bytes per Gaussian
 * and 25 per pair) on `device`; synchronises `stream` once (to size the pair buffers). */
mrh_status mrh_splat_render(const float* means_dev, const float* covs_dev, const float* opacity_dev,
                            const float* colors_dev, uint64_t n, const mrh_pinhole* K, const double* T_wc_host,
                            float* rgb_out_dev, float* trans_out_dev, uint64_t* n_pairs_out, int device, void* stream);

/* Save the map to a file (the persistence half of streaming, Sec. 3.3): the creation parameters, then every resident
 * block and every archived block (key, level, payload in the library's block layout; resident ones first, each group
 * in key order). Synchronises `stream` and the device copies it needs. MRH_ERR_INVALID_ARG when the file cannot be
 * written. */
mrh_status mrh_save_map(mrh_map* map, const char* path, void* stream);

/* Create a map on `device` from a file written by mrh_save_map, with every saved block resident (archived ones
 * included; streaming is off). MRH_ERR_INVALID_ARG for a missing or malformed file; MRH_ERR_HASH_FULL /
 * MRH_ERR_POOL_EMPTY when the saved blocks do not fit the saved capacities. *out is NULL on error. */
mrh_status mrh_load_map(const char* path, int device, mrh_map** out);

/* Number of allocated blocks and voxels (synchronises `stream`). */
mrh_status mrh_count_blocks(mrh_map* map, uint64_t* n_blocks, uint64_t* n_voxels, void* stream);

/* Copy every allocated block out, sorted by key (x, then y, then z). Outputs (device): keys_dev n x 3 int32,
 * levels_dev n uint8, voxel_offset_dev n + 1 uint64 (voxels of block b are [off[b], off[b+1])), tsdf_dev, weight_dev,
 * s2_dev V float32 each (FP16 storage is widened exactly), color_dev V x 3 float32 or NULL. Capacities are in blocks
 * and voxels; MRH_ERR_CAPACITY if too small. When counting the blocks fails (MRH_ERR_CUDA) nothing is queued;
 * MRH_ERR_INCONSISTENT when the hash table holds a different number of committed blocks than the heaps report live.
 * Synchronises `stream`. */
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
 * Every call looks up that array's device address with the map's device current (so no address survives a device
 * reset). Every call shares the one array per device and keeps the last call's contents (the call clears what must
 * start at zero itself), so calls whose GPU work overlaps in time, on any stream or map of the same device, race:
 * order them on one stream or synchronise between them. Arguments, outputs, ordering, the synchronisation of
 * `stream`, the early return on a failed count and the other status codes are those of mrh_extract_blocks; a
 * MRH_ERR_STATIC_LIMIT return writes nothing to the outputs. */
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
