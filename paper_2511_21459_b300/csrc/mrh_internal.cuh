// Internal definitions of libmrhash (not part of the C ABI).
//
// Device data layout (all in the map's own device memory, sized at map creation):
//   slots[2^k]           16-byte hash entries {packed key, value, frame stamp}: one flat table for every level
//                        (Sec. 3.2 "single hash table"; the entry's level selects the heap, Fig. 3)
//   heap[l]              block payloads of level l, struct-of-arrays inside a block so that every field is a
//                        contiguous, 16-byte aligned run: FP32 storage [D | W | S2 | R | G | B] float each,
//                        FP16 storage [D | R | G | B] half then [W | S2] float
//   dmin[l]              per heap block: least stored D over its observed voxels (raycast empty-interior skip)
//   free_stack[l]        ids of free blocks of level l (pops and pushes never share a kernel)
//   touched_all          slots touched by the current frame (unique: the slot's frame stamp dedups)
//   touched[l]           the same slots binned by level, the fusion work lists
//   retire               heap ids released by re-levelling in this frame, pushed back after fusion
//   DevState             counters, frame number and the sticky status word
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "mrhash.h"

namespace mrh {

constexpr int kFineDim = 8;                       // voxels per block side at the finest level (512-voxel blocks)
constexpr int kMaxLevels = 3;
constexpr int kFracBits = 16;                     // fixed-point fraction bits per block edge
constexpr long long kBlockUnit = 1LL << kFracBits;
constexpr long long kVoxelUnit = kBlockUnit / kFineDim;
constexpr int kBlockShift = kFracBits;      // log2 of kBlockUnit
constexpr int kVoxelShift = kFracBits - 3;  // log2 of kVoxelUnit
constexpr long long kKeyLimit = (1LL << 20) - 2;  // |block coordinate| bound of the 21-bit packed key
constexpr unsigned long long kEmptyKey = ~0ULL;
constexpr uint32_t kValPending = 0xFFFFFFFFu;     // key present, no heap block yet
constexpr uint32_t kPtrMask = 0x0FFFFFFFu;
constexpr uint32_t kValNew = 1u << 30;            // heap block not yet initialised: fusion starts from zero state
constexpr int kMaxProbeWindows = 64;              // warp-cooperative probing: 64 x 32 slots
constexpr int kMaxProbes = 2048;                  // single-thread probing
constexpr int kMaxSegmentCells = 64;
constexpr int kMaxVoxelCells = 256;
// End-point moments of a new block of a LiDAR scan (learned level predictor): n, sum q_x, sum q_y, sum q_z,
// sum q_x^2, sum q_y^2, sum q_z^2, sum q_x q_y, sum q_x q_z, sum q_y q_z, with q the end point's position in the block
// in units of E / 1024 (integers: the sums do not depend on the order of the atomic adds).
constexpr int kLidarMoments = 10;
constexpr long long kNoEndPoint = -0x7FFFFFFFFFFFFFFFLL - 1;  // lidar_end of a refused point
constexpr int kRaycastMaxIter = 8192;
constexpr int kBrickShift = 2;  // a brick is 4 x 4 x 4 blocks
constexpr int kSuperShift = 2;  // a super-brick is 4 x 4 x 4 bricks
constexpr int kStageCap = 96;   // LiDAR: staged entries per point (a run header per block + one record per voxel)
constexpr uint32_t kStageOverflow = 0xFFFFFFFFu;
constexpr uint32_t kStageHeader = 0x80000000u;

// status bits (sticky)
constexpr uint32_t kStHashFull = 1u << 0;
constexpr uint32_t kStPoolEmpty = 1u << 1;
constexpr uint32_t kStListFull = 1u << 2;
constexpr uint32_t kStSegment = 1u << 3;
constexpr uint32_t kStObsFull = 1u << 4;
constexpr uint32_t kStTimeout = 1u << 5;  // a bounded wait on an async copy gave up
constexpr uint32_t kStArchiveFull = 1u << 6;  // streaming: the archive had no slot for a block (it stayed resident)
constexpr unsigned long long kTombKey = ~1ull;  // a hash slot whose block was streamed out (never a valid key)
constexpr uint32_t kArPresent = 1u << 30;       // archive entry: its payload is in the archive (not resident)

struct __align__(16) Slot {
  unsigned long long key;
  uint32_t val;    // heap id (28 bits) | level << 28 | kValNew, or kValPending
  uint32_t stamp;  // frame number of the last frame that touched the block
};

// Per touched block, written by k_bin in binned order: everything a fusion warp needs in one 16-byte load.
struct __align__(16) BlockMeta {
  unsigned long long key;
  uint32_t val;
  uint32_t slot;
};

struct DevState {
  int free_top[4];
  uint32_t touched_all;
  uint32_t touched_count[4];
  uint32_t retire_count;
  uint32_t frame;
  uint32_t status;
  uint32_t new_blocks, merged, split, rechecks, valid_rays;
  uint32_t n_fresh;  // LiDAR with the predictor or capture: new blocks listed for prediction this frame
  unsigned long long observations;
  unsigned long long updated_voxels;
  uint32_t obs_total;  // LiDAR: observation records allocated to segments this frame
  uint32_t n_over;     // LiDAR: points in stage_over
  uint32_t item_next;  // LiDAR point fusion: next work item to hand out
  uint32_t evicted, restored;  // streaming: blocks moved to the archive before this frame, and back by it
  uint32_t n_restore;          // streaming: restore jobs of this frame
  uint32_t ar_used;            // streaming: archive slots handed out (each key keeps its slot)
  uint32_t ar_present;         // streaming: blocks currently in the archive
  uint32_t evict_go;           // streaming: this frame's capacity check (taken once, before any eviction)
  uint32_t max_vox_obs;          // LiDAR: the most observations one voxel received in this scan
  unsigned long long mesh_tris;  // triangles counted by the last mesh extraction
  uint32_t mesh_next;            // mesh extraction: next chunk of 32 hash slots to hand out
};

// Everything a kernel needs, passed by value.
struct MapDev {
  Slot* slots;
  uint32_t slot_mask;
  int L;
  int fp16, color;
  int min_obs;
  uint8_t* heap[kMaxLevels];
  // per heap block of level l: the least stored D over the block's observed voxels (+inf when none is observed),
  // written by the fusion epilogue of every frame that touches the block; NaN when unknown (a block loaded from a
  // file before its first fusion). The raycast skips the interior of blocks whose value is above zero.
  float* dmin[kMaxLevels];
  uint32_t* free_stack[kMaxLevels];
  uint32_t max_blocks[kMaxLevels];
  uint32_t block_bytes[kMaxLevels];
  uint32_t* touched_all;
  uint32_t* touched[kMaxLevels];
  BlockMeta* meta[kMaxLevels];  // parallel to touched[l]
  uint32_t max_touched;
  uint32_t* retire;
  uint32_t* slot_pos;         // per slot: level << 28 | position in touched[level] (written by k_bin)
  // LiDAR observation buffers (per frame)
  uint32_t* blk_count;        // per touched block (levels concatenated): observations
  uint32_t* blk_off;          // start of the block's observation records (its fusion item's segment, in order)
  uint32_t* blk_fill;
  struct LidarRay* rays;      // per point of the current scan: its ray, computed once by the allocation pass
  uint2* stage;               // per point: kStageCap entries, its observation runs ({flag | block, length} + records)
  uint32_t* stage_len;        // per point: entries staged, or kStageOverflow
  uint32_t* stage_over;       // points whose runs did not fit (filled by a second walk)
  uint2* obs_rec;             // LiDAR observations grouped by block: {ray << 9 | voxel index in the block, d bits}
  uint2* obs_bin;             // the same records regrouped per voxel inside each block (fusion pass)
  uint32_t max_obs;
  DevState* st;
  // Raycast occupancy (insert-only open-addressing sets, filled when blocks are created): bricks of 4 x 4 x 4 blocks
  // with a 64-bit mask of their created blocks, and super-bricks of 4 x 4 x 4 bricks with a mask of their non-empty
  // bricks. Bit of cell (x, y, z) inside its parent: x + 4 y + 16 z.
  unsigned long long* brick_keys;
  unsigned long long* brick_bits;
  unsigned long long* super_keys;
  unsigned long long* super_bits;
  uint32_t super_mask;
  const uint16_t* pred_w;          // learned level predictor: BF16 weights, or null (variance rule only)
  int* cap_keys;                   // feature capture of new blocks (3 ints per record), or null
  float* cap_feat;                 // 16 floats per record
  uint32_t* cap_count;
  uint32_t cap_max;
  // LiDAR scans with the predictor or capture on (null otherwise), per touched entry i or fresh-list position f:
  unsigned long long* lidar_mom;   // [i]: end-point moments of a new block
  long long* lidar_end;            // [point]: end point in fixed point (x, y, z), written by the allocation pass
  uint32_t* fresh;                 // [f]: touched index of the f-th new block
  uint8_t* fresh_level;            // [i]: predicted level of a new block
  uint32_t brick_mask;
  float v[kMaxLevels];  // voxel edge per level
  float inv_v[kMaxLevels];  // 1 / v, as the float division computes it
  float E;              // block edge
  float tau;
  float fix_scale;      // 65536 / E (float), camera key quantisation
  double fix_scale64;   // 65536 / E (double), LiDAR key quantisation
  double theta[2];
  double split_h;
  // per level: merge threshold theta_l and split threshold h theta_{l-1} (in double, as the oracle compares), and
  // their nearest floats for the float-side decision
  double thr_merge[3], thr_split[3];
  float thr_merge_f[3], thr_split_f[3];
  float min_range, max_range;
  // capacity-driven streaming (off when ar_keys is null): the archive index (key -> slot | level << 28 | kArPresent,
  // linear probing), the archive itself (ar_slot_bytes per slot, pinned host memory mapped into the device's address
  // space) and this frame's restore jobs {heap value, archive slot}
  float stream_fraction;
  float stream_radius;
  unsigned long long* ar_keys;
  uint32_t* ar_vals;
  uint32_t ar_mask;
  uint32_t ar_cap;
  uint32_t ar_slot_bytes;
  uint8_t* ar_data;
  uint2* restore_jobs;
};

struct CamArgs {
  float fx, fy, cx, cy;
  int width, height;
  float min_depth, max_depth;
  float R[9];  // world <- camera rotation, row-major
  float t[3];
};

// ---------------------------------------------------------------------------------------------------- payload layout

__host__ __device__ inline uint32_t block_bytes_for(int nv, int fp16, int color) {
  return fp16 ? (uint32_t)nv * (2u + (color ? 6u : 0u) + 8u) : (uint32_t)nv * (12u + (color ? 12u : 0u));
}
// byte offsets of the fields inside one block of nv voxels
__host__ __device__ inline uint32_t off_W(int nv, int fp16, int color) {
  return fp16 ? (uint32_t)nv * (color ? 8u : 2u) : (uint32_t)nv * 4u;
}
__host__ __device__ inline uint32_t off_S2(int nv, int fp16, int color) { return off_W(nv, fp16, color) + nv * 4u; }
__host__ __device__ inline uint32_t off_C(int nv, int fp16, int q) {
  return fp16 ? (uint32_t)nv * (2u + 2u * q) : (uint32_t)nv * (12u + 4u * q);
}

// ---------------------------------------------------------------------------------------------------- keys and hashing

__host__ __device__ inline unsigned long long pack_key(long long x, long long y, long long z) {
  const long long b = 1LL << 20;
  return ((unsigned long long)(x + b) << 42) | ((unsigned long long)(y + b) << 21) | (unsigned long long)(z + b);
}
__host__ __device__ inline void unpack_key(unsigned long long k, int* x, int* y, int* z) {
  const long long b = 1LL << 20;
  *x = (int)((long long)((k >> 42) & 0x1FFFFF) - b);
  *y = (int)((long long)((k >> 21) & 0x1FFFFF) - b);
  *z = (int)((long long)(k & 0x1FFFFF) - b);
}

// Eq. 4: H(x, y, z) = (x p1 xor y p2 xor z p3) mod n_hash, 32-bit unsigned arithmetic, n_hash a power of two.
__host__ __device__ inline uint32_t hash_xyz(int x, int y, int z, uint32_t mask) {
  return (((uint32_t)x * 73856093u) ^ ((uint32_t)y * 19349669u) ^ ((uint32_t)z * 83492791u)) & mask;
}
__host__ __device__ inline uint32_t hash_key(unsigned long long k, uint32_t mask) {
  int x, y, z;
  unpack_key(k, &x, &y, &z);
  return hash_xyz(x, y, z, mask);
}

__host__ __device__ inline long long floor_div(long long a, long long b) {  // b > 0
  long long q = a / b;
  if ((a % b != 0) && (a < 0)) --q;
  return q;
}
__host__ __device__ inline bool key_ok(long long x, long long y, long long z) {
  return x >= -kKeyLimit && x <= kKeyLimit && y >= -kKeyLimit && y <= kKeyLimit && z >= -kKeyLimit &&
         z <= kKeyLimit;
}

// float -> fixed point floor(v * S), refused when |v S| >= 2^40
__device__ inline bool to_fixed_f(float v, float S, long long* out) {
  float p = v * S;
  if (!(fabsf(p) < 1099511627776.0f)) return false;
  *out = (long long)floorf(p);
  return true;
}
__device__ inline bool to_fixed_d(double v, double S, long long* out) {
  double p = v * S;
  if (!(fabs(p) < 1099511627776.0)) return false;
  *out = (long long)floor(p);
  return true;
}

__device__ inline void set_status(DevState* st, uint32_t bit) { atomicOr(&st->status, bit); }

// bit of a cell inside its 4 x 4 x 4 parent
__host__ __device__ inline unsigned long long cell_bit(int x, int y, int z) {
  return 1ull << ((x & 3) + 4 * (y & 3) + 16 * (z & 3));
}

// Insert key (x, y, z) into an insert-only set (keys[], bits[], linear probing from Eq. 4's hash) and OR `bit` into
// its mask. Returns false when no slot was found within the probe limit.
__device__ inline bool occupancy_insert(unsigned long long* keys, unsigned long long* bits, uint32_t mask, int x,
                                        int y, int z, unsigned long long bit) {
  const unsigned long long key = pack_key(x, y, z);
  const uint32_t h = hash_xyz(x, y, z, mask);
  for (uint32_t p = 0; p <= mask && p < (uint32_t)kMaxProbes; ++p) {
    const uint32_t s = (h + p) & mask;
    const unsigned long long cur = *(volatile unsigned long long*)&keys[s];
    if (cur != key) {
      if (cur != kEmptyKey) continue;
      const unsigned long long old = atomicCAS(&keys[s], kEmptyKey, key);
      if (old != kEmptyKey && old != key) continue;
    }
    if ((*(volatile unsigned long long*)&bits[s] & bit) == 0) atomicOr(&bits[s], bit);
    return true;
  }
  return false;
}

// Mask of key (x, y, z) in an occupancy set, 0 when absent.
__device__ inline unsigned long long occupancy_bits(const unsigned long long* keys, const unsigned long long* bits,
                                                    uint32_t mask, int x, int y, int z) {
  const unsigned long long key = pack_key(x, y, z);
  const uint32_t h = hash_xyz(x, y, z, mask);
  for (int p = 0; p < kMaxProbes; ++p) {
    const uint32_t s = (h + (uint32_t)p) & mask;
    const unsigned long long c = keys[s];
    if (c == key) return bits[s];
    if (c == kEmptyKey) return 0;
  }
  return 0;
}

// Single-thread lookup (linear probing from H). Returns the slot index or -1.
__device__ inline int lookup_slot(const Slot* slots, uint32_t mask, unsigned long long key) {
  uint32_t h = hash_key(key, mask);
  for (int p = 0; p < kMaxProbes; ++p) {
    uint32_t s = (h + (uint32_t)p) & mask;
    unsigned long long k = slots[s].key;
    if (k == key) return (int)s;
    if (k == kEmptyKey) return -1;
  }
  return -1;
}

// Exact cell walk over cells of edge U = 2^ush from A to B (fixed point). visit(cell) is called for every cell in
// order (ties: upward crossings first, then downward). Returns false if more than max_cells cells would be visited;
// a segment longer than max_cells + 1 cells along some axis is refused before any visit. Cell coordinates are below
// 2^23 in magnitude and, after that check, the segment and the distances to the next boundaries below 2^23, so the
// walk runs in 32-bit integers with 64-bit products for the exact crossing order.
template <class F>
__device__ inline bool walk_cells(const long long A[3], const long long B[3], int ush, int max_cells, F&& visit) {
  const int U = 1 << ush;
  const long long lim = (long long)(max_cells + 1) << ush;
  int cell[3], end[3], aD[3], N[3];
  bool pos[3], neg[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const long long d = B[i] - A[i];
    if (d > lim || d < -lim) return false;
    cell[i] = (int)(A[i] >> ush);  // arithmetic shift: floor division by 2^ush
    end[i] = (int)(B[i] >> ush);
    pos[i] = d > 0;
    neg[i] = d < 0;
    aD[i] = (int)(d < 0 ? -d : d);
    const int frac = (int)(A[i] & (long long)(U - 1));  // A - cell * U
    N[i] = pos[i] ? U - frac : (neg[i] ? frac : 0);
  }
  visit(cell);
  for (int n = 1; n < max_cells; ++n) {
    if (cell[0] == end[0] && cell[1] == end[1] && cell[2] == end[2]) return true;
    int best = -1;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      if (aD[i] == 0) continue;
      if (best < 0 || (long long)N[i] * aD[best] < (long long)N[best] * aD[i]) best = i;
    }
    bool tie[3], up = false, down = false;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      tie[i] = aD[i] != 0 && (long long)N[i] * aD[best] == (long long)N[best] * aD[i];
      up |= tie[i] && pos[i];
      down |= tie[i] && neg[i];
    }
    if (up) {
#pragma unroll
      for (int i = 0; i < 3; ++i)
        if (tie[i] && pos[i]) { cell[i] += 1; N[i] += U; }
      visit(cell);
    }
    if (down) {
      if (cell[0] == end[0] && cell[1] == end[1] && cell[2] == end[2]) return true;
#pragma unroll
      for (int i = 0; i < 3; ++i)
        if (tie[i] && neg[i]) { cell[i] -= 1; N[i] += U; }
      visit(cell);
    }
  }
  return cell[0] == end[0] && cell[1] == end[1] && cell[2] == end[2];
}

struct PoseD {
  double T[16];  // world <- sensor, row-major
};

// One LiDAR ray as the allocation pass computes it (in double) and the observation passes reuse it.
struct __align__(16) LidarRay {
  long long A[3], B[3];  // band end points, fixed point
  float rho;             // range, float of the double value; negative: the point gives no ray
  float rh[3];           // unit direction, float of the double value
};

// LiDAR ray of point j in double (Sec. 3.1 "3D Point Cloud"): origin o = sensor position, p = T x_s,
// rho = |p - o|, n = (p - o) / rho; band end points o + max(rho - tau, 0) n and o + (rho + tau) n as fixed point.
// Returns false for a point outside [min_range, max_range], non-finite, or out of key range.
__device__ inline bool lidar_ray(const MapDev& m, const PoseD& P, const float* xyz, uint64_t j, long long A[3],
                                 long long B[3], double* rho_out, double rhat[3], double p_out[3] = nullptr) {
  double xs[3] = {(double)xyz[3 * j], (double)xyz[3 * j + 1], (double)xyz[3 * j + 2]};
  double n2 = xs[0] * xs[0] + xs[1] * xs[1] + xs[2] * xs[2];
  double rmin2 = (double)m.min_range * (double)m.min_range, rmax2 = (double)m.max_range * (double)m.max_range;
  if (!(n2 >= rmin2 && n2 <= rmax2)) return false;
  const double* T = P.T;
  double dv[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double p = T[4 * a + 0] * xs[0] + T[4 * a + 1] * xs[1] + T[4 * a + 2] * xs[2] + T[4 * a + 3];
    dv[a] = p - T[4 * a + 3];
    if (p_out) p_out[a] = p;
  }
  // the ray's length and direction in float: double is kept for the pose composition above and for the fixed-point
  // band ends below, whose block keys must not lose precision at 80 m
  const float d0 = (float)dv[0], d1 = (float)dv[1], d2 = (float)dv[2];
  const float rf = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
  rhat[0] = (double)(d0 / rf);
  rhat[1] = (double)(d1 / rf);
  rhat[2] = (double)(d2 / rf);
  const double rho = (double)rf, tau = (double)m.tau;
  double t0 = rho - tau;
  if (t0 < 0.0) t0 = 0.0;
  double t1 = rho + tau;
  bool ok = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    ok = ok && to_fixed_d(T[4 * a + 3] + t0 * rhat[a], m.fix_scale64, &A[a]);
    ok = ok && to_fixed_d(T[4 * a + 3] + t1 * rhat[a], m.fix_scale64, &B[a]);
  }
  *rho_out = rho;
  return ok && key_ok(floor_div(A[0], kBlockUnit), floor_div(A[1], kBlockUnit), floor_div(A[2], kBlockUnit)) &&
         key_ok(floor_div(B[0], kBlockUnit), floor_div(B[1], kBlockUnit), floor_div(B[2], kBlockUnit));
}

// ---------------------------------------------------------------------------------------------------- host side

// the device-side view of a map (mrh_map.cu), for the batched path
const MapDev* map_dev(const mrh_map* m, int* device, int* sms);

// launch helpers implemented in the .cu files
void launch_alloc_depth(const MapDev& m, const CamArgs& c, const float* depth, const uint8_t* rgb, float* rho_img,
                        uint32_t* rgb_img, cudaStream_t s);
void launch_alloc_points(const MapDev& m, const double* T, const float* xyz, uint64_t n, cudaStream_t s);
void launch_bin(const MapDev& m, cudaStream_t s, int sms);
void launch_bin_points(const MapDev& m, const double* T, const float* xyz, uint64_t n, cudaStream_t s, int sms);
// Record the failing call's text for mrh_last_cuda_error (calling thread) and return MRH_ERR_CUDA.
mrh_status cuda_fail(cudaError_t e, const char* what);
void launch_bin_camera(const MapDev& m, const CamArgs& c, const float* rho_img, cudaStream_t s, int sms);
void launch_fuse_depth(const MapDev& m, const CamArgs& c, const float* rho, const uint32_t* rgb, cudaStream_t s,
                       int sms);
void launch_fuse_points(const MapDev& m, const double* T, const float* xyz, uint64_t n, cudaStream_t s, int sms);
void launch_lidar_observations(const MapDev& m, const double* T, const float* xyz, uint64_t n, cudaStream_t s,
                               int sms);
void launch_raycast(const MapDev& m, const CamArgs& c, float* depth, float* normal, uint8_t* rgb,
                   cudaStream_t s);
// multi-resolution Marching Cubes (mrh_mesh.cu): the case table is uploaded once per device
cudaError_t mesh_table_ready(int device);
void host_case_table(uint8_t* ntri, int8_t* tri, int8_t* edge_end);
void launch_mesh(const MapDev& m, float* tris, uint64_t cap, unsigned long long* count, cudaStream_t s, int sms);
// vertex collapse of a triangle soup (mrh_mesh.cu); scratch sized by the caller
constexpr int kWeldScanBlock = 1024;
struct WeldScratch {
  unsigned long long* keys;  // table: packed cluster key, ~0 = empty
  uint32_t* mn;              // table: smallest member, 3 order-preserving encodings per slot
  uint32_t* vslot;           // per input vertex: its table slot
  uint32_t* vidx;            // table: output vertex index
  unsigned long long* ckeys; // occupied slots' keys, sorted
  uint32_t* cslots;          // ... and their slots
  uint32_t* blk;             // per scan block: kept count, then its first position
  uint32_t* counters;        // [0] clusters, [1] key out of range, [2] faces, [3] compaction cursor
  uint32_t table;
};
cudaError_t weld_clusters(const WeldScratch& w, const float* tris, uint32_t nv, float delta, cudaStream_t s, int sms);
cudaError_t weld_output(const WeldScratch& w, const float* tris, uint32_t n_clusters, float* verts, uint64_t cap_verts,
                        int32_t* faces, uint64_t cap_faces, uint64_t n_tris, size_t nblk, cudaStream_t s, int sms);
void sort_keys_vals(unsigned long long* keys, uint32_t* vals, uint32_t n_pow, cudaStream_t s, int sms);
// stream-ordered scratch from a pool owned by the library (one per device, memory kept for reuse)
cudaError_t scratch_alloc(void** p, size_t bytes, int device, cudaStream_t s);
// capacity-driven streaming (mrh_stream.cu)
void launch_evict_camera(const MapDev& m, const CamArgs& c, cudaStream_t s, int sms);
void launch_evict_lidar(const MapDev& m, const double* T, cudaStream_t s, int sms);
void launch_restore(const MapDev& m, cudaStream_t s, int sms);
// map save / load (mrh_io.cu): block payloads to and from a host blob (one staging copy each way)
cudaError_t io_blocks_to_blob(const MapDev& m, const std::vector<uint32_t>& level_ids,
                              const std::vector<uint64_t>& offsets, uint8_t* blob_host, uint64_t blob_bytes,
                              cudaStream_t s, int sms);
cudaError_t io_blob_to_blocks(const MapDev& m, const std::vector<int32_t>& keys, const std::vector<uint32_t>& levels,
                              const std::vector<uint64_t>& offsets, const uint8_t* blob_host, uint64_t blob_bytes,
                              cudaStream_t s, int sms);
// Gaussian splats (mrh_splat.cu)
struct SplatInputs {
  const float* means;    // n x 3
  const float* covs;     // n x 6: Sigma_W xx, xy, xz, yy, yz, zz
  const float* opacity;  // n
  const float* colors;   // n x 3
  uint64_t n;
};
constexpr uint64_t kSplatMaxPairs = 0x7FFFFFFFull;  // tile-Gaussian pairs of one render
cudaError_t splat_render(const SplatInputs& in, const CamArgs& c, float* rgb, float* trans, uint64_t* n_pairs,
                         int device, cudaStream_t s, int sms);

const char* io_magic();
uint32_t io_version();
// contrast quadtree (mrh_quadtree.cu)
size_t quadtree_scratch_bytes(int width, int height);
cudaError_t launch_quadtree(const uint8_t* rgb, int width, int height, double threshold, int min_size,
                            int32_t* leaves, uint64_t cap, void* scratch, unsigned long long** n_leaves_dev,
                            cudaStream_t s, int sms);

}  // namespace mrh
