// Map lifetime, per-frame orchestration and read-out: the C ABI of include/mrhash.h.
//
// A depth frame is five stream-ordered launches with no host round trip:
//   k_begin        frame number + 1, per-frame counters to zero
//   k_alloc_*      ray -> block allocation into the hash table, touched list           (mrh_alloc.cu)
//   k_bin          new blocks get a level-0 heap block; touched slots binned by level  (mrh_alloc.cu)
//   k_fuse_*       fusion + block variance + re-levelling                              (mrh_fuse.cu, mrh_lidar.cu)
//   k_release      heap blocks freed by re-levelling go back to their free stacks
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "mrh_alloc.cuh"
#include "mrh_internal.cuh"
#include "mrh_sort.cuh"

using namespace mrh;

struct mrh_map {
  int device = 0;
  int sms = 148;
  mrh_map_params p{};
  MapDev d{};
  // owned device allocations
  std::vector<void*> allocs;
  // per-kernel-group accounting
  bool profiling = false;
  double prof_ms[MRH_K_COUNT] = {};
  uint64_t launches[MRH_K_COUNT] = {};
  struct Pending {
    int kid;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> event_pool;
  // per-frame images for the camera path (range image, packed colour), grown to the largest frame seen
  // streaming archive (pinned host memory, mapped into the device's address space)
  uint8_t* archive_host = nullptr;
  float* rho_img = nullptr;
  uint32_t* rgb_img = nullptr;
  size_t img_pixels = 0;
  // per-point buffers of the LiDAR path (rays, staged observation runs), grown to the largest scan seen
  LidarRay* rays = nullptr;
  uint2* stage = nullptr;
  uint32_t* stage_len = nullptr;
  uint32_t* stage_over = nullptr;
  size_t ray_cap = 0;
  // learned level predictor weights (BF16), owned; d.pred_w points here while the predictor is on
  uint16_t* pred_buf = nullptr;
  // LiDAR scans with the predictor or capture: end-point moments, fresh list and levels of the new blocks
  // (one allocation sized by max_touched, made by the first scan that needs it) and the scan's end points (grown to
  // the largest scan)
  void* lidar_pred = nullptr;
  long long* lidar_end = nullptr;
  size_t end_cap = 0;
};

namespace mrh {

namespace {
thread_local char g_cuda_err[256] = "";
}  // namespace

mrh_status cuda_fail(cudaError_t e, const char* what) {
  std::snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", what, cudaGetErrorString(e));
  return MRH_ERR_CUDA;
}

namespace {

#define MRH_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

// Restores the caller's current device on scope exit.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess) ok = true;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

bool finite_pose(const double* T) {
  if (!T) return false;
  for (int i = 0; i < 16; ++i)
    if (!std::isfinite(T[i])) return false;
  return true;
}

mrh_status status_from_bits(uint32_t bits) {
  if (bits & kStHashFull) return MRH_ERR_HASH_FULL;
  if (bits & kStPoolEmpty) return MRH_ERR_POOL_EMPTY;
  if (bits & kStListFull) return MRH_ERR_LIST_FULL;
  if (bits & kStObsFull) return MRH_ERR_LIST_FULL;
  if (bits & kStSegment) return MRH_ERR_INVALID_ARG;
  if (bits & kStArchiveFull) return MRH_ERR_CAPACITY;
  return MRH_OK;
}

cudaEvent_t take_event(mrh_map* m) {
  if (!m->event_pool.empty()) {
    cudaEvent_t e = m->event_pool.back();
    m->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Brackets one kernel group with events when profiling; counts launches always.
struct KernelScope {
  mrh_map* m;
  int kid;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  KernelScope(mrh_map* m_, int kid_, cudaStream_t s_, int n_launches) : m(m_), kid(kid_), s(s_) {
    m->launches[kid] += (uint64_t)n_launches;
    if (m->profiling) {
      a = take_event(m);
      cudaEventRecord(a, s);
    }
  }
  ~KernelScope() {
    if (a) {
      cudaEvent_t b = take_event(m);
      cudaEventRecord(b, s);
      m->pending.push_back({kid, a, b});
    }
  }
};

mrh_status collect_profile(mrh_map* m) {
  for (auto& p : m->pending) {
    float ms = 0.f;
    cudaError_t e = cudaEventElapsedTime(&ms, p.a, p.b);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
    m->prof_ms[p.kid] += ms;
    m->event_pool.push_back(p.a);
    m->event_pool.push_back(p.b);
  }
  m->pending.clear();
  return MRH_OK;
}

__global__ void k_init_stack(uint32_t* stack, uint32_t cap) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += gridDim.x * blockDim.x) stack[i] = cap - 1 - i;
}

__global__ void k_begin(DevState* st) { begin_frame(st); }

__global__ void __launch_bounds__(256) k_release(MapDev m) {
  const uint32_t n = m.st->retire_count;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) release_one(m, i);
}

// ---- read-out kernels

__global__ void k_compact(MapDev m, unsigned long long* keys, uint32_t* slots_out, uint32_t* count, uint32_t cap) {
  const uint32_t n = m.slot_mask + 1;
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    Slot sl = m.slots[s];
    if (sl.key != kEmptyKey && sl.val != kValPending) {
      uint32_t i = atomicAdd(count, 1u);
      if (i < cap) {
        keys[i] = sl.key;
        slots_out[i] = s;
      }
    }
  }
}

__global__ void k_pad_keys(unsigned long long* keys, uint32_t from, uint32_t to) {
  for (uint32_t i = from + blockIdx.x * blockDim.x + threadIdx.x; i < to; i += gridDim.x * blockDim.x)
    keys[i] = kEmptyKey;
}

// one compare-exchange step (k, j) of a bitonic sort, ascending
__global__ void k_bitonic_step(unsigned long long* keys, uint32_t* vals, uint32_t n, uint32_t k, uint32_t j) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    uint32_t p = i ^ j;
    if (p <= i) continue;
    bool asc = (i & k) == 0;
    unsigned long long a = keys[i], b = keys[p];
    if ((a > b) == asc) {
      keys[i] = b;
      keys[p] = a;
      uint32_t t = vals[i];
      vals[i] = vals[p];
      vals[p] = t;
    }
  }
}

// exclusive scan of voxel counts over the sorted blocks (one CTA, chunks of 1024)
__global__ void __launch_bounds__(1024) k_voxel_offsets(MapDev m, const uint32_t* slots, uint32_t n,
                                                        unsigned long long* off) {
  __shared__ unsigned long long s[1024];
  __shared__ unsigned long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint32_t base = 0; base < n; base += 1024) {
    uint32_t i = base + threadIdx.x;
    unsigned long long v = 0;
    if (i < n) {
      uint32_t l = (m.slots[slots[i]].val >> 28) & 3u;
      int nl = kFineDim >> l;
      v = (unsigned long long)(nl * nl * nl);
    }
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      unsigned long long t = threadIdx.x >= (unsigned)o ? s[threadIdx.x - o] : 0;
      __syncthreads();
      s[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < n) off[i] = carry + s[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += s[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) off[n] = carry;
}

__global__ void k_extract(MapDev m, const uint32_t* slots, uint32_t n, const unsigned long long* off, int32_t* keys,
                          uint8_t* levels, unsigned long long* off_out, float* D, float* W, float* S2, float* C) {
  for (uint32_t b = blockIdx.x; b < n; b += gridDim.x) {
    Slot sl = m.slots[slots[b]];
    uint32_t l = (sl.val >> 28) & 3u, ptr = sl.val & kPtrMask;
    int nl = kFineDim >> l, nv = nl * nl * nl;
    const uint8_t* blk = m.heap[l] + (size_t)ptr * m.block_bytes[l];
    unsigned long long o = off[b];
    if (threadIdx.x == 0) {
      int x, y, z;
      unpack_key(sl.key, &x, &y, &z);
      keys[3 * b] = x;
      keys[3 * b + 1] = y;
      keys[3 * b + 2] = z;
      levels[b] = (uint8_t)l;
      off_out[b] = o;
      if (b == n - 1) off_out[n] = off[n];
    }
    for (int i = threadIdx.x; i < nv; i += blockDim.x) {
      float dv = m.fp16 ? __half2float(reinterpret_cast<const __half*>(blk)[i])
                        : reinterpret_cast<const float*>(blk)[i];
      D[o + i] = dv;
      W[o + i] = reinterpret_cast<const float*>(blk + off_W(nv, m.fp16, m.color))[i];
      S2[o + i] = reinterpret_cast<const float*>(blk + off_S2(nv, m.fp16, m.color))[i];
      if (C) {
        for (int q = 0; q < 3; ++q) {
          float cv = 0.f;
          if (m.color) {
            const uint8_t* pc = blk + off_C(nv, m.fp16, q);
            cv = m.fp16 ? __half2float(reinterpret_cast<const __half*>(pc)[i]) : reinterpret_cast<const float*>(pc)[i];
          }
          C[3 * (o + i) + q] = cv;
        }
      }
    }
  }
}

mrh_status validate_params(const mrh_map_params* p) {
  if (!p) return MRH_ERR_INVALID_ARG;
  if (p->n_levels < 1 || p->n_levels > kMaxLevels) return MRH_ERR_INVALID_ARG;
  if (!(p->base_voxel_size > 0.f) || !std::isfinite(p->base_voxel_size)) return MRH_ERR_INVALID_ARG;
  if (!(p->truncation > 0.f) || !std::isfinite(p->truncation)) return MRH_ERR_INVALID_ARG;
  float v0 = p->base_voxel_size / (float)(1 << (p->n_levels - 1));
  float E = v0 * (float)kFineDim;
  if (2.0f * p->truncation > 8.0f * E) return MRH_ERR_INVALID_ARG;
  if (p->hash_slots_log2 < 10 || p->hash_slots_log2 > 28) return MRH_ERR_INVALID_ARG;
  for (int l = 0; l < p->n_levels; ++l)
    if (p->max_blocks[l] < 1 || p->max_blocks[l] > kPtrMask) return MRH_ERR_INVALID_ARG;
  if (p->max_touched < 1 || p->max_touched > (1u << 28)) return MRH_ERR_INVALID_ARG;
  if (p->storage != MRH_STORAGE_FP32 && p->storage != MRH_STORAGE_FP16) return MRH_ERR_INVALID_ARG;
  if (p->has_color != 0 && p->has_color != 1) return MRH_ERR_INVALID_ARG;
  for (int l = 0; l < 2; ++l)
    if (!std::isfinite(p->var_threshold[l])) return MRH_ERR_INVALID_ARG;
  if (!(p->split_hysteresis >= 0.0) || !std::isfinite(p->split_hysteresis)) return MRH_ERR_INVALID_ARG;
  if (p->min_obs < 0) return MRH_ERR_INVALID_ARG;
  if (!(p->min_range >= 0.f) || !(p->max_range >= p->min_range)) return MRH_ERR_INVALID_ARG;
  return MRH_OK;
}

mrh_status validate_pinhole(const mrh_pinhole* K) {
  if (!K) return MRH_ERR_INVALID_ARG;
  if (K->width <= 0 || K->height <= 0 || (long long)K->width * K->height > (1LL << 28)) return MRH_ERR_INVALID_ARG;
  if (!(K->fx > 0.f) || !(K->fy > 0.f) || !std::isfinite(K->fx) || !std::isfinite(K->fy)) return MRH_ERR_INVALID_ARG;
  if (!std::isfinite(K->cx) || !std::isfinite(K->cy)) return MRH_ERR_INVALID_ARG;
  if (!(K->min_depth >= 0.f) || !(K->max_depth >= K->min_depth) || !std::isfinite(K->max_depth))
    return MRH_ERR_INVALID_ARG;
  return MRH_OK;
}

CamArgs cam_args(const mrh_pinhole* K, const double* T) {
  CamArgs c;
  c.fx = K->fx; c.fy = K->fy; c.cx = K->cx; c.cy = K->cy;
  c.width = K->width; c.height = K->height;
  c.min_depth = K->min_depth; c.max_depth = K->max_depth;
  for (int r = 0; r < 3; ++r) {
    for (int q = 0; q < 3; ++q) c.R[3 * r + q] = (float)T[4 * r + q];
    c.t[r] = (float)T[4 * r + 3];
  }
  return c;
}

template <class T>
mrh_status dev_alloc(mrh_map* m, T** out, size_t count) {
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, count * sizeof(T) > 0 ? count * sizeof(T) : 16);
  if (e != cudaSuccess) {
    cuda_fail(e, "cudaMalloc");
    return MRH_ERR_OUT_OF_MEMORY;
  }
  m->allocs.push_back(p);
  *out = (T*)p;
  return MRH_OK;
}

void free_capture(mrh_map* m) {
  if (m->d.cap_keys) cudaFree(m->d.cap_keys);
  if (m->d.cap_feat) cudaFree(m->d.cap_feat);
  if (m->d.cap_count) cudaFree(m->d.cap_count);
  m->d.cap_keys = nullptr;
  m->d.cap_feat = nullptr;
  m->d.cap_count = nullptr;
  m->d.cap_max = 0;
}

void free_all(mrh_map* m) {
  for (void* p : m->allocs) cudaFree(p);
  m->allocs.clear();
  if (m->archive_host) cudaFreeHost(m->archive_host);
  m->archive_host = nullptr;
  if (m->rho_img) cudaFree(m->rho_img);
  if (m->rgb_img) cudaFree(m->rgb_img);
  if (m->pred_buf) cudaFree(m->pred_buf);
  if (m->lidar_pred) cudaFree(m->lidar_pred);
  if (m->lidar_end) cudaFree(m->lidar_end);
  free_capture(m);
  m->pred_buf = nullptr;
  m->lidar_pred = nullptr;
  m->lidar_end = nullptr;
  m->end_cap = 0;
  m->d.lidar_mom = nullptr;
  m->d.lidar_end = nullptr;
  m->d.fresh = nullptr;
  m->d.fresh_level = nullptr;
  m->d.pred_w = nullptr;
  m->rho_img = nullptr;
  m->rgb_img = nullptr;
  m->img_pixels = 0;
  for (void* p : {(void*)m->rays, (void*)m->stage, (void*)m->stage_len, (void*)m->stage_over})
    if (p) cudaFree(p);
  m->rays = nullptr;
  m->stage = nullptr;
  m->stage_len = nullptr;
  m->stage_over = nullptr;
  m->ray_cap = 0;
  for (auto& p : m->pending) {
    m->event_pool.push_back(p.a);
    m->event_pool.push_back(p.b);
  }
  m->pending.clear();
  for (cudaEvent_t e : m->event_pool) cudaEventDestroy(e);
  m->event_pool.clear();
}

}  // namespace
}  // namespace mrh

namespace mrh {
namespace {
std::mutex g_pool_mutex;
cudaMemPool_t g_pool[64] = {};
}  // namespace

// The scratch of the read-out calls (mesh collapse, quadtree) comes from one memory pool per device that keeps its
// memory between calls (release threshold unlimited), so repeated calls do not map and unmap device memory.
cudaError_t scratch_alloc(void** p, size_t bytes, int device, cudaStream_t s) {
  if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
  cudaMemPool_t pool;
  {
    std::lock_guard<std::mutex> lock(g_pool_mutex);
    if (!g_pool[device]) {
      cudaMemPoolProps props{};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = device;
      cudaError_t e = cudaMemPoolCreate(&g_pool[device], &props);
      if (e != cudaSuccess) {
        g_pool[device] = nullptr;
        return e;
      }
      uint64_t keep = ~0ull;
      cudaMemPoolSetAttribute(g_pool[device], cudaMemPoolAttrReleaseThreshold, &keep);
    }
    pool = g_pool[device];
  }
  return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

// ascending sort of n_pow (a power of two) keys with their values (bitonic network, one launch per step)
void sort_keys_vals(unsigned long long* keys, uint32_t* vals, uint32_t n_pow, cudaStream_t s, int sms) {
  for (uint32_t k = 2; k <= n_pow; k <<= 1)
    for (uint32_t j = k >> 1; j > 0; j >>= 1) k_bitonic_step<<<sms * 8, 256, 0, s>>>(keys, vals, n_pow, k, j);
}

const MapDev* map_dev(const mrh_map* m, int* device, int* sms) {
  *device = m->device;
  *sms = m->sms;
  return &m->d;
}
}  // namespace mrh

// ------------------------------------------------------------------------------------------------ static scratch
//
// mrh_extract_blocks_noalloc sorts and scans inside this one array instead of allocating. Host code must not use the
// symbol as a pointer: its device address is looked up on every call (cudaGetSymbolAddress, with the map's device
// current; cheap next to the sort launches) and passed to the kernels, so no address outlives a device reset.
namespace mrh {
namespace {

constexpr uint32_t kNoallocMaxBlocks = MRH_NOALLOC_MAX_BLOCKS;
constexpr size_t kNoallocKeysOff = 0;                                               // u64 keys[max]
constexpr size_t kNoallocSlotsOff = kNoallocKeysOff + 8ull * kNoallocMaxBlocks;      // u32 slots[max]
constexpr size_t kNoallocOffsOff = kNoallocSlotsOff + 4ull * kNoallocMaxBlocks;      // u64 offsets[max + 1]
constexpr size_t kNoallocCountOff = kNoallocOffsOff + 8ull * (kNoallocMaxBlocks + 1); // u32 count
constexpr size_t kNoallocBytes = (kNoallocCountOff + 4 + 255) / 256 * 256;

static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoallocBytes];

// device address of the scratch array on the current device
mrh_status noalloc_scratch(uint8_t** out) {
  void* ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess || !ptr) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
  *out = (uint8_t*)ptr;
  return MRH_OK;
}

}  // namespace
}  // namespace mrh

// ------------------------------------------------------------------------------------------------ C ABI

extern "C" {

mrh_status mrh_map_create(const mrh_map_params* params, int device, mrh_map** out) {
  if (!out) return MRH_ERR_INVALID_ARG;
  *out = nullptr;
  mrh_status st = validate_params(params);
  if (st != MRH_OK) return st;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return MRH_ERR_INVALID_ARG;
  DeviceGuard guard(device);
  if (!guard.ok) return cuda_fail(cudaGetLastError(), "cudaSetDevice");
  mrh_map* m = new (std::nothrow) mrh_map();
  if (!m) return MRH_ERR_OUT_OF_MEMORY;
  m->device = device;
  m->p = *params;
  cudaDeviceGetAttribute(&m->sms, cudaDevAttrMultiProcessorCount, device);
  MapDev& d = m->d;
  d.L = params->n_levels;
  d.fp16 = params->storage == MRH_STORAGE_FP16;
  d.color = params->has_color;
  d.min_obs = params->min_obs;
  float v0 = params->base_voxel_size / (float)(1 << (d.L - 1));
  for (int l = 0; l < kMaxLevels; ++l) {
    d.v[l] = v0 * (float)(1 << l);
    d.inv_v[l] = 1.0f / d.v[l];
  }
  d.E = v0 * (float)kFineDim;
  d.tau = params->truncation;
  d.fix_scale = 65536.0f / d.E;
  d.fix_scale64 = 65536.0 / (double)d.E;
  d.theta[0] = params->var_threshold[0];
  d.theta[1] = params->var_threshold[1];
  d.split_h = params->split_hysteresis;
  for (int l = 0; l < kMaxLevels; ++l) {
    d.thr_merge[l] = l < 2 ? d.theta[l] : 0.0;
    d.thr_split[l] = l > 0 ? d.split_h * d.theta[l - 1] : 0.0;
    d.thr_merge_f[l] = (float)d.thr_merge[l];
    d.thr_split_f[l] = (float)d.thr_split[l];
  }
  d.min_range = params->min_range;
  d.max_range = params->max_range;
  d.max_touched = params->max_touched;
  const uint32_t n_slots = 1u << params->hash_slots_log2;
  d.slot_mask = n_slots - 1;
#define TRY(x)               \
  do {                       \
    mrh_status s_ = (x);     \
    if (s_ != MRH_OK) {      \
      free_all(m);           \
      delete m;              \
      return s_;             \
    }                        \
  } while (0)
  TRY(dev_alloc(m, &d.slots, n_slots));
  TRY(dev_alloc(m, &d.st, 1));
  TRY(dev_alloc(m, &d.touched_all, params->max_touched));
  TRY(dev_alloc(m, &d.retire, params->max_touched));
  TRY(dev_alloc(m, &d.slot_pos, n_slots));
  const uint32_t n_brick_slots = 1u << (params->hash_slots_log2 > 12 ? params->hash_slots_log2 - 2 : 10);
  d.brick_mask = n_brick_slots - 1;
  TRY(dev_alloc(m, &d.brick_keys, n_brick_slots));
  TRY(dev_alloc(m, &d.brick_bits, n_brick_slots));
  const uint32_t n_super_slots = std::max(n_brick_slots >> 3, 1024u);
  d.super_mask = n_super_slots - 1;
  TRY(dev_alloc(m, &d.super_keys, n_super_slots));
  TRY(dev_alloc(m, &d.super_bits, n_super_slots));
  TRY(dev_alloc(m, &d.blk_count, 3ull * params->max_touched));
  TRY(dev_alloc(m, &d.blk_fill, 3ull * params->max_touched));
  TRY(dev_alloc(m, &d.blk_off, 3ull * params->max_touched + 1));
  d.max_obs = params->max_observations;
  TRY(dev_alloc(m, &d.obs_rec, d.max_obs));
  TRY(dev_alloc(m, &d.obs_bin, d.max_obs));
  for (int l = 0; l < kMaxLevels; ++l) {
    int nl = kFineDim >> l;
    d.block_bytes[l] = block_bytes_for(nl * nl * nl, d.fp16, d.color);
    d.max_blocks[l] = l < d.L ? params->max_blocks[l] : 0;
    if (l < d.L) {
      TRY(dev_alloc(m, &d.heap[l], (size_t)d.max_blocks[l] * d.block_bytes[l]));
      TRY(dev_alloc(m, &d.dmin[l], d.max_blocks[l]));
      TRY(dev_alloc(m, &d.free_stack[l], d.max_blocks[l]));
      TRY(dev_alloc(m, &d.touched[l], params->max_touched));
      TRY(dev_alloc(m, &d.meta[l], params->max_touched));
    } else {
      d.heap[l] = nullptr;
      d.dmin[l] = nullptr;
      d.free_stack[l] = nullptr;
      d.touched[l] = nullptr;
      d.meta[l] = nullptr;
    }
  }
#undef TRY
  cudaError_t e = cudaMemset(d.slots, 0xFF, (size_t)n_slots * sizeof(Slot));
  if (e == cudaSuccess) e = cudaMemset(d.brick_keys, 0xFF, (size_t)n_brick_slots * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(d.brick_bits, 0, (size_t)n_brick_slots * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(d.super_keys, 0xFF, (size_t)n_super_slots * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(d.super_bits, 0, (size_t)n_super_slots * sizeof(unsigned long long));
  for (int l = 0; l < d.L && e == cudaSuccess; ++l)  // all ones: NaN, unknown until fused
    e = cudaMemset(d.dmin[l], 0xFF, (size_t)d.max_blocks[l] * sizeof(float));
  DevState hs;
  std::memset(&hs, 0, sizeof(hs));
  for (int l = 0; l < kMaxLevels; ++l) hs.free_top[l] = (int)d.max_blocks[l];
  if (e == cudaSuccess) e = cudaMemcpy(d.st, &hs, sizeof(hs), cudaMemcpyHostToDevice);
  for (int l = 0; l < d.L && e == cudaSuccess; ++l) {
    k_init_stack<<<m->sms * 4, 256>>>(d.free_stack[l], d.max_blocks[l]);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    free_all(m);
    delete m;
    return cuda_fail(e, "map initialisation");
  }
  *out = m;
  return MRH_OK;
}

mrh_status mrh_map_destroy(mrh_map* m) {
  if (!m) return MRH_OK;
  DeviceGuard guard(m->device);
  cudaDeviceSynchronize();
  free_all(m);
  delete m;
  return MRH_OK;
}

mrh_status mrh_set_streaming(mrh_map* m, float fraction, float radius, uint32_t archive_blocks) {
  if (!m || !(fraction >= 0.0f && fraction <= 1.0f) || !(radius >= 0.0f) || !std::isfinite(radius))
    return MRH_ERR_INVALID_ARG;
  if (fraction > 0.0f && (m->d.pred_w || m->d.cap_feat)) return MRH_ERR_INVALID_ARG;
  DeviceGuard guard(m->device);
  if (!guard.ok) return cuda_fail(cudaGetLastError(), "cudaSetDevice");
  MRH_CUDA(cudaDeviceSynchronize());
  MapDev& d = m->d;
  if (fraction == 0.0f) {  // off: archived blocks stay archived
    d.stream_fraction = 0.0f;
    d.ar_keys = nullptr;
    return MRH_OK;
  }
  if (!m->archive_host || archive_blocks != d.ar_cap) {
    DevState hs;
    MRH_CUDA(cudaMemcpy(&hs, d.st, sizeof(hs), cudaMemcpyDeviceToHost));
    if (m->archive_host && hs.ar_present > 0) return MRH_ERR_INVALID_ARG;  // the archive holds blocks
    if (archive_blocks == 0 || archive_blocks > (1u << 27)) return MRH_ERR_INVALID_ARG;
    if (m->archive_host) {
      cudaFreeHost(m->archive_host);
      m->archive_host = nullptr;
    }
    uint32_t entries = 1024;
    while (entries < 2u * archive_blocks) entries <<= 1;
    const size_t slot_bytes = d.block_bytes[0];
    cudaError_t e = cudaHostAlloc((void**)&m->archive_host, (size_t)archive_blocks * slot_bytes,
                                  cudaHostAllocMapped | cudaHostAllocPortable);
    if (e != cudaSuccess) {
      m->archive_host = nullptr;
      return MRH_ERR_OUT_OF_MEMORY;
    }
    void* dev_ptr = nullptr;
    MRH_CUDA(cudaHostGetDevicePointer(&dev_ptr, m->archive_host, 0));
    unsigned long long* keys = nullptr;
    uint32_t* vals = nullptr;
    uint2* jobs = nullptr;
    if (dev_alloc(m, &keys, entries) != MRH_OK || dev_alloc(m, &vals, entries) != MRH_OK ||
        dev_alloc(m, &jobs, d.max_touched) != MRH_OK)
      return MRH_ERR_OUT_OF_MEMORY;
    MRH_CUDA(cudaMemset(keys, 0xFF, (size_t)entries * sizeof(unsigned long long)));
    hs.ar_used = 0;
    hs.ar_present = 0;
    MRH_CUDA(cudaMemcpy(&d.st->ar_used, &hs.ar_used, sizeof(uint32_t), cudaMemcpyHostToDevice));
    MRH_CUDA(cudaMemcpy(&d.st->ar_present, &hs.ar_present, sizeof(uint32_t), cudaMemcpyHostToDevice));
    d.ar_keys = keys;
    d.ar_vals = vals;
    d.ar_mask = entries - 1;
    d.ar_cap = archive_blocks;
    d.ar_slot_bytes = (uint32_t)slot_bytes;
    d.ar_data = (uint8_t*)dev_ptr;
    d.restore_jobs = jobs;
  } else if (!d.ar_keys) {
    return MRH_ERR_INVALID_ARG;  // re-enabling after switching off is not supported
  }
  d.stream_fraction = fraction;
  d.stream_radius = radius;
  return MRH_OK;
}

mrh_status mrh_set_predictor(mrh_map* m, const uint16_t* bf16_weights_host, uint64_t n_params) {
  if (!m) return MRH_ERR_INVALID_ARG;
  if (bf16_weights_host && m->d.ar_keys) return MRH_ERR_INVALID_ARG;  // not combined with streaming
  if (!bf16_weights_host) {
    m->d.pred_w = nullptr;
    return MRH_OK;
  }
  if (n_params != (uint64_t)MRH_MLP_PARAMS) return MRH_ERR_INVALID_ARG;
  for (uint64_t i = 0; i < n_params; ++i)
    if ((bf16_weights_host[i] & 0x7F80u) == 0x7F80u) return MRH_ERR_INVALID_ARG;  // inf or nan
  DeviceGuard guard(m->device);
  if (!guard.ok) return cuda_fail(cudaGetLastError(), "cudaSetDevice");
  MRH_CUDA(cudaDeviceSynchronize());  // frames in flight may still read the old weights
  if (!m->pred_buf) MRH_CUDA(cudaMalloc(&m->pred_buf, sizeof(uint16_t) * MRH_MLP_PARAMS));
  MRH_CUDA(cudaMemcpy(m->pred_buf, bf16_weights_host, sizeof(uint16_t) * MRH_MLP_PARAMS, cudaMemcpyHostToDevice));
  m->d.pred_w = m->pred_buf;
  return MRH_OK;
}

mrh_status mrh_set_feature_capture(mrh_map* m, uint32_t capacity) {
  if (!m || (capacity > 0 && m->d.ar_keys)) return MRH_ERR_INVALID_ARG;
  DeviceGuard guard(m->device);
  if (!guard.ok) return cuda_fail(cudaGetLastError(), "cudaSetDevice");
  MRH_CUDA(cudaDeviceSynchronize());
  free_capture(m);
  if (capacity == 0) return MRH_OK;
  cudaError_t e = cudaMalloc(&m->d.cap_keys, sizeof(int) * 3 * (size_t)capacity);
  if (e == cudaSuccess) e = cudaMalloc(&m->d.cap_feat, sizeof(float) * MRH_MLP_IN * (size_t)capacity);
  if (e == cudaSuccess) e = cudaMalloc(&m->d.cap_count, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemset(m->d.cap_count, 0, sizeof(uint32_t));
  if (e != cudaSuccess) {
    free_capture(m);
    return e == cudaErrorMemoryAllocation ? MRH_ERR_OUT_OF_MEMORY : cuda_fail(e, "mrh_set_feature_capture");
  }
  m->d.cap_max = capacity;
  return MRH_OK;
}

mrh_status mrh_get_features(mrh_map* m, int32_t* keys_dev, float* features_dev, uint32_t capacity, uint32_t* n_out,
                            uint64_t* n_seen_out, int reset, void* stream) {
  if (!m || !n_out || !m->d.cap_count) return MRH_ERR_INVALID_ARG;
  DeviceGuard guard(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t seen = 0;
  MRH_CUDA(cudaMemcpyAsync(&seen, m->d.cap_count, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  MRH_CUDA(cudaStreamSynchronize(s));
  const uint32_t stored = std::min(seen, m->d.cap_max);
  *n_out = stored;
  if (n_seen_out) *n_seen_out = seen;
  if (stored > 0 && (!keys_dev || !features_dev || capacity < stored)) return MRH_ERR_CAPACITY;
  if (stored > 0) {
    MRH_CUDA(cudaMemcpyAsync(keys_dev, m->d.cap_keys, sizeof(int32_t) * 3 * (size_t)stored,
                             cudaMemcpyDeviceToDevice, s));
    MRH_CUDA(cudaMemcpyAsync(features_dev, m->d.cap_feat, sizeof(float) * MRH_MLP_IN * (size_t)stored,
                             cudaMemcpyDeviceToDevice, s));
  }
  if (reset) MRH_CUDA(cudaMemsetAsync(m->d.cap_count, 0, sizeof(uint32_t), s));
  MRH_CUDA(cudaStreamSynchronize(s));
  return MRH_OK;
}

mrh_status mrh_integrate_depth(mrh_map* m, const mrh_pinhole* K, const double* T_wc, const float* depth,
                               const uint8_t* rgb, void* stream) {
  if (!m || !depth || !finite_pose(T_wc)) return MRH_ERR_INVALID_ARG;
  mrh_status st = validate_pinhole(K);
  if (st != MRH_OK) return st;
  DeviceGuard guard(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  CamArgs c = cam_args(K, T_wc);
  const size_t pixels = (size_t)K->width * K->height;
  if (pixels > m->img_pixels) {
    // first frame (or a larger one): grow the per-frame images; stream-ordered, so earlier frames are unaffected
    if (m->rho_img) cudaFreeAsync(m->rho_img, s);
    if (m->rgb_img) cudaFreeAsync(m->rgb_img, s);
    m->rho_img = nullptr;
    m->rgb_img = nullptr;
    m->img_pixels = 0;
    MRH_CUDA(cudaMallocAsync(&m->rho_img, pixels * sizeof(float), s));
    MRH_CUDA(cudaMallocAsync(&m->rgb_img, pixels * sizeof(uint32_t), s));
    m->img_pixels = pixels;
  }
  const uint8_t* rgb_in = m->p.has_color ? rgb : nullptr;
  { KernelScope ks(m, MRH_K_BEGIN, s, 1); k_begin<<<1, 1, 0, s>>>(m->d.st); }
  if (m->d.ar_keys) {
    KernelScope ks(m, MRH_K_STREAM, s, 1);
    launch_evict_camera(m->d, c, s, m->sms);
  }
  { KernelScope ks(m, MRH_K_ALLOC, s, 1); launch_alloc_depth(m->d, c, depth, rgb_in, m->rho_img, m->rgb_img, s); }
  { KernelScope ks(m, MRH_K_BIN, s, 1); launch_bin_camera(m->d, c, m->rho_img, s, m->sms); }
  if (m->d.ar_keys) {
    KernelScope ks(m, MRH_K_STREAM, s, 1);
    launch_restore(m->d, s, m->sms);
  }
  {
    KernelScope ks(m, MRH_K_FUSE, s, 1);
    launch_fuse_depth(m->d, c, m->rho_img, rgb_in ? m->rgb_img : nullptr, s, m->sms);
  }
  { KernelScope ks(m, MRH_K_RELEASE, s, 1); k_release<<<m->sms, 256, 0, s>>>(m->d); }
  MRH_CUDA(cudaGetLastError());
  return MRH_OK;
}

mrh_status mrh_integrate_points(mrh_map* m, const double* T_ws, const float* xyz, uint64_t n, void* stream) {
  if (!m || (!xyz && n) || !finite_pose(T_ws) || n > (1ull << 23)) return MRH_ERR_INVALID_ARG;
  DeviceGuard guard(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (n > m->ray_cap) {
    for (void* p : {(void*)m->rays, (void*)m->stage, (void*)m->stage_len, (void*)m->stage_over})
      if (p) cudaFreeAsync(p, s);
    m->rays = nullptr;
    m->stage = nullptr;
    m->stage_len = nullptr;
    m->stage_over = nullptr;
    m->ray_cap = 0;
    MRH_CUDA(cudaMallocAsync(&m->rays, n * sizeof(LidarRay), s));
    MRH_CUDA(cudaMallocAsync(&m->stage, n * kStageCap * sizeof(uint2), s));
    MRH_CUDA(cudaMallocAsync(&m->stage_len, n * sizeof(uint32_t), s));
    MRH_CUDA(cudaMallocAsync(&m->stage_over, n * sizeof(uint32_t), s));
    m->ray_cap = n;
  }
  m->d.rays = m->rays;
  m->d.stage = m->stage;
  m->d.stage_len = m->stage_len;
  m->d.stage_over = m->stage_over;
  { KernelScope ks(m, MRH_K_BEGIN, s, 1); k_begin<<<1, 1, 0, s>>>(m->d.st); }
  if (m->d.ar_keys) {
    KernelScope ks(m, MRH_K_STREAM, s, 1);
    launch_evict_lidar(m->d, T_ws, s, m->sms);
  }
  const bool predict = m->d.pred_w || m->d.cap_feat;
  if (predict) {
    const size_t nt = m->d.max_touched;
    if (!m->lidar_pred) {
      const size_t bytes = nt * (sizeof(unsigned long long) * kLidarMoments + sizeof(uint32_t) + sizeof(uint8_t));
      MRH_CUDA(cudaMalloc(&m->lidar_pred, bytes));
    }
    char* base = (char*)m->lidar_pred;  // moments, fresh list, levels
    m->d.lidar_mom = (unsigned long long*)base;
    m->d.fresh = (uint32_t*)(base + nt * sizeof(unsigned long long) * kLidarMoments);
    m->d.fresh_level = (uint8_t*)((char*)m->d.fresh + nt * sizeof(uint32_t));
    if (n > m->end_cap) {
      if (m->lidar_end) cudaFreeAsync(m->lidar_end, s);
      m->lidar_end = nullptr;
      m->end_cap = 0;
      MRH_CUDA(cudaMallocAsync(&m->lidar_end, n * 3 * sizeof(long long), s));
      m->end_cap = n;
    }
  }
  m->d.lidar_end = predict ? m->lidar_end : nullptr;  // the allocation pass writes end points only when set
  { KernelScope ks(m, MRH_K_ALLOC, s, n ? 1 : 0); launch_alloc_points(m->d, T_ws, xyz, n, s); }
  if (predict) {
    KernelScope ks(m, MRH_K_BIN, s, n ? 4 : 3);
    launch_bin_points(m->d, T_ws, xyz, n, s, m->sms);
  } else {
    KernelScope ks(m, MRH_K_BIN, s, 1);
    launch_bin(m->d, s, m->sms);
  }
  if (m->d.ar_keys) {
    KernelScope ks(m, MRH_K_STREAM, s, 1);
    launch_restore(m->d, s, m->sms);
  }
  { KernelScope ks(m, MRH_K_LIDAR_OBS, s, n ? 4 : 2); launch_lidar_observations(m->d, T_ws, xyz, n, s, m->sms); }
  { KernelScope ks(m, MRH_K_FUSE, s, 1); launch_fuse_points(m->d, T_ws, xyz, n, s, m->sms); }
  { KernelScope ks(m, MRH_K_RELEASE, s, 1); k_release<<<m->sms, 256, 0, s>>>(m->d); }
  MRH_CUDA(cudaGetLastError());
  return MRH_OK;
}

mrh_status mrh_raycast(mrh_map* m, const mrh_pinhole* K, const double* T_wc, float* depth_out, float* normal_out,
                       uint8_t* rgb_out, void* stream) {
  if (!m || !depth_out || !finite_pose(T_wc) || (rgb_out && !m->d.color)) return MRH_ERR_INVALID_ARG;
  mrh_status st = validate_pinhole(K);
  if (st != MRH_OK) return st;
  DeviceGuard guard(m->device);
  CamArgs c = cam_args(K, T_wc);
  {
    KernelScope ks(m, MRH_K_RAYCAST, (cudaStream_t)stream, 1);
    launch_raycast(m->d, c, depth_out, normal_out, rgb_out, (cudaStream_t)stream);
  }
  MRH_CUDA(cudaGetLastError());
  return MRH_OK;
}

mrh_status mrh_extract_mesh(mrh_map* m, float* tris, uint64_t capacity, uint64_t* n_tris_out, void* stream) {
  if (!m || !n_tris_out || (capacity > 0 && !tris)) return MRH_ERR_INVALID_ARG;
  DeviceGuard guard(m->device);
  const cudaError_t te = mesh_table_ready(m->device);
  if (te != cudaSuccess) return cuda_fail(te, "mesh case table");
  const cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* count = &m->d.st->mesh_tris;
  MRH_CUDA(cudaMemsetAsync(count, 0, sizeof(*count), s));
  {
    KernelScope ks(m, MRH_K_MESH, s, 1);
    launch_mesh(m->d, tris, capacity, count, s, m->sms);
  }
  MRH_CUDA(cudaGetLastError());
  unsigned long long n = 0;
  MRH_CUDA(cudaMemcpyAsync(&n, count, sizeof(n), cudaMemcpyDeviceToHost, s));
  MRH_CUDA(cudaStreamSynchronize(s));
  *n_tris_out = n;
  return n > capacity ? MRH_ERR_CAPACITY : MRH_OK;
}

mrh_status mrh_weld_mesh(mrh_map* m, const float* tris, uint64_t n_tris, float delta, float* verts, uint64_t cap_verts,
                         int32_t* faces, uint64_t cap_faces, uint64_t* n_verts_out, uint64_t* n_faces_out,
                         void* stream) {
  if (!m || !n_verts_out || !n_faces_out || !(delta > 0.0f) || !std::isfinite(delta) || n_tris > (1ull << 28) ||
      (n_tris > 0 && !tris) || (cap_verts > 0 && !verts) || (cap_faces > 0 && !faces))
    return MRH_ERR_INVALID_ARG;
  DeviceGuard guard(m->device);
  const cudaStream_t s = (cudaStream_t)stream;
  *n_verts_out = *n_faces_out = 0;
  if (n_tris == 0) return MRH_OK;
  const uint32_t nv = (uint32_t)(3 * n_tris);
  uint32_t table = 1024;
  while (table < 2 * nv) table <<= 1;
  WeldScratch w{};
  const size_t nblk = (n_tris + kWeldScanBlock - 1) / kWeldScanBlock;
  cudaError_t e = cudaSuccess;
  auto grab = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = scratch_alloc(p, bytes, m->device, s);
  };
  grab((void**)&w.keys, 8ull * table);
  grab((void**)&w.mn, 12ull * table);
  grab((void**)&w.vslot, 4ull * nv);
  grab((void**)&w.vidx, 4ull * table);
  grab((void**)&w.ckeys, 8ull * table);
  grab((void**)&w.cslots, 4ull * table);
  // the cluster keys' radix sort: second key / value buffers, digit counts and their scan sums
  unsigned long long* ckeys2 = nullptr;
  uint32_t *cslots2 = nullptr, *hist = nullptr, *hsums = nullptr;
  const size_t nh = radix_scratch_words(table);
  grab((void**)&ckeys2, 8ull * table);
  grab((void**)&cslots2, 4ull * table);
  grab((void**)&hist, 4ull * nh);
  grab((void**)&hsums, 4ull * scan_sums_count(nh));
  unsigned long long* const ckeys_alloc = w.ckeys;
  uint32_t* const cslots_alloc = w.cslots;
  grab((void**)&w.blk, 4ull * (nblk + 1));
  grab((void**)&w.counters, 16);
  mrh_status st = MRH_OK;
  uint32_t hc[2] = {0, 0};
  if (e == cudaSuccess) {
    w.table = table;
    KernelScope ks(m, MRH_K_MESH, s, 1);
    e = weld_clusters(w, tris, nv, delta, s, m->sms);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hc, w.counters, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && hc[1] == 0) {
      // the cluster keys are distinct 63-bit values: sort them (with their slots) in key order
      unsigned long long* kk[2] = {w.ckeys, ckeys2};
      uint32_t* vv[2] = {w.cslots, cslots2};
      const int cur = radix_sort<unsigned long long>(kk, vv, hc[0], 63, hist, hsums, s);
      w.ckeys = kk[cur];
      w.cslots = vv[cur];
      e = weld_output(w, tris, hc[0], verts, cap_verts, faces, cap_faces, n_tris, nblk, s, m->sms);
    }
  }
  uint32_t nf = 0;
  if (e == cudaSuccess && hc[1] == 0) e = cudaMemcpyAsync(&nf, w.counters + 2, 4, cudaMemcpyDeviceToHost, s);
  for (void* p : {(void*)w.keys, (void*)w.mn, (void*)w.vslot, (void*)w.vidx, (void*)ckeys_alloc, (void*)cslots_alloc,
                  (void*)w.blk, (void*)w.counters, (void*)ckeys2, (void*)cslots2, (void*)hist, (void*)hsums})
    if (p) cudaFreeAsync(p, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "mrh_weld_mesh");
  if (hc[1] != 0) return MRH_ERR_INVALID_ARG;  // a vertex's cluster index is out of range for this delta
  *n_verts_out = hc[0];
  *n_faces_out = nf;
  if (hc[0] > cap_verts || nf > cap_faces) st = MRH_ERR_CAPACITY;
  return st;
}

mrh_status mrh_quadtree(const uint8_t* rgb, int width, int height, double threshold, int min_size, int32_t* leaves,
                        uint64_t capacity, uint64_t* n_leaves_out, int device, void* stream) {
  if (!rgb || !n_leaves_out || width < 1 || height < 1 || width > 16384 || height > 16384 || min_size < 1 ||
      std::isnan(threshold) || (capacity > 0 && !leaves))
    return MRH_ERR_INVALID_ARG;
  DeviceGuard guard(device);
  const cudaStream_t s = (cudaStream_t)stream;
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  void* scratch = nullptr;
  MRH_CUDA(scratch_alloc(&scratch, quadtree_scratch_bytes(width, height), device, s));
  unsigned long long* n_dev = nullptr;
  cudaError_t e = launch_quadtree(rgb, width, height, threshold, min_size, leaves, capacity, scratch, &n_dev, s, sms);
  unsigned long long n = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&n, n_dev, sizeof(n), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(scratch, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "mrh_quadtree");
  *n_leaves_out = n;
  return n > capacity ? MRH_ERR_CAPACITY : MRH_OK;
}

mrh_status mrh_splat_render(const float* means, const float* covs, const float* opacity, const float* colors,
                            uint64_t n, const mrh_pinhole* K, const double* T_wc, float* rgb_out, float* trans_out,
                            uint64_t* n_pairs_out, int device, void* stream) {
  if (!K || !T_wc || !rgb_out || n >= (1ull << 32) || (n > 0 && (!means || !covs || !opacity || !colors)) ||
      K->width < 1 || K->height < 1 || K->width > 16384 || K->height > 16384 || !(K->fx > 0.0f) || !(K->fy > 0.0f) ||
      !(K->min_depth > 0.0f) || !(K->max_depth >= K->min_depth) || !std::isfinite(K->cx) || !std::isfinite(K->cy))
    return MRH_ERR_INVALID_ARG;
  for (int i = 0; i < 16; ++i)
    if (!std::isfinite(T_wc[i])) return MRH_ERR_INVALID_ARG;
  DeviceGuard guard(device);
  if (!guard.ok) return cuda_fail(cudaGetLastError(), "cudaSetDevice");
  const cudaStream_t s = (cudaStream_t)stream;
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const SplatInputs in{means, covs, opacity, colors, n};
  uint64_t pairs = 0;
  const cudaError_t e = splat_render(in, cam_args(K, T_wc), rgb_out, trans_out, &pairs, device, s, sms);
  if (n_pairs_out) *n_pairs_out = pairs;
  if (e != cudaSuccess) return cuda_fail(e, "mrh_splat_render");
  return pairs > kSplatMaxPairs ? MRH_ERR_CAPACITY : MRH_OK;
}

mrh_status mrh_save_map(mrh_map* m, const char* path, void* stream) {
  if (!m || !path) return MRH_ERR_INVALID_ARG;
  DeviceGuard guard(m->device);
  const cudaStream_t s = (cudaStream_t)stream;
  MRH_CUDA(cudaStreamSynchronize(s));
  const MapDev& d = m->d;
  struct Rec {
    int32_t key[3];
    uint32_t level;
    uint32_t level_id;        // resident: level << 28 | heap id
    bool fresh;               // resident and not yet fused: its payload is the zero state
    const uint8_t* archived;  // archived: its payload in the host archive
  };
  std::vector<Rec> res, arc;
  {
    std::vector<Slot> slots((size_t)d.slot_mask + 1);
    MRH_CUDA(cudaMemcpy(slots.data(), d.slots, slots.size() * sizeof(Slot), cudaMemcpyDeviceToHost));
    for (const Slot& sl : slots) {
      // the blocks mrh_count_blocks / mrh_extract_blocks report; one still marked new is saved in its zero state
      if (sl.key == kEmptyKey || sl.key == kTombKey || sl.val == kValPending) continue;
      Rec r{};
      unpack_key(sl.key, &r.key[0], &r.key[1], &r.key[2]);
      r.level = (sl.val >> 28) & 3u;
      r.level_id = sl.val & (kPtrMask | (3u << 28));
      r.fresh = (sl.val & kValNew) != 0;
      res.push_back(r);
    }
  }
  if (d.ar_keys && m->archive_host) {
    std::vector<unsigned long long> keys((size_t)d.ar_mask + 1);
    std::vector<uint32_t> vals(keys.size());
    MRH_CUDA(cudaMemcpy(keys.data(), d.ar_keys, keys.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    MRH_CUDA(cudaMemcpy(vals.data(), d.ar_vals, vals.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < keys.size(); ++i) {
      if (keys[i] == kEmptyKey || !(vals[i] & kArPresent)) continue;
      Rec r{};
      unpack_key(keys[i], &r.key[0], &r.key[1], &r.key[2]);
      r.level = (vals[i] >> 28) & 3u;
      r.archived = m->archive_host + (size_t)(vals[i] & 0x0FFFFFFFu) * d.ar_slot_bytes;
      arc.push_back(r);
    }
  }
  auto by_key = [](const Rec& a, const Rec& b) {
    return std::lexicographical_compare(a.key, a.key + 3, b.key, b.key + 3);
  };
  std::sort(res.begin(), res.end(), by_key);
  std::sort(arc.begin(), arc.end(), by_key);
  std::vector<uint32_t> ids(res.size());
  std::vector<uint64_t> offs(res.size());
  uint64_t blob_bytes = 0;
  for (size_t i = 0; i < res.size(); ++i) {
    ids[i] = res[i].level_id;
    offs[i] = blob_bytes;
    blob_bytes += d.block_bytes[res[i].level];
  }
  std::vector<uint8_t> blob(blob_bytes);
  MRH_CUDA(io_blocks_to_blob(d, ids, offs, blob.data(), blob_bytes, s, m->sms));
  for (size_t i = 0; i < res.size(); ++i)
    if (res[i].fresh) std::memset(blob.data() + offs[i], 0, d.block_bytes[res[i].level]);
  FILE* f = std::fopen(path, "wb");
  if (!f) return MRH_ERR_INVALID_ARG;
  const uint32_t ver = io_version(), psz = (uint32_t)sizeof(mrh_map_params);
  const uint64_t n = res.size() + arc.size();
  bool ok = std::fwrite(io_magic(), 1, 8, f) == 8 && std::fwrite(&ver, 4, 1, f) == 1 && std::fwrite(&psz, 4, 1, f) == 1 &&
            std::fwrite(&m->p, sizeof(mrh_map_params), 1, f) == 1 && std::fwrite(&n, 8, 1, f) == 1;
  for (int part = 0; part < 2 && ok; ++part)
    for (size_t i = 0; i < (part ? arc.size() : res.size()) && ok; ++i) {
      const Rec& r = part ? arc[i] : res[i];
      const uint8_t lvl[4] = {(uint8_t)r.level, 0, 0, 0};
      const uint32_t nb = d.block_bytes[r.level];
      const uint8_t* src = part ? r.archived : blob.data() + offs[i];
      ok = std::fwrite(r.key, 4, 3, f) == 3 && std::fwrite(lvl, 1, 4, f) == 4 && std::fwrite(&nb, 4, 1, f) == 1 &&
           std::fwrite(src, 1, nb, f) == nb;
    }
  ok = (std::fclose(f) == 0) && ok;
  return ok ? MRH_OK : MRH_ERR_INVALID_ARG;
}

mrh_status mrh_load_map(const char* path, int device, mrh_map** out) {
  if (!path || !out) return MRH_ERR_INVALID_ARG;
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) return MRH_ERR_INVALID_ARG;
  char magic[8];
  uint32_t ver = 0, psz = 0;
  mrh_map_params p{};
  uint64_t n = 0;
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, io_magic(), 8) == 0 &&
            std::fread(&ver, 4, 1, f) == 1 && ver == io_version() && std::fread(&psz, 4, 1, f) == 1 &&
            psz == sizeof(mrh_map_params) && std::fread(&p, sizeof(p), 1, f) == 1 && std::fread(&n, 8, 1, f) == 1;
  mrh_map* m = nullptr;
  if (ok && mrh_map_create(&p, device, &m) != MRH_OK) ok = false;
  std::vector<int32_t> keys;
  std::vector<uint32_t> levels;
  std::vector<uint64_t> offs;
  std::vector<uint8_t> blob;
  for (uint64_t i = 0; i < n && ok; ++i) {
    int32_t k[3];
    uint8_t lvl[4];
    uint32_t nb = 0;
    ok = std::fread(k, 4, 3, f) == 3 && std::fread(lvl, 1, 4, f) == 4 && std::fread(&nb, 4, 1, f) == 1 &&
         lvl[0] < (uint32_t)m->d.L && nb == m->d.block_bytes[lvl[0]] && key_ok(k[0], k[1], k[2]);
    if (!ok) break;
    keys.insert(keys.end(), k, k + 3);
    levels.push_back(lvl[0]);
    offs.push_back(blob.size());
    blob.resize(blob.size() + nb);
    ok = std::fread(blob.data() + offs.back(), 1, nb, f) == nb;
  }
  std::fclose(f);
  if (!ok) {
    if (m) mrh_map_destroy(m);
    return MRH_ERR_INVALID_ARG;
  }
  DeviceGuard guard(device);
  const cudaError_t e = io_blob_to_blocks(m->d, keys, levels, offs, blob.data(), blob.size(), 0, m->sms);
  if (e != cudaSuccess) {
    mrh_map_destroy(m);
    return cuda_fail(e, "mrh_load_map");
  }
  DevState hs;
  if (cudaMemcpy(&hs, m->d.st, sizeof(hs), cudaMemcpyDeviceToHost) != cudaSuccess || hs.status != 0) {
    const mrh_status st = status_from_bits(hs.status);
    mrh_map_destroy(m);
    return st != MRH_OK ? st : MRH_ERR_CUDA;
  }
  *out = m;
  return MRH_OK;
}

void mrh_mesh_case_table(uint8_t* ntri, int8_t* tri, int8_t* edge_end) {
  if (ntri && tri && edge_end) host_case_table(ntri, tri, edge_end);
}

mrh_status mrh_count_blocks(mrh_map* m, uint64_t* n_blocks, uint64_t* n_voxels, void* stream) {
  if (!m) return MRH_ERR_INVALID_ARG;
  DeviceGuard guard(m->device);
  DevState hs;
  MRH_CUDA(cudaMemcpyAsync(&hs, m->d.st, sizeof(hs), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  MRH_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  uint64_t nb = 0, nv = 0;
  for (int l = 0; l < m->d.L; ++l) {
    uint64_t live = m->d.max_blocks[l] - (uint64_t)hs.free_top[l];
    int nl = kFineDim >> l;
    nb += live;
    nv += live * (uint64_t)(nl * nl * nl);
  }
  if (n_blocks) *n_blocks = nb;
  if (n_voxels) *n_voxels = nv;
  return status_from_bits(hs.status);
}

mrh_status mrh_extract_blocks(mrh_map* m, int32_t* keys, uint8_t* levels, uint64_t* voxel_offset, float* tsdf,
                              float* weight, float* s2, float* color, uint64_t cap_blocks, uint64_t cap_voxels,
                              uint64_t* n_blocks_out, uint64_t* n_voxels_out, void* stream) {
  if (!m || !keys || !levels || !voxel_offset || !tsdf || !weight || !s2) return MRH_ERR_INVALID_ARG;
  uint64_t nb = 0, nv = 0;
  mrh_status st = mrh_count_blocks(m, &nb, &nv, stream);
  if (n_blocks_out) *n_blocks_out = nb;
  if (n_voxels_out) *n_voxels_out = nv;
  if (st == MRH_ERR_CUDA) return st;
  if (nb > cap_blocks || nv > cap_voxels) return MRH_ERR_CAPACITY;
  DeviceGuard guard(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  // compacted keys and slots (two buffers each for the radix sort), digit counts and their scan sums
  const size_t cap = nb + 1, nh = radix_scratch_words((uint32_t)cap);
  unsigned long long *skeys[2] = {nullptr, nullptr}, *soff = nullptr;
  uint32_t *sslots[2] = {nullptr, nullptr}, *scount = nullptr, *hist = nullptr, *hsums = nullptr;
  cudaError_t e = cudaSuccess;
  auto grab = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMallocAsync(p, bytes, s);
  };
  for (int b = 0; b < 2; ++b) {
    grab((void**)&skeys[b], sizeof(unsigned long long) * cap);
    grab((void**)&sslots[b], sizeof(uint32_t) * cap);
  }
  grab((void**)&soff, sizeof(unsigned long long) * (nb + 1));
  grab((void**)&scount, sizeof(uint32_t));
  grab((void**)&hist, sizeof(uint32_t) * nh);
  grab((void**)&hsums, sizeof(uint32_t) * scan_sums_count(nh));
  uint32_t hcount = 0, n = 0;
  if (e == cudaSuccess) e = cudaMemsetAsync(scount, 0, sizeof(uint32_t), s);
  if (e == cudaSuccess) {
    k_compact<<<m->sms * 8, 256, 0, s>>>(m->d, skeys[0], sslots[0], scount, (uint32_t)cap);
    e = cudaMemcpyAsync(&hcount, scount, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) {
    n = std::min<uint32_t>(hcount, (uint32_t)nb);
    // the packed keys order as (x, then y, then z) and are distinct: a radix sort of all 64 bits
    const int cur = radix_sort<unsigned long long>(skeys, sslots, n, 64, hist, hsums, s);
    if (n > 0) {
      k_voxel_offsets<<<1, 1024, 0, s>>>(m->d, sslots[cur], n, soff);
      k_extract<<<m->sms * 8, 128, 0, s>>>(m->d, sslots[cur], n, soff, keys, levels,
                                            (unsigned long long*)voxel_offset, tsdf, weight, s2, color);
    } else {
      e = cudaMemsetAsync(voxel_offset, 0, sizeof(uint64_t), s);
    }
  }
  for (void* p : {(void*)skeys[0], (void*)skeys[1], (void*)sslots[0], (void*)sslots[1], (void*)soff, (void*)scount,
                  (void*)hist, (void*)hsums})
    if (p) cudaFreeAsync(p, s);
  if (e != cudaSuccess) return cuda_fail(e, "mrh_extract_blocks");
  MRH_CUDA(cudaGetLastError());
  MRH_CUDA(cudaStreamSynchronize(s));
  if (hcount != nb) return MRH_ERR_INCONSISTENT;
  return st;
}

mrh_status mrh_extract_blocks_noalloc(mrh_map* m, int32_t* keys, uint8_t* levels, uint64_t* voxel_offset,
                                      float* tsdf, float* weight, float* s2, float* color, uint64_t cap_blocks,
                                      uint64_t cap_voxels, uint64_t* n_blocks_out, uint64_t* n_voxels_out,
                                      void* stream) {
  if (!m || !keys || !levels || !voxel_offset || !tsdf || !weight || !s2) return MRH_ERR_INVALID_ARG;
  uint64_t nb = 0, nv = 0;
  mrh_status st = mrh_count_blocks(m, &nb, &nv, stream);
  if (n_blocks_out) *n_blocks_out = nb;
  if (n_voxels_out) *n_voxels_out = nv;
  if (st == MRH_ERR_CUDA) return st;
  if (nb > kNoallocMaxBlocks) return MRH_ERR_STATIC_LIMIT;
  if (nb > cap_blocks || nv > cap_voxels) return MRH_ERR_CAPACITY;
  DeviceGuard guard(m->device);
  if (!guard.ok) return cuda_fail(cudaGetLastError(), "cudaSetDevice");
  uint8_t* base = nullptr;
  mrh_status sst = noalloc_scratch(&base);
  if (sst != MRH_OK) return sst;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* skeys = (unsigned long long*)(base + kNoallocKeysOff);
  uint32_t* sslots = (uint32_t*)(base + kNoallocSlotsOff);
  unsigned long long* soff = (unsigned long long*)(base + kNoallocOffsOff);
  uint32_t* scount = (uint32_t*)(base + kNoallocCountOff);
  uint32_t npow = 1;
  while (npow < nb) npow <<= 1;
  MRH_CUDA(cudaMemsetAsync(scount, 0, sizeof(uint32_t), s));
  k_compact<<<m->sms * 8, 256, 0, s>>>(m->d, skeys, sslots, scount, npow);
  uint32_t hcount = 0;
  MRH_CUDA(cudaMemcpyAsync(&hcount, scount, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  MRH_CUDA(cudaStreamSynchronize(s));
  uint32_t n = std::min<uint32_t>(hcount, (uint32_t)nb);
  if (npow > n) k_pad_keys<<<m->sms * 4, 256, 0, s>>>(skeys, n, npow);
  for (uint32_t k = 2; k <= npow; k <<= 1)
    for (uint32_t j = k >> 1; j > 0; j >>= 1) k_bitonic_step<<<m->sms * 8, 256, 0, s>>>(skeys, sslots, npow, k, j);
  if (n > 0) {
    k_voxel_offsets<<<1, 1024, 0, s>>>(m->d, sslots, n, soff);
    k_extract<<<m->sms * 8, 128, 0, s>>>(m->d, sslots, n, soff, keys, levels, (unsigned long long*)voxel_offset,
                                          tsdf, weight, s2, color);
  } else {
    MRH_CUDA(cudaMemsetAsync(voxel_offset, 0, sizeof(uint64_t), s));
  }
  MRH_CUDA(cudaGetLastError());
  MRH_CUDA(cudaStreamSynchronize(s));
  if (hcount != nb) return MRH_ERR_INCONSISTENT;
  return st;
}

mrh_status mrh_get_stats(mrh_map* m, mrh_stats* out, void* stream) {
  if (!m || !out) return MRH_ERR_INVALID_ARG;
  DeviceGuard guard(m->device);
  DevState hs;
  MRH_CUDA(cudaMemcpyAsync(&hs, m->d.st, sizeof(hs), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  MRH_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  std::memset(out, 0, sizeof(*out));
  out->frame = hs.frame;
  out->valid_rays = hs.valid_rays;
  out->touched = std::min<uint32_t>(hs.touched_all, m->d.max_touched);
  out->new_blocks = hs.new_blocks;
  out->merged = hs.merged;
  out->split = hs.split;
  out->fp64_rechecks = hs.rechecks;
  for (int l = 0; l < m->d.L; ++l) {
    out->live_blocks[l] = m->d.max_blocks[l] - (uint64_t)hs.free_top[l];
    out->touched_level[l] = std::min<uint32_t>(hs.touched_count[l], m->d.max_touched);
  }
  out->observations = hs.observations;
  out->updated_voxels = hs.updated_voxels;
  out->lidar_restaged = hs.n_over;
  out->lidar_max_voxel_obs = hs.max_vox_obs;
  out->evicted = hs.evicted;
  out->restored = hs.restored;
  out->archived = hs.ar_present;
  out->status = hs.status;
  return status_from_bits(hs.status);
}

mrh_status mrh_sync(mrh_map* m, void* stream) {
  mrh_stats s;
  return mrh_get_stats(m, &s, stream);
}

mrh_status mrh_clear_status(mrh_map* m, void* stream) {
  if (!m) return MRH_ERR_INVALID_ARG;
  DeviceGuard guard(m->device);
  MRH_CUDA(cudaMemsetAsync(&m->d.st->status, 0, sizeof(uint32_t), (cudaStream_t)stream));
  return MRH_OK;
}

mrh_status mrh_set_profiling(mrh_map* m, int enable) {
  if (!m) return MRH_ERR_INVALID_ARG;
  m->profiling = enable != 0;
  return MRH_OK;
}

mrh_status mrh_get_profile(mrh_map* m, double* ms_out, uint64_t* launches_out, int n, int reset, void* stream) {
  if (!m || n < 0 || n > MRH_K_COUNT) return MRH_ERR_INVALID_ARG;
  DeviceGuard guard(m->device);
  MRH_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  mrh_status st = collect_profile(m);
  if (st != MRH_OK) return st;
  for (int i = 0; i < n; ++i) {
    if (ms_out) ms_out[i] = m->prof_ms[i];
    if (launches_out) launches_out[i] = m->launches[i];
  }
  if (reset) {
    for (int i = 0; i < MRH_K_COUNT; ++i) {
      m->prof_ms[i] = 0.0;
      m->launches[i] = 0;
    }
  }
  return MRH_OK;
}

uint32_t mrh_hash_slot(int32_t x, int32_t y, int32_t z, uint32_t log2_slots) {
  uint32_t mask = log2_slots >= 32 ? 0xFFFFFFFFu : ((1u << log2_slots) - 1u);
  return hash_xyz(x, y, z, mask);
}

const char* mrh_status_string(mrh_status s) {
  switch (s) {
    case MRH_OK: return "ok";
    case MRH_ERR_INVALID_ARG: return "invalid argument";
    case MRH_ERR_OUT_OF_MEMORY: return "out of device memory";
    case MRH_ERR_HASH_FULL: return "hash table probe limit reached";
    case MRH_ERR_POOL_EMPTY: return "block heap empty";
    case MRH_ERR_LIST_FULL: return "touched-block list full";
    case MRH_ERR_CUDA: return "CUDA error";
    case MRH_ERR_CAPACITY: return "output buffer too small";
    case MRH_ERR_STATIC_LIMIT: return "more blocks than the no-allocation extract's fixed scratch holds";
    case MRH_ERR_INCONSISTENT: return "hash table and block heaps disagree on the number of blocks";
  }
  return "unknown status";
}

const char* mrh_last_cuda_error(void) { return g_cuda_err; }

const char* mrh_version(void) { return "mrhash 0.1.0 sm_103a"; }

}  // extern "C"
