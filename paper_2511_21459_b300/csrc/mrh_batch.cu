// Batched multi-scene integration: one frame for each of up to 64 maps per step, with one launch per phase for all
// maps together (an addition to the paper's method, which integrates one map).
//
//   k_batch_begin     per-map frame counters
//   k_batch_alloc     one grid over every map's pixel tiles (a CTA finds its map from the tile offsets)
//   k_batch_bin       one grid row per map
//   k_batch_fuse      persistent warps share the work items of all maps laid end to end as a grid-stride loop would
//                     (each warp walks the maps in order and takes, in each, the items that loop gives it), so maps
//                     with large and small frames share the GPU without per-map launches or idle tails
//   k_batch_release   one grid row per map
//   k_batch_raycast   one grid over every map's pixel tiles (maps without a raycast output skip)
//
// Frame descriptors (pose, intrinsics, buffers) live in device memory and are refreshed by one host-to-device copy
// before each step, so the step itself is a fixed sequence of launches: it is captured once into a CUDA graph and
// replayed. Before capture, the first steps run as trials of alternative launch shapes (allocation CTA tile and probe
// width, fusion warps per CTA and persistent grid size, raycast warp tile); every shape computes the same result, and
// the fastest measured shape of each phase is kept.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "mrh_alloc.cuh"
#include "mrh_fuse.cuh"
#include "mrh_raycast.cuh"

namespace mrh {

constexpr int kBatchMaxMaps = 64;

// per map, per step (device memory)
struct BatchFrame {
  CamArgs cam;
  const float* depth;
  const uint8_t* rgb;       // null: no colour this frame
  float* rho_img;           // owned by the batch
  uint32_t* rgb_img;        // owned by the batch
  float* raycast_out;       // null: no raycast
  uint32_t alloc_tile0;     // first allocation tile of this map in the batched grid
  uint32_t ray_tile0;       // first raycast tile
  int alloc_tiles_x, ray_tiles_x;
};

struct BatchDev {
  const MapDev* maps;
  const BatchFrame* frames;
  int n;
};

namespace {

__device__ inline int find_map(const BatchFrame* frames, int n, uint32_t tile, bool raycast) {
  int m = 0;
  for (int i = 1; i < n; ++i)
    if ((raycast ? frames[i].ray_tile0 : frames[i].alloc_tile0) <= tile) m = i;
  return m;
}

__global__ void k_batch_begin(BatchDev b) {
  const int i = threadIdx.x;
  if (i < b.n) begin_frame(b.maps[i].st);
}

template <int TW, int TH, int PW>
__global__ void __launch_bounds__(256) k_batch_alloc(BatchDev b) {
  __shared__ unsigned long long s_set[kSetCap];
  __shared__ uint32_t s_valid;
  __shared__ int s_map;
  if (threadIdx.x == 0) s_map = find_map(b.frames, b.n, blockIdx.x, false);
  __syncthreads();
  const int mi = s_map;
  const BatchFrame& f = b.frames[mi];
  const uint32_t t = blockIdx.x - f.alloc_tile0;
  const int tx = (int)(t % (uint32_t)f.alloc_tiles_x), ty = (int)(t / (uint32_t)f.alloc_tiles_x);
  const CamArgs c = f.cam;
  alloc_depth_tile<TW, TH, PW>(b.maps[mi], c, f.depth, f.rgb, f.rho_img, f.rgb ? f.rgb_img : nullptr, tx, ty, s_set,
                               &s_valid);
}

__global__ void __launch_bounds__(256) k_batch_bin(BatchDev b) {
  const MapDev& m = b.maps[blockIdx.y];
  bin_entries(m, blockIdx.x * blockDim.x + (threadIdx.x & ~31u), gridDim.x * blockDim.x);
}

__global__ void __launch_bounds__(256) k_batch_release(BatchDev b) {
  const MapDev& m = b.maps[blockIdx.y];
  const uint32_t n = m.st->retire_count;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) release_one(m, i);
}

// Dynamic shared memory of k_batch_fuse: every map's MapDev and camera, copied once per CTA so that the fusion
// reads them from shared memory (a global copy could alias the payload stores, which would keep them in registers).
inline size_t fuse_smem_bytes(int n) { return (size_t)n * (sizeof(MapDev) + sizeof(CamArgs)); }

template <bool FP16, bool COLOR, int WARPS, int MINB>
__global__ void __launch_bounds__(32 * WARPS, MINB) k_batch_fuse(BatchDev b) {
  __shared__ uint32_t s_end[kBatchMaxMaps];  // inclusive prefix of work items over maps
  __shared__ ItemCounts s_ic[kBatchMaxMaps];
  extern __shared__ __align__(16) unsigned char s_dyn[];
  MapDev* s_maps = reinterpret_cast<MapDev*>(s_dyn);
  CamArgs* s_cam = reinterpret_cast<CamArgs*>(s_dyn + sizeof(MapDev) * (size_t)b.n);
  {
    static_assert(sizeof(MapDev) % 8 == 0 && sizeof(CamArgs) % 4 == 0, "copied in words");
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(b.maps);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(s_maps);
    const int words = b.n * (int)(sizeof(MapDev) / 8);
    for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
    constexpr int cw = (int)(sizeof(CamArgs) / 4);
    for (int i = threadIdx.x; i < b.n * cw; i += blockDim.x)
      reinterpret_cast<uint32_t*>(s_cam)[i] = reinterpret_cast<const uint32_t*>(&b.frames[i / cw].cam)[i % cw];
  }
  if (threadIdx.x < 32) {
    uint32_t carry = 0;
    for (int base = 0; base < b.n; base += 32) {
      const int i = base + (int)threadIdx.x;
      ItemCounts ic{};
      uint32_t items = 0;
      if (i < b.n) {
        ic = item_counts(b.maps[i]);
        items = ic.items();
        s_ic[i] = ic;
      }
      uint32_t incl = items;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(~0u, incl, o);
        if ((int)threadIdx.x >= o) incl += t;
      }
      if (i < b.n) s_end[i] = carry + incl;
      carry += __shfl_sync(~0u, incl, 31);
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t nwarps = gridDim.x * WARPS;
  // Map by map, the warp takes the items it would take in a grid-stride loop over all maps' items in order (item
  // s_end[mi - 1] + local of map mi goes to warp (s_end[mi - 1] + local) mod nwarps), with the map's counters in
  // 32 bits and added to its DevState once (a map's observations in one frame stay far below 2^32).
  const uint32_t gw = blockIdx.x * WARPS + warp;
  for (int mi = 0; mi < b.n; ++mi) {
    const uint32_t first = mi > 0 ? s_end[mi - 1] : 0u, items = s_end[mi] - first;
    const uint32_t start = (gw + nwarps - first % nwarps) % nwarps;
    if (start >= items) continue;
    const MapDev& m = s_maps[mi];
    const BatchFrame& f = b.frames[mi];
    CameraObs<FP16, COLOR, const CamArgs&> obs{s_cam[mi], f.rho_img, f.rgb ? f.rgb_img : nullptr};
    uint32_t my_obs = 0, my_vox = 0;
    for (uint32_t local = start; local < items; local += nwarps)  // warp-uniform
      fuse_item<FP16, COLOR>(m, obs, warp, s_ic[mi], local, my_obs, my_vox);
    for (int o = 16; o > 0; o >>= 1) {
      my_obs += __shfl_xor_sync(~0u, my_obs, o);
      my_vox += __shfl_xor_sync(~0u, my_vox, o);
    }
    if (lane == 0 && my_obs) atomicAdd(&m.st->observations, (unsigned long long)my_obs);
    if (lane == 0 && my_vox) atomicAdd(&m.st->updated_voxels, (unsigned long long)my_vox);
  }
}

// raycast CTA: 128 threads covering 16 x 8 pixels; each warp 8 x 4 (WIDE = false) or 16 x 2 (WIDE = true)
template <bool WIDE>
__global__ void __launch_bounds__(128) k_batch_raycast(BatchDev b) {
  __shared__ int s_map;
  if (threadIdx.x == 0) s_map = find_map(b.frames, b.n, blockIdx.x, true);
  __syncthreads();
  const int mi = s_map;
  const BatchFrame& f = b.frames[mi];
  if (!f.raycast_out) return;
  const uint32_t t = blockIdx.x - f.ray_tile0;
  const int tx = (int)(t % (uint32_t)f.ray_tiles_x), ty = (int)(t / (uint32_t)f.ray_tiles_x);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int u, v;
  if (WIDE) {
    u = tx * 16 + (lane & 15);
    v = ty * 8 + warp * 2 + (lane >> 4);
  } else {
    u = tx * 16 + (warp & 1) * 8 + (lane & 7);
    v = ty * 8 + (warp >> 1) * 4 + (lane >> 3);
  }
  const CamArgs c = f.cam;
  if (u < c.width && v < c.height) cast_ray_any(b.maps[mi], c, u, v, RayOut{f.raycast_out, nullptr, nullptr});
}

// ---- launch shapes (the autotuner's search space)
struct AllocShape {
  int tw, th, pw;
};
constexpr AllocShape kAllocShapes[] = {{32, 8, 8}, {16, 16, 8}, {32, 8, 4}, {16, 16, 4}};
struct FuseShape {
  int warps, per_sm;  // warps per CTA, CTAs per SM in the persistent grid (also the residency the registers allow)
};
constexpr FuseShape kFuseShapes[] = {{8, 4}, {8, 8}, {4, 8}, {8, 3}};
constexpr int kRayShapes = 2;  // warp tile 8 x 4, 16 x 2
constexpr int kTrials = 4;

}  // namespace
}  // namespace mrh

using namespace mrh;

struct mrh_batch {
  int device = 0, sms = 148, n = 0, flags = 0;
  int fp16 = 0, color = 0;
  std::vector<mrh_map*> maps;
  std::vector<mrh_pinhole> cams;
  MapDev* maps_dev = nullptr;
  BatchFrame* frames_dev = nullptr;
  std::vector<void*> images;
  std::vector<BatchFrame> frames_host;
  uint32_t alloc_tiles[4] = {0, 0, 0, 0};  // per allocation shape
  uint32_t ray_tiles = 0;
  // tuning state
  int steps = 0;
  int alloc_shape = 0, fuse_shape = 0, ray_shape = 0;
  bool tuned = false;
  double trial_ms[3][kTrials] = {};
  int trial_n[3][kTrials] = {};
  // phase boundaries of a step: after begin, after allocation, after binning, after fusion, after raycast (recorded
  // by every step, inside the captured graph too)
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t graph_stream = nullptr;
};

namespace {

#define MRH_BCUDA(call)                                        \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);        \
  } while (0)

struct BatchDeviceGuard {
  int prev = -1;
  explicit BatchDeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess) cudaSetDevice(dev);
  }
  ~BatchDeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

BatchDev batch_dev(const mrh_batch* b) { return BatchDev{b->maps_dev, b->frames_dev, b->n}; }

template <int TW, int TH, int PW>
void launch_alloc_shape(const mrh_batch* b, cudaStream_t s, uint32_t tiles) {
  k_batch_alloc<TW, TH, PW><<<tiles, 256, 0, s>>>(batch_dev(b));
}

void launch_alloc(const mrh_batch* b, int shape, cudaStream_t s) {
  const uint32_t tiles = b->alloc_tiles[shape];
  switch (shape) {
    case 0: launch_alloc_shape<32, 8, 8>(b, s, tiles); break;
    case 1: launch_alloc_shape<16, 16, 8>(b, s, tiles); break;
    case 2: launch_alloc_shape<32, 8, 4>(b, s, tiles); break;
    default: launch_alloc_shape<16, 16, 4>(b, s, tiles); break;
  }
}

template <int WARPS, int MINB>
void launch_fuse_warps(const mrh_batch* b, int grid, cudaStream_t s) {
  const BatchDev d = batch_dev(b);
  const size_t sm = fuse_smem_bytes(d.n);
  if (b->fp16) {
    if (b->color) k_batch_fuse<true, true, WARPS, MINB><<<grid, 32 * WARPS, sm, s>>>(d);
    else k_batch_fuse<true, false, WARPS, MINB><<<grid, 32 * WARPS, sm, s>>>(d);
  } else {
    if (b->color) k_batch_fuse<false, true, WARPS, MINB><<<grid, 32 * WARPS, sm, s>>>(d);
    else k_batch_fuse<false, false, WARPS, MINB><<<grid, 32 * WARPS, sm, s>>>(d);
  }
}

// 64 registers a thread at 32 warps per SM; the 3-CTA shape trades a quarter of the warps for 80 registers and no
// spills
void launch_fuse(const mrh_batch* b, int shape, cudaStream_t s) {
  const FuseShape fs = kFuseShapes[shape];
  const int grid = b->sms * fs.per_sm;
  if (fs.warps == 8 && fs.per_sm == 3) launch_fuse_warps<8, 3>(b, grid, s);
  else if (fs.warps == 8) launch_fuse_warps<8, 4>(b, grid, s);
  else launch_fuse_warps<4, 8>(b, grid, s);
}

void launch_raycast_shape(const mrh_batch* b, int shape, cudaStream_t s) {
  if (b->ray_tiles == 0) return;
  if (shape == 0) k_batch_raycast<false><<<b->ray_tiles, 128, 0, s>>>(batch_dev(b));
  else k_batch_raycast<true><<<b->ray_tiles, 128, 0, s>>>(batch_dev(b));
}

// one step with the given shapes; events (optional) bracket allocation, fusion and raycast
void launch_step(const mrh_batch* b, int as, int fs, int rs, cudaStream_t s, const cudaEvent_t* ev, bool capturing) {
  const BatchDev d = batch_dev(b);
  // under stream capture the records are external, so that they become event-record nodes of the graph
  auto mark = [&](int k) {
    if (!ev) return;
    if (capturing) cudaEventRecordWithFlags(ev[k], s, cudaEventRecordExternal);
    else cudaEventRecord(ev[k], s);
  };
  k_batch_begin<<<1, kBatchMaxMaps, 0, s>>>(d);
  mark(0);
  launch_alloc(b, as, s);
  mark(1);
  k_batch_bin<<<dim3(b->sms / 4 + 1, b->n), 256, 0, s>>>(d);
  mark(2);
  launch_fuse(b, fs, s);
  mark(3);
  k_batch_release<<<dim3(8, b->n), 256, 0, s>>>(d);
  launch_raycast_shape(b, rs, s);
  mark(4);
}

void destroy_graph(mrh_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

}  // namespace

extern "C" {

mrh_status mrh_batch_create(mrh_map* const* maps, const mrh_pinhole* cams, int n, int flags, mrh_batch** out) {
  if (!out || !maps || !cams || n < 1 || n > kBatchMaxMaps) return MRH_ERR_INVALID_ARG;
  *out = nullptr;
  int dev0 = -1, sms = 148;
  const MapDev* d0 = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!maps[i]) return MRH_ERR_INVALID_ARG;
    {
      int dv = 0, sm = 0;
      if (map_dev(maps[i], &dv, &sm)->ar_keys) return MRH_ERR_INVALID_ARG;  // streaming maps are not batched
    }
    int dev = 0, s = 0;
    const MapDev* d = map_dev(maps[i], &dev, &s);
    if (i == 0) {
      dev0 = dev;
      sms = s;
      d0 = d;
    } else if (dev != dev0 || d->fp16 != d0->fp16 || d->color != d0->color) {
      return MRH_ERR_INVALID_ARG;  // one device, one storage layout per batch
    }
    const mrh_pinhole& K = cams[i];
    if (K.width <= 0 || K.height <= 0 || (long long)K.width * K.height > (1LL << 26) || !(K.fx > 0.f) ||
        !(K.fy > 0.f))
      return MRH_ERR_INVALID_ARG;
  }
  BatchDeviceGuard guard(dev0);
  mrh_batch* b = new (std::nothrow) mrh_batch();
  if (!b) return MRH_ERR_OUT_OF_MEMORY;
  b->device = dev0;
  b->sms = sms;
  b->n = n;
  b->flags = flags;
  b->fp16 = d0->fp16;
  b->color = d0->color;
  b->maps.assign(maps, maps + n);
  b->cams.assign(cams, cams + n);
  std::vector<MapDev> mdev(n);
  for (int i = 0; i < n; ++i) {
    int dev, s;
    mdev[i] = *map_dev(maps[i], &dev, &s);
  }
  auto fail = [&](cudaError_t e, const char* what) {
    mrh_batch_destroy(b);
    return e == cudaErrorMemoryAllocation ? MRH_ERR_OUT_OF_MEMORY : cuda_fail(e, what);
  };
  cudaError_t e = cudaMalloc(&b->maps_dev, sizeof(MapDev) * n);
  if (e != cudaSuccess) return fail(e, "cudaMalloc");
  e = cudaMalloc(&b->frames_dev, sizeof(BatchFrame) * n);
  if (e != cudaSuccess) return fail(e, "cudaMalloc");
  e = cudaMemcpy(b->maps_dev, mdev.data(), sizeof(MapDev) * n, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(e, "cudaMemcpy");
  b->frames_host.resize(n);
  uint32_t ray_tiles = 0;
  uint32_t alloc_tiles[4] = {0, 0, 0, 0};
  for (int i = 0; i < n; ++i) {
    const mrh_pinhole& K = cams[i];
    const size_t px = (size_t)K.width * K.height;
    void *rho = nullptr, *rgbp = nullptr;
    e = cudaMalloc(&rho, px * sizeof(float));
    if (e != cudaSuccess) return fail(e, "cudaMalloc");
    b->images.push_back(rho);
    e = cudaMalloc(&rgbp, px * sizeof(uint32_t));
    if (e != cudaSuccess) return fail(e, "cudaMalloc");
    b->images.push_back(rgbp);
    BatchFrame& f = b->frames_host[i];
    std::memset(&f, 0, sizeof(f));
    f.rho_img = (float*)rho;
    f.rgb_img = (uint32_t*)rgbp;
    f.ray_tile0 = ray_tiles;
    f.ray_tiles_x = (K.width + 15) / 16;
    ray_tiles += (uint32_t)f.ray_tiles_x * (uint32_t)((K.height + 7) / 8);
    for (int sh = 0; sh < 4; ++sh)
      alloc_tiles[sh] += (uint32_t)((K.width + kAllocShapes[sh].tw - 1) / kAllocShapes[sh].tw) *
                         (uint32_t)((K.height + kAllocShapes[sh].th - 1) / kAllocShapes[sh].th);
  }
  b->ray_tiles = ray_tiles;
  for (int sh = 0; sh < 4; ++sh) b->alloc_tiles[sh] = alloc_tiles[sh];
  for (int k = 0; k < 5; ++k) cudaEventCreate(&b->ev[k]);
  b->tuned = !(flags & MRH_BATCH_AUTOTUNE);
  *out = b;
  return MRH_OK;
}

mrh_status mrh_batch_destroy(mrh_batch* b) {
  if (!b) return MRH_OK;
  BatchDeviceGuard guard(b->device);
  cudaDeviceSynchronize();
  destroy_graph(b);
  for (void* p : b->images) cudaFree(p);
  if (b->maps_dev) cudaFree(b->maps_dev);
  if (b->frames_dev) cudaFree(b->frames_dev);
  for (int k = 0; k < 5; ++k)
    if (b->ev[k]) cudaEventDestroy(b->ev[k]);
  delete b;
  return MRH_OK;
}

mrh_status mrh_batch_integrate(mrh_batch* b, const mrh_batch_frame* frames, void* stream) {
  if (!b || !frames) return MRH_ERR_INVALID_ARG;
  for (int i = 0; i < b->n; ++i) {
    const mrh_batch_frame& fr = frames[i];
    const mrh_pinhole& K = b->cams[i];
    if (!fr.depth_dev || fr.K.width != K.width || fr.K.height != K.height) return MRH_ERR_INVALID_ARG;
    if (!(fr.K.fx > 0.f) || !(fr.K.fy > 0.f) || !(fr.K.max_depth >= fr.K.min_depth)) return MRH_ERR_INVALID_ARG;
    for (int k = 0; k < 16; ++k)
      if (!std::isfinite(fr.T_wc[k])) return MRH_ERR_INVALID_ARG;
  }
  BatchDeviceGuard guard(b->device);
  cudaStream_t s = (cudaStream_t)stream;
  // frame descriptors: pageable copy, so the host array is free again when the call returns
  for (int i = 0; i < b->n; ++i) {
    const mrh_batch_frame& fr = frames[i];
    BatchFrame& f = b->frames_host[i];
    CamArgs& c = f.cam;
    c.fx = fr.K.fx; c.fy = fr.K.fy; c.cx = fr.K.cx; c.cy = fr.K.cy;
    c.width = fr.K.width; c.height = fr.K.height;
    c.min_depth = fr.K.min_depth; c.max_depth = fr.K.max_depth;
    for (int r = 0; r < 3; ++r) {
      for (int q = 0; q < 3; ++q) c.R[3 * r + q] = (float)fr.T_wc[4 * r + q];
      c.t[r] = (float)fr.T_wc[4 * r + 3];
    }
    f.depth = fr.depth_dev;
    f.rgb = b->color ? fr.rgb_dev : nullptr;
    f.raycast_out = fr.raycast_dev;
  }
  const bool trial = !b->tuned && b->steps >= 1 && b->steps <= kTrials;
  const int ts = b->steps - 1;
  const int as = trial ? ts % 4 : b->alloc_shape;
  const int fs = trial ? ts % 4 : b->fuse_shape;
  const int rs = trial ? ts % kRayShapes : b->ray_shape;
  // allocation tile offsets depend on the allocation shape of this step
  {
    uint32_t acc = 0;
    for (int i = 0; i < b->n; ++i) {
      BatchFrame& f = b->frames_host[i];
      const mrh_pinhole& K = b->cams[i];
      f.alloc_tiles_x = (K.width + kAllocShapes[as].tw - 1) / kAllocShapes[as].tw;
      f.alloc_tile0 = acc;
      acc += (uint32_t)f.alloc_tiles_x * (uint32_t)((K.height + kAllocShapes[as].th - 1) / kAllocShapes[as].th);
    }
  }
  MRH_BCUDA(cudaMemcpyAsync(b->frames_dev, b->frames_host.data(), sizeof(BatchFrame) * b->n,
                            cudaMemcpyHostToDevice, s));
  const bool use_graph = (b->flags & MRH_BATCH_GRAPH) && s != nullptr && b->tuned;
  if (trial) {
    launch_step(b, as, fs, rs, s, b->ev, false);
    MRH_BCUDA(cudaGetLastError());
    MRH_BCUDA(cudaEventSynchronize(b->ev[4]));
    float t_alloc = 0, t_fuse = 0, t_ray = 0;
    cudaEventElapsedTime(&t_alloc, b->ev[0], b->ev[1]);
    cudaEventElapsedTime(&t_fuse, b->ev[1], b->ev[3]);
    cudaEventElapsedTime(&t_ray, b->ev[3], b->ev[4]);
    b->trial_ms[0][as] += t_alloc;
    b->trial_n[0][as] += 1;
    b->trial_ms[1][fs] += t_fuse;
    b->trial_n[1][fs] += 1;
    b->trial_ms[2][rs] += t_ray;
    b->trial_n[2][rs] += 1;
    if (ts == kTrials - 1) {
      auto best = [&](int g, int count) {
        int arg = 0;
        double bv = 1e30;
        for (int k = 0; k < count; ++k) {
          if (!b->trial_n[g][k]) continue;
          const double v = b->trial_ms[g][k] / b->trial_n[g][k];
          if (v < bv) {
            bv = v;
            arg = k;
          }
        }
        return arg;
      };
      b->alloc_shape = best(0, 4);
      b->fuse_shape = best(1, 4);
      b->ray_shape = best(2, kRayShapes);
      b->tuned = true;
    }
  } else if (use_graph) {
    if (!b->exec || b->graph_stream != s) {
      destroy_graph(b);
      MRH_BCUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      launch_step(b, b->alloc_shape, b->fuse_shape, b->ray_shape, s, b->ev, true);
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(s, &g);
      if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
      b->graph = g;
      e = cudaGraphInstantiate(&b->exec, g, 0);
      if (e != cudaSuccess) {
        destroy_graph(b);
        return cuda_fail(e, "cudaGraphInstantiate");
      }
      b->graph_stream = s;
    }
    MRH_BCUDA(cudaGraphLaunch(b->exec, s));
  } else {
    launch_step(b, as, fs, rs, s, b->ev, false);
    MRH_BCUDA(cudaGetLastError());
  }
  b->steps += 1;
  return MRH_OK;
}

mrh_status mrh_batch_last_step_ms(const mrh_batch* b, float* ms_out4) {
  if (!b || !ms_out4 || b->steps == 0) return MRH_ERR_INVALID_ARG;
  BatchDeviceGuard guard(b->device);
  MRH_BCUDA(cudaEventSynchronize(b->ev[4]));
  for (int k = 0; k < 4; ++k) MRH_BCUDA(cudaEventElapsedTime(&ms_out4[k], b->ev[k], b->ev[k + 1]));
  return MRH_OK;
}

mrh_status mrh_batch_config(const mrh_batch* b, int* config_out) {
  if (!b || !config_out) return MRH_ERR_INVALID_ARG;
  const AllocShape a = kAllocShapes[b->alloc_shape];
  const FuseShape f = kFuseShapes[b->fuse_shape];
  config_out[0] = a.tw;
  config_out[1] = a.th;
  config_out[2] = a.pw;
  config_out[3] = f.warps;
  config_out[4] = f.per_sm;
  config_out[5] = b->ray_shape;
  config_out[6] = b->tuned ? 1 : 0;
  config_out[7] = b->exec ? 1 : 0;
  return MRH_OK;
}

}  // extern "C"
