// Device-wide exclusive scans and a stable least-significant-digit radix sort of (key, 32-bit value) pairs, shared
// by the splat rasteriser (depth and tile sorts) and the mesh vertex collapse (cluster keys). Header-only: each
// translation unit instantiates what it uses.
//
// Radix sort: 8-bit digits; per pass, every chunk of kRsChunk consecutive items counts its digits (k_rs_hist, stored
// digit-major so that one exclusive scan gives each (digit, chunk) its first output position), then scatters its
// items in order (k_rs_scatter: rounds of 256 items in thread order, ranked within a warp by lane among equal
// digits and across warps by warp), so equal keys keep their input order.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace mrh {
namespace {

// exclusive prefix sums of x[0, n) in place, in chunks of kScanChunk; sums[b] = total of chunk b
constexpr int kScanThreads = 1024, kScanItems = 4, kScanChunk = kScanThreads * kScanItems;

template <class T>
__device__ inline T block_exclusive(T v, T* s_warp, T* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T incl = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const T y = __shfl_up_sync(~0u, incl, d);
    if (lane >= d) incl += y;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const T w = s_warp[lane];
    T wi = w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const T y = __shfl_up_sync(~0u, wi, d);
      if (lane >= d) wi += y;
    }
    s_warp[lane] = wi - w;
    if (lane == 31) *total = wi;
  }
  __syncthreads();
  return s_warp[warp] + incl - v;
}

template <class T>
__global__ void __launch_bounds__(kScanThreads) k_scan_chunks(T* x, uint64_t n, T* sums) {
  __shared__ T s_warp[32];
  __shared__ T s_total;
  const uint64_t base = (uint64_t)blockIdx.x * kScanChunk + (uint64_t)threadIdx.x * kScanItems;
  T v[kScanItems];
  T sum = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = base + k < n ? x[base + k] : T(0);
    sum += v[k];
  }
  T run = block_exclusive<T>(sum, s_warp, &s_total);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) x[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == 0) sums[blockIdx.x] = s_total;
}

// exclusive prefix of the chunk sums (one CTA; each thread a contiguous run); *total = their sum
template <class T>
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(T* sums, uint32_t nb, T* total) {
  __shared__ T s_warp[32];
  __shared__ T s_total;
  const uint32_t per = (nb + kScanThreads - 1) / kScanThreads, lo = threadIdx.x * per;
  T sum = 0;
  for (uint32_t i = lo; i < lo + per && i < nb; ++i) sum += sums[i];
  T run = block_exclusive<T>(sum, s_warp, &s_total);
  for (uint32_t i = lo; i < lo + per && i < nb; ++i) {
    const T c = sums[i];
    sums[i] = run;
    run += c;
  }
  if (threadIdx.x == 0 && total) *total = s_total;
}

template <class T>
__global__ void __launch_bounds__(kScanThreads) k_scan_add(T* x, uint64_t n, const T* sums) {
  const uint64_t base = (uint64_t)blockIdx.x * kScanChunk + (uint64_t)threadIdx.x * kScanItems;
  const T off = sums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k)
    if (base + k < n) x[base + k] += off;
}

template <class T>
void exclusive_scan(T* x, uint64_t n, T* sums, T* total, cudaStream_t s) {
  const uint32_t nb = (uint32_t)((n + kScanChunk - 1) / kScanChunk);
  if (nb == 0) {
    if (total) cudaMemsetAsync(total, 0, sizeof(T), s);
    return;
  }
  k_scan_chunks<T><<<nb, kScanThreads, 0, s>>>(x, n, sums);
  k_scan_sums<T><<<1, kScanThreads, 0, s>>>(sums, nb, total);
  k_scan_add<T><<<nb, kScanThreads, 0, s>>>(x, n, sums);
}

inline size_t scan_sums_count(uint64_t n) { return (size_t)((n + kScanChunk - 1) / kScanChunk) + 1; }

constexpr int kRsThreads = 256, kRsItems = 16, kRsChunk = kRsThreads * kRsItems;

// digit counts of each chunk, stored digit-major (hist[d * nb + b]) so that one exclusive scan gives every
// (digit, chunk) its first output position
template <class K>
__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const K* keys, uint32_t n, int shift, uint32_t* hist,
                                                        uint32_t nb) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  const int lane = threadIdx.x & 31;
  const uint32_t base = blockIdx.x * (uint32_t)kRsChunk;
  uint32_t dig[kRsItems];  // all of the chunk's loads issued before the first count
#pragma unroll
  for (int r = 0; r < kRsItems; ++r) {
    const uint32_t i = base + r * kRsThreads + threadIdx.x;
    dig[r] = i < n ? (uint32_t)(keys[i] >> shift) & 255u : 256u;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kRsItems; ++r) {
    const uint32_t d = dig[r];
    const unsigned peers = __match_any_sync(~0u, d);  // one shared-memory add per distinct digit of the warp
    if (d < 256u && (peers & ((1u << lane) - 1u)) == 0) atomicAdd(&h[d], (uint32_t)__popc(peers));
  }
  __syncthreads();
  hist[threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

// stable scatter of one chunk: items are ranked in order (rounds of 256 in thread order; within a warp by lane,
// across warps by warp) on top of the chunk's scanned first position per digit; the chunk's keys and values are
// loaded up front
template <class K>
__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const K* kin, const uint32_t* vin, K* kout, uint32_t* vout,
                                                           uint32_t n, int shift, const uint32_t* hist, uint32_t nb) {
  __shared__ uint32_t s_base[256];
  __shared__ uint32_t s_warp[kRsThreads / 32][256];
  __shared__ uint32_t s_tot[256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  s_base[threadIdx.x] = hist[threadIdx.x * nb + blockIdx.x];
  const uint32_t base = blockIdx.x * (uint32_t)kRsChunk;
  K key[kRsItems];
  uint32_t val[kRsItems];
#pragma unroll
  for (int r = 0; r < kRsItems; ++r) {
    const uint32_t i = base + r * kRsThreads + threadIdx.x;
    key[r] = i < n ? kin[i] : K(0);
    val[r] = i < n ? vin[i] : 0u;
  }
#pragma unroll
  for (int r = 0; r < kRsItems; ++r) {
    if (base + r * kRsThreads < n) {  // uniform over the CTA
#pragma unroll
      for (int w = 0; w < kRsThreads / 32; ++w) s_warp[w][threadIdx.x] = 0;
      __syncthreads();
      const uint32_t i = base + r * kRsThreads + threadIdx.x;
      const bool live = i < n;
      const uint32_t d = live ? (uint32_t)(key[r] >> shift) & 255u : 256u;
      const unsigned peers = __match_any_sync(~0u, d);
      const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
      if (live && rank == 0) s_warp[warp][d] = (uint32_t)__popc(peers);
      __syncthreads();
      {
        uint32_t acc = 0;
#pragma unroll
        for (int w = 0; w < kRsThreads / 32; ++w) {
          const uint32_t c = s_warp[w][threadIdx.x];
          s_warp[w][threadIdx.x] = acc;
          acc += c;
        }
        s_tot[threadIdx.x] = acc;
      }
      __syncthreads();
      if (live) {
        const uint32_t pos = s_base[d] + s_warp[warp][d] + rank;
        kout[pos] = key[r];
        vout[pos] = val[r];
      }
      __syncthreads();
      s_base[threadIdx.x] += s_tot[threadIdx.x];
    }
  }
}

// Stable radix sort of (key, value) pairs over key bits [0, bits): 8-bit digits, ping-pong between the two buffers
// of keys and vals; returns the index (0 or 1) of the buffer holding the result.
template <class K>
int radix_sort(K* keys[2], uint32_t* vals[2], uint32_t n, int bits, uint32_t* hist, uint32_t* sums, cudaStream_t s) {
  const uint32_t nb = (n + kRsChunk - 1) / kRsChunk;
  int cur = 0;
  if (n == 0) return cur;
  for (int shift = 0; shift < bits; shift += 8) {
    k_rs_hist<K><<<nb, kRsThreads, 0, s>>>(keys[cur], n, shift, hist, nb);
    exclusive_scan<uint32_t>(hist, 256ull * nb, sums, nullptr, s);
    k_rs_scatter<K><<<nb, kRsThreads, 0, s>>>(keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], n, shift, hist, nb);
    cur ^= 1;
  }
  return cur;
}

inline size_t radix_scratch_words(uint32_t n) {
  const uint64_t nb = (n + kRsChunk - 1) / kRsChunk;
  return 256 * nb;
}

}  // namespace
}  // namespace mrh
