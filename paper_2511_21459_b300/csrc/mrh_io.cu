// Map save / load (the persistence half of streaming, Sec. 3.3).
//
// File: 8-byte magic, uint32 format version, uint32 size of mrh_map_params, the parameters the map was created with,
// uint64 block count, then per block (resident ones in key order, then archived ones in key order): int32 key[3],
// uint8 level, 3 bytes of padding, uint32 payload size, the payload in the library's own block layout (distance,
// weight, S2, colour planes of that level). Loading creates a map with the saved parameters and makes every saved
// block resident; streaming settings are not saved.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "mrh_internal.cuh"

namespace mrh {
namespace {

constexpr char kMagic[8] = {'M', 'R', 'H', 'M', 'A', 'P', '\0', '\1'};
constexpr uint32_t kVersion = 1;

struct IoBlock {
  uint32_t level_id;  // level << 28 | heap id (save), level << 28 (load)
  uint64_t offset;    // byte offset in the staging blob
};

// one warp per block: heap payload <-> staging blob (direction: 0 = to the blob, 1 = from the blob)
__global__ void __launch_bounds__(256) k_io_copy(MapDev m, const IoBlock* blocks, uint32_t n, uint8_t* blob, int dir) {
  const int lane = threadIdx.x & 31;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < n; b += nw) {
    const IoBlock io = blocks[b];
    if (io.level_id == 0xFFFFFFFFu) continue;  // not inserted (status set)
    const int l = (int)(io.level_id >> 28);
    uint8_t* heap = m.heap[l] + (size_t)(io.level_id & kPtrMask) * m.block_bytes[l];
    const uint32_t words = m.block_bytes[l] / 16;
    uint4* h = reinterpret_cast<uint4*>(heap);
    uint4* s = reinterpret_cast<uint4*>(blob + io.offset);
    for (uint32_t i = lane; i < words; i += 32) {
      if (dir == 0) s[i] = h[i];
      else h[i] = s[i];
    }
    // a loaded block's least D is unknown until it is fused again (NaN: the raycast does not skip it)
    if (dir == 1 && lane == 0) m.dmin[l][io.level_id & kPtrMask] = __int_as_float(0x7fffffff);
  }
}

// one thread per loaded block: insert the key, take a heap block of its level, record it in the raycaster's
// occupancy sets; the heap id goes back into blocks[b].level_id (all ones when the key could not be placed)
__global__ void __launch_bounds__(256) k_io_insert(MapDev m, const int32_t* keys, IoBlock* blocks, uint32_t n) {
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < n; b += gridDim.x * blockDim.x) {
    const int x = keys[3 * b], y = keys[3 * b + 1], z = keys[3 * b + 2];
    const int l = (int)(blocks[b].level_id >> 28);
    const unsigned long long key = pack_key(x, y, z);
    uint32_t s = hash_key(key, m.slot_mask);
    bool placed = false;
    for (uint32_t p = 0; p <= m.slot_mask; ++p, s = (s + 1) & m.slot_mask) {
      const unsigned long long old = atomicCAS(&m.slots[s].key, kEmptyKey, key);
      if (old == kEmptyKey || old == key) {
        placed = old == kEmptyKey;
        break;
      }
    }
    if (!placed) {
      set_status(m.st, kStHashFull);
      blocks[b].level_id = 0xFFFFFFFFu;
      continue;
    }
    const int t = atomicSub(&m.st->free_top[l], 1);
    if (t <= 0) {
      atomicAdd(&m.st->free_top[l], 1);
      set_status(m.st, kStPoolEmpty);
      blocks[b].level_id = 0xFFFFFFFFu;
      continue;
    }
    const uint32_t id = m.free_stack[l][t - 1];
    m.slots[s].val = id | ((uint32_t)l << 28);
    m.slots[s].stamp = 0;
    blocks[b].level_id = id | ((uint32_t)l << 28);
    const int rx = x >> kBrickShift, ry = y >> kBrickShift, rz = z >> kBrickShift;
    bool ok = occupancy_insert(m.brick_keys, m.brick_bits, m.brick_mask, rx, ry, rz, cell_bit(x, y, z));
    ok = ok && occupancy_insert(m.super_keys, m.super_bits, m.super_mask, rx >> kSuperShift, ry >> kSuperShift,
                                rz >> kSuperShift, cell_bit(rx, ry, rz));
    if (!ok) set_status(m.st, kStHashFull);
  }
}

}  // namespace

cudaError_t io_blocks_to_blob(const MapDev& m, const std::vector<uint32_t>& level_ids,
                              const std::vector<uint64_t>& offsets, uint8_t* blob_host, uint64_t blob_bytes,
                              cudaStream_t s, int sms) {
  const uint32_t n = (uint32_t)level_ids.size();
  if (n == 0) return cudaSuccess;
  std::vector<IoBlock> io(n);
  for (uint32_t i = 0; i < n; ++i) io[i] = IoBlock{level_ids[i], offsets[i]};
  IoBlock* d_io = nullptr;
  uint8_t* d_blob = nullptr;
  cudaError_t e = cudaMallocAsync(&d_io, n * sizeof(IoBlock), s);
  if (e == cudaSuccess) e = cudaMallocAsync(&d_blob, blob_bytes, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_io, io.data(), n * sizeof(IoBlock), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    k_io_copy<<<sms * 4, 256, 0, s>>>(m, d_io, n, d_blob, 0);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(blob_host, d_blob, blob_bytes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (d_io) cudaFreeAsync(d_io, s);
  if (d_blob) cudaFreeAsync(d_blob, s);
  return e;
}

cudaError_t io_blob_to_blocks(const MapDev& m, const std::vector<int32_t>& keys, const std::vector<uint32_t>& levels,
                              const std::vector<uint64_t>& offsets, const uint8_t* blob_host, uint64_t blob_bytes,
                              cudaStream_t s, int sms) {
  const uint32_t n = (uint32_t)levels.size();
  if (n == 0) return cudaSuccess;
  std::vector<IoBlock> io(n);
  for (uint32_t i = 0; i < n; ++i) io[i] = IoBlock{levels[i] << 28, offsets[i]};
  IoBlock* d_io = nullptr;
  int32_t* d_keys = nullptr;
  uint8_t* d_blob = nullptr;
  cudaError_t e = cudaMallocAsync(&d_io, n * sizeof(IoBlock), s);
  if (e == cudaSuccess) e = cudaMallocAsync(&d_keys, 3ull * n * sizeof(int32_t), s);
  if (e == cudaSuccess) e = cudaMallocAsync(&d_blob, blob_bytes, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_io, io.data(), n * sizeof(IoBlock), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_keys, keys.data(), 3ull * n * sizeof(int32_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_blob, blob_host, blob_bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    k_io_insert<<<sms * 4, 256, 0, s>>>(m, d_keys, d_io, n);
    k_io_copy<<<sms * 4, 256, 0, s>>>(m, d_io, n, d_blob, 1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (d_io) cudaFreeAsync(d_io, s);
  if (d_keys) cudaFreeAsync(d_keys, s);
  if (d_blob) cudaFreeAsync(d_blob, s);
  return e;
}

const char* io_magic() { return kMagic; }
uint32_t io_version() { return kVersion; }

}  // namespace mrh
