// Device-wide exclusive prefix sum in three passes (tile sums, scan of tile
// sums, tile scan with offsets). Values come from a load functor so callers
// can scan predicates (e.g. "byte starts a token") without materialising them.
// The element count is the host's n, or, when a device count is given,
// min(n, *n_dev + add): the grid is sized for the host capacity n and the
// blocks past the device count return at once, so a scan over the spans
// that a kernel produced costs what those spans cost, not the capacity.
#pragma once

#include "common.cuh"

namespace as {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint64_t scan_count(uint64_t n, const uint32_t* n_dev, uint32_t add) {
  return n_dev ? min(n, (uint64_t)*n_dev + add) : n;
}

template <typename T, typename Load>
__global__ void __launch_bounds__(kScanThreads)
    scan_tile_sums(Load load, uint64_t n, T* tile_sums, const uint32_t* n_dev, uint32_t add) {
  __shared__ T sm[33];
  n = scan_count(n, n_dev, add);
  if ((uint64_t)blockIdx.x * kScanTile >= n) return;  // the whole block: past the count
  uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
  T s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    uint64_t i = base + k;
    if (i < n) s += load(i);
  }
  T tot;
  block_exclusive_scan(s, sm, &tot);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

// One block scans all tile sums in place (exclusive) and writes the total.
template <typename T>
__global__ void __launch_bounds__(1024)
    scan_tile_offsets(T* tile_sums, uint64_t n, T* total, const uint32_t* n_dev, uint32_t add) {
  __shared__ T sm[33];
  const uint64_t n_tiles = (scan_count(n, n_dev, add) + kScanTile - 1) / kScanTile;
  T carry = 0;
  for (uint64_t b = 0; b < n_tiles; b += blockDim.x) {
    uint64_t i = b + threadIdx.x;
    T v = i < n_tiles ? tile_sums[i] : T(0);
    T tot;
    T ex = block_exclusive_scan(v, sm, &tot);
    if (i < n_tiles) tile_sums[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0 && total != nullptr) *total = carry;
}

template <typename T, typename Load>
__global__ void __launch_bounds__(kScanThreads)
    scan_tiles(Load load, uint64_t n, const T* tile_offsets, T* out, const uint32_t* n_dev, uint32_t add) {
  __shared__ T sm[33];
  n = scan_count(n, n_dev, add);
  if ((uint64_t)blockIdx.x * kScanTile >= n) return;  // the whole block: past the count
  uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
  T v[kScanItems];
  T s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    uint64_t i = base + k;
    v[k] = i < n ? load(i) : T(0);
    s += v[k];
  }
  T tot;
  T run = block_exclusive_scan(s, sm, &tot) + tile_offsets[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    uint64_t i = base + k;
    if (i < n) out[i] = run;
    run += v[k];
  }
}

// The last pass of a compaction: instead of the prefix of every element, the
// rank of each nonzero element goes to emit(i, rank), so no per-element
// position array is written and read back.
template <typename T, typename Load, typename Emit>
__global__ void __launch_bounds__(kScanThreads)
    scan_emit_tiles(Load load, uint64_t n, const T* tile_offsets, Emit emit) {
  __shared__ T sm[33];
  uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
  T v[kScanItems];
  T s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    uint64_t i = base + k;
    v[k] = i < n ? load(i) : T(0);
    s += v[k];
  }
  T tot;
  T run = block_exclusive_scan(s, sm, &tot) + tile_offsets[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (v[k]) emit(base + k, run);  // v[k] != 0 only for base + k < n
    run += v[k];
  }
}

inline uint64_t scan_tiles_needed(uint64_t n) { return (n + kScanTile - 1) / kScanTile; }

// out[i] = sum_{j<i} load(j); *total_dev = sum of all. tile_scratch needs
// scan_tiles_needed(n) elements. n may be 0 (then only *total_dev = 0).
// With n_dev, the count is min(n, *n_dev + add) and out[] is written for
// that many elements only.
template <typename T, typename Load>
inline void exclusive_scan(Load load, uint64_t n, T* out, T* total_dev, T* tile_scratch, cudaStream_t st,
                           const uint32_t* n_dev = nullptr, uint32_t add = 0) {
  uint64_t tiles = scan_tiles_needed(n);
  if (tiles == 0) {
    cudaMemsetAsync(total_dev, 0, sizeof(T), st);
    return;
  }
  scan_tile_sums<T, Load><<<(unsigned)tiles, kScanThreads, 0, st>>>(load, n, tile_scratch, n_dev, add);
  scan_tile_offsets<T><<<1, 1024, 0, st>>>(tile_scratch, n, total_dev, n_dev, add);
  scan_tiles<T, Load><<<(unsigned)tiles, kScanThreads, 0, st>>>(load, n, tile_scratch, out, n_dev, add);
  count_launch(3);
}

// emit(i, rank) for every i < n with load(i) != 0, rank = the number of such
// elements before i (in index order); *total_dev = their count.
template <typename T, typename Load, typename Emit>
inline void compact_emit(Load load, uint64_t n, Emit emit, T* total_dev, T* tile_scratch, cudaStream_t st) {
  uint64_t tiles = scan_tiles_needed(n);
  if (tiles == 0) {
    cudaMemsetAsync(total_dev, 0, sizeof(T), st);
    return;
  }
  scan_tile_sums<T, Load><<<(unsigned)tiles, kScanThreads, 0, st>>>(load, n, tile_scratch, nullptr, 0);
  scan_tile_offsets<T><<<1, 1024, 0, st>>>(tile_scratch, n, total_dev, nullptr, 0);
  scan_emit_tiles<T, Load, Emit><<<(unsigned)tiles, kScanThreads, 0, st>>>(load, n, tile_scratch, emit);
  count_launch(3);
}

// compact_emit when a producer kernel already wrote each tile's count of
// nonzero elements into tile_sums[0 .. scan_tiles_needed(n)): the counting
// pass is skipped.
template <typename T, typename Load, typename Emit>
inline void compact_emit_from_sums(Load load, uint64_t n, Emit emit, T* total_dev, T* tile_sums, cudaStream_t st) {
  uint64_t tiles = scan_tiles_needed(n);
  if (tiles == 0) {
    cudaMemsetAsync(total_dev, 0, sizeof(T), st);
    return;
  }
  scan_tile_offsets<T><<<1, 1024, 0, st>>>(tile_sums, n, total_dev, nullptr, 0);
  scan_emit_tiles<T, Load, Emit><<<(unsigned)tiles, kScanThreads, 0, st>>>(load, n, tile_sums, emit);
  count_launch(2);
}

}  // namespace as
