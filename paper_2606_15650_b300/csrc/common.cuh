// Shared device helpers: error plumbing, launch accounting, warp/block scans.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>

#include "../../include/anonshield.h"

namespace as {

// Number of SMs on the target part (B300: 148). The runtime reads the real
// count at start-up; this is only the fallback.
constexpr int kDefaultSMs = 148;

// Every kernel launch made by the library is counted here (host side), in
// total and per host thread (a lane's own launches, with other lanes running).
extern std::atomic<uint64_t> g_launches;
extern thread_local uint64_t t_launches;

inline void count_launch(uint64_t n = 1) {
  g_launches.fetch_add(n, std::memory_order_relaxed);
  t_launches += n;
}

// Thread-local message of the last kernel-level failure.
void set_k_error(const std::string& msg);

// Device-side error flag written by kernels whose waits are bounded.
// code 0 = fine; the first error wins (atomicCAS from 0).
struct DevError {
  uint32_t code;
  uint32_t where;
  uint32_t info0;
  uint32_t info1;
};
constexpr uint32_t kErrTimeout = 1;
constexpr uint32_t kErrCapacity = 2;
constexpr uint32_t kErrBounds = 3;

__device__ inline void report_error(DevError* e, uint32_t code, uint32_t where, uint32_t a = 0, uint32_t b = 0) {
  if (e == nullptr) return;
  if (atomicCAS(&e->code, 0u, code) == 0u) {
    e->where = where;
    e->info0 = a;
    e->info1 = b;
  }
}

inline unsigned grid_1d(uint64_t n, unsigned threads, unsigned cap = 1u << 30) {
  uint64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

__device__ __forceinline__ bool is_alnum(uint32_t c) {
  return (c - '0' < 10u) || ((c | 0x20u) - 'a' < 26u);
}

// bit i of the record-start bitmap: a record begins at byte i
__device__ __forceinline__ bool rs_bit(const uint32_t* rs, uint32_t i) { return (rs[i >> 5] >> (i & 31)) & 1u; }

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T v) {
  const unsigned lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= (unsigned)o) v += n;
  }
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide exclusive scan of one value per thread (blockDim.x <= 1024,
// multiple of 32). `smem` needs 33 slots. Returns the exclusive prefix;
// *total receives the block sum (same in every thread).
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* smem, T* total) {
  const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T inc = warp_inclusive_scan(v);
  if (lane == 31) smem[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    T s = lane < nw ? smem[lane] : T(0);
    T si = warp_inclusive_scan(s);
    if (lane < nw) smem[lane] = si - s;
    if (lane == nw - 1) smem[32] = si;
  }
  __syncthreads();
  T res = smem[warp] + inc - v;
  *total = smem[32];
  __syncthreads();
  return res;
}

// Largest i in [0, n) with a[i] <= x, or -1 (a sorted ascending).
template <typename T, typename U>
__device__ __forceinline__ int64_t upper_index(const T* a, int64_t n, U x) {
  int64_t lo = 0, hi = n;  // first index with a[i] > x
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if ((U)a[mid] <= x) lo = mid + 1; else hi = mid;
  }
  return lo - 1;
}

// Two-lane FP32 arithmetic (sm_100 and later): one instruction computes both
// lanes of a packed pair, each lane rounded exactly as the scalar instruction.
static __device__ __forceinline__ uint64_t f2pack(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
static __device__ __forceinline__ void f2unpack(uint64_t v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
static __device__ __forceinline__ uint64_t f2splat(float x) { return f2pack(x, x); }
static __device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
static __device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
static __device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

}  // namespace as

#define AS_CUDA_OK(expr)                                                              \
  do {                                                                                \
    cudaError_t _e = (expr);                                                          \
    if (_e != cudaSuccess) {                                                          \
      ::as::set_k_error(std::string(#expr) + ": " + cudaGetErrorString(_e));          \
      return AS_ERR_CUDA;                                                             \
    }                                                                                 \
  } while (0)
