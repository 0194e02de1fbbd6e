// Encoder kernels besides the tcgen05 GEMM (AnonShield §2 stage (2)):
//   - FP32 SIMT GEMM (the FP32 path and its one-record-per-launch baseline),
//   - self-attention over packed sequences: FP32 SIMT and BF16 tensor-core
//     (mma.sync m16n8k16, flash-style online softmax in FP32),
//   - embedding gather + LayerNorm, LayerNorm, LayerNorm + classifier/argmax.
// Block layout of the encoder (post-LayerNorm, learned positions, exact GELU,
// LayerNorm with biased variance and eps 1e-5, scale 1/sqrt(64)).
#include <math.h>

#include "encoder.cuh"

namespace as {

// ------------------------------------------------------------- SIMT GEMM FP32

namespace simt {
constexpr int BM = 128, BN = 128, BK = 8;

template <int EPI>
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, const float* __restrict__ A,
                                                   const float* __restrict__ B, const float* __restrict__ bias,
                                                   const float* __restrict__ resid, float* __restrict__ out) {
  __shared__ __align__(16) float As[2][BK][BM + 4];
  __shared__ __align__(16) float Bs[2][BK][BN + 4];
  const int tid = threadIdx.x;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int lrow = tid >> 1, lk = (tid & 1) * 4;
  const bool a_ok = (m0 + lrow) < M;
  const float* Ap = A + (size_t)(a_ok ? m0 + lrow : 0) * K + lk;
  const float* Bp = B + (size_t)(n0 + lrow) * K + lk;
  float4 ra = a_ok ? *reinterpret_cast<const float4*>(Ap) : make_float4(0.f, 0.f, 0.f, 0.f);
  float4 rb = *reinterpret_cast<const float4*>(Bp);
  As[0][lk + 0][lrow] = ra.x; As[0][lk + 1][lrow] = ra.y; As[0][lk + 2][lrow] = ra.z; As[0][lk + 3][lrow] = ra.w;
  Bs[0][lk + 0][lrow] = rb.x; Bs[0][lk + 1][lrow] = rb.y; Bs[0][lk + 2][lrow] = rb.z; Bs[0][lk + 3][lrow] = rb.w;
  __syncthreads();
  const int tx = tid & 15, ty = tid >> 4;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  int cur = 0;
  for (int k0 = 0; k0 < K; k0 += BK) {
    const bool more = k0 + BK < K;
    if (more) {
      ra = a_ok ? *reinterpret_cast<const float4*>(Ap + k0 + BK) : make_float4(0.f, 0.f, 0.f, 0.f);
      rb = *reinterpret_cast<const float4*>(Bp + k0 + BK);
    }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[8], b[8];
      float4 a0 = *reinterpret_cast<const float4*>(&As[cur][kk][ty * 4]);
      float4 a1 = *reinterpret_cast<const float4*>(&As[cur][kk][64 + ty * 4]);
      float4 b0 = *reinterpret_cast<const float4*>(&Bs[cur][kk][tx * 4]);
      float4 b1 = *reinterpret_cast<const float4*>(&Bs[cur][kk][64 + tx * 4]);
      a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w; a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
      b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w; b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) {
      const int nx = cur ^ 1;
      As[nx][lk + 0][lrow] = ra.x; As[nx][lk + 1][lrow] = ra.y; As[nx][lk + 2][lrow] = ra.z; As[nx][lk + 3][lrow] = ra.w;
      Bs[nx][lk + 0][lrow] = rb.x; Bs[nx][lk + 1][lrow] = rb.y; Bs[nx][lk + 2][lrow] = rb.z; Bs[nx][lk + 3][lrow] = rb.w;
    }
    __syncthreads();
    cur ^= 1;
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
    if (m >= M) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int n = n0 + h * 64 + tx * 4;
      float4 bv = bias ? *reinterpret_cast<const float4*>(bias + n) : make_float4(0.f, 0.f, 0.f, 0.f);
      float v0 = acc[i][h * 4 + 0] + bv.x, v1 = acc[i][h * 4 + 1] + bv.y;
      float v2 = acc[i][h * 4 + 2] + bv.z, v3 = acc[i][h * 4 + 3] + bv.w;
      if (EPI == AS_EPI_BIAS_GELU) {
        v0 = 0.5f * v0 * (1.f + erff(v0 * 0.70710678118654752f));
        v1 = 0.5f * v1 * (1.f + erff(v1 * 0.70710678118654752f));
        v2 = 0.5f * v2 * (1.f + erff(v2 * 0.70710678118654752f));
        v3 = 0.5f * v3 * (1.f + erff(v3 * 0.70710678118654752f));
      } else if (EPI == AS_EPI_BIAS_RESID) {
        float4 r = *reinterpret_cast<const float4*>(resid + (size_t)m * N + n);
        v0 += r.x; v1 += r.y; v2 += r.z; v3 += r.w;
      }
      *reinterpret_cast<float4*>(out + (size_t)m * N + n) = make_float4(v0, v1, v2, v3);
    }
  }
}
}  // namespace simt

as_status gemm_simt_f32(int epi, int64_t M, int64_t N, int64_t K, const float* A, const float* B, const float* bias,
                        const float* resid, float* out, cudaStream_t st) {
  if (M < 1 || N % 128 != 0 || K % 8 != 0 || K < 8 || M > (1ll << 31) - 1 || (M + 127) / 128 > 65535) {
    set_k_error("gemm_simt_f32: unsupported shape");
    return AS_ERR_ARG;
  }
  dim3 grid((unsigned)(N / 128), (unsigned)((M + 127) / 128));
  switch (epi) {
    case AS_EPI_BIAS: simt::gemm_kernel<AS_EPI_BIAS><<<grid, 256, 0, st>>>((int)M, (int)N, (int)K, A, B, bias, resid, out); break;
    case AS_EPI_BIAS_GELU: simt::gemm_kernel<AS_EPI_BIAS_GELU><<<grid, 256, 0, st>>>((int)M, (int)N, (int)K, A, B, bias, resid, out); break;
    case AS_EPI_BIAS_RESID: simt::gemm_kernel<AS_EPI_BIAS_RESID><<<grid, 256, 0, st>>>((int)M, (int)N, (int)K, A, B, bias, resid, out); break;
    default: set_k_error("gemm_simt_f32: bad epilogue"); return AS_ERR_ARG;
  }
  count_launch();
  AS_CUDA_OK(cudaGetLastError());
  return AS_OK;
}

// ------------------------------------------------------------ attention FP32

// One thread per query row (64 per block), K/V tiles of 32 keys in shared
// memory, online softmax per 32-key tile.
__global__ void __launch_bounds__(64) attn_f32_kernel(const float* __restrict__ qkv, float* __restrict__ out,
                                                      const int32_t* __restrict__ seq_start,
                                                      const int32_t* __restrict__ seq_len, int d) {
  const int s = blockIdx.x, h = blockIdx.y, L = seq_len[s], q0 = blockIdx.z * 64;
  if (q0 >= L) return;
  const size_t ld = 3 * (size_t)d;
  const float* base = qkv + (size_t)seq_start[s] * ld + h * 64;
  __shared__ float Ks[32][64];
  __shared__ float Vs[32][64];
  const int qi = q0 + threadIdx.x;
  const bool qv = qi < L;
  float q[64], acc[64];
#pragma unroll
  for (int j = 0; j < 64; ++j) {
    q[j] = qv ? base[(size_t)qi * ld + j] * 0.125f : 0.f;
    acc[j] = 0.f;
  }
  float m = -INFINITY, l = 0.f;
  for (int k0 = 0; k0 < L; k0 += 32) {
    __syncthreads();
    {
      const int key = threadIdx.x >> 1, half = (threadIdx.x & 1) * 32;
      const bool kv = k0 + key < L;
      const float* kp = base + (size_t)(k0 + key) * ld + d + half;
      const float* vp = base + (size_t)(k0 + key) * ld + 2 * d + half;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        Ks[key][half + j] = kv ? kp[j] : 0.f;
        Vs[key][half + j] = kv ? vp[j] : 0.f;
      }
    }
    __syncthreads();
    const int nk = min(32, L - k0);
    float sc[32];
    float tmax = -INFINITY;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      float a = 0.f;
#pragma unroll
      for (int c = 0; c < 64; ++c) a = fmaf(q[c], Ks[j][c], a);
      sc[j] = j < nk ? a : -INFINITY;
      tmax = fmaxf(tmax, sc[j]);
    }
    const float mn = fmaxf(m, tmax);
    const float corr = expf(m - mn);
    l *= corr;
#pragma unroll
    for (int c = 0; c < 64; ++c) acc[c] *= corr;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const float p = expf(sc[j] - mn);
      l += p;
#pragma unroll
      for (int c = 0; c < 64; ++c) acc[c] = fmaf(p, Vs[j][c], acc[c]);
    }
    m = mn;
  }
  if (!qv) return;
  const float inv = 1.f / l;
  float* o = out + (size_t)(seq_start[s] + qi) * d + h * 64;
#pragma unroll
  for (int c = 0; c < 64; c += 4)
    *reinterpret_cast<float4*>(o + c) = make_float4(acc[c] * inv, acc[c + 1] * inv, acc[c + 2] * inv, acc[c + 3] * inv);
}

as_status attention_f32(const float* qkv, float* out, const int32_t* seq_start, const int32_t* seq_len, int32_t n_seq,
                        int32_t max_len, int32_t d_model, int32_t n_heads, cudaStream_t st) {
  if (n_seq == 0 || max_len == 0) return AS_OK;
  if (d_model != n_heads * 64 || max_len > 4096 || n_heads > 65535) {
    set_k_error("attention_f32: head dim must be 64 and sequences at most 4096 tokens");
    return AS_ERR_ARG;
  }
  dim3 grid((unsigned)n_seq, (unsigned)n_heads, (unsigned)((max_len + 63) / 64));
  attn_f32_kernel<<<grid, 64, 0, st>>>(qkv, out, seq_start, seq_len, d_model);
  count_launch();
  AS_CUDA_OK(cudaGetLastError());
  return AS_OK;
}

// ------------------------------------------------------------ attention BF16

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// Two FP32 values to E4M3 (round to nearest even, saturate to +-448), first
// value in the low byte.
__device__ __forceinline__ uint16_t pack_e4m3(float lo, float hi) {
  uint16_t r;
  asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(r) : "f"(hi), "f"(lo));
  return r;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid) {
  // src-size 0 zero-fills the 16 destination bytes (keys past the sequence end)
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}
// 2^x with the hardware approximation (MUFU.EX2); exact enough for an FP32
// softmax whose inputs were rounded to BF16.
__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Flash-style attention, one block per (sequence, head, 64-query tile); the
// blocks of one (sequence, head) are consecutive so that K and V are read
// from DRAM once and then served from L2. 4 warps x 16 query rows. K and V
// tiles of 64 keys are double-buffered in shared memory with cp.async;
// B fragments come from ldmatrix (K) and ldmatrix.trans (V); S = Q K^T and
// O += P V run on m16n8k16 BF16 tensor cores; softmax statistics in FP32.
template <bool OUT8>
__global__ void __launch_bounds__(128, 4) attn_bf16_kernel(const __nv_bfloat16* __restrict__ qkv,
                                                          void* __restrict__ out_v,
                                                          const int32_t* __restrict__ seq_start,
                                                          const int32_t* __restrict__ seq_len, int d, int n_heads,
                                                          int q_tiles, float out_inv_scale) {
  constexpr int P = 72;  // padded row (bf16): 144 B, conflict-free ldmatrix rows
  __shared__ __align__(128) __nv_bfloat16 Ks[2][64][P];
  __shared__ __align__(128) __nv_bfloat16 Vs[2][64][P];
  const int qt = blockIdx.x % q_tiles;
  const int rest = blockIdx.x / q_tiles;
  const int h = rest % n_heads, s = rest / n_heads;
  const int L = seq_len[s], q0 = qt * 64;
  if (q0 >= L) return;
  const size_t ld = 3 * (size_t)d;
  const __nv_bfloat16* base = qkv + (size_t)seq_start[s] * ld + h * 64;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int mi = lane >> 3, mr = lane & 7;
  const int n_tiles = (L + 63) / 64;

  auto load_tile = [&](int buf, int k0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int idx = threadIdx.x + i * 128;
      const int key = idx >> 3, c8 = (idx & 7) * 8;
      const bool v = k0 + key < L;
      const __nv_bfloat16* src = base + (size_t)(v ? k0 + key : 0) * ld;
      cp_async16((uint32_t)__cvta_generic_to_shared(&Ks[buf][key][c8]), src + d + c8, v);
      cp_async16((uint32_t)__cvta_generic_to_shared(&Vs[buf][key][c8]), src + 2 * d + c8, v);
    }
    cp_async_commit();
  };
  load_tile(0, 0);

  const int qr0 = q0 + warp * 16 + g, qr1 = qr0 + 8;
  uint32_t qa[4][4];
#pragma unroll
  for (int ks = 0; ks < 4; ++ks) {
    const int c = ks * 16 + 2 * t;
    qa[ks][0] = qr0 < L ? *reinterpret_cast<const uint32_t*>(base + (size_t)qr0 * ld + c) : 0u;
    qa[ks][1] = qr1 < L ? *reinterpret_cast<const uint32_t*>(base + (size_t)qr1 * ld + c) : 0u;
    qa[ks][2] = qr0 < L ? *reinterpret_cast<const uint32_t*>(base + (size_t)qr0 * ld + c + 8) : 0u;
    qa[ks][3] = qr1 < L ? *reinterpret_cast<const uint32_t*>(base + (size_t)qr1 * ld + c + 8) : 0u;
  }
  float o[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i) o[i][0] = o[i][1] = o[i][2] = o[i][3] = 0.f;
  float m0 = -INFINITY, m1 = -INFINITY, l0 = 0.f, l1 = 0.f;
  const float sl2 = 0.125f * 1.4426950408889634f;  // 1/sqrt(64) * log2(e)

  for (int it = 0; it < n_tiles; ++it) {
    const int buf = it & 1, k0 = it * 64;
    if (it + 1 < n_tiles) {
      load_tile(buf ^ 1, k0 + 64);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    float sf[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) sf[nt][0] = sf[nt][1] = sf[nt][2] = sf[nt][3] = 0.f;
#pragma unroll
    for (int ks = 0; ks < 4; ++ks)
#pragma unroll
      for (int np = 0; np < 4; ++np) {
        uint32_t b0a, b1a, b0b, b1b;
        ldsm_x4((uint32_t)__cvta_generic_to_shared(&Ks[buf][np * 16 + (mi >> 1) * 8 + mr][ks * 16 + (mi & 1) * 8]),
                b0a, b1a, b0b, b1b);
        mma16816(sf[2 * np], qa[ks], b0a, b1a);
        mma16816(sf[2 * np + 1], qa[ks], b0b, b1b);
      }
    float mx0 = -INFINITY, mx1 = -INFINITY;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int key = k0 + nt * 8 + 2 * t + (e & 1);
        const float v = key < L ? sf[nt][e] * sl2 : -INFINITY;
        sf[nt][e] = v;
        if (e < 2) mx0 = fmaxf(mx0, v); else mx1 = fmaxf(mx1, v);
      }
    mx0 = fmaxf(mx0, __shfl_xor_sync(0xffffffffu, mx0, 1));
    mx0 = fmaxf(mx0, __shfl_xor_sync(0xffffffffu, mx0, 2));
    mx1 = fmaxf(mx1, __shfl_xor_sync(0xffffffffu, mx1, 1));
    mx1 = fmaxf(mx1, __shfl_xor_sync(0xffffffffu, mx1, 2));
    const float mn0 = fmaxf(m0, mx0), mn1 = fmaxf(m1, mx1);
    const float c0 = ex2(m0 - mn0), c1 = ex2(m1 - mn1);
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      sf[nt][0] = ex2(sf[nt][0] - mn0);
      sf[nt][1] = ex2(sf[nt][1] - mn0);
      sf[nt][2] = ex2(sf[nt][2] - mn1);
      sf[nt][3] = ex2(sf[nt][3] - mn1);
      s0 += sf[nt][0] + sf[nt][1];
      s1 += sf[nt][2] + sf[nt][3];
    }
    s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
    s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
    s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
    s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
    l0 = l0 * c0 + s0;
    l1 = l1 * c1 + s1;
    m0 = mn0;
    m1 = mn1;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      o[nt][0] *= c0; o[nt][1] *= c0; o[nt][2] *= c1; o[nt][3] *= c1;
    }
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      uint32_t pa[4];
      pa[0] = pack_bf16(sf[2 * kk][0], sf[2 * kk][1]);
      pa[1] = pack_bf16(sf[2 * kk][2], sf[2 * kk][3]);
      pa[2] = pack_bf16(sf[2 * kk + 1][0], sf[2 * kk + 1][1]);
      pa[3] = pack_bf16(sf[2 * kk + 1][2], sf[2 * kk + 1][3]);
#pragma unroll
      for (int dp = 0; dp < 4; ++dp) {
        uint32_t b0a, b1a, b0b, b1b;
        ldsm_x4_t((uint32_t)__cvta_generic_to_shared(&Vs[buf][kk * 16 + (mi & 1) * 8 + mr][dp * 16 + (mi >> 1) * 8]),
                  b0a, b1a, b0b, b1b);
        mma16816(o[2 * dp], pa, b0a, b1a);
        mma16816(o[2 * dp + 1], pa, b0b, b1b);
      }
    }
    __syncthreads();  // the next iteration refills this buffer
  }
  const float i0 = 1.f / l0, i1 = 1.f / l1;
  const size_t row0 = (size_t)seq_start[s];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int c = h * 64 + nt * 8 + 2 * t;
    if (OUT8) {
      uint8_t* out = static_cast<uint8_t*>(out_v);
      const float a0 = i0 * out_inv_scale, a1 = i1 * out_inv_scale;
      if (qr0 < L) *reinterpret_cast<uint16_t*>(out + (row0 + qr0) * d + c) = pack_e4m3(o[nt][0] * a0, o[nt][1] * a0);
      if (qr1 < L) *reinterpret_cast<uint16_t*>(out + (row0 + qr1) * d + c) = pack_e4m3(o[nt][2] * a1, o[nt][3] * a1);
    } else {
      __nv_bfloat16* out = static_cast<__nv_bfloat16*>(out_v);
      if (qr0 < L)
        *reinterpret_cast<uint32_t*>(out + (row0 + qr0) * d + c) = pack_bf16(o[nt][0] * i0, o[nt][1] * i0);
      if (qr1 < L)
        *reinterpret_cast<uint32_t*>(out + (row0 + qr1) * d + c) = pack_bf16(o[nt][2] * i1, o[nt][3] * i1);
    }
  }
}

as_status attention_bf16_e4m3(const __nv_bfloat16* qkv, uint8_t* out, float out_scale, const int32_t* seq_start,
                              const int32_t* seq_len, int32_t n_seq, int32_t max_len, int32_t d_model,
                              int32_t n_heads, cudaStream_t st) {
  if (n_seq == 0 || max_len == 0) return AS_OK;
  if (d_model != n_heads * 64 || max_len > 4096 || !(out_scale > 0.f)) {
    set_k_error("attention: head dim must be 64, sequences at most 4096 tokens, scale > 0");
    return AS_ERR_ARG;
  }
  const int q_tiles = (max_len + 63) / 64;
  const uint64_t blocks = (uint64_t)n_seq * n_heads * q_tiles;
  if (blocks > 0x7FFFFFFFull) {
    set_k_error("attention: too many sequences in one batch");
    return AS_ERR_ARG;
  }
  attn_bf16_kernel<true><<<(unsigned)blocks, 128, 0, st>>>(qkv, out, seq_start, seq_len, d_model, n_heads, q_tiles,
                                                           1.0f / out_scale);
  count_launch();
  AS_CUDA_OK(cudaGetLastError());
  return AS_OK;
}

as_status attention_bf16(const __nv_bfloat16* qkv, __nv_bfloat16* out, const int32_t* seq_start,
                         const int32_t* seq_len, int32_t n_seq, int32_t max_len, int32_t d_model, int32_t n_heads,
                         cudaStream_t st) {
  if (n_seq == 0 || max_len == 0) return AS_OK;
  if (d_model != n_heads * 64 || max_len > 4096) {
    set_k_error("attention_bf16: head dim must be 64 and sequences at most 4096 tokens");
    return AS_ERR_ARG;
  }
  const int q_tiles = (max_len + 63) / 64;
  const uint64_t blocks = (uint64_t)n_seq * n_heads * q_tiles;
  if (blocks > 0x7FFFFFFFull) {
    set_k_error("attention_bf16: too many sequences in one batch");
    return AS_ERR_ARG;
  }
  attn_bf16_kernel<false><<<(unsigned)blocks, 128, 0, st>>>(qkv, out, seq_start, seq_len, d_model, n_heads, q_tiles,
                                                            1.0f);
  count_launch();
  AS_CUDA_OK(cudaGetLastError());
  return AS_OK;
}

// -------------------------------------------------------------- LayerNorm

template <int CH>
__device__ __forceinline__ void ln_row(float4 (&v)[CH], int d, const float* __restrict__ g, const float* __restrict__ b,
                                       int lane) {
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += (v[c].x + v[c].y) + (v[c].z + v[c].w);
  const float mean = warp_sum(s) / (float)d;
  float q = 0.f;
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    v[c].x -= mean; v[c].y -= mean; v[c].z -= mean; v[c].w -= mean;
    q += (v[c].x * v[c].x + v[c].y * v[c].y) + (v[c].z * v[c].z + v[c].w * v[c].w);
  }
  const float rstd = rsqrtf(warp_sum(q) / (float)d + 1e-5f);
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int col = (c * 32 + lane) * 4;
    const float4 gg = __ldg(reinterpret_cast<const float4*>(g + col));
    const float4 bb = __ldg(reinterpret_cast<const float4*>(b + col));
    v[c].x = v[c].x * rstd * gg.x + bb.x;
    v[c].y = v[c].y * rstd * gg.y + bb.y;
    v[c].z = v[c].z * rstd * gg.z + bb.z;
    v[c].w = v[c].w * rstd * gg.w + bb.w;
  }
}

// Second output copy of a normalized row: BF16, or E4M3 of value * inv8.
struct Out2 {
  __nv_bfloat16* bf16;
  uint8_t* e4m3;
  float inv8;
};

template <int CH>
__device__ __forceinline__ void store_row(const float4 (&v)[CH], float* out_f32, Out2 o2, int64_t row, int d, int lane) {
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int col = (c * 32 + lane) * 4;
    if (out_f32) *reinterpret_cast<float4*>(out_f32 + row * d + col) = v[c];
    if (o2.bf16) {
      uint2 w;
      w.x = pack_bf16(v[c].x, v[c].y);
      w.y = pack_bf16(v[c].z, v[c].w);
      *reinterpret_cast<uint2*>(o2.bf16 + row * d + col) = w;
    }
    if (o2.e4m3) {
      const uint32_t w = (uint32_t)pack_e4m3(v[c].x * o2.inv8, v[c].y * o2.inv8) |
                         ((uint32_t)pack_e4m3(v[c].z * o2.inv8, v[c].w * o2.inv8) << 16);
      *reinterpret_cast<uint32_t*>(o2.e4m3 + row * d + col) = w;
    }
  }
}

template <int CH>
__global__ void __launch_bounds__(256) ln_kernel(const float* in, const float* __restrict__ g,
                                                 const float* __restrict__ b, float* out_f32, Out2 o2,
                                                 int64_t rows, int d) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (row >= rows) return;
  float4 v[CH];
  const float* x = in + row * d;
#pragma unroll
  for (int c = 0; c < CH; ++c) v[c] = *reinterpret_cast<const float4*>(x + (c * 32 + lane) * 4);
  ln_row<CH>(v, d, g, b, lane);
  store_row<CH>(v, out_f32, o2, row, d, lane);
}

template <int CH>
__global__ void __launch_bounds__(256) embed_ln_kernel(const int32_t* __restrict__ tok_ids,
                                                       const int32_t* __restrict__ row_tok,
                                                       const int32_t* __restrict__ row_pos,
                                                       const float* __restrict__ E, const float* __restrict__ P,
                                                       const float* __restrict__ g, const float* __restrict__ b,
                                                       float* out_f32, Out2 o2, int64_t rows, int d) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (row >= rows) return;
  const int id = tok_ids[row_tok[row]];
  const int pos = row_pos[row];
  float4 v[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int col = (c * 32 + lane) * 4;
    const float4 e = __ldg(reinterpret_cast<const float4*>(E + (size_t)id * d + col));
    const float4 p = __ldg(reinterpret_cast<const float4*>(P + (size_t)pos * d + col));
    v[c] = make_float4(e.x + p.x, e.y + p.y, e.z + p.z, e.w + p.w);
  }
  ln_row<CH>(v, d, g, b, lane);
  store_row<CH>(v, out_f32, o2, row, d, lane);
}

template <int CH>
__global__ void __launch_bounds__(256) ln_classify_kernel(const float* in, const float* __restrict__ g,
                                                          const float* __restrict__ b, const float* __restrict__ W,
                                                          const float* __restrict__ bc, int C,
                                                          const int32_t* __restrict__ row_tok,
                                                          const uint8_t* __restrict__ row_own, float* logits,
                                                          uint8_t* labels, int64_t rows, int d) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (row >= rows) return;
  if (row_own && !row_own[row]) return;
  float4 v[CH];
  const float* x = in + row * d;
#pragma unroll
  for (int c = 0; c < CH; ++c) v[c] = *reinterpret_cast<const float4*>(x + (c * 32 + lane) * 4);
  ln_row<CH>(v, d, g, b, lane);
  float my = 0.f;  // lane c keeps logit c
  for (int k = 0; k < C; ++k) {
    const float* w = W + (size_t)k * d;
    float a = 0.f;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const float4 ww = __ldg(reinterpret_cast<const float4*>(w + (c * 32 + lane) * 4));
      a += (v[c].x * ww.x + v[c].y * ww.y) + (v[c].z * ww.z + v[c].w * ww.w);
    }
    a = warp_sum(a) + bc[k];
    if (lane == k) my = a;
  }
  // argmax, lowest label on ties
  float best = lane < C ? my : -INFINITY;
  int bi = lane < C ? lane : 255;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  const int64_t tok = row_tok[row];
  if (lane < C && logits) logits[tok * C + lane] = my;
  if (lane == 0) labels[tok] = (uint8_t)bi;
}

#define AS_CH_DISPATCH(D, ...)                                   \
  switch ((D) / 128) {                                           \
    case 1: { constexpr int CH = 1; __VA_ARGS__; } break;        \
    case 2: { constexpr int CH = 2; __VA_ARGS__; } break;        \
    case 4: { constexpr int CH = 4; __VA_ARGS__; } break;        \
    case 6: { constexpr int CH = 6; __VA_ARGS__; } break;        \
    case 8: { constexpr int CH = 8; __VA_ARGS__; } break;        \
    default: set_k_error("unsupported d_model"); return AS_ERR_UNSUPPORTED; \
  }

as_status layernorm_rows(const float* in, const float* g, const float* b, float* out_f32, __nv_bfloat16* out_bf16,
                         int64_t rows, int32_t d, cudaStream_t st) {
  return layernorm_rows_ex(in, g, b, out_f32, out_bf16, nullptr, 1.0f, rows, d, st);
}

as_status layernorm_rows_ex(const float* in, const float* g, const float* b, float* out_f32, __nv_bfloat16* out_bf16,
                            uint8_t* out_e4m3, float e4m3_scale, int64_t rows, int32_t d, cudaStream_t st) {
  if (rows == 0) return AS_OK;
  if (d % 128) { set_k_error("layernorm: d must be a multiple of 128"); return AS_ERR_ARG; }
  const unsigned grid = (unsigned)((rows + 7) / 8);
  const Out2 o2{out_bf16, out_e4m3, 1.0f / e4m3_scale};
  AS_CH_DISPATCH(d, ln_kernel<CH><<<grid, 256, 0, st>>>(in, g, b, out_f32, o2, rows, d));
  count_launch();
  AS_CUDA_OK(cudaGetLastError());
  return AS_OK;
}

as_status embed_ln(const int32_t* tok_ids, const int32_t* row_tok, const int32_t* row_pos, const float* tok_emb,
                   const float* pos_emb, const float* g, const float* b, float* out_f32, __nv_bfloat16* out_bf16,
                   int64_t rows, int32_t d, cudaStream_t st) {
  return embed_ln_ex(tok_ids, row_tok, row_pos, tok_emb, pos_emb, g, b, out_f32, out_bf16, nullptr, 1.0f, rows, d, st);
}

as_status embed_ln_ex(const int32_t* tok_ids, const int32_t* row_tok, const int32_t* row_pos, const float* tok_emb,
                      const float* pos_emb, const float* g, const float* b, float* out_f32, __nv_bfloat16* out_bf16,
                      uint8_t* out_e4m3, float e4m3_scale, int64_t rows, int32_t d, cudaStream_t st) {
  if (rows == 0) return AS_OK;
  const unsigned grid = (unsigned)((rows + 7) / 8);
  const Out2 o2{out_bf16, out_e4m3, 1.0f / e4m3_scale};
  AS_CH_DISPATCH(d, embed_ln_kernel<CH><<<grid, 256, 0, st>>>(tok_ids, row_tok, row_pos, tok_emb, pos_emb, g, b,
                                                              out_f32, o2, rows, d));
  count_launch();
  AS_CUDA_OK(cudaGetLastError());
  return AS_OK;
}

as_status layernorm_classify(const float* in, const float* g, const float* b, const float* cls_w, const float* cls_b,
                             int32_t C, const int32_t* row_tok, const uint8_t* row_own, float* logits,
                             uint8_t* labels, int64_t rows, int32_t d, cudaStream_t st) {
  if (rows == 0) return AS_OK;
  if (C < 1 || C > 32) { set_k_error("classifier: 1..32 labels"); return AS_ERR_ARG; }
  const unsigned grid = (unsigned)((rows + 7) / 8);
  AS_CH_DISPATCH(d, ln_classify_kernel<CH><<<grid, 256, 0, st>>>(in, g, b, cls_w, cls_b, C, row_tok, row_own,
                                                                 logits, labels, rows, d));
  count_launch();
  AS_CUDA_OK(cudaGetLastError());
  return AS_OK;
}

// Largest |x| over a buffer, folded into *amax_bits with atomicMax on the
// IEEE bit pattern (non-negative floats order like unsigned integers).
template <typename T>
__global__ void amax_kernel(const T* __restrict__ x, uint64_t n, unsigned int* amax_bits) {
  float m = 0.f;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf((float)x[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(amax_bits, __float_as_uint(m));
}

void amax_f32(const float* x, uint64_t n, unsigned int* amax_bits, cudaStream_t st) {
  if (n == 0) return;
  amax_kernel<float><<<grid_1d(n, 256, 148 * 16), 256, 0, st>>>(x, n, amax_bits);
  count_launch();
}

void amax_bf16(const __nv_bfloat16* x, uint64_t n, unsigned int* amax_bits, cudaStream_t st) {
  if (n == 0) return;
  amax_kernel<__nv_bfloat16><<<grid_1d(n, 256, 148 * 16), 256, 0, st>>>(x, n, amax_bits);
  count_launch();
}

// y = E4M3(x / scale), round to nearest even with saturation.
__global__ void quantize_e4m3_kernel(const float* __restrict__ x, uint8_t* __restrict__ y, uint64_t n2, float inv) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n2; i += (uint64_t)gridDim.x * blockDim.x) {
    const float2 v = reinterpret_cast<const float2*>(x)[i];
    reinterpret_cast<uint16_t*>(y)[i] = pack_e4m3(v.x * inv, v.y * inv);
  }
}

void quantize_e4m3(const float* x, uint8_t* y, uint64_t n, float scale, cudaStream_t st) {
  if (n == 0) return;
  quantize_e4m3_kernel<<<grid_1d(n / 2, 256, 148 * 64), 256, 0, st>>>(x, y, n / 2, 1.0f / scale);
  count_launch();
}

__global__ void f32_to_bf16_kernel(const float* in, __nv_bfloat16* out, uint64_t n) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = __float2bfloat16_rn(in[i]);
}

void convert_f32_bf16(const float* in, __nv_bfloat16* out, uint64_t n, cudaStream_t st) {
  if (n == 0) return;
  f32_to_bf16_kernel<<<grid_1d(n, 256, 148 * 64), 256, 0, st>>>(in, out, n);
  count_launch();
}

}  // namespace as
