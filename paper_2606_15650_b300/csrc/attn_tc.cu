// Self-attention on the 5th-generation tensor cores (sm_103a), BF16 in,
// FP32 softmax statistics and accumulation (encoder of AnonShield §2 stage (2)).
//
// One CTA computes one (sequence, head, 128-query tile):
//   S_j = Q K_j^T           tcgen05.mma M=128 N=128 K=64, S in TMEM
//   P_j = exp2(S_j*c - m)   four softmax warps, one query row per thread,
//                           online max / sum in FP32, P rounded to BF16 and
//                           written to shared memory (128-byte swizzle)
//   O  += P_j V_j           tcgen05.mma M=128 N=64 K=128, O in TMEM, O
//                           rescaled in TMEM when the row maximum grows
// Both MMAs read K-major operands: Q and K rows come straight from the packed
// QKV buffer; V is read from a transposed copy (feature-major, tokens
// contiguous), written by vt_transpose_kernel. TMA loads need the token
// coordinate of V^T on a 16-byte boundary, so every sequence starts on a row
// that is a multiple of 8 (the batch packer inserts padding rows).
// Keys past the sequence end are masked to -inf; query rows past it are not
// stored. Every mbarrier wait is bounded (see gemm_tc.cu).
#include <atomic>
#include <cuda.h>
#include <cudaTypedefs.h>

#include "encoder.cuh"

namespace as {
namespace atc {

constexpr int kQ = 128;        // query rows per CTA
constexpr int kKT = 128;       // keys per tile
constexpr int kThreads = 192;  // loader, MMA, 4 softmax warps
constexpr uint64_t kTimeoutNs = 2000000000ull;

struct Params {
  const int32_t* seq_start;
  const int32_t* seq_len;
  __nv_bfloat16* out;
  int d, n_heads, q_tiles;
  DevError* err;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, DevError* err,
                                          uint32_t where) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  uint32_t n = 0;
  while (!mbar_try_wait(bar, parity)) {
    if ((++n & 255u) == 0) {
      if (*abort_flag) return false;
      if (globaltimer() - t0 > kTimeoutNs) {
        report_error(err, kErrTimeout, where, blockIdx.x, parity);
        *abort_flag = 1;
        return false;
      }
    }
  }
  return true;
}
// Warp-uniform wait: every lane gets the same answer, so the warp stays
// converged for the warp-collective tcgen05.ld / tcgen05.st that follow.
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, DevError* err,
                                          uint32_t where) {
  const bool ok = mbar_wait(bar, parity, abort_flag, err, where);
  return __all_sync(0xffffffffu, ok);
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* tm, uint32_t bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(bar), "r"(c0), "r"(c1)
      : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]),
      "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]),
      "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Shared memory (offsets from a 1024-aligned base)
constexpr int kQBytes = kQ * 64 * 2;                 // 16 KB, one swizzle panel
constexpr int kKBytes = kKT * 64 * 2;                // 16 KB per stage
constexpr int kVBytes = 64 * kKT * 2;                // 16 KB per stage: two 64x64 panels
constexpr int kPBytes = kQ * kKT * 2;                // 32 KB: two 128x64 panels
constexpr int kOffQ = 0;
constexpr int kOffK = kOffQ + kQBytes;               // 2 stages
constexpr int kOffV = kOffK + 2 * kKBytes;           // 2 stages
constexpr int kOffP = kOffV + 2 * kVBytes;
constexpr int kOffBar = kOffP + kPBytes;
// bars: q_full, kv_full[2], kv_empty[2], s_full, s_empty, p_full, o_done
constexpr int kNumBars = 9;
constexpr int kSmemBytes = kOffBar + kNumBars * 8 + 16;
constexpr int kSmemAlloc = kSmemBytes;             // two CTAs fit on one SM
constexpr uint32_t kTmemCols = 256;                  // S: cols 0..127, O: cols 128..191
constexpr uint32_t kColO = 128;

__global__ void __launch_bounds__(kThreads, 1)
    attn_tc_kernel(const __grid_constant__ CUtensorMap tmQK, const __grid_constant__ CUtensorMap tmVt, Params p) {
  const int qt = blockIdx.x % p.q_tiles;
  const int rest = blockIdx.x / p.q_tiles;
  const int h = rest % p.n_heads, s = rest / p.n_heads;
  const int L = p.seq_len[s], q0 = qt * kQ;
  if (q0 >= L) return;  // whole CTA leaves before any barrier or TMEM use
  const int row0 = p.seq_start[s];
  const int n_tiles = (L + kKT - 1) / kKT;

  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = smem_raw;
  // A V^T tile load starts at token row0 + 128 j: TMA needs that coordinate on a
  // 16-byte boundary (8 tokens), and the swizzled panels need a 1024-byte
  // aligned base. Record and skip instead of issuing a misaligned copy.
  if ((row0 & 7) || (smem_u32(smem) & 1023)) {
    if (threadIdx.x == 0) report_error(p.err, kErrBounds, 70, (uint32_t)row0, smem_u32(smem));
    return;
  }
  const uint32_t sb = smem_u32(smem);
  const uint32_t bar0 = sb + kOffBar;
  const uint32_t q_full = bar0, kv_full0 = bar0 + 8, kv_empty0 = bar0 + 24, s_full = bar0 + 40, s_empty = bar0 + 48,
                 p_full = bar0 + 56, o_done = bar0 + 64;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kOffBar + kNumBars * 8);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    mbar_init(q_full, 1);
    mbar_init(kv_full0, 1);
    mbar_init(kv_full0 + 8, 1);
    mbar_init(kv_empty0, 1);
    mbar_init(kv_empty0 + 8, 1);
    mbar_init(s_full, 1);
    mbar_init(s_empty, 128);
    mbar_init(p_full, 128);
    mbar_init(o_done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const int d = p.d;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- loader
      mbar_expect_tx(q_full, kQBytes);
      tma_load_2d(sb + kOffQ, &tmQK, q_full, h * 64, row0 + q0);
      for (int j = 0; j < n_tiles; ++j) {
        const int st = j & 1;
        if (!mbar_wait(kv_empty0 + 8 * st, ((j >> 1) & 1) ^ 1u, abort_flag, p.err, 40)) goto done;
        mbar_expect_tx(kv_full0 + 8 * st, kKBytes + kVBytes);
        const int k0 = row0 + j * kKT;
        tma_load_2d(sb + kOffK + st * kKBytes, &tmQK, kv_full0 + 8 * st, d + h * 64, k0);
        tma_load_2d(sb + kOffV + st * kVBytes, &tmVt, kv_full0 + 8 * st, k0, h * 64);
        tma_load_2d(sb + kOffV + st * kVBytes + kVBytes / 2, &tmVt, kv_full0 + 8 * st, k0 + 64, h * 64);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      constexpr uint32_t idS = idesc_bf16(kQ, kKT), idO = idesc_bf16(kQ, 64);
      if (!mbar_wait(q_full, 0, abort_flag, p.err, 50)) goto done;
      const uint64_t qdesc = sw128_desc(sb + kOffQ);
      for (int j = 0; j < n_tiles; ++j) {
        const int st = j & 1;
        if (!mbar_wait(kv_full0 + 8 * st, (j >> 1) & 1, abort_flag, p.err, 51)) goto done;
        if (j > 0 && !mbar_wait(s_empty, (j - 1) & 1, abort_flag, p.err, 52)) goto done;
        fence_after();
        const uint64_t kdesc = sw128_desc(sb + kOffK + st * kKBytes);
#pragma unroll
        for (int k = 0; k < 4; ++k) mma_bf16(tmem, qdesc + 2 * k, kdesc + 2 * k, idS, k > 0 ? 1u : 0u);
        mma_commit(s_full);
        if (!mbar_wait(p_full, j & 1, abort_flag, p.err, 53)) goto done;
        fence_after();
        const uint32_t vb = sb + kOffV + st * kVBytes;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const uint64_t pdesc = sw128_desc(sb + kOffP + (k >> 2) * (kPBytes / 2)) + 2 * (k & 3);
          const uint64_t vdesc = sw128_desc(vb + (k >> 2) * (kVBytes / 2)) + 2 * (k & 3);
          mma_bf16(tmem + kColO, pdesc, vdesc, idO, (j > 0 || k > 0) ? 1u : 0u);
        }
        mma_commit(o_done);
        mma_commit(kv_empty0 + 8 * st);
      }
    }
  } else {
    // ---------------- softmax: warp w owns TMEM lanes (query rows) 32*(w%4)..
    const int sub = warp & 3;
    const int r = sub * 32 + lane;               // query row in the tile
    const uint32_t trow = tmem + ((uint32_t)(sub * 32) << 16);
    const float c = 0.125f * 1.4426950408889634f;  // 1/sqrt(64) * log2(e)
    float m = -INFINITY, l = 0.f;
    bool ok = true;
    for (int j = 0; j < n_tiles && ok; ++j) {
      const int valid = min(kKT, L - j * kKT);   // keys of this tile inside the sequence
      if (!warp_wait(s_full, j & 1, abort_flag, p.err, 60)) { ok = false; break; }
      fence_after();
      // pass 1: row maximum of the scaled scores
      float mx = -INFINITY;
#pragma unroll 1
      for (int cc = 0; cc < kKT / 32; ++cc) {
        uint32_t v[32];
        tmem_ld32(trow + cc * 32, v);
#pragma unroll
        for (int i = 0; i < 32; ++i)
          if (cc * 32 + i < valid) mx = fmaxf(mx, __uint_as_float(v[i]) * c);
      }
      const float mn = fmaxf(m, mx);
      const float corr = ex2_approx(m - mn);     // 0 on the first tile (m = -inf)
      // pass 2: P = exp2(s*c - mn), row sum, BF16 into the swizzled P panels.
      // P is written only after the previous P.V has finished reading it.
      if (j > 0 && !warp_wait(o_done, (j - 1) & 1, abort_flag, p.err, 61)) { ok = false; break; }
      float sum = 0.f;
#pragma unroll 1
      for (int cc = 0; cc < kKT / 32; ++cc) {
        uint32_t v[32];
        tmem_ld32(trow + cc * 32, v);
        uint32_t pk[16];
#pragma unroll
        for (int i = 0; i < 32; i += 2) {
          const float p0 = (cc * 32 + i < valid) ? ex2_approx(__uint_as_float(v[i]) * c - mn) : 0.f;
          const float p1 = (cc * 32 + i + 1 < valid) ? ex2_approx(__uint_as_float(v[i + 1]) * c - mn) : 0.f;
          sum += p0 + p1;
          __nv_bfloat162 b = __floats2bfloat162_rn(p0, p1);
          pk[i >> 1] = *reinterpret_cast<uint32_t*>(&b);
        }
        // 32 keys = 64 bytes = four 16-byte pieces of row r in panel cc/2
        uint8_t* panel = smem + kOffP + (cc >> 1) * (kPBytes / 2);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int piece = (cc & 1) * 4 + q;
          *reinterpret_cast<uint4*>(panel + r * 128 + ((piece ^ (r & 7)) << 4)) =
              make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
        }
      }
      fence_before();
      mbar_arrive(s_empty);                      // S may be overwritten by S_{j+1}
      l = l * corr + sum;
      // tcgen05.ld / st are warp-collective: the whole warp rescales when any
      // of its rows needs it (rows whose maximum did not grow multiply by 1)
      if (j > 0 && __any_sync(0xffffffffu, corr < 1.f)) {
        // rescale the running output O (its last update, P_{j-1} V_{j-1}, is done)
#pragma unroll 1
        for (int cc = 0; cc < 2; ++cc) {
          uint32_t v[32];
          tmem_ld32(trow + kColO + cc * 32, v);
#pragma unroll
          for (int i = 0; i < 32; ++i) v[i] = __float_as_uint(__uint_as_float(v[i]) * corr);
          tmem_st32(trow + kColO + cc * 32, v);
        }
      }
      m = mn;
      fence_proxy_async();
      fence_before();
      mbar_arrive(p_full);
    }
    if (ok && warp_wait(o_done, (n_tiles - 1) & 1, abort_flag, p.err, 62)) {
      fence_after();
      const float inv = 1.f / l;
      const bool row_ok = q0 + r < L;
      __nv_bfloat16* o = p.out + (size_t)(row0 + q0 + r) * d + h * 64;
#pragma unroll 1
      for (int cc = 0; cc < 2; ++cc) {
        uint32_t v[32];
        tmem_ld32(trow + kColO + cc * 32, v);
        if (row_ok) {
#pragma unroll
          for (int i = 0; i < 32; i += 8) {
            uint4 w;
            __nv_bfloat162 a0 = __floats2bfloat162_rn(__uint_as_float(v[i]) * inv, __uint_as_float(v[i + 1]) * inv);
            __nv_bfloat162 a1 = __floats2bfloat162_rn(__uint_as_float(v[i + 2]) * inv, __uint_as_float(v[i + 3]) * inv);
            __nv_bfloat162 a2 = __floats2bfloat162_rn(__uint_as_float(v[i + 4]) * inv, __uint_as_float(v[i + 5]) * inv);
            __nv_bfloat162 a3 = __floats2bfloat162_rn(__uint_as_float(v[i + 6]) * inv, __uint_as_float(v[i + 7]) * inv);
            w.x = *reinterpret_cast<uint32_t*>(&a0);
            w.y = *reinterpret_cast<uint32_t*>(&a1);
            w.z = *reinterpret_cast<uint32_t*>(&a2);
            w.w = *reinterpret_cast<uint32_t*>(&a3);
            *reinterpret_cast<uint4*>(o + cc * 32 + i) = w;
          }
        }
      }
    }
  }
done:
  fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// Vt[c][r] = V[r][c] = qkv[r][2d + c] for c < d, r < rows (32x32 smem tiles).
__global__ void vt_transpose_kernel(const __nv_bfloat16* __restrict__ qkv, __nv_bfloat16* __restrict__ vt, int rows,
                                    int d, int ldt) {
  __shared__ __nv_bfloat16 t[32][33];
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  for (int i = ty; i < 32; i += 8) {
    const int r = r0 + i;
    t[i][tx] = r < rows ? qkv[(size_t)r * 3 * d + 2 * d + c0 + tx] : __float2bfloat16(0.f);
  }
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    const int r = r0 + tx;
    if (r < ldt) vt[(size_t)(c0 + i) * ldt + r] = t[tx][i];
  }
}

}  // namespace atc

namespace {
// Set once per process / device; concurrent callers write the same values.
std::atomic<PFN_cuTensorMapEncodeTiled_v12000> g_enc{nullptr};
std::atomic<bool> g_attn_attr_set[64] = {};

as_status make_map_bf16(CUtensorMap* tm, const void* ptr, uint64_t rows, uint64_t cols, uint64_t ld_elems,
                        uint32_t box_cols, uint32_t box_rows) {
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld_elems * 2)};
  cuuint32_t box[2] = {box_cols, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_enc.load()(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_k_error("attention_tcgen05: cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
    return AS_ERR_CUDA;
  }
  return AS_OK;
}
}  // namespace

uint64_t attention_vt_elems(int64_t rows, int32_t d_model) { return (uint64_t)d_model * (uint64_t)((rows + 7) & ~7ll); }

as_status attention_tcgen05(const __nv_bfloat16* qkv, __nv_bfloat16* vt, __nv_bfloat16* out, const int32_t* seq_start,
                            const int32_t* seq_len, int32_t n_seq, int32_t max_len, int64_t rows, int32_t d_model,
                            int32_t n_heads, DevError* err, cudaStream_t st) {
  if (n_seq == 0 || max_len == 0 || rows == 0) return AS_OK;
  if (d_model != n_heads * 64 || d_model % 64 || max_len > 4096 || rows > (1ll << 31) - 8 ||
      (reinterpret_cast<uintptr_t>(qkv) & 15) || (reinterpret_cast<uintptr_t>(vt) & 15)) {
    set_k_error("attention_tcgen05: head dim 64, sequences <= 4096 tokens, 16-byte aligned buffers");
    return AS_ERR_ARG;
  }
  if (!g_enc.load()) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    AS_CUDA_OK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !fn) {
      set_k_error("cuTensorMapEncodeTiled not available from the driver");
      return AS_ERR_CUDA;
    }
    g_enc.store(reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn));
  }
  int dev = 0;
  cudaGetDevice(&dev);
  if (!g_attn_attr_set[dev & 63].load()) {
    AS_CUDA_OK(cudaFuncSetAttribute(atc::attn_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, atc::kSmemAlloc));
    g_attn_attr_set[dev & 63].store(true);
  }
  const int ldt = (int)((rows + 7) & ~7ll);
  dim3 tg((unsigned)((ldt + 31) / 32), (unsigned)(d_model / 32));
  atc::vt_transpose_kernel<<<tg, 256, 0, st>>>(qkv, vt, (int)rows, d_model, ldt);
  count_launch();
  CUtensorMap tmQK, tmVt;
  as_status s = make_map_bf16(&tmQK, qkv, (uint64_t)rows, 3ull * d_model, 3ull * d_model, 64, atc::kQ);
  if (s == AS_OK) s = make_map_bf16(&tmVt, vt, (uint64_t)d_model, (uint64_t)ldt, (uint64_t)ldt, 64, 64);
  if (s != AS_OK) return s;
  atc::Params p;
  p.seq_start = seq_start;
  p.seq_len = seq_len;
  p.out = out;
  p.d = d_model;
  p.n_heads = n_heads;
  p.q_tiles = (max_len + atc::kQ - 1) / atc::kQ;
  p.err = err;
  const uint64_t blocks = (uint64_t)n_seq * n_heads * p.q_tiles;
  if (blocks > 0x7FFFFFFFull) {
    set_k_error("attention_tcgen05: too many sequences in one batch");
    return AS_ERR_ARG;
  }
  atc::attn_tc_kernel<<<(unsigned)blocks, atc::kThreads, atc::kSmemAlloc, st>>>(tmQK, tmVt, p);
  count_launch();
  AS_CUDA_OK(cudaGetLastError());
  return AS_OK;
}

}  // namespace as
