// BF16 GEMM on the 5th-generation tensor cores (sm_103a): C = epi(A . B^T).
//
// Encoder projections (QKV, output, FFN in/out) of the token classifier
// (AnonShield §2 stage (2)). A = activations [M][K] BF16 row-major, B =
// nn.Linear weight [N][K] BF16 row-major: both K-major, which is what the
// tensor core reads directly.
//
// Structure (one CTA per SM, persistent over 128 x BN output tiles):
//   warp 0, one lane : TMA producer, A and B tiles (64 K-elements, 128-byte
//                      swizzle) into a STAGES-deep shared-memory ring
//   warp 1           : issues tcgen05.mma (M=128, N=BN, K=16) into a TMEM
//                      accumulator; tcgen05.commit frees ring slots and
//                      signals a finished accumulator (the whole warp runs
//                      the loop and waits, one elected lane issues: issuing
//                      from a single divergent lane took longer than the
//                      64-cycle MMAs of BN = 128 tiles)
//   warps 2..9       : epilogue; two warps per TMEM lane quarter (32 rows),
//                      each taking half of the tile's columns: tcgen05.ld,
//                      bias / GELU / residual in FP32, then 32x32 chunks
//                      through swizzled shared memory and TMA tensor stores
//                      (the FP32 residual comes in by TMA the same way)
// Two TMEM accumulators (2 x BN columns) let the epilogue of tile i overlap
// the main loop of tile i+1. Every mbarrier wait is bounded (globaltimer):
// on timeout the kernel records the failure, every role leaves its loop,
// TMEM is freed and the kernel returns.
//
// Residual + LayerNorm epilogue (kEpiResidLN: X = LN(X + alpha A.B^T + bias),
// the post-LN block of the encoder): a row of N = C x BN columns is split over
// a cluster of C CTAs (C <= 4), which walk the same 128-row blocks. Each
// epilogue warp (32 rows x BN/2 columns) writes y = alpha acc + bias + X back
// into TMEM, takes the mean and the centred sum of squares of its part of each
// row, and stores them into every CTA of the cluster (distributed shared
// memory) with a release-arrive on that CTA's exchange barrier. Once all 2C
// partials of its rows are in, a warp combines them (Chan et al.'s pairwise
// update), normalizes y from TMEM and writes X in place (FP32) and its BF16
// or E4M3 copy.
#include <atomic>
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "encoder.cuh"

namespace as {
namespace tc {

constexpr int kBM = 128;
// Operand / output element types of one instantiation
constexpr int kInBF16 = 0, kInE4M3 = 1;
constexpr int kOutBF16 = 0, kOutF32 = 1, kOutE4M3 = 2;
// Epilogue code of the fused residual + LayerNorm (next to the public AS_EPI_*)
constexpr int kEpiResidLN = 3;
constexpr int kMaxLnCluster = 4;
// elements per k-block: a 128-byte swizzled row holds 64 BF16 or 128 E4M3
__host__ __device__ constexpr int bk_elems(int in) { return in == kInE4M3 ? 128 : 64; }
constexpr int kEpiWarps = 8;
constexpr int kThreads = 64 + 32 * kEpiWarps;   // producer + MMA + epilogue warps
constexpr uint64_t kTimeoutNs = 2000000000ull;

struct Params {
  int M, N, K;
  int n_tiles_n, n_tiles;
  int raster;           // tile order: 0 = along N within a row block, 1 = along M within a column block
  int epi;
  const float* bias;
  const float* resid;
  void* out;
  DevError* err;
  float alpha;          // accumulator scale (product of the FP8 operand scales; 1 for BF16)
  float out_scale_inv;  // 1 / scale of an FP8 output
  // kEpiResidLN: LN gain / bias; out (= resid) gets the FP32 rows, out16 / out8 the copy
  const float* ln_g;
  const float* ln_b;
  __nv_bfloat16* out16;
  uint8_t* out8;
  int copy;             // kEpiResidLN: 0 none, 1 BF16 (out16), 2 E4M3 (out8); tensor map tmC
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Output tile t -> (first row, first column).
__device__ __forceinline__ void tile_origin(const Params& p, int t, int bn, int& m0, int& n0) {
  if (p.raster == 0) {
    m0 = (t / p.n_tiles_n) * 128;
    n0 = (t % p.n_tiles_n) * bn;
  } else {
    const int n_tiles_m = p.n_tiles / p.n_tiles_n;
    m0 = (t % n_tiles_m) * 128;
    n0 = (t / n_tiles_m) * bn;
  }
}

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

// Bounded wait. Returns false when the kernel is aborting (timeout here or
// elsewhere in the CTA).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, DevError* err,
                                          uint32_t where) {
  if (mbar_try_wait(bar, parity)) return true;
  uint64_t t0 = globaltimer();
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

// Warp-uniform wait for warps that go on to the warp-collective tcgen05.ld.
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, DevError* err,
                                          uint32_t where) {
  const bool ok = mbar_wait(bar, parity, abort_flag, err, where);
  return __all_sync(0xffffffffu, ok);
}

// One lane of a converged warp (the same lane on every call).
__device__ __forceinline__ bool elect_one() {
  uint32_t pred = 0;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "elect.sync _|p, 0xffffffff;\n\t"
      "selp.b32 %0, 1, 0, p;\n\t}"
      : "=r"(pred));
  return pred != 0;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* tm, uint32_t bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(bar), "r"(c0), "r"(c1)
      : "memory");
}

// TMA load into this CTA's shared memory whose transaction completes on an
// mbarrier of either CTA of the pair (a shared::cluster address).
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap* tm, uint32_t cluster_bar, int c0,
                                                 int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(cluster_bar), "r"(c0), "r"(c1)
      : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor, K-major operand with 128-byte swizzle:
// 8-row groups 1024 bytes apart (SBO), descriptor version 1 (tcgen05).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;              // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
  d |= (uint64_t)1 << 46;              // version
  d |= (uint64_t)2 << 61;              // SWIZZLE_128B
  return d;
}

// Instruction descriptor: D FP32, A/B BF16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// kind::f8f6f4 with A and B in E4M3 (format code 0), D in FP32.
__host__ __device__ constexpr uint32_t idesc_e4m3(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_e4m3(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// 2-SM forms (a CTA pair, the even rank issuing): M = 256 over the two CTAs'
// TMEM, A rows and B columns split between their shared memories; commits
// arrive on the mbarrier at this offset in both CTAs.
__device__ __forceinline__ void mma_bf16_pair(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_e4m3_pair(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
// mask: the pair's two cluster ranks (0x3 << rank of the even CTA)
__device__ __forceinline__ void mma_commit_pair(uint32_t bar, uint16_t mask) {
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::
                   "r"(bar), "h"(mask)
               : "memory");
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

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// GELU 0.5 x (1 + erf(x / sqrt 2)) for the BF16 epilogue. erf uses the
// rational approximation of Abramowitz & Stegun, Handbook of Mathematical
// Functions, eq. 7.1.26 (|error| <= 1.5e-7): erf(z) = 1 - t (a1 + t (a2 + t (a3
// + t (a4 + t a5)))) exp(-z^2), t = 1 / (1 + p z), z >= 0, odd extension. The
// result is rounded to BF16 (relative 2^-9) right after, so the approximation
// error does not show; it costs about a third of a full-precision erf.
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float gelu_erf(float x) {
  const float z = fabsf(x) * 0.70710678118654752f;
  const float t = rcp_approx(fmaf(0.3275911f, z, 1.0f));
  float poly = fmaf(t, 1.061405429f, -1.453152027f);
  poly = fmaf(t, poly, 1.421413741f);
  poly = fmaf(t, poly, -0.284496736f);
  poly = fmaf(t, poly, 0.254829592f);
  const float e = ex2_approx(-z * z * 1.4426950408889634f);
  const float erf_abs = fmaf(-poly * t, e, 1.0f);
  const float erf_x = copysignf(erf_abs, x);
  return 0.5f * x * (1.0f + erf_x);
}

// gelu_erf2 (below) computes gelu_erf of two values with the two-lane FP32
// instructions of common.cuh: each lane rounds exactly as the scalar
// instruction would, so the result is bit for bit that of gelu_erf with about
// half the issue slots (the epilogue of the GELU projection is issue-bound).
// gelu_erf of two values, the same operations in the same order.
__device__ __forceinline__ void gelu_erf2(float& x0, float& x1) {
  const uint64_t x = f2pack(x0, x1);
  const uint64_t z = mul2(f2pack(fabsf(x0), fabsf(x1)), f2splat(0.70710678118654752f));
  float d0, d1;
  f2unpack(fma2(f2splat(0.3275911f), z, f2splat(1.0f)), d0, d1);
  const uint64_t t = f2pack(rcp_approx(d0), rcp_approx(d1));
  uint64_t poly = fma2(t, f2splat(1.061405429f), f2splat(-1.453152027f));
  poly = fma2(t, poly, f2splat(1.421413741f));
  poly = fma2(t, poly, f2splat(-0.284496736f));
  poly = fma2(t, poly, f2splat(0.254829592f));
  float z0, z1, a0, a1, p0, p1, r0, r1, y0, y1;
  f2unpack(z, z0, z1);
  f2unpack(mul2(mul2(f2pack(-z0, -z1), z), f2splat(1.4426950408889634f)), a0, a1);
  const uint64_t e = f2pack(ex2_approx(a0), ex2_approx(a1));
  f2unpack(poly, p0, p1);
  f2unpack(fma2(mul2(f2pack(-p0, -p1), t), e, f2splat(1.0f)), r0, r1);
  const uint64_t erf = f2pack(copysignf(r0, x0), copysignf(r1, x1));
  f2unpack(mul2(mul2(f2splat(0.5f), x), add2(f2splat(1.0f), erf)), y0, y1);
  x0 = y0;
  x1 = y1;
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// ---- thread-block cluster helpers (the LayerNorm epilogue)
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_size() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_index() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_count() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return r;
}
// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t mapa(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_cluster_v2(uint32_t addr, float a, float b) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(a), "f"(b) : "memory");
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t remote_bar) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(remote_bar) : "memory");
}
// A release made of one cluster-scope fence and relaxed arrivals: after
// several remote stores, one fence orders them all before each of the
// following arrivals (instead of one release, and its wait, per arrival).
__device__ __forceinline__ void fence_acq_rel_cluster() { asm volatile("fence.acq_rel.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_cluster_relaxed(uint32_t remote_bar) {
  asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(remote_bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_cluster(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded, warp-uniform wait with cluster-scope acquire (the partials of the peers).
__device__ __forceinline__ bool warp_wait_cluster(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                                  DevError* err, uint32_t where) {
  bool ok = mbar_try_wait_cluster(bar, parity);
  if (!ok) {
    const uint64_t t0 = globaltimer();
    uint32_t n = 0;
    while (!(ok = mbar_try_wait_cluster(bar, parity))) {
      if ((++n & 255u) == 0) {
        if (*abort_flag) break;
        if (globaltimer() - t0 > kTimeoutNs) {
          report_error(err, kErrTimeout, where, blockIdx.x, parity);
          *abort_flag = 1;
          break;
        }
      }
    }
  }
  return __all_sync(0xffffffffu, ok);
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

// TMA tensor store of one box from shared memory (bulk-group completion).
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* tm, uint32_t src, int c0, int c1) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(tm)),
               "r"(src), "r"(c0), "r"(c1)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Epilogue staging: each epilogue warp owns two chunk buffers of 32 rows.
// BF16 chunks are 32 columns with 64-byte rows stored with the 64-byte TMA
// swizzle (16-byte piece j of row r at j ^ ((r >> 1) & 3)); FP32 chunks are
// 16 columns, also 64-byte rows with the 64-byte swizzle (2 KB per buffer, so
// the residual GEMMs keep room for four pipeline stages); E4M3 chunks are 32
// columns, 32-byte rows with the 32-byte swizzle (piece j at j ^ ((r >> 2) &
// 1)). The warp writes (and, for the residual, reads) one row per lane without
// bank conflicts, and the TMA engine moves whole lines to and from global memory.
template <int OUT>
struct EpiTraits {
  static constexpr bool kF32 = OUT == kOutF32;
  static constexpr int kEsize = OUT == kOutF32 ? 4 : (OUT == kOutBF16 ? 2 : 1);
  static constexpr int kCols = OUT == kOutF32 ? 16 : 32;   // columns per chunk
  static constexpr int kChunkBytes = 32 * kCols * kEsize;
};

// Residual / output staging buffers per epilogue warp: 4 for the LayerNorm
// epilogue on a short main-loop ring (2 stages, or 3 half-B stages of a 2-SM
// pair), which the attention-output block can afford (K = d) and which keeps
// more of its residual and output bytes in flight; else 2.
__host__ __device__ constexpr int stg_bufs(bool ln, int stages, bool bhalf) {
  return ln && (stages == 2 || (bhalf && stages == 3)) ? 4 : 2;
}

template <int BN, int STAGES, int OUT, bool LN = false, bool BHALF = false>
struct Smem {
  static constexpr int kRB = stg_bufs(LN, STAGES, BHALF);
  static constexpr int kABytes = kBM * 128;       // 16 KB: 128 rows x 128 bytes
  static constexpr int kBBytes = BN * (BHALF ? 64 : 128);  // B rows of this CTA (half of them in a 2-SM pair)
  static constexpr int kStageBytes = kABytes + kBBytes;
  static constexpr int kStgOff = STAGES * kStageBytes;                       // 1024-aligned
  static constexpr int kStgBytes = kEpiWarps * kRB * EpiTraits<OUT>::kChunkBytes;
  // LayerNorm copy staging (BF16 or E4M3 chunks of 16 columns x 32 rows, two per warp)
  static constexpr int kStg2Off = kStgOff + kStgBytes;
  static constexpr int kStg2Bytes = LN ? kEpiWarps * kRB * 1024 : 0;
  // LayerNorm partials: [2 tile parities][2 * kMaxLnCluster parts][128 rows] x (mean, m2)
  static constexpr int kXOff = kStg2Off + kStg2Bytes;
  static constexpr int kXBytes = LN ? 2 * 2 * kMaxLnCluster * kBM * 8 : 0;
  // LayerNorm: bias, gain and LayerNorm bias of this CTA's BN columns (fixed
  // per CTA) in shared memory when they fit, else read from global memory
  static constexpr int kVecOff = kXOff + kXBytes;
  static constexpr int kNumBarsPre = 2 * STAGES + 4 + kRB * kEpiWarps + 2;
  static constexpr bool kVecSmem = LN && kVecOff + 3 * BN * 4 + kNumBarsPre * 8 + 16 + 1024 <= 232448;
  static constexpr int kVecBytes = kVecSmem ? 3 * BN * 4 : 0;
  static constexpr int kBarOff = kVecOff + kVecBytes;
  // full[S], empty[S], tfull[2], tempty[2], resid[kEpiWarps][kRB], xbar[2]; tmem slot + abort flag
  static constexpr int kNumBars = 2 * STAGES + 4 + kRB * kEpiWarps + 2;
  static constexpr int kBytes = kBarOff + kNumBars * 8 + 16;
  static constexpr int kAlloc = kBytes + 1024;    // room to align the base to 1024
};

template <int BN, int STAGES, int EPI, int IN, int OUT, int PAIR = 1>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                const __grid_constant__ CUtensorMap tmC, const __grid_constant__ CUtensorMap tmR, Params p) {
  constexpr bool LN = EPI == kEpiResidLN;
  // PAIR = 2: 2-SM MMA. A cluster of two CTAs computes a 256 x BN tile: each
  // loads its 128 A rows and half of the B rows; the even CTA issues
  // tcgen05.mma.cta_group::2 (M = 256) reading both CTAs' shared memory and
  // writing each CTA's 128 rows into its own TMEM; both CTAs' loads complete
  // on the even CTA's full barrier; its commits free the stage and hand over
  // the accumulator in both CTAs; both epilogues release the accumulator on
  // the even CTA's barrier.
  // With both (LayerNorm + pairs): cluster rank = 2 x column block + row half;
  // ranks 2j, 2j+1 form a 2-SM pair, the LayerNorm exchange runs among the
  // ranks of the same row half.
  constexpr bool MC = PAIR == 2;
  using L = Smem<BN, STAGES, OUT, LN, MC>;
  using E = EpiTraits<OUT>;
  static_assert((EPI == AS_EPI_BIAS_RESID || LN) == (OUT == kOutF32), "the residual epilogues write FP32");
  constexpr uint32_t kTmemCols = 2 * BN;   // power of two: 256 or 512
  constexpr int kMmaM = MC ? 2 * kBM : kBM;
  constexpr uint32_t kIdesc = IN == kInE4M3 ? idesc_e4m3(kMmaM, BN) : idesc_bf16(kMmaM, BN);
  constexpr int kBKe = bk_elems(IN);
  constexpr int CW = E::kCols;             // columns per chunk
  constexpr int CH = BN / 2 / CW;          // chunks per epilogue warp and tile (a warp owns half the columns)
  static_assert(CH % 2 == 0, "chunks alternate between two staging buffers");
  static_assert(CH % L::kRB == 0, "chunks cycle through the staging buffers");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sbase = smem_u32(smem);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::kBarOff);
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (STAGES + s); };
  auto tfull_bar = [&](int a) { return bar0 + 8u * (2 * STAGES + a); };
  auto tempty_bar = [&](int a) { return bar0 + 8u * (2 * STAGES + 2 + a); };
  constexpr int RB = L::kRB;   // staging buffers per epilogue warp
  auto resid_bar = [&](int w, int b) { return bar0 + 8u * (2 * STAGES + 4 + RB * w + b); };
  auto xbar = [&](int b) { return bar0 + 8u * (2 * STAGES + 4 + RB * kEpiWarps + b); };
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L::kBarOff + L::kNumBars * 8);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int KB = p.K / kBKe;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(tfull_bar(a), 1);
      mbar_init(tempty_bar(a), (MC ? 2 : 1) * kEpiWarps * 32);   // a pair: both CTAs' epilogues
    }
    for (int w = 0; w < kEpiWarps; ++w)
      for (int b = 0; b < RB; ++b) mbar_init(resid_bar(w, b), 1);
    if (LN) {
      // every epilogue thread of every CTA of the exchange group arrives once per tile
      const uint32_t group = MC ? cluster_size() / 2 : cluster_size();
      mbar_init(xbar(0), group * kEpiWarps * 32);
      mbar_init(xbar(1), group * kEpiWarps * 32);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmC)) : "memory");
    if (E::kF32) asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmR)) : "memory");
  }
  if (warp == 1) {
    if constexpr (MC) {
      // collective over the pair: the same columns in both CTAs' TMEM
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                   "r"(kTmemCols)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                   "r"(kTmemCols)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if constexpr (LN || MC) cluster_sync_all();  // the peers' barriers are initialised before anyone arrives on them
  const uint32_t tmem_base = *tmem_slot;
  // Tile walk: all output tiles, or (LayerNorm) the 128-row blocks, one per
  // cluster at a time, each CTA taking the column block of its cluster rank.
  int t_first = blockIdx.x, t_step = gridDim.x, t_count = p.n_tiles;
  // crank: the row half in a 2-SM pair (0 = the CTA that issues the MMAs);
  // lrank / csize: position and size of the LayerNorm exchange group;
  // lead: cluster rank of the pair's issuing CTA
  uint32_t crank = 0, csize = 1, lrank = 0, lead = 0;
  const int n_mblocks = p.n_tiles / p.n_tiles_n;
  const int n_mpairs = (n_mblocks + 1) / 2;
  if constexpr (LN || MC) {
    const uint32_t cr = cluster_rank();
    crank = MC ? (cr & 1u) : 0u;
    lead = cr & ~1u;
    lrank = MC ? (cr >> 1) : cr;
    csize = MC ? cluster_size() / 2 : cluster_size();
    t_first = (int)cluster_index();
    t_step = (int)cluster_count();
    t_count = LN ? (MC ? n_mpairs : n_mblocks) : n_mpairs * p.n_tiles_n;
  }
  auto origin = [&](int t, int& m0, int& n0) {
    if constexpr (LN) {
      m0 = (MC ? 2 * t + (int)crank : t) * kBM;
      n0 = (int)lrank * BN;
    } else if constexpr (MC) {
      // pair tiles: 256 rows x BN columns, the CTA of row half h takes rows 128 h ..
      const int mp = p.raster == 0 ? t / p.n_tiles_n : t % n_mpairs;
      const int nt = p.raster == 0 ? t % p.n_tiles_n : t / n_mpairs;
      m0 = (2 * mp + (int)crank) * kBM;
      n0 = nt * BN;
    } else {
      tile_origin(p, t, BN, m0, n0);
    }
  };
  if constexpr (L::kVecSmem) {
    // the column block is fixed per CTA: its bias / gain / LayerNorm bias go to shared memory once
    float* vec = reinterpret_cast<float*>(smem + L::kVecOff);
    const int nb = (int)lrank * BN;
    for (int j = threadIdx.x; j < BN; j += blockDim.x) {
      vec[j] = p.bias ? p.bias[nb + j] : 0.f;
      vec[BN + j] = p.ln_g[nb + j];
      vec[2 * BN + j] = p.ln_b[nb + j];
    }
    __syncthreads();
  }

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer
      uint32_t it = 0;
      for (int tile = t_first; tile < t_count; tile += t_step) {
        int m0, n0;
        origin(tile, m0, n0);
        for (int kb = 0; kb < KB; ++kb, ++it) {
          const int s = it % STAGES;
          const uint32_t ph = (it / STAGES) & 1u;
          if (!mbar_wait(empty_bar(s), ph ^ 1u, abort_flag, p.err, 10)) goto done;
          const uint32_t a_dst = sbase + s * L::kStageBytes;
          if constexpr (MC) {
            // both CTAs' halves complete on the even CTA's full barrier
            const uint32_t fb = mapa(full_bar(s), lead);
            if (crank == 0) mbar_expect_tx(full_bar(s), 2 * L::kStageBytes);
            tma_load_2d_pair(a_dst, &tmA, fb, kb * kBKe, m0);
            tma_load_2d_pair(a_dst + L::kABytes, &tmB, fb, kb * kBKe, n0 + (int)crank * (BN / 2));
          } else {
            mbar_expect_tx(full_bar(s), L::kStageBytes);
            tma_load_2d(a_dst, &tmA, full_bar(s), kb * kBKe, m0);
            tma_load_2d(a_dst + L::kABytes, &tmB, full_bar(s), kb * kBKe, n0);
          }
        }
      }
    }
  } else if (warp == 1) {
    if (!MC || crank == 0) {
      // ---------------- MMA issuer (the even CTA of a 2-SM pair): the whole warp
      // runs the loop (warp-uniform waits), one elected lane issues each group
      uint32_t it = 0, lt = 0;
      for (int tile = t_first; tile < t_count; tile += t_step, ++lt) {
        const uint32_t acc = lt & 1u, aph = (lt >> 1) & 1u;
        if (!warp_wait(tempty_bar(acc), aph ^ 1u, abort_flag, p.err, 20)) goto done;
        fence_after();
        const uint32_t d_tmem = tmem_base + acc * BN;
        for (int kb = 0; kb < KB; ++kb, ++it) {
          const int s = it % STAGES;
          const uint32_t ph = (it / STAGES) & 1u;
          if (!warp_wait(full_bar(s), ph, abort_flag, p.err, 21)) goto done;
          fence_after();
          const uint32_t a_addr = sbase + s * L::kStageBytes;
          const uint64_t adesc = sw128_desc(a_addr), bdesc = sw128_desc(a_addr + L::kABytes);
          if (elect_one()) {
            // four MMAs per 128-byte k-block (K = 16 BF16 or 32 E4M3 each): 32 bytes apart
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const uint32_t en = (kb > 0 || k > 0) ? 1u : 0u;
              if constexpr (MC) {
                if (IN == kInE4M3) mma_e4m3_pair(d_tmem, adesc + 2 * k, bdesc + 2 * k, kIdesc, en);
                else mma_bf16_pair(d_tmem, adesc + 2 * k, bdesc + 2 * k, kIdesc, en);
              } else {
                if (IN == kInE4M3) mma_e4m3(d_tmem, adesc + 2 * k, bdesc + 2 * k, kIdesc, en);
                else mma_bf16(d_tmem, adesc + 2 * k, bdesc + 2 * k, kIdesc, en);
              }
            }
            if constexpr (MC) mma_commit_pair(empty_bar(s), (uint16_t)(0x3u << lead));
            else mma_commit(empty_bar(s));
          }
          __syncwarp();
        }
        if (elect_one()) {
          if constexpr (MC) mma_commit_pair(tfull_bar(acc), (uint16_t)(0x3u << lead));
          else mma_commit(tfull_bar(acc));
        }
        __syncwarp();
      }
    }
  } else {
    // ---------------- epilogue: warp w owns TMEM lanes 32*(w%4) .. +31 (a
    // warp can reach only its own lane quarter) and column half (w-2)/4
    const int ew = warp - 2;
    const int sub = warp & 3;
    const int half = ew >> 2;
    const uint32_t stg = sbase + L::kStgOff + ew * RB * E::kChunkBytes;
    uint8_t* stg_ptr = smem + L::kStgOff + ew * RB * E::kChunkBytes;
    const int r = lane;
    uint32_t lt = 0;
    for (int tile = t_first; tile < t_count; tile += t_step, ++lt) {
      const uint32_t acc = lt & 1u, aph = (lt >> 1) & 1u;
      int m0, n0;
      origin(tile, m0, n0);
      const int row0 = m0 + sub * 32;
      if (E::kF32) {
        // residual chunks of this tile: fetched before the accumulator is ready
        if (lane == 0) {
          bulk_wait_read<0>();  // earlier stores have left the staging buffers
#pragma unroll
          for (int i = 0; i < RB; ++i) {
            mbar_expect_tx(resid_bar(ew, i), E::kChunkBytes);
            tma_load_2d(stg + i * E::kChunkBytes, &tmR, resid_bar(ew, i), n0 + (half * CH + i) * CW, row0);
          }
        }
        __syncwarp();
      }
      if (!warp_wait(tfull_bar(acc), aph, abort_flag, p.err, 30)) break;
      fence_after();
      if constexpr (LN) {
        const uint32_t t_row = tmem_base + ((uint32_t)(sub * 32) << 16) + acc * BN;
        const uint64_t alpha2 = f2splat(p.alpha);
        // pass 1: y = alpha acc + bias + x, written back to TMEM; sums of y - y0 and
        // (y - y0)^2 over this warp's columns, y0 = the first y of the row (a shift
        // that keeps the one-pass variance free of cancellation)
        float s1 = 0.f, s2 = 0.f, y0 = 0.f;
        bool ok = true;
#pragma unroll 1
        for (int i = 0; i < CH; ++i) {
          const int c = half * CH + i;
          const int buf = i % RB;
          const int n = n0 + c * CW;
          uint32_t rr[16];
          tmem_ld16(t_row + c * CW, rr);
          const uint32_t par = (lt * (CH / RB) + i / RB) & 1u;
          if (!warp_wait(resid_bar(ew, buf), par, abort_flag, p.err, 32)) {
            ok = false;
            break;
          }
          const uint8_t* cb = stg_ptr + buf * E::kChunkBytes;
          const float4* vb = L::kVecSmem ? reinterpret_cast<const float4*>(smem + L::kVecOff) + (c * CW) / 4 : nullptr;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float4 b = L::kVecSmem ? vb[j]
                             : (p.bias ? __ldg(reinterpret_cast<const float4*>(p.bias + n + 4 * j))
                                       : make_float4(0.f, 0.f, 0.f, 0.f));
            const float4 x = *reinterpret_cast<const float4*>(cb + r * 64 + ((j ^ ((r >> 1) & 3)) << 4));
            float y[4];
            f2unpack(add2(fma2(f2pack(__uint_as_float(rr[4 * j]), __uint_as_float(rr[4 * j + 1])), alpha2,
                               f2pack(b.x, b.y)), f2pack(x.x, x.y)), y[0], y[1]);
            f2unpack(add2(fma2(f2pack(__uint_as_float(rr[4 * j + 2]), __uint_as_float(rr[4 * j + 3])), alpha2,
                               f2pack(b.z, b.w)), f2pack(x.z, x.w)), y[2], y[3]);
            if (i == 0 && j == 0) y0 = y[0];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float dy = y[e] - y0;
              s1 += dy;
              s2 = fmaf(dy, dy, s2);
              rr[4 * j + e] = __float_as_uint(y[e]);
            }
          }
          tmem_st16(t_row + c * CW, rr);
          // the residual chunk RB ahead into this buffer, once every lane has read it
          // (the warp barrier orders the reads before the copy is issued)
          __syncwarp();
          if (lane == 0 && i + RB < CH) {
            mbar_expect_tx(resid_bar(ew, buf), E::kChunkBytes);
            tma_load_2d(stg + buf * E::kChunkBytes, &tmR, resid_bar(ew, buf), n + RB * CW, row0);
          }
        }
        if (!ok) break;
        tmem_wait_st();
        constexpr float kPart = (float)(CH * CW);
        const float mean_h = y0 + s1 / kPart;
        const float m2 = fmaxf(s2 - s1 * s1 / kPart, 0.f);
        // exchange: (mean, m2) of part (rank, half) of row sub*32+lane into every CTA of the cluster
        const uint32_t pb = lt & 1u;
        const int prow = sub * 32 + lane;
        const uint32_t xaddr =
            sbase + L::kXOff + ((pb * (2 * kMaxLnCluster) + lrank * 2 + half) * kBM + prow) * 8;
        for (uint32_t q = 0; q < csize; ++q)   // cluster rank of group member q: 2q + crank with pairs
          st_cluster_v2(mapa(xaddr, MC ? 2 * q + crank : q), mean_h, m2);
        fence_acq_rel_cluster();
        for (uint32_t q = 0; q < csize; ++q) mbar_arrive_cluster_relaxed(mapa(xbar(pb), MC ? 2 * q + crank : q));
        if (!warp_wait_cluster(xbar(pb), (lt >> 1) & 1u, abort_flag, p.err, 33)) break;
        // combine the 2C partials of equal size (Chan et al.)
        const int nparts = 2 * (int)csize;
        const float2* xs = reinterpret_cast<const float2*>(smem + L::kXOff) + pb * (2 * kMaxLnCluster) * kBM + prow;
        float msum = 0.f;
        for (int k = 0; k < nparts; ++k) msum += xs[k * kBM].x;
        const float mean = msum / (float)nparts;
        float m2t = 0.f;
        for (int k = 0; k < nparts; ++k) {
          const float2 pk = xs[k * kBM];
          const float dm = pk.x - mean;
          m2t += pk.y + kPart * dm * dm;
        }
        const float rstd = rsqrtf(m2t / ((float)nparts * kPart) + 1e-5f);
        // pass 2: normalize; FP32 rows (in place) and the copy leave through
        // swizzled staging and TMA tensor stores (rows past M are clipped)
        uint8_t* c2_ptr = smem + L::kStg2Off + ew * RB * 1024;
        const uint32_t c2 = sbase + L::kStg2Off + ew * RB * 1024;
#pragma unroll 1
        for (int i = 0; i < CH; ++i) {
          const int c = half * CH + i;
          const int n = n0 + c * CW;
          const int buf = i % RB;
          uint32_t rr[16];
          tmem_ld16(t_row + c * CW, rr);
          float o[16];
          const float4* vg = reinterpret_cast<const float4*>(smem + L::kVecOff + BN * 4) + (c * CW) / 4;
          const float4* vbb = reinterpret_cast<const float4*>(smem + L::kVecOff + 2 * BN * 4) + (c * CW) / 4;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float4 g = L::kVecSmem ? vg[j] : __ldg(reinterpret_cast<const float4*>(p.ln_g + n + 4 * j));
            const float4 b = L::kVecSmem ? vbb[j] : __ldg(reinterpret_cast<const float4*>(p.ln_b + n + 4 * j));
            o[4 * j + 0] = (__uint_as_float(rr[4 * j + 0]) - mean) * rstd * g.x + b.x;
            o[4 * j + 1] = (__uint_as_float(rr[4 * j + 1]) - mean) * rstd * g.y + b.y;
            o[4 * j + 2] = (__uint_as_float(rr[4 * j + 2]) - mean) * rstd * g.z + b.z;
            o[4 * j + 3] = (__uint_as_float(rr[4 * j + 3]) - mean) * rstd * g.w + b.w;
          }
          if (lane == 0) bulk_wait_read<RB - 1>();  // the stores RB chunks back have read this buffer pair
          __syncwarp();
          uint8_t* cb = stg_ptr + buf * E::kChunkBytes;
#pragma unroll
          for (int j = 0; j < 4; ++j)
            *reinterpret_cast<float4*>(cb + r * 64 + ((j ^ ((r >> 1) & 3)) << 4)) =
                make_float4(o[4 * j], o[4 * j + 1], o[4 * j + 2], o[4 * j + 3]);
          uint8_t* cc = c2_ptr + buf * 1024;
          if (p.copy == 1) {
            // BF16: 32-byte rows, 32-byte swizzle (piece j of row r at j ^ ((r >> 2) & 1))
            uint32_t w[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              __nv_bfloat162 h = __floats2bfloat162_rn(o[2 * j], o[2 * j + 1]);
              w[j] = *reinterpret_cast<uint32_t*>(&h);
            }
#pragma unroll
            for (int j = 0; j < 2; ++j)
              *reinterpret_cast<uint4*>(cc + r * 32 + ((j ^ ((r >> 2) & 1)) << 4)) =
                  make_uint4(w[4 * j], w[4 * j + 1], w[4 * j + 2], w[4 * j + 3]);
          } else if (p.copy == 2) {
            // E4M3: 16-byte rows, no swizzle
            uint32_t q[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              uint16_t lo, hi;
              asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;"
                  : "=h"(lo) : "f"(o[4 * j + 1] * p.out_scale_inv), "f"(o[4 * j] * p.out_scale_inv));
              asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;"
                  : "=h"(hi) : "f"(o[4 * j + 3] * p.out_scale_inv), "f"(o[4 * j + 2] * p.out_scale_inv));
              q[j] = (uint32_t)lo | ((uint32_t)hi << 16);
            }
            *reinterpret_cast<uint4*>(cc + r * 16) = make_uint4(q[0], q[1], q[2], q[3]);
          }
          fence_proxy_async();
          __syncwarp();
          if (lane == 0) {
            tma_store_2d(&tmR, stg + buf * E::kChunkBytes, n, row0);
            if (p.copy) tma_store_2d(&tmC, c2 + buf * 1024, n, row0);
            bulk_commit();
          }
        }
        fence_before();
        if (MC && crank != 0) mbar_arrive_cluster(mapa(tempty_bar(acc), lead));
        else mbar_arrive(tempty_bar(acc));
      } else {
#pragma unroll 1
      for (int i = 0; i < CH; ++i) {
        const int c = half * CH + i;
        const int buf = i & 1;
        uint32_t rr[CW];
        {
          const uint32_t ta = tmem_base + ((uint32_t)(sub * 32) << 16) + acc * BN + c * CW;
          if constexpr (CW == 32) tmem_ld32(ta, rr); else tmem_ld16(ta, rr);
        }
        const int n = n0 + c * CW;
        float v[CW];
        const uint64_t alpha2 = f2splat(p.alpha);
#pragma unroll
        for (int j = 0; j < CW; j += 4) {
          float4 b = p.bias ? __ldg(reinterpret_cast<const float4*>(p.bias + n + j)) : make_float4(0.f, 0.f, 0.f, 0.f);
          f2unpack(fma2(f2pack(__uint_as_float(rr[j + 0]), __uint_as_float(rr[j + 1])), alpha2, f2pack(b.x, b.y)),
                   v[j + 0], v[j + 1]);
          f2unpack(fma2(f2pack(__uint_as_float(rr[j + 2]), __uint_as_float(rr[j + 3])), alpha2, f2pack(b.z, b.w)),
                   v[j + 2], v[j + 3]);
        }
        uint8_t* cb = stg_ptr + buf * E::kChunkBytes;
        if (E::kF32) {
          // residual rows arrived by TMA; each buffer is filled CH/2 times per tile
          const uint32_t par = (lt * (CH / 2) + (i >> 1)) & 1u;
          if (!warp_wait(resid_bar(ew, buf), par, abort_flag, p.err, 31)) break;
#pragma unroll
          for (int j = 0; j < CW / 4; ++j) {
            float4* q = reinterpret_cast<float4*>(cb + r * 64 + ((j ^ ((r >> 1) & 3)) << 4));
            float4 x = *q;
            float4 y;
            f2unpack(add2(f2pack(v[4 * j], v[4 * j + 1]), f2pack(x.x, x.y)), y.x, y.y);
            f2unpack(add2(f2pack(v[4 * j + 2], v[4 * j + 3]), f2pack(x.z, x.w)), y.z, y.w);
            *q = y;
          }
        } else {
          if (EPI == AS_EPI_BIAS_GELU) {
#pragma unroll
            for (int j = 0; j < CW; j += 2) gelu_erf2(v[j], v[j + 1]);
          }
          if (lane == 0) bulk_wait_read<1>();  // the store two chunks back has read this buffer
          __syncwarp();
          if (OUT == kOutE4M3) {
            // E4M3 with saturation, round to nearest even: 32 bytes = 2 pieces
            uint32_t q[8];
            const uint64_t inv2 = f2splat(p.out_scale_inv);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              uint16_t lo, hi;
              float s0, s1, s2, s3;
              f2unpack(mul2(f2pack(v[4 * j], v[4 * j + 1]), inv2), s0, s1);
              f2unpack(mul2(f2pack(v[4 * j + 2], v[4 * j + 3]), inv2), s2, s3);
              asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(lo) : "f"(s1), "f"(s0));
              asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(hi) : "f"(s3), "f"(s2));
              q[j] = (uint32_t)lo | ((uint32_t)hi << 16);
            }
#pragma unroll
            for (int j = 0; j < 2; ++j)
              *reinterpret_cast<uint4*>(cb + r * 32 + ((j ^ ((r >> 2) & 1)) << 4)) =
                  make_uint4(q[4 * j], q[4 * j + 1], q[4 * j + 2], q[4 * j + 3]);
          } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              uint4 w;
              __nv_bfloat162 h0 = __floats2bfloat162_rn(v[8 * j + 0], v[8 * j + 1]);
              __nv_bfloat162 h1 = __floats2bfloat162_rn(v[8 * j + 2], v[8 * j + 3]);
              __nv_bfloat162 h2 = __floats2bfloat162_rn(v[8 * j + 4], v[8 * j + 5]);
              __nv_bfloat162 h3 = __floats2bfloat162_rn(v[8 * j + 6], v[8 * j + 7]);
              w.x = *reinterpret_cast<uint32_t*>(&h0);
              w.y = *reinterpret_cast<uint32_t*>(&h1);
              w.z = *reinterpret_cast<uint32_t*>(&h2);
              w.w = *reinterpret_cast<uint32_t*>(&h3);
              *reinterpret_cast<uint4*>(cb + r * 64 + ((j ^ ((r >> 1) & 3)) << 4)) = w;
            }
          }
        }
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) {
          tma_store_2d(&tmC, stg + buf * E::kChunkBytes, n, row0);
          bulk_commit();
          if (E::kF32 && i + 2 < CH) {
            // refill this buffer with the residual of chunk i + 2 once the
            // store has read it
            bulk_wait_read<0>();
            mbar_expect_tx(resid_bar(ew, buf), E::kChunkBytes);
            tma_load_2d(stg + buf * E::kChunkBytes, &tmR, resid_bar(ew, buf), n + 2 * CW, row0);
          }
        }
      }
      fence_before();
      if constexpr (MC) {
        if (crank == 0) mbar_arrive(tempty_bar(acc));
        else mbar_arrive_cluster(mapa(tempty_bar(acc), lead));
      } else {
        mbar_arrive(tempty_bar(acc));
      }
      }
    }
    if (lane == 0) bulk_wait_all();
  }
done:
  fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    fence_after();
    if constexpr (MC)
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kTmemCols) : "memory");
    else
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kTmemCols) : "memory");
  }
  // no CTA leaves while a peer may still write into its shared memory or barriers
  if constexpr (LN || MC) cluster_sync_all();
}

}  // namespace tc

// ------------------------------------------------------------------ host side

namespace {

// Set once; several host threads (serving lanes) may race to set them, each
// writing the same value.
std::atomic<PFN_cuTensorMapEncodeTiled_v12000> g_encode{nullptr};
std::atomic<int> g_num_sms{0};

as_status ensure_driver() {
  if (g_encode.load()) return AS_OK;
  cudaDriverEntryPointQueryResult q;
  void* fn = nullptr;
  AS_CUDA_OK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
  if (q != cudaDriverEntryPointSuccess || !fn) {
    set_k_error("cuTensorMapEncodeTiled not available from the driver");
    return AS_ERR_CUDA;
  }
  g_encode.store(reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn));
  return AS_OK;
}

// 2D row-major tensor map [rows][cols] of `dtype` with box {box_cols, box_rows}.
as_status make_map(CUtensorMap* tm, const void* ptr, CUtensorMapDataType dtype, uint32_t esize, uint64_t rows,
                   uint64_t cols, uint32_t box_cols, uint32_t box_rows, CUtensorMapSwizzle swz) {
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(cols * esize)};
  cuuint32_t box[2] = {box_cols, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode.load()(tm, dtype, 2, const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_k_error("cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
    return AS_ERR_CUDA;
  }
  return AS_OK;
}

template <int BN, int STAGES, int EPI, int IN, int OUT, int PAIR>
as_status launch_bn(const tc::Params& p0, const void* A, const void* B, cudaStream_t st) {
  using L = tc::Smem<BN, STAGES, OUT, false, PAIR == 2>;
  static_assert(L::kAlloc <= 232448, "shared memory per CTA");
  static std::atomic<bool> attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (!attr_set[dev & 63]) {
    AS_CUDA_OK(cudaFuncSetAttribute(tc::gemm_kernel<BN, STAGES, EPI, IN, OUT, PAIR>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, L::kAlloc));
    attr_set[dev & 63] = true;
  }
  CUtensorMap tmA, tmB, tmC, tmR;
  const auto bf = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const auto u8 = CU_TENSOR_MAP_DATA_TYPE_UINT8;
  const auto ein = IN == tc::kInE4M3 ? u8 : bf;
  const uint32_t isz = IN == tc::kInE4M3 ? 1 : 2, bke = tc::bk_elems(IN);
  as_status s = make_map(&tmA, A, ein, isz, (uint64_t)p0.M, (uint64_t)p0.K, bke, tc::kBM, CU_TENSOR_MAP_SWIZZLE_128B);
  // B boxes: the whole BN-row tile, or half of it per CTA of a 2-SM pair
  if (s == AS_OK)
    s = make_map(&tmB, B, ein, isz, (uint64_t)p0.N, (uint64_t)p0.K, bke, BN / PAIR, CU_TENSOR_MAP_SWIZZLE_128B);
  if (s == AS_OK) {
    if (OUT == tc::kOutF32) {
      s = make_map(&tmC, p0.out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (uint64_t)p0.M, (uint64_t)p0.N, 16, 32,
                   CU_TENSOR_MAP_SWIZZLE_64B);
      if (s == AS_OK)
        s = make_map(&tmR, p0.resid, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (uint64_t)p0.M, (uint64_t)p0.N, 16, 32,
                     CU_TENSOR_MAP_SWIZZLE_64B);
    } else if (OUT == tc::kOutE4M3) {
      s = make_map(&tmC, p0.out, u8, 1, (uint64_t)p0.M, (uint64_t)p0.N, 32, 32, CU_TENSOR_MAP_SWIZZLE_32B);
      tmR = tmC;  // unused
    } else {
      s = make_map(&tmC, p0.out, bf, 2, (uint64_t)p0.M, (uint64_t)p0.N, 32, 32, CU_TENSOR_MAP_SWIZZLE_64B);
      tmR = tmC;  // unused
    }
  }
  if (s != AS_OK) return s;
  tc::Params p = p0;
  p.n_tiles_n = p.N / BN;
  p.n_tiles = p.n_tiles_n * ((p.M + tc::kBM - 1) / tc::kBM);
  const int n_sms = g_num_sms.load();
  if (PAIR == 1) {
    int grid = p.n_tiles < n_sms ? p.n_tiles : n_sms;
    tc::gemm_kernel<BN, STAGES, EPI, IN, OUT, PAIR><<<grid, tc::kThreads, L::kAlloc, st>>>(tmA, tmB, tmC, tmR, p);
    count_launch();
    AS_CUDA_OK(cudaGetLastError());
    return AS_OK;
  }
  // pairs of CTAs (a cluster of two), persistent over 256 x BN pair tiles
  const int m_blocks = (p.M + tc::kBM - 1) / tc::kBM;
  const int pair_tiles = (m_blocks + 1) / 2 * p.n_tiles_n;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(tc::kThreads);
  cfg.dynamicSmemBytes = L::kAlloc;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const int pairs = std::max(1, std::min(pair_tiles, n_sms / 2));
  cfg.gridDim = dim3((unsigned)(2 * pairs));
  AS_CUDA_OK(cudaLaunchKernelEx(&cfg, tc::gemm_kernel<BN, STAGES, EPI, IN, OUT, PAIR>, tmA, tmB, tmC, tmR, p));
  count_launch();
  return AS_OK;
}

// Residual + LayerNorm GEMM: a cluster of C = N / BN CTAs per 128-row block,
// or (PAIR = 2) of 2C CTAs per 256-row block, 2-SM pairs along M.
template <int BN, int STAGES, int IN, int PAIR>
as_status launch_ln(const tc::Params& p0, const void* A, const void* B, int C, cudaStream_t st) {
  using L = tc::Smem<BN, STAGES, tc::kOutF32, true, PAIR == 2>;
  static_assert(L::kAlloc <= 232448, "shared memory per CTA");
  auto kern = tc::gemm_kernel<BN, STAGES, tc::kEpiResidLN, IN, tc::kOutF32, PAIR>;
  static std::atomic<bool> attr_set[64] = {};
  static std::atomic<int> max_clusters[64][2 * tc::kMaxLnCluster + 1] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (!attr_set[dev & 63]) {
    AS_CUDA_OK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L::kAlloc));
    attr_set[dev & 63] = true;
  }
  CUtensorMap tmA, tmB, tmR;
  const auto bf = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const auto u8 = CU_TENSOR_MAP_DATA_TYPE_UINT8;
  const auto ein = IN == tc::kInE4M3 ? u8 : bf;
  const uint32_t isz = IN == tc::kInE4M3 ? 1 : 2, bke = tc::bk_elems(IN);
  as_status s = make_map(&tmA, A, ein, isz, (uint64_t)p0.M, (uint64_t)p0.K, bke, tc::kBM, CU_TENSOR_MAP_SWIZZLE_128B);
  if (s == AS_OK)
    s = make_map(&tmB, B, ein, isz, (uint64_t)p0.N, (uint64_t)p0.K, bke, BN / PAIR, CU_TENSOR_MAP_SWIZZLE_128B);
  if (s == AS_OK)
    s = make_map(&tmR, p0.resid, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (uint64_t)p0.M, (uint64_t)p0.N, 16, 32,
                 CU_TENSOR_MAP_SWIZZLE_64B);
  // the copy: BF16 chunks with 32-byte rows (32-byte swizzle), E4M3 with 16-byte rows
  CUtensorMap tmO = tmR;
  if (s == AS_OK && p0.copy == 1)
    s = make_map(&tmO, p0.out16, bf, 2, (uint64_t)p0.M, (uint64_t)p0.N, 16, 32, CU_TENSOR_MAP_SWIZZLE_32B);
  if (s == AS_OK && p0.copy == 2)
    s = make_map(&tmO, p0.out8, u8, 1, (uint64_t)p0.M, (uint64_t)p0.N, 16, 32, CU_TENSOR_MAP_SWIZZLE_NONE);
  if (s != AS_OK) return s;
  tc::Params p = p0;
  p.n_tiles_n = C;
  const int m_blocks = (p.M + tc::kBM - 1) / tc::kBM;
  p.n_tiles = C * m_blocks;
  const int csz = C * PAIR;
  const int units = (m_blocks + PAIR - 1) / PAIR;   // row blocks (or block pairs) to walk
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)csz;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(tc::kThreads);
  cfg.dynamicSmemBytes = L::kAlloc;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // persistent: as many clusters as fit on the GPU at once (asked once per device and size)
  int mc = max_clusters[dev & 63][csz].load();
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cap);
  if (mc == 0 && cap != cudaStreamCaptureStatusNone) {
    mc = g_num_sms.load() > 0 ? g_num_sms.load() / csz : 1;  // not asked while capturing a graph
  } else if (mc == 0) {
    cfg.gridDim = dim3((unsigned)(csz * units));
    int q = 0;
    AS_CUDA_OK(cudaOccupancyMaxActiveClusters(&q, kern, &cfg));
    mc = q > 0 ? q : 1;
    max_clusters[dev & 63][csz].store(mc);
  }
  cfg.gridDim = dim3((unsigned)(csz * std::min(units, mc)));
  AS_CUDA_OK(cudaLaunchKernelEx(&cfg, kern, tmA, tmB, tmO, tmR, p));
  count_launch();
  return AS_OK;
}

// Tile configurations (the autotuner's choices): cfg & 1 = raster order,
// cfg & 2 = 128-column tiles (6 stages) instead of 256-column tiles (4 stages),
// cfg & 4 = 2-SM MMA (CTA pairs, 256-row tiles, half the B rows per CTA).
template <int IN, int PAIR>
as_status dispatch_pair(const tc::Params& p, int epi, bool out_e4m3, bool wide, const void* A, const void* B,
                        cudaStream_t st) {
  // a 2-SM pair keeps half the B rows per CTA: 32 KB (wide) / 24 KB stages, so 6 / 8 of them
  constexpr int SW = PAIR == 2 ? 6 : 4, SN = PAIR == 2 ? 8 : 6;
  switch (epi) {
    case AS_EPI_BIAS:
      if (out_e4m3) break;
      return wide ? launch_bn<256, SW, AS_EPI_BIAS, IN, tc::kOutBF16, PAIR>(p, A, B, st)
                  : launch_bn<128, SN, AS_EPI_BIAS, IN, tc::kOutBF16, PAIR>(p, A, B, st);
    case AS_EPI_BIAS_GELU:
      if (out_e4m3)
        return wide ? launch_bn<256, SW, AS_EPI_BIAS_GELU, IN, tc::kOutE4M3, PAIR>(p, A, B, st)
                    : launch_bn<128, SN, AS_EPI_BIAS_GELU, IN, tc::kOutE4M3, PAIR>(p, A, B, st);
      return wide ? launch_bn<256, SW, AS_EPI_BIAS_GELU, IN, tc::kOutBF16, PAIR>(p, A, B, st)
                  : launch_bn<128, SN, AS_EPI_BIAS_GELU, IN, tc::kOutBF16, PAIR>(p, A, B, st);
    case AS_EPI_BIAS_RESID:
      if (out_e4m3) break;
      return wide ? launch_bn<256, SW, AS_EPI_BIAS_RESID, IN, tc::kOutF32, PAIR>(p, A, B, st)
                  : launch_bn<128, SN, AS_EPI_BIAS_RESID, IN, tc::kOutF32, PAIR>(p, A, B, st);
    default:
      break;
  }
  set_k_error("gemm_tcgen05: unsupported epilogue / output combination");
  return AS_ERR_ARG;
}

template <int IN>
as_status dispatch(const tc::Params& p0, int epi, bool out_e4m3, const void* A, const void* B, cudaStream_t st,
                   int cfg) {
  tc::Params p = p0;
  bool wide = p.N % 256 == 0;
  bool pair = false;
  if (cfg >= 0) {
    p.raster = cfg & 1;
    if (cfg & 2) wide = false;
    pair = (cfg & 4) != 0;
  }
  return pair ? dispatch_pair<IN, 2>(p, epi, out_e4m3, wide, A, B, st)
              : dispatch_pair<IN, 1>(p, epi, out_e4m3, wide, A, B, st);
}

}  // namespace

bool gemm_tcgen05_cfg_valid(int cfg, int64_t N) { return cfg >= 0 && cfg < kGemmCfgs && ((cfg & 2) || N % 256 == 0); }

as_status gemm_tcgen05_ex(int epi, bool in_e4m3, bool out_e4m3, int64_t M, int64_t N, int64_t K, const void* A,
                          const void* B, const float* bias, const float* resid, void* out, float alpha,
                          float out_scale, DevError* err, cudaStream_t st, int cfg) {
  as_status s = ensure_driver();
  if (s != AS_OK) return s;
  if (g_num_sms.load() == 0) {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    g_num_sms.store(n > 0 ? n : kDefaultSMs);
  }
  const int bke = tc::bk_elems(in_e4m3 ? tc::kInE4M3 : tc::kInBF16);
  if (M < 1 || N % 128 != 0 || K % bke != 0 || K < bke || M > (1ll << 31) - 1 ||
      (reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15) ||
      (reinterpret_cast<uintptr_t>(out) & 15) || (epi == AS_EPI_BIAS_RESID && (reinterpret_cast<uintptr_t>(resid) & 15)) ||
      (bias && (reinterpret_cast<uintptr_t>(bias) & 15)) || (out_e4m3 && !(out_scale > 0.f))) {
    set_k_error("gemm_tcgen05: unsupported shape, alignment or scale");
    return AS_ERR_ARG;
  }
  tc::Params p{};
  p.M = (int)M;
  p.N = (int)N;
  p.K = (int)K;
  p.epi = epi;
  p.bias = bias;
  p.resid = resid;
  p.out = out;
  p.err = err;
  p.alpha = alpha;
  p.out_scale_inv = out_e4m3 ? 1.0f / out_scale : 1.0f;
  if (cfg >= 0 && !gemm_tcgen05_cfg_valid(cfg, N)) {
    set_k_error("gemm_tcgen05: tile configuration not valid for this shape");
    return AS_ERR_ARG;
  }
  return in_e4m3 ? dispatch<tc::kInE4M3>(p, epi, out_e4m3, A, B, st, cfg)
                 : dispatch<tc::kInBF16>(p, epi, out_e4m3, A, B, st, cfg);
}

int gemm_resid_ln_cluster(int64_t N) {
  const int bn = N % 256 == 0 ? 256 : 128;
  const int64_t c = N % 128 == 0 ? N / bn : 0;
  return (c >= 1 && c <= tc::kMaxLnCluster) ? (int)c : 0;
}

as_status gemm_tcgen05_resid_ln(bool in_e4m3, int64_t M, int64_t N, int64_t K, const void* A, const void* B,
                                const float* bias, float* x32, const float* ln_g, const float* ln_b,
                                __nv_bfloat16* out16, uint8_t* out8, float out8_scale, float alpha, DevError* err,
                                cudaStream_t st, bool pair, bool deep) {
  as_status s = ensure_driver();
  if (s != AS_OK) return s;
  if (g_num_sms.load() == 0) {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    g_num_sms.store(n > 0 ? n : kDefaultSMs);
  }
  const int C = gemm_resid_ln_cluster(N);
  const int bke = tc::bk_elems(in_e4m3 ? tc::kInE4M3 : tc::kInBF16);
  auto mis = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) != 0; };
  if (C == 0 || M < 1 || K % bke != 0 || K < bke || M > (1ll << 31) - 1 || mis(A) || mis(B) || mis(x32) ||
      !ln_g || !ln_b || mis(ln_g) || mis(ln_b) || (bias && mis(bias)) || (out16 && mis(out16)) ||
      (out8 && (mis(out8) || !(out8_scale > 0.f))) || (out16 && out8)) {
    set_k_error("gemm_tcgen05_resid_ln: unsupported shape, alignment or scale");
    return AS_ERR_ARG;
  }
  tc::Params p{};
  p.M = (int)M;
  p.N = (int)N;
  p.K = (int)K;
  p.epi = tc::kEpiResidLN;
  p.bias = bias;
  p.resid = x32;
  p.out = x32;
  p.err = err;
  p.alpha = alpha;
  p.out_scale_inv = out8 ? 1.0f / out8_scale : 1.0f;
  p.ln_g = ln_g;
  p.ln_b = ln_b;
  p.out16 = out16;
  p.out8 = out8;
  p.copy = out16 ? 1 : (out8 ? 2 : 0);
  const bool wide = N % 256 == 0;
  // deep: a short main-loop ring and four staging buffers per epilogue warp
  if (pair) {
    if (deep) {
      if (in_e4m3)
        return wide ? launch_ln<256, 3, tc::kInE4M3, 2>(p, A, B, C, st) : launch_ln<128, 3, tc::kInE4M3, 2>(p, A, B, C, st);
      return wide ? launch_ln<256, 3, tc::kInBF16, 2>(p, A, B, C, st) : launch_ln<128, 3, tc::kInBF16, 2>(p, A, B, C, st);
    }
    if (in_e4m3)
      return wide ? launch_ln<256, 5, tc::kInE4M3, 2>(p, A, B, C, st) : launch_ln<128, 6, tc::kInE4M3, 2>(p, A, B, C, st);
    return wide ? launch_ln<256, 5, tc::kInBF16, 2>(p, A, B, C, st) : launch_ln<128, 6, tc::kInBF16, 2>(p, A, B, C, st);
  }
  if (deep) {
    if (in_e4m3)
      return wide ? launch_ln<256, 2, tc::kInE4M3, 1>(p, A, B, C, st) : launch_ln<128, 2, tc::kInE4M3, 1>(p, A, B, C, st);
    return wide ? launch_ln<256, 2, tc::kInBF16, 1>(p, A, B, C, st) : launch_ln<128, 2, tc::kInBF16, 1>(p, A, B, C, st);
  }
  if (in_e4m3)
    return wide ? launch_ln<256, 3, tc::kInE4M3, 1>(p, A, B, C, st) : launch_ln<128, 4, tc::kInE4M3, 1>(p, A, B, C, st);
  return wide ? launch_ln<256, 3, tc::kInBF16, 1>(p, A, B, C, st) : launch_ln<128, 4, tc::kInBF16, 1>(p, A, B, C, st);
}

as_status gemm_tcgen05(int epi, int64_t M, int64_t N, int64_t K, const void* A, const void* B, const float* bias,
                       const float* resid, void* out, DevError* err, cudaStream_t st) {
  return gemm_tcgen05_ex(epi, false, false, M, N, K, A, B, bias, resid, out, 1.0f, 1.0f, err, st, -1);
}

}  // namespace as
