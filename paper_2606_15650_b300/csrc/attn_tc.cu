// Self-attention on the 5th-generation tensor cores (sm_103a), BF16 in,
// FP32 softmax statistics and accumulation (encoder of AnonShield §2 stage (2)).
//
// Persistent: two CTAs per SM, each looping over work units (one 128-query
// tile of one sequence, one head); keys in tiles of 64, numbered globally
// across a CTA's units (g), which fixes every buffer index and barrier phase.
//   S_g = Q K_g^T           tcgen05.mma M=128 N=64 K=64 into one of two S
//                           buffers in TMEM, issued right after O_{g-2}
//                           (so, a whole softmax ahead of its use)
//   P_g = exp2(S_g*c - m)   four softmax warps, one query row per thread: the
//                           64-key row of S is read in one pass and released,
//                           P rounded to BF16 and stored back into one of two
//                           P buffers in TMEM
//   O  += P_g V_g           tcgen05.mma with A (P) from TMEM and B (V) from
//                           shared memory; O in TMEM, read by the same warps
//                           at the end of the unit (epilogue)
// The maximum m that P is taken against is raised only when a row's true
// maximum exceeds it by more than 2^8 (P stays <= 256), so O is rescaled in
// TMEM only on those raises instead of on every growth of the maximum.
// Q, K and V tiles come straight from the packed QKV rows by TMA: Q and K as
// K-major operands, V as an MN-major B operand (keys along K, features
// contiguous), so no transposed copy of V is made. K (4 stages) and V (4
// stages) have rings of their own; Q is double-buffered across units.
// Warps: Q/K loader, V loader (one thread each, blocking on their own
// barriers), MMA issuer (one warp, warp-uniform loop, one elected lane issues),
// four softmax warps. 104 KB shared memory, 256 TMEM columns.
// Every MMA is issued from that warp, in the order S_0, S_1, O_0, S_2, O_1,
// S_3, ..., and tcgen05 MMAs of one thread complete in issue order: once S_g is
// complete (the softmax warps wait for it anyway) so is O_{g-2}, which frees P
// buffer g&1 for P_g without a wait of its own. And S_{g+2} is issued only
// after P_g is full, which the softmax warps signal after reading S_g, so the S
// buffer needs no release barrier either. Per key tile the issuer tests three
// barriers together (V_g, K of S_{g+2}, and P_g, the only one the softmax
// warps hold up; the tests' shared-memory round trips overlap) and commits
// twice (S-full, O-done); the loaders refill a stage on those.
// Keys past the sequence end are masked to -inf; query rows past it are not
// stored. Every mbarrier wait is bounded (see gemm_tc.cu); on a timeout each
// issuing thread waits (bounded) for its copies and MMAs in flight before the
// CTA frees its TMEM.
#include <algorithm>
#include <atomic>
#include <vector>
#include <cuda.h>
#include <cudaTypedefs.h>

#include "encoder.cuh"

namespace as {
namespace atc {

constexpr int kQ = 128;        // query rows per CTA
constexpr int kKT = 64;        // keys per tile
constexpr int kThreads = 224;  // Q/K loader, V loader, MMA issuer, 4 softmax warps
constexpr uint64_t kTimeoutNs = 2000000000ull;

// Work item = one 128-query tile of one sequence, self-contained so that one
// 8-byte load describes it: x = the sequence's first row, y = L | (q0 << 16)
// (L = 0: a padding item). A work unit is an (item, head) pair; CTA b takes
// units b, b + grid, ...
struct Params {
  const int2* items;
  int n_items;
  void* out;            // BF16, or E4M3 of value * out_inv_scale
  float out_inv_scale;
  int d, n_heads;
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
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
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
// Warp-uniform wait for three barrier phases (none of which can be lapped
// while the warp waits): the three tests are issued back to back, so their
// shared-memory round trips overlap, and only the phases not yet complete
// are then waited for one by one.
__device__ __forceinline__ bool warp_wait3(uint32_t b0, uint32_t p0, uint32_t b1, uint32_t p1, uint32_t b2,
                                           uint32_t p2, volatile int* abort_flag, DevError* err, uint32_t where) {
  const bool r0 = mbar_test(b0, p0), r1 = mbar_test(b1, p1), r2 = mbar_test(b2, p2);
  const bool a0 = __all_sync(0xffffffffu, r0), a1 = __all_sync(0xffffffffu, r1), a2 = __all_sync(0xffffffffu, r2);
  return (a0 || warp_wait(b0, p0, abort_flag, err, where)) && (a1 || warp_wait(b1, p1, abort_flag, err, where + 1)) &&
         (a2 || warp_wait(b2, p2, abort_flag, err, where + 2));
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
// The same 128-byte-swizzle descriptor for an MN-major operand whose swizzle
// atoms (8 K-rows of 128 bytes) follow each other along K: both strides are
// 1024 bytes (the MN stride is unused with N = 64, one atom wide).
__device__ __forceinline__ uint64_t sw128_desc_mn(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)(1024 >> 4) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
constexpr uint32_t kIdescTransposeB = 1u << 16;  // B operand MN-major
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
// A operand from TMEM (M lanes x K/2 columns, two 16-bit values per column,
// the lower K index in the low half), B from shared memory.
__device__ __forceinline__ void mma_bf16_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
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
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void tmem_ld64(uint32_t taddr, uint32_t (&r)[64]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared memory (offsets from a 1024-aligned base): 104 KB, two CTAs per SM.
constexpr int kQBytes = kQ * 64 * 2;                 // 16 KB per buffer: Q tile, one 128-byte-swizzle panel
constexpr int kKBytes = kKT * 64 * 2;                // 8 KB per stage: 64 keys x 64 features
constexpr int kVBytes = kKT * 64 * 2;                // 8 KB per stage: 64 keys x 64 features
// K and V have rings of their own: a K stage is free as soon as S_g = Q K_g^T
// is done, a V stage only after O += P_g V_g, which comes a softmax later.
// The loaders wait on the S-full and O-done barriers themselves (one per ring
// slot, so indexed by g % 4 like the stages): no separate release barriers,
// and the MMA issuer commits twice per key tile instead of four times.
constexpr int kRing = 4;
constexpr int kKStages = kRing;
constexpr int kVStages = kRing;
constexpr int kOffQ = 0;                             // 2 buffers (consecutive work units)
constexpr int kOffK = kOffQ + 2 * kQBytes;
constexpr int kOffV = kOffK + kKStages * kKBytes;
// Epilogue staging, 2 KB per softmax warp: a warp's output rows pass through
// it so that each global store writes whole rows (a lane per 16-byte piece)
// instead of one 16-byte piece of 32 different rows
constexpr int kStgBytes = 2048;
constexpr int kOffStg = kOffV + kVStages * kVBytes;
constexpr int kOffBar = kOffStg + 4 * kStgBytes;
// mbarriers (8 bytes each)
enum {
  kBarQFull = 0,     // [2] Q of a unit landed
  kBarQEmpty = 2,    // [2] the S MMAs of a unit are done with its Q
  kBarKFull = 4,     // [kRing] K_g landed (by g % kRing)
  kBarVFull = 8,     // [kRing] V_g landed
  kBarSFull = 12,    // [kRing] S_g = Q K_g^T in TMEM; K stage g % kRing free again
  kBarPFull = 16,    // [2] P_g in TMEM, S_g read (128 arrivals; by P buffer)
  kBarODone = 18,    // [kRing] O += P_g V_g done; V stage g % kRing free again
  kBarDrain = 22,
  kNumBars = 23
};
// A barrier indexed by g % kRing completes phase g / kRing with tile g. No
// waiter can lag a full ring behind: tile g + kRing needs K or V stage
// g % kRing refilled, which its loader does only after that wait.
constexpr int kSmemBytes = kOffBar + kNumBars * 8 + 16;
constexpr int kSmemAlloc = kSmemBytes + 1024;        // room to align the base to 1024 bytes
// TMEM: S buffers at columns 0 and 64, O at 128, P buffers at 192 and 224.
// One O suffices: the softmax warps read a unit's O (epilogue) before they
// produce the next unit's first P, which the next O MMA waits for.
constexpr uint32_t kTmemCols = 256;
constexpr uint32_t kColO = 128;
constexpr uint32_t kColP = 192;                      // P_g: 64 BF16 keys per row = 32 columns
// P is exp2(t - m) against a row maximum m that is raised only when the true
// maximum exceeds it by more than this (log2 units): P <= 2^8, and O and the
// row sum are rescaled only on those rare raises.
constexpr float kRescaleSlack = 8.0f;

struct Work {
  int L, row0, q0, h, n_t;
};
__device__ __forceinline__ bool item_empty(int2 it) { return (it.y & 0xFFFF) == 0; }

// A CTA's walk over its units (u = b, b + grid, ...), skipping padding items
// the same way in every role. Unit u is (item u / heads, head u % heads); the
// pair is carried along the walk (two divisions at the start, none after).
// The descriptor of the unit after the current one is loaded when the current
// one starts, so that a unit boundary does not wait on a global load (it is
// only read a whole unit later).
struct UnitWalk {
  int u = 0, n = 0, step = 0;
  int item = 0, h = 0, nh = 1, step_item = 0, step_h = 0;
  int2 cur{0, 0}, nxt{0, 0};
  __device__ __forceinline__ void fwd() {
    u += step;
    item += step_item;
    h += step_h;
    if (h >= nh) {
      h -= nh;
      ++item;
    }
  }
  // item of unit u + step
  __device__ __forceinline__ int next_item() const { return item + step_item + (h + step_h >= nh ? 1 : 0); }
  __device__ __forceinline__ void start(const Params& p, int n_units) {
    n = n_units;
    nh = p.n_heads;
    step = (int)gridDim.x;
    step_item = step / nh;
    step_h = step - step_item * nh;
    u = (int)blockIdx.x;
    item = u / nh;
    h = u - item * nh;
    while (u < n && item_empty(cur = __ldg(p.items + item))) fwd();
    if (u < n && u + step < n) nxt = __ldg(p.items + next_item());
  }
  __device__ __forceinline__ void advance(const Params& p) {
    fwd();
    if (u >= n) return;
    cur = nxt;
    if (item_empty(cur)) {
      do fwd();
      while (u < n && item_empty(cur = __ldg(p.items + item)));
      if (u >= n) return;
    }
    if (u + step < n) nxt = __ldg(p.items + next_item());
  }
  __device__ __forceinline__ bool done() const { return u >= n; }
  __device__ __forceinline__ Work work(const Params&) const {
    Work w;
    w.h = h;
    w.row0 = cur.x;
    w.L = cur.y & 0xFFFF;
    w.q0 = cur.y >> 16;
    w.n_t = (w.L + kKT - 1) / kKT;
    return w;
  }
};

__device__ __forceinline__ uint16_t e4m3x2(float lo, float hi) {
  uint16_t r;
  asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(r) : "f"(hi), "f"(lo));
  return r;
}

// Persistent: a CTA loops over its work units; tiles are numbered globally
// across units (g), which fixes every buffer index and barrier phase.
template <bool OUT8>
__global__ void __launch_bounds__(kThreads, 2)
    attn_tc_kernel(const __grid_constant__ CUtensorMap tmQ, const __grid_constant__ CUtensorMap tmKV, Params p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const uint32_t sb = smem_u32(smem);
  const uint32_t bar0 = sb + kOffBar;
  auto bar = [&](int i) { return bar0 + 8u * (uint32_t)i; };
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kOffBar + kNumBars * 8);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_units = p.n_items * p.n_heads;

  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(bar(kBarQFull + i), 1);
      mbar_init(bar(kBarQEmpty + i), 1);
      mbar_init(bar(kBarPFull + i), 128);
    }
    for (int i = 0; i < kRing; ++i) {
      mbar_init(bar(kBarKFull + i), 1);
      mbar_init(bar(kBarVFull + i), 1);
      mbar_init(bar(kBarSFull + i), 1);
      mbar_init(bar(kBarODone + i), 1);
    }
    mbar_init(bar(kBarDrain), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
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
      // ---------------- Q and K loads, in unit order
      int i = 0, g = 0;
      bool ok = true;
      UnitWalk uw;
      for (uw.start(p, n_units); !uw.done() && ok; uw.advance(p), ++i) {
        const Work w = uw.work(p);
        const int b = i & 1;
        if (i >= 2 && !mbar_wait(bar(kBarQEmpty + b), ((i >> 1) - 1) & 1, abort_flag, p.err, 40)) { ok = false; break; }
        mbar_expect_tx(bar(kBarQFull + b), kQBytes);
        tma_load_2d(sb + kOffQ + b * kQBytes, &tmQ, bar(kBarQFull + b), w.h * 64, w.row0 + w.q0);
        for (int t = 0; t < w.n_t; ++t, ++g) {
          const int st = g % kKStages;
          // S_{g - kRing} done with this stage (passes at once for g < kRing)
          if (!mbar_wait(bar(kBarSFull + st), ((g / kKStages) & 1) ^ 1u, abort_flag, p.err, 41)) { ok = false; break; }
          mbar_expect_tx(bar(kBarKFull + st), kKBytes);
          tma_load_2d(sb + kOffK + st * kKBytes, &tmKV, bar(kBarKFull + st), d + w.h * 64, w.row0 + t * kKT);
        }
      }
      if (!ok) {
        // wait (bounded) for the loads still in flight: the last ones of each ring
        const uint64_t t0 = globaltimer();
        for (int j = max(0, g - kKStages); j < g; ++j)
          while (!mbar_test(bar(kBarKFull + j % kKStages), (j / kKStages) & 1) && globaltimer() - t0 < kTimeoutNs) {
          }
        for (int j = max(0, i - 1); j <= i; ++j)
          while (!mbar_test(bar(kBarQFull + (j & 1)), (j >> 1) & 1) && globaltimer() - t0 < kTimeoutNs) {
          }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- V loads, in unit order (a ring of their own: a V stage
      // frees only after O += P V, later than the K stage of the same tile)
      int g = 0;
      bool ok = true;
      UnitWalk uw;
      for (uw.start(p, n_units); !uw.done() && ok; uw.advance(p)) {
        const Work w = uw.work(p);
        for (int t = 0; t < w.n_t; ++t, ++g) {
          const int st = g % kVStages;
          // O += P_{g - kRing} V_{g - kRing} done with this stage
          if (!mbar_wait(bar(kBarODone + st), ((g / kVStages) & 1) ^ 1u, abort_flag, p.err, 42)) { ok = false; break; }
          mbar_expect_tx(bar(kBarVFull + st), kVBytes);
          tma_load_2d(sb + kOffV + st * kVBytes, &tmKV, bar(kBarVFull + st), 2 * d + w.h * 64, w.row0 + t * kKT);
        }
      }
      if (!ok) {
        const uint64_t t0 = globaltimer();
        for (int j = max(0, g - kVStages); j < g; ++j)
          while (!mbar_test(bar(kBarVFull + j % kVStages), (j / kVStages) & 1) && globaltimer() - t0 < kTimeoutNs) {
          }
      }
    }
  } else if (warp == 2) {
    // ---------------- MMA issuer: the whole warp runs the loop (its waits and
    // cursors are warp-uniform) and one elected lane issues each group of MMAs.
    // Order: S_0, S_1, then O_g followed by S_{g+2} for every g, so S_{g+1} is
    // computed while the softmax warps work on S_g. The waits that do not
    // depend on the softmax (V_g, and Q and K of S_{g+2}) come before the wait
    // for P_g, which is then followed at once by the eight MMAs.
    constexpr uint32_t idS = idesc_bf16(kQ, kKT), idO = idesc_bf16(kQ, 64) | kIdescTransposeB;
    UnitWalk cs, co;                          // S and O cursors
    cs.start(p, n_units);
    co.start(p, n_units);
    int is = 0, ts = 0, gs = 0, to = 0, go = 0;
    Work ws{}, wo{};
    if (!cs.done()) ws = wo = cs.work(p);
    bool ok = true, issued = false;
    auto wait_s = [&]() -> bool {             // Q and K_gs landed
      if (ts == 0 && !warp_wait(bar(kBarQFull + (is & 1)), (is >> 1) & 1, abort_flag, p.err, 50)) return false;
      return warp_wait(bar(kBarKFull + gs % kKStages), (gs / kKStages) & 1, abort_flag, p.err, 51);
    };
    auto issue_s = [&]() {
      const int st = gs % kKStages;
      const int sbuf = gs & 1;  // free: S_{gs-2} was read before P_{gs-2}, which O_{gs-2} waited for
      const uint64_t qdesc = sw128_desc(sb + kOffQ + (is & 1) * kQBytes);
      const uint64_t kdesc = sw128_desc(sb + kOffK + st * kKBytes);
      const bool last = ts + 1 == ws.n_t;
      if (elect_one()) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          mma_bf16(tmem + 64u * (uint32_t)sbuf, qdesc + 2 * k, kdesc + 2 * k, idS, k > 0 ? 1u : 0u);
        mma_commit(bar(kBarSFull + st));
        if (last) mma_commit(bar(kBarQEmpty + (is & 1)));
      }
      __syncwarp();
      issued = true;
      ++gs;
      if (++ts == ws.n_t) {
        cs.advance(p);
        ++is;
        ts = 0;
        if (!cs.done()) ws = cs.work(p);
      }
    };
    auto issue_o = [&]() {
      const int st = go % kVStages;
      const uint32_t pcol = tmem + kColP + 32u * (uint32_t)(go & 1);
      const uint64_t vdesc = sw128_desc_mn(sb + kOffV + st * kVBytes);
      const uint32_t ocol = tmem + kColO;
      const uint32_t acc0 = to > 0 ? 1u : 0u;
      if (elect_one()) {
#pragma unroll
        for (int k = 0; k < 4; ++k) mma_bf16_ta(ocol, pcol + 8 * k, vdesc + 128 * k, idO, k > 0 ? 1u : acc0);
        mma_commit(bar(kBarODone + st));
      }
      __syncwarp();
      ++go;
      if (++to == wo.n_t) {
        co.advance(p);
        to = 0;
        if (!co.done()) wo = co.work(p);
      }
    };
    for (int k = 0; k < 2 && ok && !cs.done(); ++k) {
      ok = wait_s();
      if (ok) {
        fence_after();
        issue_s();
      }
    }
    while (ok && !co.done()) {
      const bool more_s = !cs.done();
      // V_g, K of S_{g+2} (V_g again when no S follows) and P_g, tested together
      const uint32_t bv = bar(kBarVFull + go % kVStages), pv = (go / kVStages) & 1;
      uint32_t bk = bv, pk = pv;
      if (more_s) {
        if (ts == 0 && !warp_wait(bar(kBarQFull + (is & 1)), (is >> 1) & 1, abort_flag, p.err, 50)) { ok = false; break; }
        bk = bar(kBarKFull + gs % kKStages);
        pk = (gs / kKStages) & 1;
      }
      ok = warp_wait3(bv, pv, bk, pk, bar(kBarPFull + (go & 1)), (go >> 1) & 1, abort_flag, p.err, 55);
      if (!ok) break;
      fence_after();
      issue_o();
      if (more_s) issue_s();
    }
    if (!ok && issued) {
      // wait (bounded) for the MMAs in flight before the TMEM is freed
      if (elect_one()) mma_commit(bar(kBarDrain));
      __syncwarp();
      const uint64_t t0 = globaltimer();
      while (!mbar_test(bar(kBarDrain), 0) && globaltimer() - t0 < kTimeoutNs) {
      }
    }
  } else {
    // ---------------- softmax + epilogue: warp w owns TMEM lanes (query rows) 32*(w%4)..
    const int sub = warp & 3;
    const uint32_t trow = tmem + ((uint32_t)(sub * 32) << 16);
    const float c = 0.125f * 1.4426950408889634f;  // 1/sqrt(64) * log2(e)
    // O += P_k V_k completes phase k/2 of o_done[k&1]
    auto wait_o = [&](int k, uint32_t where) {
      return warp_wait(bar(kBarODone + (k % kRing)), (k / kRing) & 1, abort_flag, p.err, where);
    };
    int g = 0, i = 0;
    bool ok = true;
    UnitWalk uw;
    for (uw.start(p, n_units); !uw.done() && ok; uw.advance(p), ++i) {
      const Work w = uw.work(p);
      const uint32_t ocol = kColO;
      float m = -INFINITY, l = 0.f;              // m: the maximum P is taken against
      // a warp whose 32 query rows all lie past the sequence end (the ragged last
      // query tile) computes nothing: its P and O rows only feed output rows that
      // are never stored, and MMA rows do not mix; it keeps the barrier protocol
      // and its share of the V-tail zeroing
      const bool live = w.q0 + sub * 32 < w.L;
      for (int t = 0; t < w.n_t; ++t, ++g) {
        const int valid = min(kKT, w.L - t * kKT);  // keys of this tile inside the sequence
        if (!warp_wait(bar(kBarSFull + (g % kRing)), (g / kRing) & 1, abort_flag, p.err, 60)) { ok = false; break; }
        fence_after();
        // keys past the sequence end have P = 0, but the MMA still multiplies
        // their V rows: zero those rows of the landed V tile (a 128-byte row
        // holds all its swizzled pieces), so that whatever lies past the
        // sequence (another sequence's rows, padding, non-finite data)
        // contributes exactly nothing (every softmax warp takes a share)
        auto zero_v_tail = [&]() -> bool {
          if (valid >= kKT) return true;
          const int vst = g % kVStages;
          if (!warp_wait(bar(kBarVFull + vst), (g / kVStages) & 1, abort_flag, p.err, 64)) return false;
          uint4* vt = reinterpret_cast<uint4*>(smem + kOffV + vst * kVBytes);
          for (int q = valid * 8 + (warp - 3) * 32 + lane; q < kKT * 8; q += 128) vt[q] = make_uint4(0u, 0u, 0u, 0u);
          fence_proxy_async();
          return true;
        };
        if (!live) {
          if (!zero_v_tail()) { ok = false; break; }
          // S_g being complete, so are O_{g-2} and the P-full phase of tile g-2:
          // this arrival lands in tile g's phase even from a warp that computes
          // nothing and could otherwise run ahead
          fence_before();
          mbar_arrive(bar(kBarPFull + (g & 1)));
          continue;
        }
        uint32_t v[64];
        tmem_ld64(trow + 64u * (uint32_t)(g & 1), v);
        // row maximum of the raw scores (keys past the end masked to -inf); the
        // scale c > 0 is applied in the exp2 argument: t = s * c - m
        if (valid < kKT) {
#pragma unroll
          for (int q = 0; q < 64; ++q)
            if (q >= valid) v[q] = __float_as_uint(-INFINITY);
        }
        // eight independent running maxima, then a tree: short dependency chains
        float m8[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) m8[q] = __uint_as_float(v[q]);
#pragma unroll
        for (int q = 8; q < 64; ++q) m8[q & 7] = fmaxf(m8[q & 7], __uint_as_float(v[q]));
        const float mx =
            fmaxf(fmaxf(fmaxf(m8[0], m8[1]), fmaxf(m8[2], m8[3])), fmaxf(fmaxf(m8[4], m8[5]), fmaxf(m8[6], m8[7]))) * c;
        // tcgen05.ld / st are warp-collective: the warp raises together when any
        // of its rows needs it (a row that does not multiplies by <= 1, exactly)
        if (__any_sync(0xffffffffu, mx > m + kRescaleSlack)) {
          const float mn = fmaxf(m, mx);
          const float corr = ex2_approx(m - mn);  // 0 on the first tile of a unit (m = -inf)
          l *= corr;
          if (t > 0) {
            // rescale the running output once its last update O_{g-1} is done
            if (!wait_o(g - 1, 61)) { ok = false; break; }
            fence_after();
#pragma unroll 1
            for (int half = 0; half < 2; ++half) {
              uint32_t ov[32];
              tmem_ld32(trow + ocol + 32 * half, ov);
#pragma unroll
              for (int q = 0; q < 32; ++q) ov[q] = __float_as_uint(__uint_as_float(ov[q]) * corr);
              tmem_st32(trow + ocol + 32 * half, ov);
            }
          }
          m = mn;
        }
        // P packed in place: the pair (2q, 2q+1) goes to v[q], already read
        // exp2 argument s*c - m and the row sum in two-lane FP32 (four packed
        // partial sums = eight independent chains)
        const uint64_t c2 = f2splat(c), nm2 = f2splat(-m);
        uint64_t s2[4] = {0ull, 0ull, 0ull, 0ull};
#pragma unroll
        for (int q = 0; q < 64; q += 2) {
          float a0, a1;
          f2unpack(fma2(f2pack(__uint_as_float(v[q]), __uint_as_float(v[q + 1])), c2, nm2), a0, a1);
          const float p0 = ex2_approx(a0), p1 = ex2_approx(a1);
          s2[(q >> 1) & 3] = add2(s2[(q >> 1) & 3], f2pack(p0, p1));
          __nv_bfloat162 b = __floats2bfloat162_rn(p0, p1);
          v[q >> 1] = *reinterpret_cast<uint32_t*>(&b);
        }
        float sl[8];
        f2unpack(add2(s2[0], s2[1]), sl[0], sl[1]);
        f2unpack(add2(s2[2], s2[3]), sl[2], sl[3]);
        l += (sl[0] + sl[1]) + (sl[2] + sl[3]);
        if (!zero_v_tail()) { ok = false; break; }
        // P_g goes to TMEM buffer g&1: O += P_{g-2} V_{g-2} has read it, since
        // it completed before S_g (issue order), which these warps waited for
        tmem_st32(trow + kColP + 32u * (uint32_t)(g & 1), *reinterpret_cast<uint32_t(*)[32]>(&v[0]));
        fence_before();
        mbar_arrive(bar(kBarPFull + (g & 1)));
      }
      if (!ok) break;
      if (!live) continue;
      // epilogue: O_{g-1} is this unit's last update (the next unit's first
      // O MMA waits for P, which these warps write only after this read)
      if (!wait_o(g - 1, 63)) { ok = false; break; }
      fence_after();
      uint32_t v[64];
      tmem_ld64(trow + ocol, v);
      // rows of this warp inside the sequence (at least one: the warp is live)
      const int rows_here = min(32, w.L - (w.q0 + sub * 32));
      uint8_t* stg = smem + kOffStg + sub * kStgBytes;
      const size_t row_base = (size_t)(w.row0 + w.q0 + sub * 32);
      if (OUT8) {
        // 64-byte rows: 32 rows x 4 pieces of 16 bytes, one pass; piece c of row
        // r sits at slot c ^ ((r >> 1) & 3) (conflict-free both ways)
        const uint64_t inv2 = f2splat(p.out_inv_scale / l);
        // O / l times the output scale in two-lane FP32, rounded to E4M3 pairs
        auto e4m3_pair = [&](int q) -> uint32_t {
          float a0, a1;
          f2unpack(mul2(f2pack(__uint_as_float(v[q]), __uint_as_float(v[q + 1])), inv2), a0, a1);
          return e4m3x2(a0, a1);
        };
#pragma unroll
        for (int q = 0; q < 64; q += 16) {
          uint4 x;
          uint32_t* xw = reinterpret_cast<uint32_t*>(&x);
#pragma unroll
          for (int k = 0; k < 4; ++k) xw[k] = e4m3_pair(q + 4 * k) | (e4m3_pair(q + 4 * k + 2) << 16);
          *reinterpret_cast<uint4*>(stg + lane * 64 + (((q >> 4) ^ ((lane >> 1) & 3)) << 4)) = x;
        }
        __syncwarp();
        uint8_t* o = static_cast<uint8_t*>(p.out) + w.h * 64;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int rr = (lane >> 2) + 8 * j, c = lane & 3;
          const uint4 x = *reinterpret_cast<const uint4*>(stg + rr * 64 + ((c ^ ((rr >> 1) & 3)) << 4));
          if (rr < rows_here) *reinterpret_cast<uint4*>(o + (row_base + rr) * d + c * 16) = x;
        }
        __syncwarp();
      } else {
        // 128-byte rows: every lane converts its row at once (O / l in two-lane
        // FP32, rounded to BF16 pairs), then two passes of 16 rows x 8 pieces
        // through the staging buffer; piece c of row r sits at slot c ^ (r & 7)
        const uint64_t inv2 = f2splat(1.f / l);
        uint32_t pk[32];
#pragma unroll
        for (int q = 0; q < 64; q += 2) {
          float a0, a1;
          f2unpack(mul2(f2pack(__uint_as_float(v[q]), __uint_as_float(v[q + 1])), inv2), a0, a1);
          __nv_bfloat162 b = __floats2bfloat162_rn(a0, a1);
          pk[q >> 1] = *reinterpret_cast<uint32_t*>(&b);
        }
        __nv_bfloat16* o = static_cast<__nv_bfloat16*>(p.out) + w.h * 64;
#pragma unroll
        for (int pass = 0; pass < 2; ++pass) {
          if ((lane >> 4) == pass) {
#pragma unroll
            for (int c = 0; c < 8; ++c)
              *reinterpret_cast<uint4*>(stg + (lane & 15) * 128 + ((c ^ (lane & 7)) << 4)) =
                  make_uint4(pk[4 * c], pk[4 * c + 1], pk[4 * c + 2], pk[4 * c + 3]);
          }
          __syncwarp();
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int rr = (lane >> 3) + 4 * j, c = lane & 7;
            const uint4 x = *reinterpret_cast<const uint4*>(stg + rr * 128 + ((c ^ (rr & 7)) << 4));
            const int row = pass * 16 + rr;
            if (row < rows_here) *reinterpret_cast<uint4*>(o + (row_base + row) * d + c * 8) = x;
          }
          __syncwarp();
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 2) {
    __syncwarp();
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

}  // namespace atc

namespace {
// Set once per process / device; concurrent callers write the same values.
std::atomic<PFN_cuTensorMapEncodeTiled_v12000> g_enc{nullptr};
std::atomic<bool> g_attn_attr_set[64] = {};
std::atomic<int> g_attn_sms[64] = {};

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

void attention_items(const int32_t* seq_start, const int32_t* seq_len, int32_t n_seq, std::vector<int32_t>& items) {
  // longest sequences first: CTAs take units round-robin, and a descending
  // cost order evens out their totals (the q-tiles of one sequence stay
  // adjacent, so its K and V rows are read by CTAs working at the same time)
  std::vector<int32_t> order(n_seq > 0 ? n_seq : 0);
  for (int32_t s = 0; s < n_seq; ++s) order[s] = s;
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return seq_len[a] > seq_len[b]; });
  for (int32_t s : order)
    for (int32_t q0 = 0; q0 < seq_len[s]; q0 += atc::kQ) {
      items.push_back(seq_start[s]);
      items.push_back(seq_len[s] | (q0 << 16));
    }
}

namespace {
as_status attention_tc_launch(bool out8, const __nv_bfloat16* qkv, void* out, float out_scale, const int32_t* items,
                              int32_t n_items, int32_t max_len,
                              int64_t rows, int32_t d_model, int32_t n_heads, DevError* err, cudaStream_t st) {
  if (n_items == 0 || max_len == 0 || rows == 0) return AS_OK;
  if (d_model != n_heads * 64 || d_model % 64 || max_len > 4096 || rows > (1ll << 31) - 8 ||
      (reinterpret_cast<uintptr_t>(qkv) & 15) || (reinterpret_cast<uintptr_t>(out) & 15) ||
      (reinterpret_cast<uintptr_t>(items) & 7)) {
    set_k_error("attention_tcgen05: head dim 64, sequences <= 4096 tokens, 16-byte aligned buffers, 8-byte aligned items");
    return AS_ERR_ARG;
  }
  if ((int64_t)n_items * n_heads > 0x7FFFFFFFll - 65536) {
    set_k_error("attention_tcgen05: too many work items in one batch");
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
    AS_CUDA_OK(cudaFuncSetAttribute(atc::attn_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    atc::kSmemAlloc));
    AS_CUDA_OK(cudaFuncSetAttribute(atc::attn_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    atc::kSmemAlloc));
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    g_attn_sms[dev & 63].store(n > 0 ? n : 148);
    g_attn_attr_set[dev & 63].store(true);
  }
  CUtensorMap tmQ, tmKV;
  as_status s = make_map_bf16(&tmQ, qkv, (uint64_t)rows, 3ull * d_model, 3ull * d_model, 64, atc::kQ);
  if (s == AS_OK) s = make_map_bf16(&tmKV, qkv, (uint64_t)rows, 3ull * d_model, 3ull * d_model, 64, atc::kKT);
  if (s != AS_OK) return s;
  atc::Params p;
  p.items = reinterpret_cast<const int2*>(items);
  p.n_items = n_items;
  p.out = out;
  p.out_inv_scale = out8 ? 1.0f / out_scale : 1.0f;
  p.d = d_model;
  p.n_heads = n_heads;
  p.err = err;
  const int64_t units = (int64_t)n_items * n_heads;
  const int grid = (int)std::min<int64_t>(units, 2ll * g_attn_sms[dev & 63].load());  // two CTAs per SM, persistent
  if (out8)
    atc::attn_tc_kernel<true><<<grid, atc::kThreads, atc::kSmemAlloc, st>>>(tmQ, tmKV, p);
  else
    atc::attn_tc_kernel<false><<<grid, atc::kThreads, atc::kSmemAlloc, st>>>(tmQ, tmKV, p);
  count_launch();
  AS_CUDA_OK(cudaGetLastError());
  return AS_OK;
}

}  // namespace

as_status attention_tcgen05(const __nv_bfloat16* qkv, __nv_bfloat16* out, const int32_t* items, int32_t n_items,
                            int32_t max_len, int64_t rows, int32_t d_model, int32_t n_heads, DevError* err,
                            cudaStream_t st) {
  return attention_tc_launch(false, qkv, out, 1.0f, items, n_items, max_len, rows, d_model, n_heads, err, st);
}

as_status attention_tcgen05_e4m3(const __nv_bfloat16* qkv, uint8_t* out, float out_scale, const int32_t* items,
                                 int32_t n_items, int32_t max_len, int64_t rows, int32_t d_model, int32_t n_heads,
                                 DevError* err, cudaStream_t st) {
  if (!(out_scale > 0.f)) {
    set_k_error("attention_tcgen05_e4m3: out_scale must be positive");
    return AS_ERR_ARG;
  }
  return attention_tc_launch(true, qkv, out, out_scale, items, n_items, max_len, rows, d_model, n_heads, err, st);
}

}  // namespace as
