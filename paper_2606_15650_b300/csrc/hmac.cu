// HMAC-SHA256 pseudonym digests (AnonShield §2 stage (3)).
//
// SHA-256 follows FIPS 180-4; HMAC follows RFC 2104 (block 64 bytes, keys
// longer than a block are hashed first). The key is preprocessed once per
// call into the two midstates after absorbing K^ipad and K^opad, so each
// entity costs ceil((len + 9) / 64) inner compressions plus one outer. One
// thread per entity occurrence; the message is read straight from the
// record bytes. The round constants are derived at start-up from their
// definition (fractional bits of cube / square roots of the first primes)
// with exact integer arithmetic.
#include <mutex>

#include "stages.cuh"

namespace as {

__constant__ uint32_t c_K[64];
__constant__ uint32_t c_H0[8];

namespace {

// floor(x^(1/r)) for x < 2^120, r in {2, 3}, by bisection on 128-bit integers.
uint64_t iroot_u128(unsigned __int128 x, int r) {
  uint64_t lo = 0, hi = 1ull << 41;
  while (hi - lo > 1) {
    uint64_t mid = lo + (hi - lo) / 2;
    unsigned __int128 p = (unsigned __int128)mid * mid;
    if (r == 3) p *= mid;
    if (p <= x) lo = mid; else hi = mid;
  }
  return lo;
}

void derive_constants(uint32_t K[64], uint32_t H0[8]) {
  int primes[64];
  int n = 0;
  for (int c = 2; n < 64; ++c) {
    bool p = true;
    for (int d = 2; d * d <= c; ++d)
      if (c % d == 0) { p = false; break; }
    if (p) primes[n++] = c;
  }
  for (int i = 0; i < 64; ++i) K[i] = (uint32_t)iroot_u128((unsigned __int128)primes[i] << 96, 3);
  for (int i = 0; i < 8; ++i) H0[i] = (uint32_t)iroot_u128((unsigned __int128)primes[i] << 64, 2);
}

int g_const_device_mask = 0;
std::mutex g_const_mu;

}  // namespace

void sha256_init_constants() {
  // __constant__ memory is per device: upload on each device first used.
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_const_mu);
  if (dev < 31 && (g_const_device_mask >> dev) & 1) return;
  uint32_t K[64], H0[8];
  derive_constants(K, H0);
  cudaMemcpyToSymbol(c_K, K, sizeof(K));
  cudaMemcpyToSymbol(c_H0, H0, sizeof(H0));
  if (dev < 31) g_const_device_mask |= 1 << dev;
}

__device__ __forceinline__ uint32_t rotr(uint32_t x, int n) { return __funnelshift_r(x, x, n); }

__device__ void sha256_compress(uint32_t st[8], const uint32_t w_in[16]) {
  uint32_t w[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) w[i] = w_in[i];
  uint32_t a = st[0], b = st[1], c = st[2], d = st[3], e = st[4], f = st[5], g = st[6], h = st[7];
#pragma unroll
  for (int t = 0; t < 64; ++t) {
    uint32_t wt;
    if (t < 16) {
      wt = w[t];
    } else {
      uint32_t w15 = w[(t - 15) & 15], w2 = w[(t - 2) & 15];
      uint32_t s0 = rotr(w15, 7) ^ rotr(w15, 18) ^ (w15 >> 3);
      uint32_t s1 = rotr(w2, 17) ^ rotr(w2, 19) ^ (w2 >> 10);
      wt = w[t & 15] + s0 + w[(t - 7) & 15] + s1;
      w[t & 15] = wt;
    }
    uint32_t S1 = rotr(e, 6) ^ rotr(e, 11) ^ rotr(e, 25);
    uint32_t ch = (e & f) ^ (~e & g);
    uint32_t t1 = h + S1 + ch + c_K[t] + wt;
    uint32_t S0 = rotr(a, 2) ^ rotr(a, 13) ^ rotr(a, 22);
    uint32_t mj = (a & b) ^ (a & c) ^ (b & c);
    uint32_t t2 = S0 + mj;
    h = g; g = f; f = e; e = d + t1; d = c; c = b; b = a; a = t1 + t2;
  }
  st[0] += a; st[1] += b; st[2] += c; st[3] += d; st[4] += e; st[5] += f; st[6] += g; st[7] += h;
}

// Hash `len` message bytes that follow `prefix_blocks` already-absorbed
// 64-byte blocks, starting from state `st` (SHA-256 padding appended).
__device__ void sha256_tail(uint32_t st[8], const uint8_t* msg, uint32_t len, uint64_t prefix_blocks) {
  uint64_t total_bits = (prefix_blocks * 64 + len) * 8;
  uint32_t nblocks = (len + 9 + 63) / 64;
  for (uint32_t bk = 0; bk < nblocks; ++bk) {
    uint32_t w[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      uint32_t v = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        uint32_t p = bk * 64 + i * 4 + j;
        uint32_t byte = p < len ? msg[p] : (p == len ? 0x80u : 0u);
        v = (v << 8) | byte;
      }
      w[i] = v;
    }
    if (bk == nblocks - 1) {
      w[14] = (uint32_t)(total_bits >> 32);
      w[15] = (uint32_t)total_bits;
    }
    sha256_compress(st, w);
  }
}

__global__ void hmac_key_setup_kernel(const uint8_t* key, uint32_t key_len, uint32_t* key_state) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  uint8_t k[64];
  for (int i = 0; i < 64; ++i) k[i] = 0;
  if (key_len > 64) {
    uint32_t st[8];
    for (int i = 0; i < 8; ++i) st[i] = c_H0[i];
    sha256_tail(st, key, key_len, 0);
    for (int i = 0; i < 8; ++i)
      for (int j = 0; j < 4; ++j) k[4 * i + j] = (uint8_t)(st[i] >> (24 - 8 * j));
  } else {
    for (uint32_t i = 0; i < key_len; ++i) k[i] = key[i];
  }
  for (int pass = 0; pass < 2; ++pass) {
    uint8_t pad = pass == 0 ? 0x36 : 0x5c;
    uint32_t w[16];
    for (int i = 0; i < 16; ++i) {
      uint32_t v = 0;
      for (int j = 0; j < 4; ++j) v = (v << 8) | (uint32_t)(k[4 * i + j] ^ pad);
      w[i] = v;
    }
    uint32_t st[8];
    for (int i = 0; i < 8; ++i) st[i] = c_H0[i];
    sha256_compress(st, w);
    for (int i = 0; i < 8; ++i) key_state[pass * 8 + i] = st[i];
  }
}

void launch_hmac_key_setup(const uint8_t* key, uint32_t key_len, uint32_t* key_state, cudaStream_t st) {
  hmac_key_setup_kernel<<<1, 32, 0, st>>>(key, key_len, key_state);
  count_launch();
}

__global__ void hmac_spans_kernel(const uint8_t* __restrict__ bytes, const uint32_t* __restrict__ sp_start,
                                  const uint32_t* __restrict__ sp_len, const uint32_t* n_dev,
                                  const uint32_t* __restrict__ key_state, uint32_t* __restrict__ digests) {
  uint32_t n = *n_dev;
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    uint32_t inner[8], outer[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      inner[i] = key_state[i];
      outer[i] = key_state[8 + i];
    }
    sha256_tail(inner, bytes + sp_start[k], sp_len[k], 1);
    uint32_t w[16];
#pragma unroll
    for (int i = 0; i < 8; ++i) w[i] = inner[i];
    w[8] = 0x80000000u;
#pragma unroll
    for (int i = 9; i < 15; ++i) w[i] = 0;
    w[15] = (64 + 32) * 8;
    sha256_compress(outer, w);
#pragma unroll
    for (int i = 0; i < 8; ++i) digests[(size_t)k * 8 + i] = outer[i];
  }
}

// ok[i] = 1 when map slot i holds an entry whose stored digest is the HMAC of
// its stored original under the key (re-identification trusts only those).
__global__ void hmac_verify_slots_kernel(MapView m, const uint32_t* __restrict__ key_state, uint8_t* __restrict__ ok) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i <= m.mask; i += (uint64_t)gridDim.x * blockDim.x) {
    const MapSlot& s = m.slots[i];
    uint8_t good = 0;
    if (s.key != 0 && s.arena_off != ~0ull) {
      uint32_t inner[8], outer[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        inner[k] = key_state[k];
        outer[k] = key_state[8 + k];
      }
      sha256_tail(inner, m.arena + s.arena_off, s.len, 1);
      uint32_t w[16];
#pragma unroll
      for (int k = 0; k < 8; ++k) w[k] = inner[k];
      w[8] = 0x80000000u;
#pragma unroll
      for (int k = 9; k < 15; ++k) w[k] = 0;
      w[15] = (64 + 32) * 8;
      sha256_compress(outer, w);
      good = 1;
#pragma unroll
      for (int k = 0; k < 8; ++k) good &= outer[k] == s.digest[k];
    }
    ok[i] = good;
  }
}

void launch_hmac_verify_slots(MapView m, const uint32_t* key_state, uint8_t* ok, cudaStream_t st) {
  hmac_verify_slots_kernel<<<grid_1d(m.mask + 1, 128, 148 * 32), 128, 0, st>>>(m, key_state, ok);
  count_launch();
}

void launch_hmac_spans(const uint8_t* bytes, const uint32_t* sp_start, const uint32_t* sp_len, const uint32_t* n_dev,
                       uint32_t cap, const uint32_t* key_state, uint32_t* digests, cudaStream_t st) {
  if (cap == 0) return;
  hmac_spans_kernel<<<grid_1d(cap, 128, 148 * 32), 128, 0, st>>>(bytes, sp_start, sp_len, n_dev, key_state, digests);
  count_launch();
}

}  // namespace as
