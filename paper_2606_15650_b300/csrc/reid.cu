// Controlled re-identification (AnonShield §2 stage (4): the mapping lets an
// administrator holding the database and the key reverse the pseudonyms).
//
// A pseudonym "[NAME_h]" (h = L lower-case hex characters, NAME a type name,
// inside one record) resolves to the map entry of that type whose digest
// begins with h, when exactly one does and that entry verifies under the key
// (hmac_verify_slots_kernel). The entries are first indexed by (type, the
// first min(4L, 56) digest bits) in an open-addressing table whose value is
// the map slot, or kReidAmbiguous when two entries share the key. Then one
// thread per '[' parses a pseudonym and looks it up; resolved ones become
// spans, and the forward substitution's copy / offsets kernels write the
// output, with reid_replace_kernel copying each entry's original bytes in
// place of its pseudonym.
#include "scan.cuh"
#include "stages.cuh"

namespace as {

__device__ __forceinline__ uint64_t reid_home(unsigned long long k, uint64_t mask) {
  return ((k * 0x9E3779B97F4A7C15ull) >> 17) & mask;
}

// first p (<= 56) bits of a digest
__device__ __forceinline__ unsigned long long digest_prefix(const uint32_t* d, uint32_t p) {
  const unsigned long long top56 = ((unsigned long long)d[0] << 24) | (d[1] >> 8);
  return top56 >> (56 - p);
}

__global__ void reid_index_kernel(MapView m, uint32_t p_bits, ReidTab tab) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i <= m.mask; i += (uint64_t)gridDim.x * blockDim.x) {
    const MapSlot& s = m.slots[i];
    if (s.key == 0) continue;
    const unsigned long long k = ((unsigned long long)(s.type & 0xFFu) << 56) | digest_prefix(s.digest, p_bits);
    uint64_t h = reid_home(k, tab.mask);
    for (uint64_t probe = 0; probe <= tab.mask; ++probe) {
      const unsigned long long cur = atomicCAS(&tab.key[h], 0ull, k);
      if (cur == 0) {
        atomicCAS(&tab.val[h], kReidEmpty, (uint32_t)i);  // fails only when a twin already marked it ambiguous
        break;
      }
      if (cur == k) {
        atomicExch(&tab.val[h], kReidAmbiguous);
        break;
      }
      h = (h + 1) & tab.mask;
    }
  }
}

void launch_reid_index(MapView m, uint32_t p_bits, ReidTab tab, cudaStream_t st) {
  reid_index_kernel<<<grid_1d(m.mask + 1, 256, 148 * 32), 256, 0, st>>>(m, p_bits, tab);
  count_launch();
}

__device__ __forceinline__ uint32_t hex_val(uint32_t c) { return c - '0' < 10u ? c - '0' : c - 'a' < 6u ? c - 'a' + 10 : 16u; }

// plen[i] = pseudonym length and pslot[i] = its map slot for each resolved
// pseudonym starting at byte i, else 0; ctr[0..3] += pseudonyms, resolved,
// ambiguous, unverified.
__global__ void reid_mark_kernel(const uint8_t* __restrict__ bytes, uint32_t N, const uint32_t* __restrict__ rs,
                                 const char* __restrict__ names, const uint32_t* __restrict__ name_off,
                                 uint32_t n_types, uint32_t L, ReidTab tab, MapView m, const uint8_t* __restrict__ ok,
                                 uint32_t* __restrict__ plen, uint32_t* __restrict__ pslot, uint8_t* __restrict__ flag,
                                 unsigned long long* ctr) {
  const uint32_t p_hex = L < 14 ? L : 14;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    uint32_t len = 0, slot = 0;
    if (bytes[i] == '[') {
      for (uint32_t t = 1; t <= n_types; ++t) {
        const uint32_t a = name_off[t], nl = name_off[t + 1] - a;
        const uint64_t close = (uint64_t)i + 2 + nl + L;  // position of ']'
        if (close >= N) continue;
        bool match = true;
        for (uint32_t p = i + 1; p <= (uint32_t)close && match; ++p) {
          const uint32_t q = p - i - 1;  // offset inside "NAME_h]"
          const uint32_t c = bytes[p];
          if (rs_bit(rs, p)) match = false;
          else if (q < nl) match = c == (uint8_t)names[a + q];
          else if (q == nl) match = c == '_';
          else if (p < close) match = hex_val(c) < 16u;
          else match = c == ']';
        }
        if (!match) continue;
        atomicAdd(&ctr[0], 1ull);
        const uint8_t* h = bytes + i + 2 + nl;
        unsigned long long pre = 0;
        for (uint32_t k = 0; k < p_hex; ++k) pre = (pre << 4) | hex_val(h[k]);
        const unsigned long long key = ((unsigned long long)t << 56) | pre;
        uint32_t v = kReidEmpty;
        uint64_t e = reid_home(key, tab.mask);
        for (uint64_t probe = 0; probe <= tab.mask; ++probe) {
          const unsigned long long cur = tab.key[e];
          if (cur == 0) break;
          if (cur == key) {
            v = tab.val[e];
            break;
          }
          e = (e + 1) & tab.mask;
        }
        if (v == kReidAmbiguous) {
          atomicAdd(&ctr[2], 1ull);
        } else if (v != kReidEmpty) {
          const MapSlot& s = m.slots[v];
          bool same = s.type == t;
          for (uint32_t k = p_hex; k < L && same; ++k) same = hex_val(h[k]) == ((s.digest[k >> 3] >> (28 - 4 * (k & 7))) & 15u);
          if (same && !ok[v]) {
            atomicAdd(&ctr[3], 1ull);
          } else if (same) {
            atomicAdd(&ctr[1], 1ull);
            len = (uint32_t)(close - i + 1);
            slot = v;
          }
        }
        break;  // at most one type name fits at a position
      }
    }
    plen[i] = len;
    pslot[i] = slot;
    flag[i] = len != 0;
  }
}

void launch_reid_mark(const uint8_t* bytes, uint32_t N, const uint32_t* rs, const char* names, const uint32_t* name_off,
                      uint32_t n_types, uint32_t L, ReidTab tab, MapView m, const uint8_t* ok, uint32_t* plen,
                      uint32_t* pslot, uint8_t* flag, unsigned long long* ctr, cudaStream_t st) {
  if (N == 0) return;
  reid_mark_kernel<<<grid_1d(N, 256, 148 * 64), 256, 0, st>>>(bytes, N, rs, names, name_off, n_types, L, tab, m, ok,
                                                              plen, pslot, flag, ctr);
  count_launch();
}

__global__ void reid_emit_kernel(const uint32_t* __restrict__ plen, const uint32_t* __restrict__ pslot,
                                 const uint8_t* __restrict__ flag, const uint32_t* __restrict__ pos, uint32_t N,
                                 uint32_t* __restrict__ sp_s, uint32_t* __restrict__ sp_l, uint32_t* __restrict__ sp_k) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    if (flag[i]) {
      const uint32_t k = pos[i];
      sp_s[k] = i;
      sp_l[k] = plen[i];
      sp_k[k] = pslot[i];
    }
  }
}

void launch_reid_emit(const uint32_t* plen, const uint32_t* pslot, const uint8_t* flag, const uint32_t* pos, uint32_t N,
                      uint32_t* sp_s, uint32_t* sp_l, uint32_t* sp_k, cudaStream_t st) {
  if (N == 0) return;
  reid_emit_kernel<<<grid_1d(N, 256, 148 * 64), 256, 0, st>>>(plen, pslot, flag, pos, N, sp_s, sp_l, sp_k);
  count_launch();
}

// delta[k] = original length - pseudonym length for k < n; 0 up to cap.
__global__ void reid_delta_kernel(const uint32_t* __restrict__ sp_l, const uint32_t* __restrict__ sp_k, uint32_t n,
                                  MapView m, int64_t* __restrict__ delta, uint32_t cap) {
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < cap; k += gridDim.x * blockDim.x)
    delta[k] = k < n ? (int64_t)m.slots[sp_k[k]].len - (int64_t)sp_l[k] : 0;
}

void launch_reid_delta(const uint32_t* sp_l, const uint32_t* sp_k, uint32_t n, MapView m, int64_t* delta, uint32_t cap,
                       cudaStream_t st) {
  reid_delta_kernel<<<grid_1d(cap, 256, 148 * 64), 256, 0, st>>>(sp_l, sp_k, n, m, delta, cap);
  count_launch();
}

// One warp per resolved pseudonym copies the entry's original bytes.
__global__ void reid_replace_kernel(const uint32_t* __restrict__ sp_s, const uint32_t* __restrict__ sp_k, uint32_t n,
                                    const int64_t* __restrict__ shift, MapView m, uint8_t* __restrict__ out) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t k = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < n; k += nwarps) {
    const MapSlot& s = m.slots[sp_k[k]];
    uint8_t* o = out + ((int64_t)sp_s[k] + shift[k]);
    const uint8_t* src = m.arena + s.arena_off;
    for (uint32_t b = lane; b < s.len; b += 32) o[b] = src[b];
  }
}

void launch_reid_replace(const uint32_t* sp_s, const uint32_t* sp_k, uint32_t n, const int64_t* shift, MapView m,
                         uint8_t* out, cudaStream_t st) {
  if (n == 0) return;
  const uint64_t blocks = std::min<uint64_t>((n + 7) / 8, 148 * 32);
  reid_replace_kernel<<<(unsigned)blocks, 256, 0, st>>>(sp_s, sp_k, n, shift, m, out);
  count_launch();
}

}  // namespace as
