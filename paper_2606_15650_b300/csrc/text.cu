// Byte tokenizer and pattern recognizers (AnonShield §2 stage (2)).
//
// Tokenizer: maximal runs of [0-9A-Za-z] are split greedily into the longest
// vocabulary strings (2..12 bytes), falling back to single bytes; every other
// byte is a token of its own (id = byte + 1). One thread walks each run; the
// starts are then compacted in byte order by a prefix sum, so token order is
// byte order and every record owns a contiguous token range.
//
// Recognizers: a word is a maximal run of [A-Za-z0-9.:-]; trailing '.', '-'
// and a ':' that does not close a final '::' are stripped; the whole word is
// then tested as MAC, IPv6, IPv4(:port), CVE id, host name(:port), first
// match wins, port excluded from the span. One thread per word start.
#include "scan.cuh"
#include "stages.cuh"

namespace as {

__device__ __forceinline__ bool rs_bit(const uint32_t* rs, uint32_t i) { return (rs[i >> 5] >> (i & 31)) & 1u; }

__global__ void mark_record_starts_kernel(const uint64_t* offsets, uint64_t n, uint32_t N, uint32_t* rs) {
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < n; r += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t o = offsets[r];
    if (o < N) atomicOr(&rs[o >> 5], 1u << (o & 31));
  }
}

void launch_mark_record_starts(const uint64_t* offsets, uint64_t n, uint32_t N, uint32_t* rs, cudaStream_t st) {
  cudaMemsetAsync(rs, 0, ((size_t)N / 32 + 1) * 4, st);
  if (n == 0) return;
  mark_record_starts_kernel<<<grid_1d(n, 256, 65535), 256, 0, st>>>(offsets, n, N, rs);
  count_launch();
}

__device__ __forceinline__ uint32_t vocab_lookup(VocabTable vt, const uint32_t b[kMaxPiece], uint32_t len) {
  uint32_t w[3] = {0, 0, 0};
#pragma unroll
  for (int k = 0; k < kMaxPiece; ++k)
    if ((uint32_t)k < len) w[k >> 2] |= b[k] << (8 * (k & 3));
  uint32_t h = vocab_hash(w[0], w[1], w[2], len) & vt.mask;
  for (uint32_t probe = 0; probe <= vt.mask; ++probe) {
    uint4 s = __ldg(&vt.slots[h]);
    if (s.w == 0) return 0;
    if ((s.w & 0xFFFFu) == len && s.x == w[0] && s.y == w[1] && s.z == w[2]) return s.w >> 16;
    h = (h + 1) & vt.mask;
  }
  return 0;
}

__global__ void tokenize_mark_kernel(const uint8_t* __restrict__ bytes, uint32_t N, const uint32_t* __restrict__ rs,
                                     VocabTable vt, uint16_t* __restrict__ tok_at) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    uint32_t c = bytes[i];
    if (!is_alnum(c)) {
      tok_at[i] = (uint16_t)(c + 1);
      continue;
    }
    if (!rs_bit(rs, i) && i > 0 && is_alnum(bytes[i - 1])) continue;  // written by the run's first thread
    uint32_t p = i;
    while (true) {
      uint32_t b[kMaxPiece];
      uint32_t avail = 0;
#pragma unroll
      for (int k = 0; k < kMaxPiece; ++k) b[k] = 0;
      for (uint32_t k = 0; k < (uint32_t)kMaxPiece; ++k) {
        uint32_t q = p + k;
        if (q >= N) break;
        uint32_t ch = bytes[q];
        if (!is_alnum(ch) || (k > 0 && rs_bit(rs, q))) break;
        b[k] = ch;
        avail = k + 1;
      }
      uint32_t take = 1, id = b[0] + 1;
      for (uint32_t L = avail; L >= 2; --L) {
        uint32_t v = vocab_lookup(vt, b, L);
        if (v) { take = L; id = v; break; }
      }
      tok_at[p] = (uint16_t)id;
      for (uint32_t k = 1; k < take; ++k) tok_at[p + k] = 0;
      p += take;
      if (p >= N || !is_alnum(bytes[p]) || rs_bit(rs, p)) break;
    }
  }
}

void launch_tokenize_mark(const uint8_t* bytes, uint32_t N, const uint32_t* rs, VocabTable vt, uint16_t* tok_at,
                          cudaStream_t st) {
  if (N == 0) return;
  tokenize_mark_kernel<<<grid_1d(N, 256, 148 * 64), 256, 0, st>>>(bytes, N, rs, vt, tok_at);
  count_launch();
}

__global__ void tokenize_emit_kernel(const uint16_t* __restrict__ tok_at, const uint32_t* __restrict__ pos, uint32_t N,
                                     int32_t* __restrict__ ids, uint32_t* __restrict__ off) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    uint32_t v = tok_at[i];
    if (v) {
      uint32_t t = pos[i];
      ids[t] = (int32_t)v;
      off[t] = i;
    }
  }
}

void launch_tokenize_emit(const uint16_t* tok_at, const uint32_t* pos, uint32_t N, int32_t* ids, uint32_t* off,
                          cudaStream_t st) {
  if (N == 0) return;
  tokenize_emit_kernel<<<grid_1d(N, 256, 148 * 64), 256, 0, st>>>(tok_at, pos, N, ids, off);
  count_launch();
}

__global__ void token_lengths_kernel(const uint32_t* __restrict__ off, uint32_t T, uint32_t N, uint32_t* __restrict__ len) {
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x)
    len[t] = (t + 1 < T ? off[t + 1] : N) - off[t];
}

void launch_token_lengths(const uint32_t* off, uint32_t T, uint32_t N, uint32_t* len, cudaStream_t st) {
  if (T == 0) return;
  token_lengths_kernel<<<grid_1d(T, 256, 148 * 64), 256, 0, st>>>(off, T, N, len);
  count_launch();
}

__global__ void record_token_offsets_kernel(const uint64_t* offsets, uint64_t n, const uint32_t* pos, uint32_t N,
                                            const uint32_t* total_T, uint64_t* rec_tok) {
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r <= n; r += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t o = offsets[r];
    rec_tok[r] = o < N ? pos[o] : *total_T;
  }
}

void launch_record_token_offsets(const uint64_t* offsets, uint64_t n, const uint32_t* pos, uint32_t N,
                                 const uint32_t* total_T, uint64_t* rec_tok, cudaStream_t st) {
  record_token_offsets_kernel<<<grid_1d(n + 1, 256, 65535), 256, 0, st>>>(offsets, n, pos, N, total_T, rec_tok);
  count_launch();
}

// ---------------------------------------------------------------- recognizers

__device__ __forceinline__ bool in_word(uint32_t c) { return is_alnum(c) || c == '.' || c == ':' || c == '-'; }
__device__ __forceinline__ bool is_digit(uint32_t c) { return c - '0' < 10u; }
__device__ __forceinline__ bool is_alpha(uint32_t c) { return (c | 0x20u) - 'a' < 26u; }
__device__ __forceinline__ bool is_hex(uint32_t c) { return is_digit(c) || (c | 0x20u) - 'a' < 6u; }

constexpr uint8_t kTypeIP = 1, kTypeHost = 2, kTypeCVE = 3, kTypeMAC = 4;

__device__ bool rx_is_mac(const uint8_t* w, uint32_t n) {
  if (n != 17) return false;
  uint32_t sep = w[2];
  if (sep != ':' && sep != '-') return false;
  for (int g = 0; g < 6; ++g) {
    if (!is_hex(w[3 * g]) || !is_hex(w[3 * g + 1])) return false;
    if (g < 5 && w[3 * g + 2] != sep) return false;
  }
  return true;
}

// Groups of 1..4 hex digits separated by single ':' over w[0..n); 0 when n == 0; -1 if invalid.
__device__ int rx_hex_groups(const uint8_t* w, uint32_t n) {
  if (n == 0) return 0;
  int groups = 0;
  uint32_t run = 0;
  for (uint32_t i = 0; i <= n; ++i) {
    if (i == n || w[i] == ':') {
      if (run < 1 || run > 4) return -1;
      ++groups;
      run = 0;
    } else {
      if (!is_hex(w[i])) return -1;
      ++run;
    }
  }
  return groups;
}

__device__ bool rx_is_ipv6(const uint8_t* w, uint32_t n) {
  int dbl = 0;
  uint32_t dpos = 0;
  bool colon = false;
  for (uint32_t i = 0; i < n; ++i) {
    if (w[i] != ':') continue;
    colon = true;
    if (i + 1 < n && w[i + 1] == ':') {
      if (i + 2 < n && w[i + 2] == ':') return false;  // ":::"
      if (dbl == 0) dpos = i;
      ++dbl;
      ++i;
    }
  }
  if (!colon) return false;
  if (dbl == 0) return rx_hex_groups(w, n) == 8;
  if (dbl != 1) return false;
  int l = rx_hex_groups(w, dpos), r = rx_hex_groups(w + dpos + 2, n - dpos - 2);
  return l >= 0 && r >= 0 && l + r <= 7;
}

// ':' followed by 1..5 digits exactly filling w[at..n); true also when at == n.
__device__ bool rx_port_ok(const uint8_t* w, uint32_t at, uint32_t n) {
  if (at == n) return true;
  uint32_t k = n - at;
  if (w[at] != ':' || k < 2 || k > 6) return false;
  for (uint32_t i = at + 1; i < n; ++i)
    if (!is_digit(w[i])) return false;
  return true;
}

__device__ uint32_t rx_core_len(const uint8_t* w, uint32_t n) {
  for (uint32_t i = 0; i < n; ++i)
    if (w[i] == ':') return i;
  return n;
}

__device__ uint32_t rx_ipv4_len(const uint8_t* w, uint32_t n) {
  uint32_t core = rx_core_len(w, n);
  uint32_t parts = 0, digits = 0, val = 0;
  bool lead0 = false;
  for (uint32_t i = 0; i <= core; ++i) {
    if (i == core || w[i] == '.') {
      if (digits < 1 || digits > 3 || (lead0 && digits > 1) || val > 255) return 0;
      ++parts;
      digits = 0;
      val = 0;
      lead0 = false;
    } else {
      if (!is_digit(w[i])) return 0;
      if (digits == 0) lead0 = w[i] == '0';
      val = val * 10 + (w[i] - '0');
      ++digits;
      if (digits > 3) return 0;
    }
  }
  if (parts != 4) return 0;
  return rx_port_ok(w, core, n) ? core : 0;
}

__device__ bool rx_is_cve(const uint8_t* w, uint32_t n) {
  if (n < 13 || w[0] != 'C' || w[1] != 'V' || w[2] != 'E' || w[3] != '-') return false;
  for (int i = 4; i < 8; ++i)
    if (!is_digit(w[i])) return false;
  if (w[8] != '-') return false;
  for (uint32_t i = 9; i < n; ++i)
    if (!is_digit(w[i])) return false;
  return true;
}

__device__ uint32_t rx_host_len(const uint8_t* w, uint32_t n) {
  uint32_t core = rx_core_len(w, n);
  if (!rx_port_ok(w, core, n) || core > 253) return 0;
  uint32_t labels = 0, start = 0;
  bool last_alpha = true;
  for (uint32_t i = 0; i <= core; ++i) {
    if (i == core || w[i] == '.') {
      uint32_t L = i - start;
      if (L < 1 || L > 63) return 0;
      if (w[start] == '-' || w[i - 1] == '-') return 0;
      ++labels;
      last_alpha = L >= 2;
      for (uint32_t k = start; k < i; ++k) last_alpha = last_alpha && is_alpha(w[k]);
      start = i + 1;
    } else if (!(is_alnum(w[i]) || w[i] == '-')) {
      return 0;
    }
  }
  return (labels >= 2 && last_alpha) ? core : 0;
}

__global__ void recognize_mark_kernel(const uint8_t* __restrict__ bytes, uint32_t N, const uint32_t* __restrict__ rs,
                                      uint32_t* __restrict__ rx_len, uint8_t* __restrict__ rx_type) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    uint32_t len = 0;
    uint8_t type = 0;
    uint32_t c = bytes[i];
    if (in_word(c) && (i == 0 || rs_bit(rs, i) || !in_word(bytes[i - 1]))) {
      uint32_t e = i + 1;
      while (e < N && in_word(bytes[e]) && !rs_bit(rs, e)) ++e;
      while (e > i) {
        uint32_t t = bytes[e - 1];
        if (t == '.' || t == '-') --e;
        else if (t == ':' && !(e >= i + 2 && bytes[e - 2] == ':')) --e;
        else break;
      }
      const uint8_t* w = bytes + i;
      uint32_t n = e - i;
      if (n > 0) {
        uint32_t k;
        if (rx_is_mac(w, n)) { len = n; type = kTypeMAC; }
        else if (rx_is_ipv6(w, n)) { len = n; type = kTypeIP; }
        else if ((k = rx_ipv4_len(w, n)) > 0) { len = k; type = kTypeIP; }
        else if (rx_is_cve(w, n)) { len = n; type = kTypeCVE; }
        else if ((k = rx_host_len(w, n)) > 0) { len = k; type = kTypeHost; }
      }
    }
    rx_len[i] = len;
    rx_type[i] = type;
  }
}

void launch_recognize_mark(const uint8_t* bytes, uint32_t N, const uint32_t* rs, uint32_t* rx_len, uint8_t* rx_type,
                           cudaStream_t st) {
  if (N == 0) return;
  recognize_mark_kernel<<<grid_1d(N, 256, 148 * 64), 256, 0, st>>>(bytes, N, rs, rx_len, rx_type);
  count_launch();
}

__global__ void recognize_emit_kernel(const uint32_t* __restrict__ rx_len, const uint8_t* __restrict__ rx_type,
                                      const uint32_t* __restrict__ pos, uint32_t N, uint32_t* sp_start,
                                      uint32_t* sp_len, uint8_t* sp_type) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    uint8_t t = rx_type[i];
    if (t) {
      uint32_t k = pos[i];
      sp_start[k] = i;
      sp_len[k] = rx_len[i];
      sp_type[k] = t;
    }
  }
}

void launch_recognize_emit(const uint32_t* rx_len, const uint8_t* rx_type, const uint32_t* pos, uint32_t N,
                           uint32_t* sp_start, uint32_t* sp_len, uint8_t* sp_type, cudaStream_t st) {
  if (N == 0) return;
  recognize_emit_kernel<<<grid_1d(N, 256, 148 * 64), 256, 0, st>>>(rx_len, rx_type, pos, N, sp_start, sp_len, sp_type);
  count_launch();
}

}  // namespace as
