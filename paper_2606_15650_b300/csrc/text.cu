// Byte tokenizer and pattern recognizers (AnonShield §2 stage (2)).
//
// Tokenizer: maximal runs of [0-9A-Za-z] are split greedily into the longest
// vocabulary strings (2..12 bytes), falling back to single bytes; every other
// byte is a token of its own (id = byte + 1). A block collects the run
// starts of a tile and one thread walks each run, marking each token's id at
// its first byte and counting the tile's tokens; the tile counts are scanned,
// and one block per tile ranks its tokens in shared memory and writes the id
// / offset / length table in order. So token order is byte order and every
// record owns a contiguous token range. (as_tokenize_static keeps the scan +
// emit pair over a per-byte position array, which lives in its fixed
// scratch.)
//
// Recognizers: a word is a maximal run of [A-Za-z0-9.:-]; trailing '.', '-'
// and a ':' that does not close a final '::' are stripped; the whole word is
// then tested as MAC, IPv6, IPv4(:port), CVE id, host name(:port), hash,
// UUID, certificate fingerprint, OID, first enabled match wins, port excluded
// from the span. Before the word tests, the multi-word recognizers (PEM
// certificate at a line start, URL, CPE name) are tried at the word start.
// One thread per word start (collected per tile, as for the tokenizer). A
// second pass, one warp per record, takes the candidates left to right and
// drops those that start inside an accepted multi-word span (the behaviour
// of a scanning regex engine).
#include <algorithm>
#include <atomic>

#include "scan.cuh"
#include "stages.cuh"

namespace as {

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

// Bytes of a mark tile (also one scan tile: the mark kernels can write the
// scan's tile counts).
constexpr uint32_t kMarkTileBytes = 4096;
static_assert(kMarkTileBytes == (uint32_t)kScanTile, "a mark tile is one scan tile");

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

// Greedy longest-match split of the alphanumeric run that starts at byte i:
// the id of each piece at its first byte, 0 at its other bytes.
// Returns the number of pieces that start before tile_end; with tile_sums,
// each piece that starts past it is added to its own tile's count.
__device__ __forceinline__ uint32_t tokenize_run(const uint8_t* __restrict__ bytes, uint32_t N,
                                                 const uint32_t* __restrict__ rs, VocabTable vt,
                                                 uint16_t* __restrict__ tok_at, uint32_t i, uint64_t tile_end,
                                                 uint32_t* __restrict__ tile_sums) {
  uint32_t p = i, in_tile = 0;
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
    // longest vocabulary prefix: only lengths that some string starting
    // with b[0] b[1] has, at most avail, longest first
    uint32_t take = 1, id = b[0] + 1;
    if (avail >= 2) {
      uint32_t lens = __ldg(&vt.lenmask[alnum_code(b[0]) * kAlnumCodes + alnum_code(b[1])]);
      lens &= (2u << avail) - 1u;
      while (lens) {
        const uint32_t L = 31u - __clz(lens);
        const uint32_t v = vocab_lookup(vt, b, L);
        if (v) { take = L; id = v; break; }
        lens &= ~(1u << L);
      }
    }
    tok_at[p] = (uint16_t)id;
    for (uint32_t k = 1; k < take; ++k) tok_at[p + k] = 0;
    if (p < tile_end) ++in_tile;
    else if (tile_sums) atomicAdd(&tile_sums[p / kMarkTileBytes], 1u);
    p += take;
    if (p >= N || !is_alnum(bytes[p]) || rs_bit(rs, p)) break;
  }
  return in_tile;
}

// A block takes tiles of kMarkTile bytes. It first writes the id of every
// non-alphanumeric byte and collects the tile's run starts in shared memory
// (one ballot per warp and step), then its threads split whole runs, one run
// per thread: every lane of a warp has a run to work on, where one thread per
// byte would leave most lanes idle while a few walk their runs. A run that
// continues past the tile is finished by its own thread. With tile_sums
// (zeroed by the caller) the block also adds the number of tokens that start
// in each tile, so the compaction needs no counting pass.
constexpr uint32_t kMarkThreads = 256;
constexpr uint32_t kMarkTile = kMarkTileBytes;

// Blocks of a mark kernel that fit on the device at once (the kernels loop
// over tiles with a grid stride, so a second wave of blocks would start late
// with a full share of tiles), looked up once per kernel and device (the
// current one: every launcher runs with the ctx's device current).
template <typename Kernel>
unsigned resident_blocks(Kernel kernel, uint64_t tiles) {
  constexpr int kMaxDevices = 64;
  static std::atomic<int> cap[kMaxDevices] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  const int slot = dev >= 0 && dev < kMaxDevices ? dev : 0;
  int c = cap[slot].load();
  if (c == 0) {
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kMarkThreads, 0);
    c = std::max(1, per_sm * sms);
    if (dev >= 0 && dev < kMaxDevices) cap[slot].store(c);
  }
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(tiles, (uint64_t)c));
}

__device__ __forceinline__ void collect_start(bool start, uint32_t i, uint32_t* starts, uint32_t* n_starts) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t m = __ballot_sync(0xffffffffu, start);
  uint32_t at = 0;
  if (lane == 0 && m) at = atomicAdd(n_starts, (uint32_t)__popc(m));
  at = __shfl_sync(0xffffffffu, at, 0);
  if (start) starts[at + __popc(m & ((1u << lane) - 1u))] = i;  // < kMarkTile: one start per byte at most
}

__global__ void __launch_bounds__(kMarkThreads, 4)
    tokenize_mark_kernel(const uint8_t* __restrict__ bytes, uint32_t N, const uint32_t* __restrict__ rs, VocabTable vt,
                         uint16_t* __restrict__ tok_at, uint32_t* __restrict__ tile_sums) {
  __shared__ uint32_t starts[kMarkTile];
  __shared__ uint32_t n_starts, n_tok;
  for (uint64_t base = (uint64_t)blockIdx.x * kMarkTile; base < N; base += (uint64_t)gridDim.x * kMarkTile) {
    if (threadIdx.x == 0) {
      n_starts = 0;
      n_tok = 0;
    }
    __syncthreads();
    uint32_t my_tok = 0;
    for (uint32_t k = 0; k < kMarkTile / kMarkThreads; ++k) {
      const uint64_t i = base + k * kMarkThreads + threadIdx.x;
      bool start = false;
      if (i < N) {
        const uint32_t c = bytes[i];
        if (!is_alnum(c)) {
          tok_at[i] = (uint16_t)(c + 1);
          ++my_tok;
        } else {
          start = i == 0 || rs_bit(rs, (uint32_t)i) || !is_alnum(bytes[i - 1]);
        }
      }
      collect_start(start, (uint32_t)i, starts, &n_starts);
    }
    __syncthreads();
    const uint32_t ns = n_starts;
    for (uint32_t j = threadIdx.x; j < ns; j += kMarkThreads)
      my_tok += tokenize_run(bytes, N, rs, vt, tok_at, starts[j], base + kMarkTile, tile_sums);
    if (tile_sums && my_tok) atomicAdd(&n_tok, my_tok);
    __syncthreads();  // starts and n_starts are reused by the next tile
    if (tile_sums && threadIdx.x == 0 && n_tok) atomicAdd(&tile_sums[base / kMarkTile], n_tok);
  }
}

void launch_tokenize_mark(const uint8_t* bytes, uint32_t N, const uint32_t* rs, VocabTable vt, uint16_t* tok_at,
                          cudaStream_t st, uint32_t* tile_sums) {
  if (N == 0) return;
  const unsigned grid = resident_blocks(tokenize_mark_kernel, (N + kMarkTile - 1) / kMarkTile);
  tokenize_mark_kernel<<<grid, kMarkThreads, 0, st>>>(bytes, N, rs, vt, tok_at, tile_sums);
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

// Token table straight from the marks: one compaction whose last pass writes
// each token's id and first byte at its rank (no per-byte position array).
struct TokStart {
  const uint16_t* tok_at;
  __device__ uint32_t operator()(uint64_t i) const { return tok_at[i] != 0; }
};
struct EmitToken {
  const uint16_t* tok_at;
  int32_t* ids;
  uint32_t* off;
  __device__ void operator()(uint64_t i, uint32_t t) const {
    ids[t] = (int32_t)tok_at[i];
    off[t] = (uint32_t)i;
  }
};

void launch_tokenize_compact(const uint16_t* tok_at, uint32_t N, int32_t* ids, uint32_t* off, uint32_t* n_tokens,
                             uint32_t* tile_scratch, cudaStream_t st) {
  compact_emit<uint32_t>(TokStart{tok_at}, N, EmitToken{tok_at, ids, off}, n_tokens, tile_scratch, st);
}

// Token table of one 4,096-byte tile per block, from the marks and the tile
// offsets (the exclusive scan of the tile counts): the tile's tokens are
// ranked in shared memory and then written out in rank order, so that the
// id / offset / length stores of a warp are contiguous. The last token of a
// tile takes its length from the next token start past the tile (at most
// kMaxPiece bytes on: no token is longer), or N.
__global__ void __launch_bounds__(kScanThreads)
    token_emit_tiles_kernel(const uint16_t* __restrict__ tok_at, uint32_t N, const uint32_t* __restrict__ tile_off,
                            int32_t* __restrict__ ids, uint32_t* __restrict__ off, uint32_t* __restrict__ len) {
  __shared__ uint32_t s_pos[kMarkTile];
  __shared__ uint16_t s_id[kMarkTile];
  __shared__ uint32_t sm[33];
  __shared__ uint32_t next_start;
  const uint64_t base = (uint64_t)blockIdx.x * kMarkTile;
  if (base >= N) return;
  const uint32_t n_here = (uint32_t)min((uint64_t)kMarkTile, (uint64_t)N - base);
  const uint32_t j0 = threadIdx.x * kScanItems;
  uint16_t v[kScanItems];
  if (j0 + kScanItems <= n_here) {
    const uint4* src = reinterpret_cast<const uint4*>(tok_at + base + j0);
    const uint4 a = src[0], b = src[1];
    const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) v[k] = (uint16_t)(w[k >> 1] >> (16 * (k & 1)));
  } else {
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) v[k] = j0 + k < n_here ? tok_at[base + j0 + k] : (uint16_t)0;
  }
  uint32_t cnt = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) cnt += v[k] != 0;
  if (threadIdx.x == 0) {
    uint64_t q = base + n_here;
    while (q < N && tok_at[q] == 0) ++q;
    next_start = (uint32_t)q;
  }
  uint32_t tot;
  uint32_t r = block_exclusive_scan(cnt, sm, &tot);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (v[k]) {
      s_id[r] = v[k];
      s_pos[r] = j0 + k;
      ++r;
    }
  }
  __syncthreads();
  const uint32_t t0 = tile_off[blockIdx.x];
  for (uint32_t q = threadIdx.x; q < tot; q += kScanThreads) {
    const uint32_t o = (uint32_t)base + s_pos[q];
    const uint32_t e = q + 1 < tot ? (uint32_t)base + s_pos[q + 1] : next_start;
    ids[t0 + q] = (int32_t)s_id[q];
    off[t0 + q] = o;
    len[t0 + q] = e - o;
  }
}

void launch_tokenize_table(const uint16_t* tok_at, uint32_t N, int32_t* ids, uint32_t* off, uint32_t* len,
                           uint32_t* n_tokens, uint32_t* tile_sums, cudaStream_t st) {
  const uint64_t tiles = scan_tiles_needed(N);
  if (tiles == 0) {
    cudaMemsetAsync(n_tokens, 0, sizeof(uint32_t), st);
    return;
  }
  scan_tile_offsets<uint32_t><<<1, 1024, 0, st>>>(tile_sums, N, n_tokens, nullptr, 0);
  token_emit_tiles_kernel<<<(unsigned)tiles, kScanThreads, 0, st>>>(tok_at, N, tile_sums, ids, off, len);
  count_launch(2);
}

// First token of each record from the token table: a record start is always
// a token start, so it is the number of tokens that start before the record
// (binary search of the sorted token offsets); offsets at N give T.
__global__ void record_token_starts_kernel(const uint64_t* __restrict__ offsets, uint64_t n,
                                           const uint32_t* __restrict__ off, const uint32_t* total_T, uint32_t N,
                                           uint64_t* __restrict__ rec_tok) {
  const uint32_t T = *total_T;
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r <= n; r += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t o = offsets[r];
    rec_tok[r] = o >= N ? T : o == 0 ? 0 : (uint64_t)(upper_index(off, (int64_t)T, (uint32_t)(o - 1)) + 1);
  }
}

void launch_record_token_starts(const uint64_t* offsets, uint64_t n, const uint32_t* tok_off, const uint32_t* total_T,
                                uint32_t N, uint64_t* rec_tok, cudaStream_t st) {
  record_token_starts_kernel<<<grid_1d(n + 1, 256, 65535), 256, 0, st>>>(offsets, n, tok_off, total_T, N, rec_tok);
  count_launch();
}

// ---------------------------------------------------------------- recognizers

__device__ __forceinline__ bool in_word(uint32_t c) { return is_alnum(c) || c == '.' || c == ':' || c == '-'; }
__device__ __forceinline__ bool is_digit(uint32_t c) { return c - '0' < 10u; }
__device__ __forceinline__ bool is_alpha(uint32_t c) { return (c | 0x20u) - 'a' < 26u; }
__device__ __forceinline__ bool is_hex(uint32_t c) { return is_digit(c) || (c | 0x20u) - 'a' < 6u; }

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

__device__ bool rx_is_hash(const uint8_t* w, uint32_t n) {
  if (n != 32 && n != 40 && n != 64 && n != 128) return false;
  for (uint32_t k = 0; k < n; ++k)
    if (!is_hex(w[k])) return false;
  return true;
}

__device__ bool rx_is_uuid(const uint8_t* w, uint32_t n) {
  if (n != 36) return false;
  for (uint32_t k = 0; k < n; ++k) {
    const bool dash = k == 8 || k == 13 || k == 18 || k == 23;
    if (dash ? w[k] != '-' : !is_hex(w[k])) return false;
  }
  return true;
}

// 16, 20 or 32 groups of two hex digits joined by ':'
__device__ bool rx_is_cert_fp(const uint8_t* w, uint32_t n) {
  if ((n + 1) % 3) return false;
  const uint32_t g = (n + 1) / 3;
  if (g != 16 && g != 20 && g != 32) return false;
  for (uint32_t k = 0; k < g; ++k) {
    if (!is_hex(w[3 * k]) || !is_hex(w[3 * k + 1])) return false;
    if (k + 1 < g && w[3 * k + 2] != ':') return false;
  }
  return true;
}

// >= 5 decimal arcs joined by '.', no leading zeros; first arc 0..2, second
// arc <= 39 below first arc 2
__device__ bool rx_is_oid(const uint8_t* w, uint32_t n) {
  uint32_t arcs = 0, start = 0;
  for (uint32_t k = 0; k <= n; ++k) {
    if (k == n || w[k] == '.') {
      const uint32_t L = k - start;
      if (L == 0 || (L > 1 && w[start] == '0')) return false;
      if (arcs == 0 && (L != 1 || w[start] > '2')) return false;
      if (arcs == 1 && w[0] < '2' && (L > 2 || (L == 2 && (w[start] - '0') * 10 + (w[start + 1] - '0') > 39)))
        return false;
      ++arcs;
      start = k + 1;
    } else if (!is_digit(w[k])) {
      return false;
    }
  }
  return arcs >= 5;
}

// byte sets of the multi-word recognizers, as 128-bit masks over ASCII
constexpr uint64_t set_lo(const char* s, uint64_t m = 0) {
  return *s ? set_lo(s + 1, (unsigned char)*s < 64 ? m | (1ull << (unsigned char)*s) : m) : m;
}
constexpr uint64_t set_hi(const char* s, uint64_t m = 0) {
  return *s ? set_hi(s + 1, (unsigned char)*s >= 64 && (unsigned char)*s < 128 ? m | (1ull << ((unsigned char)*s - 64)) : m)
            : m;
}
// a byte set is two scalar masks (lo: bytes 0..63, hi: 64..127), passed by value
#define AS_ALNUM "0123456789ABCDEFGHIJKLMNOPQRSTUVWXYZabcdefghijklmnopqrstuvwxyz"
#define AS_BYTE_SET(name, chars) \
  constexpr uint64_t name##_lo = set_lo(chars), name##_hi = set_hi(chars);
AS_BYTE_SET(kUrlBytes, AS_ALNUM "-._~:/?#[]@!$&*+,;=%")
AS_BYTE_SET(kUrlTrail, ".,:;!?")
AS_BYTE_SET(kCpeFsBytes, AS_ALNUM "._~%!*?-")
AS_BYTE_SET(kCpeUriBytes, AS_ALNUM "._~%-")
AS_BYTE_SET(kB64Space, AS_ALNUM "+/=\t\n\v\f\r ")
#undef AS_BYTE_SET
#undef AS_ALNUM
#define AS_SET(name) name##_lo, name##_hi
__device__ __forceinline__ bool in_set(uint32_t c, uint64_t lo, uint64_t hi) {
  return c < 64 ? (lo >> c) & 1u : c < 128 ? (hi >> (c - 64)) & 1u : false;
}

__constant__ char kPemBegin[] = "-----BEGIN CERTIFICATE-----";
__constant__ char kPemEnd[] = "-----END CERTIFICATE-----";

// Scanning helpers for a candidate starting at record position i: a byte
// p > i belongs to the record while p < N and no record starts at p.
struct RecScan {
  const uint8_t* b;
  uint32_t N;
  const uint32_t* rs;
  uint32_t i;
  __device__ __forceinline__ bool in(uint32_t p) const { return p < N && (p == i || !rs_bit(rs, p)); }
  __device__ __forceinline__ uint32_t run(uint32_t p, uint64_t lo, uint64_t hi) const {
    while (in(p) && in_set(b[p], lo, hi)) ++p;
    return p;
  }
  __device__ __forceinline__ bool lit(uint32_t p, const char* s, uint32_t n) const {
    for (uint32_t k = 0; k < n; ++k)
      if (!in(p + k) || b[p + k] != (uint8_t)s[k]) return false;
    return true;
  }
};

// End of a PEM certificate block starting at i (a line start), else 0.
__device__ uint32_t rx_pem_end(const RecScan& r) {
  const uint32_t i = r.i;
  if (!(i == 0 || rs_bit(r.rs, i) || r.b[i - 1] == '\n')) return 0;
  if (!r.lit(i, kPemBegin, sizeof(kPemBegin) - 1)) return 0;
  const uint32_t j = r.run(i + sizeof(kPemBegin) - 1, AS_SET(kB64Space));
  if (!r.lit(j, kPemEnd, sizeof(kPemEnd) - 1)) return 0;
  return j + sizeof(kPemEnd) - 1;
}

// End of a URL starting at i, else 0.
__device__ uint32_t rx_url_end(const RecScan& r) {
  const uint32_t i = r.i;
  if (!is_alpha(r.b[i])) return 0;
  uint32_t j = i + 1;
  while (r.in(j) && is_alnum(r.b[j])) {
    if (++j - i > 16) return 0;
  }
  if (j - i < 2 || !r.lit(j, "://", 3)) return 0;
  const uint32_t body = j + 3;
  uint32_t e = r.run(body, AS_SET(kUrlBytes));
  while (e > body && in_set(r.b[e - 1], AS_SET(kUrlTrail))) --e;
  return e > body ? e : 0;
}

// End of a CPE name (formatted string or URI form) starting at i, else 0.
__device__ uint32_t rx_cpe_end(const RecScan& r) {
  const uint32_t i = r.i;
  if (r.lit(i, "cpe:2.3:", 8)) {
    uint32_t j = i + 8, last = j;
    for (int comp = 0; comp < 11; ++comp) {
      if (comp > 0) {
        if (!r.in(j) || r.b[j] != ':') return 0;
        ++j;
      }
      const uint32_t e = r.run(j, AS_SET(kCpeFsBytes));
      if (e == j) return 0;
      if (comp == 0) {
        const uint32_t p = r.b[j];
        if (e - j != 1 || !(p == 'a' || p == 'o' || p == 'h' || p == '*' || p == '-')) return 0;
      }
      last = j;
      j = e;
    }
    while (j > last + 1 && r.b[j - 1] == '.') --j;
    return r.b[j - 1] == '.' ? 0 : j;
  }
  if (r.lit(i, "cpe:/", 5) && r.in(i + 5) && (r.b[i + 5] == 'a' || r.b[i + 5] == 'o' || r.b[i + 5] == 'h')) {
    uint32_t j = i + 6;
    for (int comp = 0; comp < 6 && r.in(j) && r.b[j] == ':'; ++comp) j = r.run(j + 1, AS_SET(kCpeUriBytes));
    while (r.b[j - 1] == '.' || r.b[j - 1] == ':') --j;
    return j;
  }
  return 0;
}

#undef AS_SET

// The recognizers at the word that starts at byte i: the entity length and
// type (kRxLong set for a multi-word match), 0 and 0 when nothing matches.
__device__ __forceinline__ void recognize_word(const uint8_t* __restrict__ bytes, uint32_t N,
                                               const uint32_t* __restrict__ rs, const RxTypes& T, uint32_t i,
                                               uint32_t& len, uint8_t& type) {
  len = 0;
  type = 0;
  const uint32_t c = bytes[i];
  if (T.t[kRxPem] | T.t[kRxUrl] | T.t[kRxCpe]) {
    const RecScan r{bytes, N, rs, i};
    uint32_t le = 0;
    if (T.t[kRxPem] && (le = rx_pem_end(r)) > i) type = T.t[kRxPem];
    else if (T.t[kRxUrl] && (le = rx_url_end(r)) > i) type = T.t[kRxUrl];
    else if (T.t[kRxCpe] && (le = rx_cpe_end(r)) > i) type = T.t[kRxCpe];
    if (type) {
      len = le - i;
      type |= kRxLong;
    }
  }
  // which separators the stripped word holds ('.' 1, ':' 2, '-' 4): every
  // test below except the hash needs one inside the word it tests, so words
  // without them skip it. The first position of each separator is kept, so
  // that a separator the strip removes (a sentence's final '.') does not count.
  uint32_t first_sep[3] = {UINT32_MAX, UINT32_MAX, UINT32_MAX};
  auto note_sep = [&](uint32_t ch, uint32_t at) {
    const int k = ch == '.' ? 0 : ch == ':' ? 1 : ch == '-' ? 2 : -1;
    if (k >= 0 && first_sep[k] == UINT32_MAX) first_sep[k] = at;
  };
  note_sep(c, i);
  uint32_t e = i + 1;
  while (e < N && !rs_bit(rs, e)) {
    const uint32_t ch = bytes[e];
    if (!in_word(ch)) break;
    note_sep(ch, e);
    ++e;
  }
  while (e > i) {
    uint32_t t = bytes[e - 1];
    if (t == '.' || t == '-') --e;
    else if (t == ':' && !(e >= i + 2 && bytes[e - 2] == ':')) --e;
    else break;
  }
  const uint32_t sep = (first_sep[0] < e ? 1u : 0u) | (first_sep[1] < e ? 2u : 0u) | (first_sep[2] < e ? 4u : 0u);
  const uint8_t* w = bytes + i;
  uint32_t n = e - i;
  if (n > 0 && !type) {
    uint32_t k;
    // a test skipped for want of its separator would have failed (MAC: ':'
    // or '-'; IPv6, fingerprint: ':'; IPv4, host name, OID: '.'; CVE,
    // UUID: '-'), so the first match is the same
    if (T.t[kRxMac] && (sep & 6u) && rx_is_mac(w, n)) { len = n; type = T.t[kRxMac]; }
    else if (T.t[kRxIpv6] && (sep & 2u) && rx_is_ipv6(w, n)) { len = n; type = T.t[kRxIpv6]; }
    else if (T.t[kRxIpv4] && (sep & 1u) && (k = rx_ipv4_len(w, n)) > 0) { len = k; type = T.t[kRxIpv4]; }
    else if (T.t[kRxCve] && (sep & 4u) && rx_is_cve(w, n)) { len = n; type = T.t[kRxCve]; }
    else if (T.t[kRxHost] && (sep & 1u) && (k = rx_host_len(w, n)) > 0) { len = k; type = T.t[kRxHost]; }
    else if (T.t[kRxHash] && rx_is_hash(w, n)) { len = n; type = T.t[kRxHash]; }
    else if (T.t[kRxUuid] && (sep & 4u) && rx_is_uuid(w, n)) { len = n; type = T.t[kRxUuid]; }
    else if (T.t[kRxCertFp] && (sep & 2u) && rx_is_cert_fp(w, n)) { len = n; type = T.t[kRxCertFp]; }
    else if (T.t[kRxOid] && (sep & 1u) && rx_is_oid(w, n)) { len = n; type = T.t[kRxOid]; }
  }
}

// Tiles of kMarkTile bytes as in the tokenizer: the block writes type 0 for
// every byte that starts no word and collects the word starts, then one
// thread per word runs the recognizers. A candidate's length is written only
// where its type is not 0 (the only places it is read). With tile_sums
// (zeroed by the caller) the block adds its number of candidates, so the
// compaction needs no counting pass; that count is final only when no
// multi-word kind is on (the resolve pass may drop candidates).
__global__ void __launch_bounds__(kMarkThreads)
    recognize_mark_kernel(const uint8_t* __restrict__ bytes, uint32_t N, const uint32_t* __restrict__ rs, RxTypes T,
                          uint32_t* __restrict__ rx_len, uint8_t* __restrict__ rx_type,
                          uint32_t* __restrict__ tile_sums) {
  __shared__ uint32_t starts[kMarkTile];
  __shared__ uint32_t n_starts, n_cand;
  for (uint64_t base = (uint64_t)blockIdx.x * kMarkTile; base < N; base += (uint64_t)gridDim.x * kMarkTile) {
    if (threadIdx.x == 0) {
      n_starts = 0;
      n_cand = 0;
    }
    __syncthreads();
    for (uint32_t k = 0; k < kMarkTile / kMarkThreads; ++k) {
      const uint64_t i = base + k * kMarkThreads + threadIdx.x;
      bool start = false;
      if (i < N) {
        start = in_word(bytes[i]) && (i == 0 || rs_bit(rs, (uint32_t)i) || !in_word(bytes[i - 1]));
        if (!start) rx_type[i] = 0;
      }
      collect_start(start, (uint32_t)i, starts, &n_starts);
    }
    __syncthreads();
    const uint32_t ns = n_starts;
    uint32_t my_cand = 0;
    for (uint32_t j = threadIdx.x; j < ns; j += kMarkThreads) {
      const uint32_t i = starts[j];
      uint32_t len;
      uint8_t type;
      recognize_word(bytes, N, rs, T, i, len, type);
      rx_type[i] = type;
      if (type) {
        rx_len[i] = len;  // read only where the type is not 0
        ++my_cand;
      }
    }
    if (tile_sums && my_cand) atomicAdd(&n_cand, my_cand);
    __syncthreads();  // starts and n_starts are reused by the next tile
    if (tile_sums && threadIdx.x == 0 && n_cand) atomicAdd(&tile_sums[base / kMarkTile], n_cand);
  }
}

void launch_recognize_mark(const uint8_t* bytes, uint32_t N, const uint32_t* rs, RxTypes types, uint32_t* rx_len,
                           uint8_t* rx_type, cudaStream_t st, uint32_t* tile_sums) {
  if (N == 0) return;
  const unsigned grid = resident_blocks(recognize_mark_kernel, (N + kMarkTile - 1) / kMarkTile);
  recognize_mark_kernel<<<grid, kMarkThreads, 0, st>>>(bytes, N, rs, types, rx_len, rx_type, tile_sums);
  count_launch();
}

// One warp per record, 512 bytes of rx_type per step (16 per lane, one
// aligned 16-byte load; rx_type has 16 bytes of slack past N). kept_end is
// the end of the last accepted multi-word span. Within a step the accepted
// spans are taken in byte order: the lowest lane holding an open multi-word
// candidate accepts its first one and every lane drops its candidates that
// start inside it. Writes touch only this record's bytes.
__global__ void recognize_resolve_kernel(const uint64_t* __restrict__ offsets, uint64_t n,
                                         const uint32_t* __restrict__ rx_len, uint8_t* __restrict__ rx_type) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t r = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n; r += nwarps) {
    const uint32_t a = (uint32_t)offsets[r], b = (uint32_t)offsets[r + 1];
    uint32_t kept_end = a;
    for (uint32_t base = a & ~15u; base < b; base += 512) {
      const uint32_t q = base + lane * 16;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (q < b) v = *reinterpret_cast<const uint4*>(rx_type + q);
      const uint32_t words[4] = {v.x, v.y, v.z, v.w};
      uint32_t cand = 0, open = 0;
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const uint32_t t = (words[k >> 2] >> (8 * (k & 3))) & 0xffu;
        const uint32_t p = q + k;
        if (t && p >= a && p < b) {
          cand |= 1u << k;
          if (t & kRxLong) open |= 1u << k;
        }
      }
      uint32_t drop = 0, accepted = 0;
#pragma unroll
      for (int k = 0; k < 16; ++k)
        if (((cand >> k) & 1u) && q + k < kept_end) drop |= 1u << k;
      open &= ~drop;
      for (;;) {
        const uint32_t lanes = __ballot_sync(0xffffffffu, open != 0);
        if (!lanes) break;
        const int j = __ffs(lanes) - 1;
        uint32_t s = 0, e = 0;
        if ((int)lane == j) {
          const int k = __ffs(open) - 1;
          s = q + k;
          e = s + rx_len[s];
          accepted |= 1u << k;
          open &= ~(1u << k);
        }
        s = __shfl_sync(0xffffffffu, s, j);
        e = __shfl_sync(0xffffffffu, e, j);
        kept_end = e;
#pragma unroll
        for (int k = 0; k < 16; ++k)
          if (((cand >> k) & 1u) && q + k > s && q + k < e) drop |= 1u << k;
        open &= ~drop;
      }
      const uint32_t touch = drop | accepted;
      if (touch) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          if ((touch >> k) & 1u) {
            const uint32_t t = (words[k >> 2] >> (8 * (k & 3))) & 0x7fu;
            rx_type[q + k] = ((drop >> k) & 1u) ? 0 : (uint8_t)t;
          }
        }
      }
    }
  }
}

void launch_recognize_resolve(const uint64_t* offsets, uint64_t n, const uint32_t* rx_len, uint8_t* rx_type,
                              cudaStream_t st) {
  if (n == 0) return;
  const uint64_t blocks = std::min<uint64_t>((n + 7) / 8, 148 * 16);
  recognize_resolve_kernel<<<(unsigned)blocks, 256, 0, st>>>(offsets, n, rx_len, rx_type);
  count_launch();
}

// Recognizer spans in byte order: one compaction of the per-byte marks whose
// last pass writes each span at its rank.
struct RxStart {
  const uint8_t* rx_type;
  __device__ uint32_t operator()(uint64_t i) const { return rx_type[i] != 0; }
};
struct EmitRxSpan {
  const uint32_t* rx_len;
  const uint8_t* rx_type;
  uint32_t *sp_start, *sp_len;
  uint8_t* sp_type;
  __device__ void operator()(uint64_t i, uint32_t k) const {
    sp_start[k] = (uint32_t)i;
    sp_len[k] = rx_len[i];
    sp_type[k] = rx_type[i];
  }
};

void launch_recognize_compact(const uint32_t* rx_len, const uint8_t* rx_type, uint32_t N, uint32_t* sp_start,
                              uint32_t* sp_len, uint8_t* sp_type, uint32_t* n_spans, uint32_t* tile_scratch,
                              cudaStream_t st, bool sums_given) {
  const EmitRxSpan emit{rx_len, rx_type, sp_start, sp_len, sp_type};
  if (sums_given)
    compact_emit_from_sums<uint32_t>(RxStart{rx_type}, N, emit, n_spans, tile_scratch, st);
  else
    compact_emit<uint32_t>(RxStart{rx_type}, N, emit, n_spans, tile_scratch, st);
}

}  // namespace as
