// From per-token labels to the final entity spans of each record.
//
// BIO decoding is lenient: a span starts at B-t, or at I-t whose predecessor
// in the record is not B-t/I-t, and continues while the next label is I-t.
// Token spans become byte spans [off(first), off(last)+len(last)) with ASCII
// whitespace trimmed. Overlaps: every NER span sharing a byte with a pattern
// recognizer span is dropped (recognizers win; the paper's standalone path
// has no overlap resolution and truncates entities, Appendix D). Types in
// the preserve mask are dropped after that (§2, --entities-to-preserve).
// Every step is one thread per token or per span; lists stay sorted by byte
// offset, and merging two sorted lists is done by rank (binary search).
#include "scan.cuh"
#include "stages.cuh"

namespace as {

__global__ void token_flags_kernel(const uint64_t* rec_tok, uint64_t n, uint8_t* flags) {
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < n; r += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t a = rec_tok[r], b = rec_tok[r + 1];
    if (a < b) {
      if (b - a == 1) {
        flags[a] = 3;
      } else {
        flags[a] = 1;
        flags[b - 1] = 2;
      }
    }
  }
}

void launch_token_flags(const uint64_t* rec_tok, uint64_t n, uint8_t* flags, cudaStream_t st) {
  if (n == 0) return;
  token_flags_kernel<<<grid_1d(n, 256, 65535), 256, 0, st>>>(rec_tok, n, flags);
  count_launch();
}

__device__ __forceinline__ uint32_t ltype(uint32_t l) { return (l + 1) >> 1; }
__device__ __forceinline__ bool lbegin(uint32_t l) { return l & 1u; }

__global__ void bio_mark_kernel(const uint8_t* __restrict__ labels, const uint8_t* __restrict__ flags, uint32_t T,
                                uint8_t* __restrict__ is_start, uint8_t* __restrict__ is_end) {
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
    uint32_t l = labels[t], ty = ltype(l), f = flags[t];
    uint8_t s = 0, e = 0;
    if (ty) {
      s = lbegin(l) || (f & 1u) || ltype(labels[t - 1]) != ty;
      e = (f & 2u) || !(ltype(labels[t + 1]) == ty && !lbegin(labels[t + 1]));
    }
    is_start[t] = s;
    is_end[t] = e;
  }
}

void launch_bio_mark(const uint8_t* labels, const uint8_t* flags, uint32_t T, uint8_t* is_start, uint8_t* is_end,
                     cudaStream_t st) {
  if (T == 0) return;
  bio_mark_kernel<<<grid_1d(T, 256, 148 * 64), 256, 0, st>>>(labels, flags, T, is_start, is_end);
  count_launch();
}

__device__ __forceinline__ bool is_ws(uint32_t c) { return c == 0x20 || (c - 0x09u) < 5u; }

// Start tokens write their span's first token and type; end tokens its last.
// Spans pair in order: span k = number of starts before t (+1 at a start).
__global__ void bio_emit_kernel(const uint8_t* __restrict__ labels, const uint8_t* __restrict__ is_start,
                                const uint8_t* __restrict__ is_end, const uint32_t* __restrict__ pos, uint32_t T,
                                uint32_t* first_tok, uint32_t* last_tok, uint8_t* type) {
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
    uint32_t s = is_start[t], e = is_end[t];
    if (s) {
      first_tok[pos[t]] = t;
      type[pos[t]] = (uint8_t)ltype(labels[t]);
    }
    if (e) last_tok[pos[t] + s - 1] = t;
  }
}

void launch_bio_emit(const uint8_t* labels, const uint8_t* is_start, const uint8_t* is_end, const uint32_t* pos,
                     uint32_t T, const uint32_t* tok_off, const uint32_t* tok_len, const uint8_t* bytes,
                     uint32_t* ner_start, uint32_t* ner_len, uint8_t* ner_type, cudaStream_t st) {
  // ner_start / ner_len first hold the first / last token of each span.
  if (T == 0) return;
  bio_emit_kernel<<<grid_1d(T, 256, 148 * 64), 256, 0, st>>>(labels, is_start, is_end, pos, T, ner_start, ner_len,
                                                             ner_type);
  count_launch();
}

__global__ void bio_to_bytes_kernel(uint32_t* ner_a, uint32_t* ner_b, const uint32_t* n_dev,
                                    const uint32_t* __restrict__ tok_off, const uint32_t* __restrict__ tok_len,
                                    const uint8_t* __restrict__ bytes) {
  uint32_t n = *n_dev;
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    uint32_t ft = ner_a[k], lt = ner_b[k];
    uint32_t a = tok_off[ft];
    uint32_t b = tok_off[lt] + tok_len[lt];
    while (a < b && is_ws(bytes[a])) ++a;
    while (b > a && is_ws(bytes[b - 1])) --b;
    ner_a[k] = a;
    ner_b[k] = b - a;
  }
}

void launch_bio_to_bytes(uint32_t* ner_start, uint32_t* ner_len, const uint32_t* n_dev, uint32_t cap,
                         const uint32_t* tok_off, const uint32_t* tok_len, const uint8_t* bytes, cudaStream_t st) {
  if (cap == 0) return;
  bio_to_bytes_kernel<<<grid_1d(cap, 256, 148 * 64), 256, 0, st>>>(ner_start, ner_len, n_dev, tok_off, tok_len, bytes);
  count_launch();
}

__global__ void ner_keep_kernel(const uint32_t* __restrict__ ns, const uint32_t* __restrict__ nl,
                                const uint8_t* __restrict__ nt, const uint32_t* n_ner_dev,
                                const uint32_t* __restrict__ rs, const uint32_t* __restrict__ rl,
                                const uint32_t* n_rx_dev, uint64_t preserve, uint8_t* keep, uint32_t cap) {
  uint32_t n = *n_ner_dev, nr = *n_rx_dev;
  // keep[0..n): the scan and the compaction after it read no further
  const uint32_t end = min(cap, n);
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < end; k += gridDim.x * blockDim.x) {
    uint8_t kp = 0;
    if (k < n && nl[k] > 0) {
      uint32_t s = ns[k], e = s + nl[k];
      // last recognizer span starting before e: the only candidate overlap
      int64_t j = upper_index(rs, (int64_t)nr, (uint32_t)(e - 1));
      bool overlap = j >= 0 && rs[j] + rl[j] > s;
      kp = !overlap && !((preserve >> nt[k]) & 1ull);
    }
    keep[k] = kp;
  }
}

void launch_ner_keep(const uint32_t* ns, const uint32_t* nl, const uint8_t* nt, const uint32_t* n_ner_dev,
                     uint32_t cap, const uint32_t* rs, const uint32_t* rl, const uint32_t* n_rx_dev, uint64_t preserve,
                     uint8_t* keep, cudaStream_t st) {
  if (cap == 0) return;
  ner_keep_kernel<<<grid_1d(cap, 256, 148 * 64), 256, 0, st>>>(ns, nl, nt, n_ner_dev, rs, rl, n_rx_dev, preserve,
                                                               keep, cap);
  count_launch();
}

__global__ void rx_keep_kernel(const uint8_t* __restrict__ t, const uint32_t* n_dev, uint64_t preserve, uint8_t* keep,
                               uint32_t cap) {
  uint32_t n = *n_dev;
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < cap; k += gridDim.x * blockDim.x)
    keep[k] = k < n && !((preserve >> t[k]) & 1ull);
}

void launch_rx_keep(const uint8_t* t, const uint32_t* n_dev, uint32_t cap, uint64_t preserve, uint8_t* keep,
                    cudaStream_t st) {
  if (cap == 0) return;
  rx_keep_kernel<<<grid_1d(cap, 256, 148 * 64), 256, 0, st>>>(t, n_dev, preserve, keep, cap);
  count_launch();
}

__global__ void compact_spans_kernel(const uint32_t* s, const uint32_t* l, const uint8_t* t, const uint8_t* keep,
                                     const uint32_t* pos, const uint32_t* n_dev, uint32_t* os, uint32_t* ol,
                                     uint8_t* ot) {
  uint32_t n = *n_dev;
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    if (keep[k]) {
      uint32_t p = pos[k];
      os[p] = s[k];
      ol[p] = l[k];
      ot[p] = t[k];
    }
  }
}

void launch_compact_spans(const uint32_t* s, const uint32_t* l, const uint8_t* t, const uint8_t* keep,
                          const uint32_t* pos, const uint32_t* n_dev, uint32_t cap, uint32_t* os, uint32_t* ol,
                          uint8_t* ot, cudaStream_t st) {
  if (cap == 0) return;
  compact_spans_kernel<<<grid_1d(cap, 256, 148 * 64), 256, 0, st>>>(s, l, t, keep, pos, n_dev, os, ol, ot);
  count_launch();
}

// Output rank of an element = its index in its own list + number of elements
// of the other list that start before it (the lists are disjoint).
__global__ void merge_spans_kernel(const uint32_t* a_s, const uint32_t* a_l, const uint8_t* a_t, const uint32_t* n_a_dev,
                                   const uint32_t* b_s, const uint32_t* b_l, const uint8_t* b_t,
                                   const uint32_t* n_b_dev, uint32_t* o_s, uint32_t* o_l, uint8_t* o_t,
                                   uint32_t total_cap) {
  uint32_t na = *n_a_dev, nb = *n_b_dev;
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < total_cap; k += gridDim.x * blockDim.x) {
    if (k < na) {
      uint32_t s = a_s[k];
      int64_t r = s == 0 ? 0 : upper_index(b_s, (int64_t)nb, s - 1) + 1;
      uint32_t p = k + (uint32_t)r;
      o_s[p] = s; o_l[p] = a_l[k]; o_t[p] = a_t[k];
    } else if (k - na < nb) {
      uint32_t j = k - na;
      uint32_t s = b_s[j];
      int64_t r = s == 0 ? 0 : upper_index(a_s, (int64_t)na, s - 1) + 1;
      uint32_t p = j + (uint32_t)r;
      o_s[p] = s; o_l[p] = b_l[j]; o_t[p] = b_t[j];
    }
  }
}

void launch_merge_spans(const uint32_t* a_s, const uint32_t* a_l, const uint8_t* a_t, const uint32_t* n_a_dev,
                        uint32_t a_cap, const uint32_t* b_s, const uint32_t* b_l, const uint8_t* b_t,
                        const uint32_t* n_b_dev, uint32_t b_cap, uint32_t* o_s, uint32_t* o_l, uint8_t* o_t,
                        cudaStream_t st) {
  uint32_t cap = a_cap + b_cap;
  if (cap == 0) return;
  merge_spans_kernel<<<grid_1d(cap, 256, 148 * 64), 256, 0, st>>>(a_s, a_l, a_t, n_a_dev, b_s, b_l, b_t, n_b_dev, o_s,
                                                                  o_l, o_t, cap);
  count_launch();
}

}  // namespace as
