// Structure-preserving substitution (AnonShield §2 stages (3) and (5)).
//
// Each final span becomes "[TYPE_slug]" ("[TYPE]" when the slug length is
// 0), the slug being the first L lower-case hex characters of the span's
// HMAC; every other byte is copied unchanged. With delta_k = replacement
// length - span length and shift_k = sum of delta over spans before k (one
// exclusive scan over the sorted global span list), an input byte b outside
// all spans lands at b + shift_j, j = number of spans starting before b;
// span k's replacement starts at start_k + shift_k; record r starts at
// offsets[r] + shift_j(offsets[r]). So the whole batch is written in one
// pass over the input plus one thread per span, with no per-record loop.
#include "scan.cuh"
#include "stages.cuh"

namespace as {

__global__ void sub_delta_kernel(const uint32_t* __restrict__ sp_len, const uint8_t* __restrict__ sp_type,
                                 const uint32_t* n_dev, const uint32_t* __restrict__ name_len, uint32_t slug_len,
                                 int64_t* __restrict__ delta, uint32_t cap) {
  uint32_t n = *n_dev;
  // delta[0..n] (delta[n] = 0): the shift scan reads no further
  const uint32_t end = min(cap, n + 1);
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < end; k += gridDim.x * blockDim.x) {
    int64_t d = 0;
    if (k < n) {
      int64_t rep = 2 + (int64_t)name_len[sp_type[k]] + (slug_len ? 1 + (int64_t)slug_len : 0);
      d = rep - (int64_t)sp_len[k];
    }
    delta[k] = d;
  }
}

void launch_sub_delta(const uint32_t* sp_len, const uint8_t* sp_type, const uint32_t* n_dev, uint32_t cap,
                      const uint32_t* name_len, uint32_t slug_len, int64_t* delta, cudaStream_t st) {
  if (cap == 0) return;
  sub_delta_kernel<<<grid_1d(cap, 256, 148 * 64), 256, 0, st>>>(sp_len, sp_type, n_dev, name_len, slug_len, delta, cap);
  count_launch();
}

constexpr uint32_t kCopyBytes = 16;  // input bytes per thread

// shift[] has n+1 entries: shift[n] = total delta.
__global__ void sub_copy_kernel(const uint8_t* __restrict__ bytes, uint32_t N, const uint32_t* __restrict__ sp_s,
                                const uint32_t* __restrict__ sp_l, const uint32_t* n_dev,
                                const int64_t* __restrict__ shift, uint8_t* __restrict__ out) {
  uint32_t n = *n_dev;
  uint64_t nchunks = (N + kCopyBytes - 1) / kCopyBytes;
  for (uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c < nchunks; c += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t b0 = (uint32_t)(c * kCopyBytes);
    uint32_t b1 = min(N, b0 + kCopyBytes);
    // j = number of spans starting at or before b0
    int64_t j = upper_index(sp_s, (int64_t)n, b0) + 1;
    uint8_t v[kCopyBytes];
    if (b1 - b0 == kCopyBytes && ((uintptr_t)(bytes + b0) & 15u) == 0) {
      *reinterpret_cast<uint4*>(v) = __ldg(reinterpret_cast<const uint4*>(bytes + b0));
    } else {
      for (uint32_t b = b0; b < b1; ++b) v[b - b0] = bytes[b];
    }
    for (uint32_t b = b0; b < b1; ++b) {
      while (j < (int64_t)n && sp_s[j] <= b) ++j;
      // span j-1 is the last starting at or before b
      if (j > 0 && b < sp_s[j - 1] + sp_l[j - 1]) continue;
      out[(int64_t)b + shift[j]] = v[b - b0];
    }
  }
}

void launch_sub_copy(const uint8_t* bytes, uint32_t N, const uint32_t* sp_start, const uint32_t* sp_len,
                     const uint32_t* n_dev, const int64_t* shift, uint8_t* out, cudaStream_t st) {
  if (N == 0) return;
  uint64_t chunks = (N + kCopyBytes - 1) / kCopyBytes;
  sub_copy_kernel<<<grid_1d(chunks, 256, 148 * 64), 256, 0, st>>>(bytes, N, sp_start, sp_len, n_dev, shift, out);
  count_launch();
}

__global__ void sub_replace_kernel(const uint32_t* __restrict__ sp_s, const uint8_t* __restrict__ sp_t,
                                   const uint32_t* n_dev, const int64_t* __restrict__ shift,
                                   const uint32_t* __restrict__ digests, const char* __restrict__ names,
                                   const uint32_t* __restrict__ name_off, uint32_t slug_len, uint8_t* __restrict__ out) {
  uint32_t n = *n_dev;
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    uint8_t* o = out + ((int64_t)sp_s[k] + shift[k]);
    uint32_t t = sp_t[k];
    uint32_t a = name_off[t], b = name_off[t + 1];
    uint32_t p = 0;
    o[p++] = '[';
    for (uint32_t i = a; i < b; ++i) o[p++] = (uint8_t)names[i];
    if (slug_len) {
      o[p++] = '_';
      const uint32_t* d = digests + (size_t)k * 8;
      for (uint32_t i = 0; i < slug_len; ++i) {
        uint32_t nib = (d[i >> 3] >> (28 - 4 * (i & 7))) & 15u;
        o[p++] = (uint8_t)(nib < 10 ? '0' + nib : 'a' + nib - 10);
      }
    }
    o[p] = ']';
  }
}

void launch_sub_replace(const uint32_t* sp_start, const uint8_t* sp_type, const uint32_t* n_dev, uint32_t cap,
                        const int64_t* shift, const uint32_t* digests, const char* names, const uint32_t* name_off,
                        uint32_t slug_len, uint8_t* out, cudaStream_t st) {
  if (cap == 0) return;
  sub_replace_kernel<<<grid_1d(cap, 256, 148 * 64), 256, 0, st>>>(sp_start, sp_type, n_dev, shift, digests, names,
                                                                  name_off, slug_len, out);
  count_launch();
}

__global__ void sub_offsets_kernel(const uint64_t* __restrict__ offsets, uint64_t n_records,
                                   const uint32_t* __restrict__ sp_s, const uint32_t* n_dev,
                                   const int64_t* __restrict__ shift, uint64_t* __restrict__ out_off) {
  uint32_t n = *n_dev;
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r <= n_records; r += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t o = offsets[r];
    // spans starting strictly before o end at or before o (they never cross records)
    int64_t j = o == 0 ? 0 : upper_index(sp_s, (int64_t)n, (uint64_t)(o - 1)) + 1;
    out_off[r] = (uint64_t)((int64_t)o + shift[j]);
  }
}

void launch_sub_offsets(const uint64_t* offsets, uint64_t n_records, const uint32_t* sp_start, const uint32_t* n_dev,
                        const int64_t* shift, uint64_t* out_off, cudaStream_t st) {
  sub_offsets_kernel<<<grid_1d(n_records + 1, 256, 65535), 256, 0, st>>>(offsets, n_records, sp_start, n_dev, shift,
                                                                         out_off);
  count_launch();
}

}  // namespace as
