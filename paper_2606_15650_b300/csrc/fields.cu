// Per-field policy (the schema-aware configuration of AnonShield §2:
// force_anonymize, fields_to_anonymize, fields_to_exclude), device side.
//
// A call with fields builds a compact arena of the fields to detect in (each
// field is a sub-record of its own, empty unless the field is detected in),
// runs the detection steps on it, translates the resulting spans back to the
// records (field start + offset inside the field) and merges them with the
// spans of the forced fields (field value with ASCII whitespace trimmed, one
// entity of the field's forced type). Excluded fields and bytes outside every
// field are never read by the detection steps and pass through unchanged.
#include "scan.cuh"
#include "stages.cuh"

namespace as {

namespace {

__device__ __forceinline__ bool field_ws(uint32_t c) { return c == 0x20 || (c - 0x09u) < 5u; }

// One warp per field: copy the bytes of a detected field to its sub-record
// (fields that are not detected have an empty sub-record: nothing to copy).
__global__ void field_gather_kernel(const uint8_t* __restrict__ bytes, const uint32_t* __restrict__ f_start,
                                    const uint64_t* __restrict__ sub_off, uint64_t nf, uint8_t* __restrict__ sub) {
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  const uint32_t lane = threadIdx.x & 31;
  for (uint64_t k = blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); k < nf; k += warps) {
    const uint64_t o = sub_off[k], len = sub_off[k + 1] - o;
    const uint8_t* src = bytes + f_start[k];
    for (uint64_t i = lane; i < len; i += 32) sub[o + i] = src[i];
  }
}

// Forced fields: trim ASCII whitespace at both ends; keep[i] = non-empty.
__global__ void field_force_trim_kernel(const uint8_t* __restrict__ bytes, uint32_t* __restrict__ s,
                                        uint32_t* __restrict__ l, uint8_t* __restrict__ keep, uint32_t n) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    uint32_t a = s[i], b = s[i] + l[i];
    while (a < b && field_ws(bytes[a])) ++a;
    while (b > a && field_ws(bytes[b - 1])) --b;
    s[i] = a;
    l[i] = b - a;
    keep[i] = b > a;
  }
}

// Spans found in the compact arena -> record coordinates: the span lies in
// sub-record k (the last k with sub_off[k] <= start); it moves by
// f_start[k] - sub_off[k].
__global__ void field_translate_kernel(uint32_t* __restrict__ sp_s, const uint32_t* __restrict__ n_dev,
                                       const uint64_t* __restrict__ sub_off, uint64_t nf,
                                       const uint32_t* __restrict__ f_start) {
  const uint32_t n = *n_dev;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint64_t p = sp_s[i];
    // upper bound over sub_off[0..nf]: first index with sub_off > p, minus one;
    // empty sub-records share their offset with the next one, and the search
    // lands on the non-empty sub-record that holds p
    uint64_t lo = 0, hi = nf + 1;
    while (lo < hi) {
      const uint64_t mid = (lo + hi) >> 1;
      if (sub_off[mid] <= p) lo = mid + 1; else hi = mid;
    }
    const uint64_t k = lo - 1;
    sp_s[i] = (uint32_t)(f_start[k] + (p - sub_off[k]));
  }
}

__global__ void add_count_kernel(uint32_t* dst, const uint32_t* add) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *dst += *add;
}

}  // namespace

void launch_field_gather(const uint8_t* bytes, const uint32_t* f_start, const uint64_t* sub_off, uint64_t nf,
                         uint8_t* sub, cudaStream_t st) {
  if (nf == 0) return;
  field_gather_kernel<<<grid_1d((nf + 7) / 8, 1, 148 * 16), 256, 0, st>>>(bytes, f_start, sub_off, nf, sub);
  count_launch();
}

void launch_field_force_trim(const uint8_t* bytes, uint32_t* s, uint32_t* l, uint8_t* keep, uint32_t n,
                             cudaStream_t st) {
  if (n == 0) return;
  field_force_trim_kernel<<<grid_1d(n, 256, 148 * 16), 256, 0, st>>>(bytes, s, l, keep, n);
  count_launch();
}

void launch_field_translate(uint32_t* sp_s, const uint32_t* n_dev, uint32_t cap, const uint64_t* sub_off, uint64_t nf,
                            const uint32_t* f_start, cudaStream_t st) {
  if (cap == 0) return;
  field_translate_kernel<<<grid_1d(cap, 256, 148 * 16), 256, 0, st>>>(sp_s, n_dev, sub_off, nf, f_start);
  count_launch();
}

void launch_add_count(uint32_t* dst, const uint32_t* add, cudaStream_t st) {
  add_count_kernel<<<1, 32, 0, st>>>(dst, add);
  count_launch();
}

}  // namespace as
