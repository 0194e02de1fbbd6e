// Device-resident entity -> pseudonym map (AnonShield §2 stage (4)).
//
// Open addressing over a power-of-two slot array. The slot key packs the
// entity type (top 8 bits) with 56 bits of the entity's HMAC digest; the
// digest is a keyed hash of the exact entity bytes, so equal keys mean equal
// (type, bytes) except for a 2^-56 collision chance per pair. A slot is
// claimed by one atomicCAS; the claiming thread alone writes the payload
// (full digest, type, a copy of the original bytes in the arena), while the
// counters are updated by every occurrence with atomics (min first_seen,
// max last_seen, count). Nobody ever waits on another thread's write.
#include "scan.cuh"
#include "stages.cuh"

namespace as {

__device__ __forceinline__ unsigned long long map_key(uint32_t type, const uint32_t* d) {
  unsigned long long k = ((unsigned long long)(d[0] & 0x00FFFFFFu) << 32) | d[1];
  return ((unsigned long long)(type & 0xFFu) << 56) | k;
}

__device__ __forceinline__ uint64_t map_home(const uint32_t* d, uint64_t mask) {
  return (((uint64_t)d[2] << 32) ^ ((uint64_t)d[3] * 0x9E3779B97F4A7C15ull) ^ d[4]) & mask;
}

__global__ void map_init_kernel(MapView m) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i <= m.mask; i += (uint64_t)gridDim.x * blockDim.x) {
    MapSlot& s = m.slots[i];
    s.key = 0;
    s.first_seen = ~0ull;
    s.last_seen = 0;
    s.count = 0;
    s.arena_off = 0;
    s.len = 0;
    s.type = 0;
    s.first_call = 0;
    s.last_call = 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *m.arena_used = 0;
    *m.n_entries = 0;
  }
}

void launch_map_init(MapView m, cudaStream_t st) {
  map_init_kernel<<<grid_1d(m.mask + 1, 256, 148 * 64), 256, 0, st>>>(m);
  count_launch();
}

// Returns the slot index, or -1 when the table is full / the arena is full.
__device__ int64_t map_upsert(MapView m, uint32_t type, const uint32_t* digest, const uint8_t* orig, uint32_t len,
                              uint32_t call_id, DevError* err) {
  unsigned long long key = map_key(type, digest);
  uint64_t h = map_home(digest, m.mask);
  for (uint64_t probe = 0; probe <= m.mask; ++probe) {
    MapSlot& s = m.slots[h];
    unsigned long long cur = atomicAdd(&s.key, 0ull);
    if (cur == 0) {
      cur = atomicCAS(&s.key, 0ull, key);
      if (cur == 0) {
        // claimed: write the payload
        unsigned long long off = atomicAdd(m.arena_used, (unsigned long long)len);
        if (off + len > m.arena_cap) {
          report_error(err, kErrCapacity, 2, (uint32_t)(m.arena_cap >> 20), len);
          s.arena_off = ~0ull;
        } else {
          for (uint32_t i = 0; i < len; ++i) m.arena[off + i] = orig[i];
          s.arena_off = off;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) s.digest[i] = digest[i];
        s.len = len;
        s.type = type;
        s.first_call = call_id;
        atomicAdd(m.n_entries, 1ull);
        return (int64_t)h;
      }
    }
    if (cur == key) return (int64_t)h;
    h = (h + 1) & m.mask;
  }
  report_error(err, kErrCapacity, 1, (uint32_t)(m.mask + 1), 0);
  return -1;
}

__global__ void map_insert_spans_kernel(MapView m, const uint8_t* __restrict__ bytes, const uint32_t* __restrict__ sp_s,
                                        const uint32_t* __restrict__ sp_l, const uint8_t* __restrict__ sp_t,
                                        const uint32_t* __restrict__ digests, const uint32_t* n_dev,
                                        const uint64_t* __restrict__ offsets, uint64_t n_records, uint64_t rec_base,
                                        uint32_t call_id, DevError* err) {
  uint32_t n = *n_dev;
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    uint32_t s = sp_s[k];
    int64_t h = map_upsert(m, sp_t[k], digests + (size_t)k * 8, bytes + s, sp_l[k], call_id, err);
    if (h < 0) continue;
    uint64_t rec = rec_base + (uint64_t)upper_index(offsets, (int64_t)n_records, (uint64_t)s);
    MapSlot& sl = m.slots[h];
    atomicMin(&sl.first_seen, (unsigned long long)rec);
    atomicMax(&sl.last_seen, (unsigned long long)rec);
    atomicAdd(&sl.count, 1ull);
    atomicMax(&sl.last_call, call_id);
  }
}

void launch_map_insert_spans(MapView m, const uint8_t* bytes, const uint32_t* sp_start, const uint32_t* sp_len,
                             const uint8_t* sp_type, const uint32_t* digests, const uint32_t* n_dev, uint32_t cap,
                             const uint64_t* offsets, uint64_t n_records, uint64_t rec_base, uint32_t call_id,
                             DevError* err, cudaStream_t st) {
  if (cap == 0) return;
  map_insert_spans_kernel<<<grid_1d(cap, 256, 148 * 32), 256, 0, st>>>(m, bytes, sp_start, sp_len, sp_type, digests,
                                                                       n_dev, offsets, n_records, rec_base, call_id,
                                                                       err);
  count_launch();
}

__global__ void map_import_kernel(MapView m, const uint8_t* orig, const uint64_t* orig_off, const uint32_t* orig_len,
                                  const uint32_t* type, const uint32_t* digests, const uint64_t* first,
                                  const uint64_t* last, const uint64_t* count, uint64_t n, uint32_t call_id,
                                  DevError* err) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x) {
    int64_t h = map_upsert(m, type[k], digests + k * 8, orig + orig_off[k], orig_len[k], call_id, err);
    if (h < 0) continue;
    MapSlot& sl = m.slots[h];
    atomicMin(&sl.first_seen, (unsigned long long)first[k]);
    atomicMax(&sl.last_seen, (unsigned long long)last[k]);
    atomicAdd(&sl.count, (unsigned long long)count[k]);
    atomicMax(&sl.last_call, call_id);
  }
}

void launch_map_import(MapView m, const uint8_t* orig, const uint64_t* orig_off, const uint32_t* orig_len,
                       const uint32_t* type, const uint32_t* digests, const uint64_t* first, const uint64_t* last,
                       const uint64_t* count, uint64_t n, uint32_t call_id, DevError* err, cudaStream_t st) {
  if (n == 0) return;
  map_import_kernel<<<grid_1d(n, 256, 148 * 32), 256, 0, st>>>(m, orig, orig_off, orig_len, type, digests, first,
                                                               last, count, n, call_id, err);
  count_launch();
}

__global__ void map_select_kernel(MapView m, uint32_t call_lo, uint32_t call_hi, uint8_t* keep) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i <= m.mask; i += (uint64_t)gridDim.x * blockDim.x) {
    const MapSlot& s = m.slots[i];
    keep[i] = s.key != 0 && (call_lo == 0 || (s.last_call >= call_lo && s.last_call <= call_hi));
  }
}

void launch_map_select(MapView m, uint32_t call_lo, uint32_t call_hi, uint8_t* keep, cudaStream_t st) {
  map_select_kernel<<<grid_1d(m.mask + 1, 256, 148 * 64), 256, 0, st>>>(m, call_lo, call_hi, keep);
  count_launch();
}

__global__ void map_gather_kernel(MapView m, const uint8_t* keep, const uint32_t* pos, uint32_t* idx) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i <= m.mask; i += (uint64_t)gridDim.x * blockDim.x)
    if (keep[i]) idx[pos[i]] = (uint32_t)i;
}

void launch_map_gather(MapView m, const uint8_t* keep, const uint32_t* pos, uint32_t* idx, cudaStream_t st) {
  map_gather_kernel<<<grid_1d(m.mask + 1, 256, 148 * 64), 256, 0, st>>>(m, keep, pos, idx);
  count_launch();
}

__global__ void map_gather_slots_kernel(MapView m, const uint32_t* idx, uint32_t n, MapSlot* out) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = m.slots[idx[i]];
}

void launch_map_gather_slots(MapView m, const uint32_t* idx, uint32_t n, MapSlot* out, cudaStream_t st) {
  if (n == 0) return;
  map_gather_slots_kernel<<<grid_1d(n, 256, 148 * 32), 256, 0, st>>>(m, idx, n, out);
  count_launch();
}

}  // namespace as
