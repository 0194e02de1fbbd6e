// JSON Lines ingest (AnonShield §2 stages (1) and (5): JSON / JSONL inputs
// keep their structure and only sensitive values are replaced, with
// per-field control through the schema-aware configuration).
//
// Each record is one line. A line that is one JSON value (RFC 8259) with
// optional white space, nested at most kJsonMaxDepth containers deep, gives
// one field per run of a string VALUE's raw bytes outside escape sequences
// (so a replacement never cuts an escape); the field id is the index of the
// innermost enclosing member's key among the listed key names (raw bytes),
// n_keys when none matches or there is no member. A line that does not parse
// is one field over the whole line with id n_keys + 1 (the caller detects
// it as free text); an empty or all-white-space line has none.
//
// One thread per line walks it once to count its fields (and to decide
// whether it parses) and, after a prefix sum over the counts, once more to
// write them. The parser is iterative with a per-thread stack of container
// kinds and the field id of each open array.
#include "scan.cuh"
#include "stages.cuh"

namespace as {

namespace {

__device__ __forceinline__ bool jws(uint32_t c) { return c == ' ' || c == '\t' || c == '\n' || c == '\r'; }
__device__ __forceinline__ bool jdig(uint32_t c) { return c - '0' < 10u; }
__device__ __forceinline__ bool jhex(uint32_t c) { return c - '0' < 10u || (c | 0x20u) - 'a' < 6u; }

struct FieldSink {
  uint32_t count = 0;
  uint64_t base = 0;          // arena offset of the line
  uint64_t* start = nullptr;  // null: count only
  uint32_t* len = nullptr;
  uint32_t* id = nullptr;
  __device__ __forceinline__ void put(uint32_t a, uint32_t b, uint32_t fid) {
    if (start) {
      start[count] = base + a;
      len[count] = b - a;
      id[count] = fid;
    }
    ++count;
  }
};

// String starting with the quote at i; returns the position after the closing
// quote, or 0 when malformed. emit: runs outside escapes go to the sink.
__device__ uint32_t jstring(const uint8_t* s, uint32_t n, uint32_t i, bool emit, uint32_t fid, FieldSink& sink) {
  ++i;
  uint32_t run0 = i;
  while (i < n) {
    const uint32_t c = s[i];
    if (c == '"') {
      if (emit && i > run0) sink.put(run0, i, fid);
      return i + 1;
    }
    if (c < 0x20u) return 0;
    if (c == '\\') {
      if (emit && i > run0) sink.put(run0, i, fid);
      if (i + 1 >= n) return 0;
      const uint32_t e = s[i + 1];
      if (e == 'u') {
        if (i + 6 > n || !jhex(s[i + 2]) || !jhex(s[i + 3]) || !jhex(s[i + 4]) || !jhex(s[i + 5])) return 0;
        i += 6;
      } else if (e == '"' || e == '\\' || e == '/' || e == 'b' || e == 'f' || e == 'n' || e == 'r' || e == 't') {
        i += 2;
      } else {
        return 0;
      }
      run0 = i;
      continue;
    }
    ++i;
  }
  return 0;
}

// Number or literal at i; position after it, or 0.
__device__ uint32_t jscalar(const uint8_t* s, uint32_t n, uint32_t i) {
  const uint32_t c = s[i];
  const char* lit = c == 't' ? "true" : c == 'f' ? "false" : c == 'n' ? "null" : nullptr;
  if (lit) {
    uint32_t k = 0;
    for (; lit[k]; ++k)
      if (i + k >= n || s[i + k] != (uint8_t)lit[k]) return 0;
    return i + k;
  }
  uint32_t j = i;
  if (j < n && s[j] == '-') ++j;
  if (j < n && s[j] == '0') {
    ++j;
  } else if (j < n && jdig(s[j])) {
    while (j < n && jdig(s[j])) ++j;
  } else {
    return 0;
  }
  if (j < n && s[j] == '.') {
    ++j;
    if (!(j < n && jdig(s[j]))) return 0;
    while (j < n && jdig(s[j])) ++j;
  }
  if (j < n && (s[j] | 0x20u) == 'e') {
    ++j;
    if (j < n && (s[j] == '+' || s[j] == '-')) ++j;
    if (!(j < n && jdig(s[j]))) return 0;
    while (j < n && jdig(s[j])) ++j;
  }
  return j;
}

__device__ uint32_t jkey_id(const uint8_t* k, uint32_t len, JsonKeys K) {
  for (uint32_t t = 0; t < K.n; ++t) {
    const uint32_t a = K.off[t], b = K.off[t + 1];
    if (b - a != len) continue;
    uint32_t q = 0;
    while (q < len && k[q] == (uint8_t)K.names[a + q]) ++q;
    if (q == len) return t;
  }
  return K.n;
}

// Walks one line; false when it does not parse. Fields go to the sink.
__device__ bool jline(const uint8_t* s, uint32_t n, JsonKeys K, FieldSink& sink) {
  enum { kVal, kAfter, kObjFirst, kKey, kArrFirst };
  uint8_t is_obj[kJsonMaxDepth];
  uint32_t arr_id[kJsonMaxDepth];
  int depth = 0;
  uint32_t vid = K.n, i = 0;
  int st = kVal;
  for (;;) {
    while (i < n && jws(s[i])) ++i;
    if (st == kObjFirst) {
      if (i < n && s[i] == '}') {
        --depth;
        ++i;
        st = kAfter;
        continue;
      }
      st = kKey;
    }
    if (st == kArrFirst) {
      if (i < n && s[i] == ']') {
        --depth;
        ++i;
        st = kAfter;
        continue;
      }
      st = kVal;
    }
    if (st == kKey) {
      if (i >= n || s[i] != '"') return false;
      const uint32_t e = jstring(s, n, i, false, 0, sink);
      if (!e) return false;
      vid = jkey_id(s + i + 1, e - i - 2, K);
      i = e;
      while (i < n && jws(s[i])) ++i;
      if (i >= n || s[i] != ':') return false;
      ++i;
      st = kVal;
      continue;
    }
    if (st == kVal) {
      if (i >= n) return false;
      const uint32_t c = s[i];
      if (c == '"') {
        i = jstring(s, n, i, true, vid, sink);
        if (!i) return false;
        st = kAfter;
      } else if (c == '{' || c == '[') {
        if (depth == kJsonMaxDepth) return false;
        is_obj[depth] = c == '{';
        arr_id[depth] = vid;
        ++depth;
        ++i;
        st = c == '{' ? kObjFirst : kArrFirst;
      } else {
        i = jscalar(s, n, i);
        if (!i) return false;
        st = kAfter;
      }
      continue;
    }
    // kAfter: a value ended
    if (depth == 0) return i == n;
    if (i >= n) return false;
    const uint32_t c = s[i++];
    if (is_obj[depth - 1]) {
      if (c == ',') st = kKey;
      else if (c == '}') --depth;
      else return false;
    } else {
      if (c == ',') {
        st = kVal;
        vid = arr_id[depth - 1];
      } else if (c == ']') {
        --depth;
      } else {
        return false;
      }
    }
  }
}

}  // namespace

__global__ void jsonl_count_kernel(const uint8_t* __restrict__ bytes, const uint64_t* __restrict__ off, uint64_t n,
                                   JsonKeys K, uint32_t* __restrict__ cnt, uint8_t* __restrict__ bad,
                                   unsigned long long* n_bad) {
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < n; r += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t a = off[r];
    const uint32_t len = (uint32_t)(off[r + 1] - a);
    const uint8_t* s = bytes + a;
    uint32_t i = 0;
    while (i < len && jws(s[i])) ++i;
    FieldSink sink;
    bool ok = true;
    if (i < len) ok = jline(s, len, K, sink);
    cnt[r] = ok ? sink.count : 1u;
    bad[r] = ok ? 0 : 1;
    if (!ok) atomicAdd(n_bad, 1ull);
  }
}

__global__ void jsonl_emit_kernel(const uint8_t* __restrict__ bytes, const uint64_t* __restrict__ off, uint64_t n,
                                  JsonKeys K, const uint32_t* __restrict__ pos, const uint8_t* __restrict__ bad,
                                  uint64_t* __restrict__ f_start, uint32_t* __restrict__ f_len,
                                  uint32_t* __restrict__ f_id) {
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < n; r += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t a = off[r];
    const uint32_t len = (uint32_t)(off[r + 1] - a);
    const uint32_t k = pos[r];
    if (bad[r]) {
      f_start[k] = a;
      f_len[k] = len;
      f_id[k] = K.n + 1;
      continue;
    }
    const uint8_t* s = bytes + a;
    uint32_t i = 0;
    while (i < len && jws(s[i])) ++i;
    if (i == len) continue;
    FieldSink sink;
    sink.base = a;
    sink.start = f_start + k;
    sink.len = f_len + k;
    sink.id = f_id + k;
    jline(s, len, K, sink);
  }
}

void launch_jsonl_count(const uint8_t* bytes, const uint64_t* off, uint64_t n, JsonKeys K, uint32_t* cnt, uint8_t* bad,
                        unsigned long long* n_bad, cudaStream_t st) {
  if (n == 0) return;
  jsonl_count_kernel<<<grid_1d(n, 128, 148 * 64), 128, 0, st>>>(bytes, off, n, K, cnt, bad, n_bad);
  count_launch();
}

void launch_jsonl_emit(const uint8_t* bytes, const uint64_t* off, uint64_t n, JsonKeys K, const uint32_t* pos,
                       const uint8_t* bad, uint64_t* f_start, uint32_t* f_len, uint32_t* f_id, cudaStream_t st) {
  if (n == 0) return;
  jsonl_emit_kernel<<<grid_1d(n, 128, 148 * 64), 128, 0, st>>>(bytes, off, n, K, pos, bad, f_start, f_len, f_id);
  count_launch();
}

}  // namespace as
