// Host runtime behind the C ABI (include/anonshield.h).
//
// One as_anonymize call runs the whole path on the ctx's stream:
//   H2D (host inputs) -> tokenizer + recognizers -> [sync: token counts]
//   -> windows / packing into encoder batches -> encoder per batch
//   -> BIO decode -> overlap rule + preserve -> HMAC -> entity map
//   -> substitution -> [sync: output size] -> D2H (host inputs).
// Device buffers are owned by the ctx and only grow, so a steady stream of
// calls allocates nothing after warm-up.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <thread>
#include <unordered_map>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "encoder.cuh"
#include "scan.cuh"
#include "stages.cuh"

namespace as {

std::atomic<uint64_t> g_launches{0};
thread_local uint64_t t_launches = 0;
static thread_local std::string t_k_error;
void set_k_error(const std::string& msg) { t_k_error = msg; }

}  // namespace as

using namespace as;

namespace {

struct DBuf {
  void* p = nullptr;
  size_t cap = 0;
  template <typename T>
  T* as() const { return reinterpret_cast<T*>(p); }
};

as_status grow(DBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.cap >= bytes) return AS_OK;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
  size_t want = bytes + bytes / 8;
  if (cudaMalloc(&b.p, want) != cudaSuccess) {
    cudaGetLastError();
    set_k_error("cudaMalloc of " + std::to_string(want) + " bytes failed");
    return AS_ERR_OOM;
  }
  b.cap = want;
  return AS_OK;
}

void release(DBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
}

struct LayerW {
  const float *w_qkv, *b_qkv, *w_o, *b_o, *ln1_g, *ln1_b, *w_1, *b_1, *w_2, *b_2, *ln2_g, *ln2_b;
  __nv_bfloat16 *w_qkv16, *w_o16, *w_1_16, *w_2_16;
  uint8_t *w_qkv8, *w_o8, *w_1_8, *w_2_8;   // E4M3 copies (FP8 precision)
  float s_qkv, s_o, s_1, s_2;                // their per-tensor scales: amax / 448
};

// Encoder arithmetic of one call.
enum EncMode { kEncF32 = 0, kEncBF16 = 1, kEncFP8 = 2, kEncCalib = 3 };
// Activation scales of the FP8 path, four per layer: inputs of the QKV, output,
// FFN-in and FFN-out projections.
constexpr int kActPerLayer = 4;

struct NonZeroU8 {
  const uint8_t* p;
  __device__ uint32_t operator()(uint64_t i) const { return p[i] != 0; }
};
struct LoadI64 {
  const int64_t* p;
  __device__ int64_t operator()(uint64_t i) const { return p[i]; }
};
struct LoadU32 {
  const uint32_t* p;
  __device__ uint32_t operator()(uint64_t i) const { return p[i]; }
};

// A call with a per-field policy: the detection steps run on `rec` (the
// compact arena of fields, one sub-record per field); the rest of the path on
// the original records described here.
struct FieldJob {
  const uint8_t* bytes;           // original records (device)
  const uint64_t* offsets;        // n + 1
  uint64_t n, N;
  const uint32_t* field_start;    // nf (device)
  const uint64_t* sub_off;        // nf + 1 sub-record offsets (device)
  uint64_t nf;
  const uint32_t *fs_s, *fs_l;    // forced spans, sorted (device)
  const uint8_t* fs_t;
  const uint32_t* n_force_dev;
  uint32_t force_cap;
  bool on_device;                 // the caller's records (and so the output) are on the device
};

struct SeqDesc {
  uint32_t src_tok;  // first token of the window (global token index)
  uint32_t len;
  uint32_t row;      // first encoder row, relative to its batch
  uint16_t own_lo, own_hi;
};

struct Chunk {
  uint64_t s0, s1;   // sequences
  uint64_t rows;     // rows of the batch (sequences start on multiples of 8)
  uint32_t max_len;
  uint64_t tokens;   // rows that hold a token (the sum of the sequence lengths)
};

// cnt[5] = cnt[3] + cnt[4] (kept spans: recognizer + NER), on the device.
__global__ void sum_kept_kernel(uint32_t* cnt) {
  if (threadIdx.x == 0 && blockIdx.x == 0) cnt[5] = cnt[3] + cnt[4];
}

__global__ void expand_rows_kernel(const SeqDesc* __restrict__ seqs, int32_t* row_tok, int32_t* row_pos,
                                   uint8_t* row_own, int32_t* seq_start, int32_t* seq_len) {
  const SeqDesc d = seqs[blockIdx.x];
  if (threadIdx.x == 0) {
    seq_start[blockIdx.x] = (int32_t)d.row;
    seq_len[blockIdx.x] = (int32_t)d.len;
  }
  for (uint32_t j = threadIdx.x; j < d.len; j += blockDim.x) {
    row_tok[d.row + j] = (int32_t)(d.src_tok + j);
    row_pos[d.row + j] = (int32_t)j;
    row_own[d.row + j] = (j >= d.own_lo && j < d.own_hi) ? 1 : 0;
  }
}

}  // namespace

// Everything one in-flight call owns: its stream, device error flag, the
// per-call buffers (grown, never shrunk), the trace of its last call and its
// launch timing. as_anonymize uses the ctx's main lane; each serving worker
// has a lane of its own, so batches overlap on the device.
struct Lane {
  cudaStream_t stream = nullptr;
  DBuf dev_err;
  DBuf in_bytes, in_off, rs_bits, tok_at, scan_tiles, counters, delta_total;
  DBuf tok_ids, tok_off, tok_len, rec_tok;
  DBuf rx_len_b, rx_type_b, rx_s, rx_l, rx_t;
  DBuf labels, logits, tok_flags, bio_start, bio_end, pos_t;
  DBuf ner_s, ner_l, ner_t, keep, pos_k, nk_s, nk_l, nk_t, rk_s, rk_l, rk_t;
  DBuf fin_s, fin_l, fin_t, digests, delta, shift;
  DBuf names, name_off, name_len;
  DBuf seqs, row_tok, row_pos, row_own, seq_start, seq_len, attn_items, attn_cur;
  DBuf f_bytes, f_off, f_start, f_sub_off, f_sub, fs_s, fs_l, fs_t, fr_s, fr_l, fr_t, f_keep, f_pos, f_cnt, ff_s, ff_l,
      ff_t;
  DBuf rid_ok, rid_tk, rid_tv, rid_len, rid_slot, rid_flag, rid_pos, rid_s, rid_l, rid_k;
  DBuf j_names, j_koff, j_cnt, j_bad, j_pos, j_fs, j_fl, j_fid;
  DBuf X32, X16, QKV, ATT, Y32, H, X8, ATT8, H8;
  // last call results kept for as_debug_trace
  uint64_t last_n = 0, last_T = 0, last_nrx = 0, last_nfin = 0;
  bool last_logits = false;
  std::vector<uint64_t> h_rec_tok;
  std::vector<int32_t> h_tok_ids;
  std::vector<uint32_t> h_tok_off, h_tok_len, h_rx_s, h_rx_l, h_fin_s, h_fin_l;
  std::vector<uint8_t> h_rx_t, h_labels, h_fin_t;
  std::vector<float> h_logits;
  // launch timing (as_profile)
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<std::pair<int, double>> ev_pending;  // (kind, flops) per event pair
  as_profile_stats prof_acc{};
  // captured encoder graphs (small batches), keyed by shape, buffers and parameters
  struct EncGraph {
    std::vector<uint64_t> sig;
    cudaGraphExec_t exec = nullptr;
    uint64_t kernels = 0, used = 0;
  };
  std::vector<EncGraph> graphs;
  uint64_t graph_clock = 0, graph_replays = 0;
  bool enc_warm = false;  // an encoder batch ran kernel by kernel on this lane
  // encoder batches of this lane hold at most row_cap rows (0: the ctx's
  // max_chunk_tokens); serving lanes take it from the activation budget
  uint64_t row_cap = 0;
  std::atomic<uint64_t> act_bytes{0};  // bytes of the encoder activation buffers now held
  // pinned host staging (streaming): one batch's bytes and rebased offsets
  uint8_t* h_in = nullptr;
  size_t h_in_cap = 0;
  uint64_t* h_in_off = nullptr;
  size_t h_in_off_cap = 0;

  void release_all();
};

struct Server;

struct as_ctx {
  as_config cfg{};
  int device = 0;
  Lane main;
  // weights
  DBuf w32, w16, w8, amax_dev;
  std::vector<float> act_scale;   // kActPerLayer per layer (FP8); empty until calibrated
  bool calibrating = false;
  const float *tok_emb = nullptr, *pos_emb = nullptr, *emb_g = nullptr, *emb_b = nullptr;
  const float *cls_w = nullptr, *cls_b = nullptr;
  std::vector<LayerW> layers;
  // vocab
  DBuf vocab_slots;
  DBuf vocab_lenmask;
  uint32_t vocab_mask = 0;
  // map
  DBuf map_slots, map_arena, map_ctr;  // map_ctr: arena_used, n_entries
  uint64_t map_mask = 0;
  std::vector<uint8_t> key;
  bool key_set = false;
  DBuf key_dev, key_state;
  std::atomic<uint32_t> call_id{0};
  uint64_t records_done = 0;
  uint32_t slug_len = 10;
  std::atomic<uint64_t> n_entries_seen{0};  // map size after the previous call
  Server* server = nullptr;                 // serving loop (as_serve_start)
  int gemm_cfg[AS_TUNE_ROLES] = {-1, -1, -1, -1};  // tile configuration per projection (as_autotune)
  std::vector<std::unique_ptr<Lane>> stream_lanes;  // as_anonymize_stream workers, kept between calls
};

struct as_output {
  as_ctx* ctx = nullptr;  // used only by as_output_map (the ctx must be alive then)
  int device = 0;         // where d_bytes / d_off live: freeing needs no ctx
  uint32_t call_id = 0;
  uint32_t call_lo = 0;  // streaming outputs span the calls call_lo..call_id
  uint32_t on_device = 0;
  std::vector<uint8_t> h_bytes;
  std::vector<uint64_t> h_off;
  void* d_bytes = nullptr;
  uint64_t* d_off = nullptr;
  uint64_t n = 0;
  as_stats stats{};
  bool map_loaded = false;
  std::vector<as_entity> map;
  std::vector<uint8_t> map_orig;
};

void Lane::release_all() {
  DBuf* all[] = {&dev_err, &in_bytes, &in_off, &rs_bits, &tok_at, &scan_tiles, &counters, &delta_total,
                 &tok_ids, &tok_off, &tok_len, &rec_tok, &rx_len_b, &rx_type_b, &rx_s, &rx_l, &rx_t, &labels, &logits,
                 &tok_flags, &bio_start, &bio_end, &pos_t, &ner_s, &ner_l, &ner_t, &keep, &pos_k, &nk_s,
                 &nk_l, &nk_t, &rk_s, &rk_l, &rk_t, &fin_s, &fin_l, &fin_t, &digests, &delta, &shift, &names,
                 &name_off, &name_len, &seqs, &attn_items, &attn_cur, &f_bytes, &f_off, &f_start, &f_sub_off, &f_sub, &fs_s,
                 &fs_l, &fs_t, &fr_s, &fr_l, &fr_t, &f_keep, &f_pos, &f_cnt, &ff_s, &ff_l, &ff_t, &row_tok, &row_pos, &row_own, &seq_start, &seq_len, &X32, &X16, &QKV,
                 &ATT, &Y32, &H, &X8, &ATT8, &H8,
                  &rid_ok, &rid_tk, &rid_tv, &rid_len, &rid_slot, &rid_flag, &rid_pos, &rid_s, &rid_l, &rid_k,
                  &j_names, &j_koff, &j_cnt, &j_bad, &j_pos, &j_fs, &j_fl, &j_fid};
  for (DBuf* b : all) release(*b);
  for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
  ev_pool.clear();
  for (EncGraph& gr : graphs)
    if (gr.exec) cudaGraphExecDestroy(gr.exec);
  graphs.clear();
  enc_warm = false;
  if (h_in) cudaFreeHost(h_in);
  if (h_in_off) cudaFreeHost(h_in_off);
  h_in = nullptr;
  h_in_off = nullptr;
  h_in_cap = h_in_off_cap = 0;
}

namespace {

// Message of the last failure on the calling thread (one ctx per thread is
// the ABI convention; serving workers are threads of their own).
thread_local std::string t_err;

as_status fail(as_ctx*, as_status s, const std::string& msg) {
  t_err = msg;
  return s;
}

#define CK(expr)                                                                                   \
  do {                                                                                             \
    cudaError_t _e = (expr);                                                                       \
    if (_e != cudaSuccess) return fail(c, AS_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
  } while (0)

#define CKS(expr)                                                      \
  do {                                                                 \
    as_status _s = (expr);                                             \
    if (_s != AS_OK) return fail(c, _s, t_k_error_or(#expr));          \
  } while (0)

#define CKI(expr)                  \
  do {                             \
    as_status _s = (expr);         \
    if (_s != AS_OK) return _s;    \
  } while (0)

std::string t_k_error_or(const char* what) {
  const char* e = as_k_last_error();
  return std::string(what) + ": " + (e ? e : "");
}

MapView map_view(as_ctx* c) {
  MapView m;
  m.slots = c->map_slots.as<MapSlot>();
  m.mask = c->map_mask;
  m.arena = c->map_arena.as<uint8_t>();
  m.arena_used = c->map_ctr.as<unsigned long long>();
  m.arena_cap = c->map_arena.cap;
  m.n_entries = c->map_ctr.as<unsigned long long>() + 1;
  return m;
}

as_status check_dev_error(as_ctx* c, Lane* ln) {
  DevError e{};
  CK(cudaMemcpyAsync(&e, ln->dev_err.p, sizeof(e), cudaMemcpyDeviceToHost, ln->stream));
  CK(cudaStreamSynchronize(ln->stream));
  if (e.code == 0) return AS_OK;
  cudaMemsetAsync(ln->dev_err.p, 0, sizeof(DevError), ln->stream);
  if (e.code == kErrTimeout)
    return fail(c, AS_ERR_TIMEOUT, "a bounded device wait ran out (site " + std::to_string(e.where) + ")");
  if (e.code == kErrCapacity)
    return fail(c, AS_ERR_CAPACITY, "entity map full (site " + std::to_string(e.where) + "); raise map_capacity / map_arena_bytes");
  return fail(c, AS_ERR_CUDA, "device error code " + std::to_string(e.code));
}

uint64_t pow2_at_least(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

as_status build_vocab(as_ctx* c) {
  const as_config& g = c->cfg;
  uint64_t n = g.n_vocab_words;
  // about 8 slots per string: a lookup of a string that is not there
  // usually ends at its first slot
  uint64_t size = std::max<uint64_t>(1024, pow2_at_least(8 * n + 1));
  std::vector<uint4> slots(size, make_uint4(0, 0, 0, 0));
  std::vector<uint16_t> lenmask((size_t)kAlnumCodes * kAlnumCodes, 0);
  for (uint64_t k = 0; k < n; ++k) {
    uint32_t a = g.vocab_offsets[k], b = g.vocab_offsets[k + 1];
    if (b <= a) return fail(c, AS_ERR_ARG, "vocab offsets must increase");
    uint32_t len = b - a;
    if (len < 2 || len > (uint32_t)kMaxPiece) return fail(c, AS_ERR_ARG, "vocab strings must be 2..12 bytes");
    uint32_t w[3] = {0, 0, 0};
    for (uint32_t i = 0; i < len; ++i) {
      uint8_t ch = g.vocab_bytes[a + i];
      bool an = (ch >= '0' && ch <= '9') || (ch >= 'A' && ch <= 'Z') || (ch >= 'a' && ch <= 'z');
      if (!an) return fail(c, AS_ERR_ARG, "vocab strings must be [0-9A-Za-z]");
      w[i >> 2] |= (uint32_t)ch << (8 * (i & 3));
    }
    uint32_t id = (uint32_t)(257 + k);
    lenmask[alnum_code(g.vocab_bytes[a]) * kAlnumCodes + alnum_code(g.vocab_bytes[a + 1])] |= (uint16_t)(1u << len);
    uint32_t h = vocab_hash(w[0], w[1], w[2], len) & (uint32_t)(size - 1);
    while (true) {
      uint4& s = slots[h];
      if (s.w == 0) {
        s = make_uint4(w[0], w[1], w[2], len | (id << 16));
        break;
      }
      if ((s.w & 0xFFFFu) == len && s.x == w[0] && s.y == w[1] && s.z == w[2])
        return fail(c, AS_ERR_ARG, "duplicate vocab string at id " + std::to_string(id));
      h = (h + 1) & (uint32_t)(size - 1);
    }
  }
  CKS(grow(c->vocab_slots, size * sizeof(uint4)));
  CK(cudaMemcpy(c->vocab_slots.p, slots.data(), size * sizeof(uint4), cudaMemcpyHostToDevice));
  CKS(grow(c->vocab_lenmask, lenmask.size() * sizeof(uint16_t)));
  CK(cudaMemcpy(c->vocab_lenmask.p, lenmask.data(), lenmask.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
  c->vocab_mask = (uint32_t)(size - 1);
  return AS_OK;
}

uint64_t expected_weights(const as_config& g) {
  uint64_t d = g.d_model, f = g.d_ffn;
  uint64_t per_layer = 3 * d * d + 3 * d + d * d + d + 2 * d + f * d + f + d * f + d + 2 * d;
  return (uint64_t)g.vocab * d + (uint64_t)g.max_pos * d + 2 * d + g.n_layers * per_layer + (uint64_t)g.n_labels * d +
         g.n_labels;
}

as_status load_weights(as_ctx* c) {
  const as_config& g = c->cfg;
  uint64_t n = g.weights_len;
  CKS(grow(c->w32, n * 4));
  CK(cudaMemcpy(c->w32.p, g.weights, n * 4, cudaMemcpyHostToDevice));
  const float* p = c->w32.as<float>();
  uint64_t d = g.d_model, f = g.d_ffn;
  auto take = [&](uint64_t k) { const float* q = p; p += k; return q; };
  c->tok_emb = take((uint64_t)g.vocab * d);
  c->pos_emb = take((uint64_t)g.max_pos * d);
  c->emb_g = take(d);
  c->emb_b = take(d);
  c->layers.resize(g.n_layers);
  for (auto& L : c->layers) {
    L.w_qkv = take(3 * d * d); L.b_qkv = take(3 * d);
    L.w_o = take(d * d); L.b_o = take(d);
    L.ln1_g = take(d); L.ln1_b = take(d);
    L.w_1 = take(f * d); L.b_1 = take(f);
    L.w_2 = take(d * f); L.b_2 = take(d);
    L.ln2_g = take(d); L.ln2_b = take(d);
  }
  c->cls_w = take((uint64_t)g.n_labels * d);
  c->cls_b = take(g.n_labels);
  if (g.precision == AS_BF16 || g.precision == AS_FP8) {
    uint64_t per = 3 * d * d + d * d + f * d + d * f;
    CKS(grow(c->w16, per * g.n_layers * 2));
    __nv_bfloat16* q = c->w16.as<__nv_bfloat16>();
    for (auto& L : c->layers) {
      L.w_qkv16 = q; convert_f32_bf16(L.w_qkv, q, 3 * d * d, c->main.stream); q += 3 * d * d;
      L.w_o16 = q; convert_f32_bf16(L.w_o, q, d * d, c->main.stream); q += d * d;
      L.w_1_16 = q; convert_f32_bf16(L.w_1, q, f * d, c->main.stream); q += f * d;
      L.w_2_16 = q; convert_f32_bf16(L.w_2, q, d * f, c->main.stream); q += d * f;
    }
    CK(cudaStreamSynchronize(c->main.stream));
  }
  if (g.precision == AS_FP8) {
    // per-tensor weight scales s = amax / 448, then E4M3 copies
    uint64_t per = 3 * d * d + d * d + f * d + d * f;
    CKS(grow(c->w8, per * g.n_layers));
    CKS(grow(c->amax_dev, 4 * g.n_layers * 4));
    CK(cudaMemsetAsync(c->amax_dev.p, 0, 4 * g.n_layers * 4, c->main.stream));
    unsigned int* am = c->amax_dev.as<unsigned int>();
    for (uint32_t l = 0; l < g.n_layers; ++l) {
      const LayerW& L = c->layers[l];
      amax_f32(L.w_qkv, 3 * d * d, am + 4 * l + 0, c->main.stream);
      amax_f32(L.w_o, d * d, am + 4 * l + 1, c->main.stream);
      amax_f32(L.w_1, f * d, am + 4 * l + 2, c->main.stream);
      amax_f32(L.w_2, d * f, am + 4 * l + 3, c->main.stream);
    }
    std::vector<unsigned int> bits(4 * g.n_layers);
    CK(cudaMemcpyAsync(bits.data(), am, bits.size() * 4, cudaMemcpyDeviceToHost, c->main.stream));
    CK(cudaStreamSynchronize(c->main.stream));
    auto scale_of = [](unsigned int b) {
      float a;
      memcpy(&a, &b, 4);
      return a > 0.f ? a / 448.0f : 1.0f;
    };
    uint8_t* q = c->w8.as<uint8_t>();
    for (uint32_t l = 0; l < g.n_layers; ++l) {
      LayerW& L = c->layers[l];
      L.s_qkv = scale_of(bits[4 * l + 0]);
      L.s_o = scale_of(bits[4 * l + 1]);
      L.s_1 = scale_of(bits[4 * l + 2]);
      L.s_2 = scale_of(bits[4 * l + 3]);
      L.w_qkv8 = q; quantize_e4m3(L.w_qkv, q, 3 * d * d, L.s_qkv, c->main.stream); q += 3 * d * d;
      L.w_o8 = q; quantize_e4m3(L.w_o, q, d * d, L.s_o, c->main.stream); q += d * d;
      L.w_1_8 = q; quantize_e4m3(L.w_1, q, f * d, L.s_1, c->main.stream); q += f * d;
      L.w_2_8 = q; quantize_e4m3(L.w_2, q, d * f, L.s_2, c->main.stream); q += d * f;
    }
    CK(cudaStreamSynchronize(c->main.stream));
  }
  return AS_OK;
}

// ---------------------------------------------------------------- encoder

// Event pair around one launch when profiling is on (kind 0 GEMM, 1 attention),
// or around one integer stage of a batch call (kinds 2..5, the order of
// as_profile_stats.stage_ms). Scopes never nest: event i of the pool belongs
// to pending entry i / 2.
// A stage scope is also an NVTX range (named below, whether or not event
// timing is on), so that a profiler can select a stage's kernels by name.
constexpr int kProfGemm = 0, kProfAttn = 1, kProfText = 2, kProfSpans = 3, kProfHash = 4, kProfSubst = 5;
constexpr const char* kStageRange[4] = {"as.text", "as.spans", "as.hash_map", "as.substitution"};
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};
struct ProfScope {
  Lane* ln;
  bool on;
  bool range = false;
  ProfScope(Lane* ln_, int kind, double flops) : ln(ln_), on(ln_->prof) {
    if (kind >= kProfText) {
      nvtxRangePushA(kStageRange[kind - kProfText]);
      range = true;
    }
    if (!on) return;
    if (ln->ev_used + 2 > ln->ev_pool.size()) {
      for (int i = 0; i < 64; ++i) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        ln->ev_pool.push_back(e);
      }
    }
    cudaEventRecord(ln->ev_pool[ln->ev_used], ln->stream);
    ln->ev_pending.push_back({kind, flops});
  }
  // records the closing event (once; the destructor closes a scope still open)
  void end() {
    if (range) {
      nvtxRangePop();
      range = false;
    }
    if (!on) return;
    on = false;
    cudaEventRecord(ln->ev_pool[ln->ev_used + 1], ln->stream);
    ln->ev_used += 2;
  }
  ~ProfScope() { end(); }
};

// After a stream sync: fold the recorded event pairs into the totals.
void prof_collect(Lane* ln) {
  for (size_t i = 0; i < ln->ev_pending.size(); ++i) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ln->ev_pool[2 * i], ln->ev_pool[2 * i + 1]);
    const int kind = ln->ev_pending[i].first;
    if (kind == kProfGemm) {
      ln->prof_acc.gemm_launches++;
      ln->prof_acc.gemm_ms += ms;
      ln->prof_acc.gemm_flops += ln->ev_pending[i].second;
    } else if (kind == kProfAttn) {
      ln->prof_acc.attn_launches++;
      ln->prof_acc.attn_ms += ms;
      ln->prof_acc.attn_flops += ln->ev_pending[i].second;
    } else {
      if (kind == kProfText) ln->prof_acc.stage_calls++;
      ln->prof_acc.stage_ms[kind - kProfText] += ms;
    }
  }
  ln->ev_pending.clear();
  ln->ev_used = 0;
}

constexpr uint64_t kGraphSmallRows = AS_GRAPH_MAX_ROWS;
constexpr size_t kGraphCache = 16;

uint64_t pow2_at_least(uint64_t x, uint64_t lo) {
  uint64_t v = lo;
  while (v < x) v <<= 1;
  return v;
}

// Graph shape bucket of a count x (rows or attention work items): a power of
// two (at least lo) up to kGraphSmallRows, above that the next multiple of
// 1/16 of the next power of two (at most 6.25 % padding), so that one
// captured graph serves every batch of the same bucket. Full packed batches
// (just under the row cap, a power of two by default) share one bucket.
uint64_t graph_bucket(uint64_t x, uint64_t lo) {
  const uint64_t p = pow2_at_least(x, lo);
  if (p <= kGraphSmallRows) return p;
  const uint64_t q = p / 16;
  return (x + q - 1) / q * q;
}

// Encoder batches of BF16 / FP8 contexts with the tcgen05 attention run as
// graphs (graphs on); their rows are padded to the bucket.
bool graphable(const as_config& g) {
  return !g.no_graphs && g.precision != AS_FP32 && g.attention == AS_ATTN_TCGEN05;
}
uint64_t encoder_rows(const as_config& g, uint64_t rows) { return graphable(g) ? graph_bucket(rows, 128) : rows; }

// Post-LN residual block `block` (0 attention, 1 feed-forward) as one
// clustered GEMM + LayerNorm kernel, and whether that kernel runs on 2-SM
// pairs (tile configuration bit 2 of its projection; default: pairs for the
// feed-forward block, whose K = d_ffn is long enough to pay for them).
bool ln_fused(const as_config& g, int block) {
  return g.precision != AS_FP32 && gemm_resid_ln_cluster(g.d_model) > 0 && !(g.no_fused_ln & (1u << block));
}
bool ln_pair(const int cfg, int block) { return cfg < 0 ? block == 1 : (cfg & 4) != 0; }
// deep epilogue staging (tile configuration bit 1 of a fused block; off by default)
bool ln_deep(const int cfg, int) { return cfg >= 0 && (cfg & 2) != 0; }

// Embedding, the layers and the classifier over R rows (everything of an
// encoder batch whose launch shapes depend only on R and n_items).
as_status encoder_body(as_ctx* c, Lane* ln, int64_t R, int32_t ns, uint32_t max_len, double attn_flops,
                       bool want_logits, const int32_t* attn_items, int32_t n_items, int64_t R_alg) {
  const as_config& g = c->cfg;
  const int32_t d = (int32_t)g.d_model, f = (int32_t)g.d_ffn;
  cudaStream_t st = ln->stream;
  float* X32 = ln->X32.as<float>();
  float* Y32 = ln->Y32.as<float>();
  const int mode = g.precision == AS_FP32 ? kEncF32
                   : g.precision == AS_BF16 ? kEncBF16
                                            : (c->calibrating ? kEncCalib : kEncFP8);
  const bool bf = mode == kEncBF16 || mode == kEncCalib;
  const bool f8 = mode == kEncFP8;
  __nv_bfloat16* X16 = bf ? ln->X16.as<__nv_bfloat16>() : nullptr;
  uint8_t* X8 = f8 ? ln->X8.as<uint8_t>() : nullptr;
  unsigned int* amax = c->amax_dev.as<unsigned int>();
  const float* as8 = f8 ? c->act_scale.data() : nullptr;
  const uint64_t Rd = (uint64_t)R * d;
  CKS(embed_ln_ex(ln->tok_ids.as<int32_t>(), ln->row_tok.as<int32_t>(), ln->row_pos.as<int32_t>(), c->tok_emb,
                  c->pos_emb, c->emb_g, c->emb_b, X32, X16, X8, f8 ? as8[0] : 1.0f, R, d, st));
  if (mode == kEncCalib) amax_bf16(X16, Rd, amax + 0, st);
  DevError* err = ln->dev_err.as<DevError>();
  // post-LN residual blocks as one clustered kernel (BF16 / FP8)
  const bool fuse_ln = ln_fused(g, 0), fuse_ln2 = ln_fused(g, 1);
  const bool pair1 = ln_pair(c->gemm_cfg[1], 0), pair2 = ln_pair(c->gemm_cfg[3], 1);
  const bool deep1 = ln_deep(c->gemm_cfg[1], 0), deep2 = ln_deep(c->gemm_cfg[3], 1);
  for (uint32_t l = 0; l < g.n_layers; ++l) {
    const LayerW& L = c->layers[l];
    const bool last = l + 1 == g.n_layers;
    if (f8) {
      const float* sc = as8 + kActPerLayer * l;
      __nv_bfloat16* QKV = ln->QKV.as<__nv_bfloat16>();
      uint8_t* ATT8 = ln->ATT8.as<uint8_t>();
      uint8_t* H8 = ln->H8.as<uint8_t>();
      { ProfScope ps(ln, 0, 2.0 * R_alg * 3 * d * d);
        CKS(gemm_tcgen05_ex(AS_EPI_BIAS, true, false, R, 3 * d, d, X8, L.w_qkv8, L.b_qkv, nullptr, QKV,
                            sc[0] * L.s_qkv, 1.0f, err, st, c->gemm_cfg[0])); }
      { ProfScope ps(ln, 1, attn_flops);
        if (g.attention == AS_ATTN_TCGEN05)
          CKS(attention_tcgen05_e4m3(QKV, ATT8, sc[1], attn_items, n_items, (int32_t)max_len, R, d,
                                     (int32_t)g.n_heads, err, st));
        else
          CKS(attention_bf16_e4m3(QKV, ATT8, sc[1], ln->seq_start.as<int32_t>(), ln->seq_len.as<int32_t>(), ns,
                                  (int32_t)max_len, d, (int32_t)g.n_heads, st)); }
      if (fuse_ln) {
        ProfScope ps(ln, 0, 2.0 * R_alg * d * d);
        CKS(gemm_tcgen05_resid_ln(true, R, d, d, ATT8, L.w_o8, L.b_o, X32, L.ln1_g, L.ln1_b, nullptr, X8, sc[2],
                                  sc[1] * L.s_o, err, st, pair1, deep1));
      } else {
        { ProfScope ps(ln, 0, 2.0 * R_alg * d * d);
          CKS(gemm_tcgen05_ex(AS_EPI_BIAS_RESID, true, false, R, d, d, ATT8, L.w_o8, L.b_o, X32, Y32, sc[1] * L.s_o,
                              1.0f, err, st, c->gemm_cfg[1])); }
        CKS(layernorm_rows_ex(Y32, L.ln1_g, L.ln1_b, X32, nullptr, X8, sc[2], R, d, st));
      }
      { ProfScope ps(ln, 0, 2.0 * R_alg * f * d);
        CKS(gemm_tcgen05_ex(AS_EPI_BIAS_GELU, true, true, R, f, d, X8, L.w_1_8, L.b_1, nullptr, H8, sc[2] * L.s_1,
                            sc[3], err, st, c->gemm_cfg[2])); }
      if (fuse_ln2 && !last) {
        ProfScope ps(ln, 0, 2.0 * R_alg * d * f);
        CKS(gemm_tcgen05_resid_ln(true, R, d, f, H8, L.w_2_8, L.b_2, X32, L.ln2_g, L.ln2_b, nullptr, X8,
                                  as8[kActPerLayer * (l + 1)], sc[3] * L.s_2, err, st, pair2, deep2));
        continue;
      }
      { ProfScope ps(ln, 0, 2.0 * R_alg * d * f);
        CKS(gemm_tcgen05_ex(AS_EPI_BIAS_RESID, true, false, R, d, f, H8, L.w_2_8, L.b_2, X32, Y32, sc[3] * L.s_2,
                            1.0f, err, st, c->gemm_cfg[3])); }
    } else if (bf) {
      __nv_bfloat16* QKV = ln->QKV.as<__nv_bfloat16>();
      __nv_bfloat16* ATT = ln->ATT.as<__nv_bfloat16>();
      __nv_bfloat16* H = ln->H.as<__nv_bfloat16>();
      { ProfScope ps(ln, 0, 2.0 * R_alg * 3 * d * d); CKS(gemm_tcgen05_ex(AS_EPI_BIAS, false, false, R, 3 * d, d, X16, L.w_qkv16, L.b_qkv, nullptr, QKV, 1.0f, 1.0f, err, st, c->gemm_cfg[0])); }
      if (g.attention == AS_ATTN_TCGEN05) {
        ProfScope ps(ln, 1, attn_flops);
        CKS(attention_tcgen05(QKV, ATT, attn_items, n_items, (int32_t)max_len, R, d, (int32_t)g.n_heads, err, st));
      } else {
        ProfScope ps(ln, 1, attn_flops);
        CKS(attention_bf16(QKV, ATT, ln->seq_start.as<int32_t>(), ln->seq_len.as<int32_t>(), ns, (int32_t)max_len, d,
                           (int32_t)g.n_heads, st));
      }
      if (mode == kEncCalib) amax_bf16(ATT, Rd, amax + kActPerLayer * l + 1, st);
      if (fuse_ln) {
        ProfScope ps(ln, 0, 2.0 * R_alg * d * d);
        CKS(gemm_tcgen05_resid_ln(false, R, d, d, ATT, L.w_o16, L.b_o, X32, L.ln1_g, L.ln1_b, X16, nullptr, 1.0f,
                                  1.0f, err, st, pair1, deep1));
      } else {
        { ProfScope ps(ln, 0, 2.0 * R_alg * d * d); CKS(gemm_tcgen05_ex(AS_EPI_BIAS_RESID, false, false, R, d, d, ATT, L.w_o16, L.b_o, X32, Y32, 1.0f, 1.0f, err, st, c->gemm_cfg[1])); }
        CKS(layernorm_rows(Y32, L.ln1_g, L.ln1_b, X32, X16, R, d, st));
      }
      if (mode == kEncCalib) amax_bf16(X16, Rd, amax + kActPerLayer * l + 2, st);
      { ProfScope ps(ln, 0, 2.0 * R_alg * f * d); CKS(gemm_tcgen05_ex(AS_EPI_BIAS_GELU, false, false, R, f, d, X16, L.w_1_16, L.b_1, nullptr, H, 1.0f, 1.0f, err, st, c->gemm_cfg[2])); }
      if (mode == kEncCalib) amax_bf16(H, (uint64_t)R * f, amax + kActPerLayer * l + 3, st);
      if (fuse_ln2 && !last) {
        { ProfScope ps(ln, 0, 2.0 * R_alg * d * f);
          CKS(gemm_tcgen05_resid_ln(false, R, d, f, H, L.w_2_16, L.b_2, X32, L.ln2_g, L.ln2_b, X16, nullptr, 1.0f,
                                    1.0f, err, st, pair2, deep2)); }
        if (mode == kEncCalib) amax_bf16(X16, Rd, amax + kActPerLayer * (l + 1), st);
        continue;
      }
      { ProfScope ps(ln, 0, 2.0 * R_alg * d * f); CKS(gemm_tcgen05_ex(AS_EPI_BIAS_RESID, false, false, R, d, f, H, L.w_2_16, L.b_2, X32, Y32, 1.0f, 1.0f, err, st, c->gemm_cfg[3])); }
    } else {
      float* QKV = ln->QKV.as<float>();
      float* ATT = ln->ATT.as<float>();
      float* H = ln->H.as<float>();
      { ProfScope ps(ln, 0, 2.0 * R_alg * 3 * d * d); CKS(gemm_simt_f32(AS_EPI_BIAS, R, 3 * d, d, X32, L.w_qkv, L.b_qkv, nullptr, QKV, st)); }
      { ProfScope ps(ln, 1, attn_flops);
        CKS(attention_f32(QKV, ATT, ln->seq_start.as<int32_t>(), ln->seq_len.as<int32_t>(), ns, (int32_t)max_len, d,
                          (int32_t)g.n_heads, st)); }
      { ProfScope ps(ln, 0, 2.0 * R_alg * d * d); CKS(gemm_simt_f32(AS_EPI_BIAS_RESID, R, d, d, ATT, L.w_o, L.b_o, X32, Y32, st)); }
      CKS(layernorm_rows(Y32, L.ln1_g, L.ln1_b, X32, nullptr, R, d, st));
      { ProfScope ps(ln, 0, 2.0 * R_alg * f * d); CKS(gemm_simt_f32(AS_EPI_BIAS_GELU, R, f, d, X32, L.w_1, L.b_1, nullptr, H, st)); }
      { ProfScope ps(ln, 0, 2.0 * R_alg * d * f); CKS(gemm_simt_f32(AS_EPI_BIAS_RESID, R, d, f, H, L.w_2, L.b_2, X32, Y32, st)); }
    }
    if (!last) {
      CKS(layernorm_rows_ex(Y32, L.ln2_g, L.ln2_b, X32, X16, X8, f8 ? as8[kActPerLayer * (l + 1)] : 1.0f, R, d, st));
      if (mode == kEncCalib) amax_bf16(X16, Rd, amax + kActPerLayer * (l + 1), st);
    } else {
      CKS(layernorm_classify(Y32, L.ln2_g, L.ln2_b, c->cls_w, c->cls_b, (int32_t)g.n_labels, ln->row_tok.as<int32_t>(),
                             ln->row_own.as<uint8_t>(), want_logits ? ln->logits.as<float>() : nullptr,
                             ln->labels.as<uint8_t>(), R, d, st));
    }
  }
  return AS_OK;
}

as_status run_encoder_chunk(as_ctx* c, Lane* ln, const Chunk& ch, const SeqDesc* seq_dev, double attn_flops,
                            bool want_logits, const int32_t* attn_items, int32_t n_items) {
  const as_config& g = c->cfg;
  const int64_t R = (int64_t)ch.rows;
  const int64_t Rb = (int64_t)encoder_rows(g, ch.rows);  // R, or its graph bucket
  const int64_t R_alg = (int64_t)ch.tokens;              // rows that hold a token (FLOP accounting)
  const int32_t ns = (int32_t)(ch.s1 - ch.s0);
  cudaStream_t st = ln->stream;
  // padding rows between sequences (and up to the bucket): token 0, position 0, owned by nobody
  CK(cudaMemsetAsync(ln->row_tok.p, 0, Rb * 4, st));
  CK(cudaMemsetAsync(ln->row_pos.p, 0, Rb * 4, st));
  CK(cudaMemsetAsync(ln->row_own.p, 0, Rb, st));
  // sequence ns is empty: padded attention work items point at it
  CK(cudaMemsetAsync(ln->seq_start.as<int32_t>() + ns, 0, 4, st));
  CK(cudaMemsetAsync(ln->seq_len.as<int32_t>() + ns, 0, 4, st));
  expand_rows_kernel<<<ns, 128, 0, st>>>(seq_dev + ch.s0, ln->row_tok.as<int32_t>(), ln->row_pos.as<int32_t>(),
                                         ln->row_own.as<uint8_t>(), ln->seq_start.as<int32_t>(), ln->seq_len.as<int32_t>());
  count_launch();
  const bool graph = graphable(g);
  if (!graph || !ln->enc_warm || ln->prof || c->calibrating) {
    CKS(encoder_body(c, ln, graph ? Rb : R, ns, ch.max_len, attn_flops, want_logits, attn_items, n_items, R_alg));
    ln->enc_warm = true;
    return AS_OK;
  }
  // the batch's work items go to one fixed lane buffer, so that every batch of
  // a call (and of later calls) with the same shape bucket replays one graph
  CKS(grow(ln->attn_cur, std::max<size_t>(1, (size_t)n_items) * 8));
  if (n_items) CK(cudaMemcpyAsync(ln->attn_cur.p, attn_items, (size_t)n_items * 8, cudaMemcpyDeviceToDevice, st));
  attn_items = ln->attn_cur.as<int32_t>();
  // one graph launch per batch: look up (or capture) the graph of this shape
  std::vector<uint64_t> sig = {(uint64_t)Rb, (uint64_t)n_items, (uint64_t)want_logits, (uint64_t)g.precision};
  for (const DBuf* b : {&ln->X32, &ln->Y32, &ln->X16, &ln->X8, &ln->QKV, &ln->ATT, &ln->ATT8, &ln->H, &ln->H8,
                        &ln->row_tok, &ln->row_pos, &ln->row_own, &ln->seq_start, &ln->seq_len, &ln->tok_ids,
                        &ln->logits, &ln->labels})
    sig.push_back(reinterpret_cast<uint64_t>(b->p));
  sig.push_back(reinterpret_cast<uint64_t>(attn_items));
  for (int r = 0; r < AS_TUNE_ROLES; ++r) sig.push_back((uint64_t)(int64_t)c->gemm_cfg[r]);
  for (float x : c->act_scale) {  // FP8 scales are kernel arguments
    uint32_t u;
    memcpy(&u, &x, 4);
    sig.push_back(u);
  }
  Lane::EncGraph* hit = nullptr;
  for (Lane::EncGraph& gr : ln->graphs)
    if (gr.sig == sig) hit = &gr;
  if (!hit) {
    if (ln->graphs.size() >= kGraphCache) {  // evict the least recently used
      auto lru = std::min_element(ln->graphs.begin(), ln->graphs.end(),
                                  [](const Lane::EncGraph& a, const Lane::EncGraph& b) { return a.used < b.used; });
      cudaGraphExecDestroy(lru->exec);
      ln->graphs.erase(lru);
    }
    cudaGraph_t gr = nullptr;
    const uint64_t l0 = t_launches;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      CKS(encoder_body(c, ln, Rb, ns, ch.max_len, attn_flops, want_logits, attn_items, n_items, R_alg));
      return AS_OK;
    }
    const as_status bs = encoder_body(c, ln, Rb, ns, ch.max_len, attn_flops, want_logits, attn_items, n_items, R_alg);
    const cudaError_t ce = cudaStreamEndCapture(st, &gr);
    const uint64_t kernels = t_launches - l0;
    g_launches.fetch_sub(kernels);  // captured, not run: counted when the graph is launched
    t_launches -= kernels;
    cudaGraphExec_t exec = nullptr;
    if (bs != AS_OK || ce != cudaSuccess || !gr || cudaGraphInstantiate(&exec, gr, 0) != cudaSuccess) {
      if (gr) cudaGraphDestroy(gr);
      cudaGetLastError();
      // capture refused: run this batch kernel by kernel
      CKS(encoder_body(c, ln, Rb, ns, ch.max_len, attn_flops, want_logits, attn_items, n_items, R_alg));
      return AS_OK;
    }
    cudaGraphDestroy(gr);
    ln->graphs.push_back(Lane::EncGraph{std::move(sig), exec, kernels, 0});
    hit = &ln->graphs.back();
  }
  hit->used = ++ln->graph_clock;
  CK(cudaGraphLaunch(hit->exec, st));
  count_launch(hit->kernels);
  ++ln->graph_replays;
  return AS_OK;
}

as_status ensure_encoder_buffers(as_ctx* c, Lane* ln, uint64_t rows, uint64_t n_seq) {
  const as_config& g = c->cfg;
  const uint64_t d = g.d_model, f = g.d_ffn;
  const bool bf = g.precision != AS_FP32;   // FP8 keeps BF16 buffers for calibration and QKV
  const bool f8 = g.precision == AS_FP8;
  const size_t act = bf ? 2 : 4;
  CKS(grow(ln->row_tok, rows * 4));
  CKS(grow(ln->row_pos, rows * 4));
  CKS(grow(ln->row_own, rows));
  CKS(grow(ln->seq_start, n_seq * 4));
  CKS(grow(ln->seq_len, n_seq * 4));
  CKS(grow(ln->X32, rows * d * 4));
  CKS(grow(ln->Y32, rows * d * 4));
  if (bf) CKS(grow(ln->X16, rows * d * 2));
  CKS(grow(ln->QKV, rows * 3 * d * act));
  const void* att_before = ln->ATT.p;
  CKS(grow(ln->ATT, rows * d * act));
  // rows no sequence covers are never written by attention: keep them finite
  if (ln->ATT.p != att_before) CK(cudaMemsetAsync(ln->ATT.p, 0, ln->ATT.cap, ln->stream));
  CKS(grow(ln->H, rows * f * act));
  if (f8) {
    CKS(grow(ln->X8, rows * d));
    const void* before = ln->ATT8.p;
    CKS(grow(ln->ATT8, rows * d));
    if (ln->ATT8.p != before) CK(cudaMemsetAsync(ln->ATT8.p, 0, ln->ATT8.cap, ln->stream));
    CKS(grow(ln->H8, rows * f));
  }
  uint64_t held = 0;
  for (const DBuf* b : {&ln->row_tok, &ln->row_pos, &ln->row_own, &ln->X32, &ln->Y32, &ln->X16, &ln->QKV, &ln->ATT,
                        &ln->H, &ln->X8, &ln->ATT8, &ln->H8})
    held += b->cap;
  ln->act_bytes.store(held);
  return AS_OK;
}

// Bytes the encoder activation buffers of a lane hold for `rows` rows: the
// buffers ensure_encoder_buffers sizes by rows, each allocated with the 1/8
// slack of grow().
uint64_t encoder_held_bytes(const as_config& g, uint64_t rows) {
  const uint64_t d = g.d_model, f = g.d_ffn;
  const bool bf = g.precision != AS_FP32, f8 = g.precision == AS_FP8;
  const uint64_t act = bf ? 2 : 4;
  const uint64_t per_buffer[] = {4, 4, 1, 4 * d, 4 * d, bf ? 2 * d : 0, 3 * d * act, d * act, f * act,
                                 f8 ? d : 0, f8 ? d : 0, f8 ? f : 0};
  uint64_t held = 0;
  for (uint64_t b : per_buffer)
    if (b) held += rows * b + rows * b / 8;
  return held;
}

RxTypes recognizer_table(const as_schema* s) {
  static_assert(AS_RX_KINDS == kRxKinds && AS_RX_URL == kRxUrl && AS_RX_CPE == kRxCpe && AS_RX_PEM == kRxPem &&
                    AS_RX_MAC == kRxMac && AS_RX_OID == kRxOid && AS_RX_CERT_FP == kRxCertFp,
                "recognizer kinds of the ABI and the kernels agree");
  RxTypes r{};
  if (s->recognizer_types) {
    for (int k = 0; k < kRxKinds; ++k) r.t[k] = s->recognizer_types[k];
  } else {
    r.t[kRxMac] = 4;
    r.t[kRxIpv6] = r.t[kRxIpv4] = 1;
    r.t[kRxCve] = 3;
    r.t[kRxHost] = 2;
  }
  return r;
}

as_status validate_schema(as_ctx* c, const as_schema* s) {
  if (!s) return fail(c, AS_ERR_ARG, "schema is NULL");
  const as_config& g = c->cfg;
  if (s->n_types < 1 || s->n_types > 62) return fail(c, AS_ERR_ARG, "n_types must be 1..62");
  if (2 * s->n_types + 1 != g.n_labels)
    return fail(c, AS_ERR_ARG, "n_labels must equal 2 * n_types + 1 (O, B-t, I-t)");
  if (!s->recognizer_types && s->n_types < 4)
    return fail(c, AS_ERR_ARG, "the default pattern recognizers need entity types 1..4");
  if (s->recognizer_types)
    for (int k = 0; k < AS_RX_KINDS; ++k)
      if (s->recognizer_types[k] > s->n_types)
        return fail(c, AS_ERR_ARG, "recognizer_types[" + std::to_string(k) + "] exceeds n_types");
  if (!s->type_names) return fail(c, AS_ERR_ARG, "type_names is NULL");
  for (uint32_t t = 0; t < s->n_types; ++t)
    if (!s->type_names[t] || !s->type_names[t][0]) return fail(c, AS_ERR_ARG, "empty type name");
  if (s->slug_hex_len > 64) return fail(c, AS_ERR_ARG, "slug_hex_len must be 0..64");
  if (s->window) {
    if (s->window > g.max_pos) return fail(c, AS_ERR_ARG, "window exceeds max_pos");
    if (s->stride == 0 || s->stride > s->window || (s->window - s->stride) % 2)
      return fail(c, AS_ERR_ARG, "need 0 < stride <= window and window - stride even");
  }
  return AS_OK;
}

as_status set_key(as_ctx* c, const uint8_t* key, size_t key_len) {
  if (!key && key_len) return fail(c, AS_ERR_ARG, "key is NULL");
  std::vector<uint8_t> k(key, key + key_len);
  if (c->key_set && k == c->key) return AS_OK;
  uint64_t n_entries = 0;
  CK(cudaMemcpyAsync(&n_entries, c->map_ctr.as<unsigned long long>() + 1, 8, cudaMemcpyDeviceToHost, c->main.stream));
  CK(cudaStreamSynchronize(c->main.stream));
  if (c->key_set && n_entries > 0)
    return fail(c, AS_ERR_STATE, "key differs from the key of the non-empty entity map (clear the map first)");
  c->key = k;
  c->key_set = true;
  CKS(grow(c->key_dev, key_len + 1));
  if (key_len) CK(cudaMemcpyAsync(c->key_dev.p, key, key_len, cudaMemcpyHostToDevice, c->main.stream));
  CKS(grow(c->key_state, 16 * 4));
  launch_hmac_key_setup(c->key_dev.as<uint8_t>(), (uint32_t)key_len, c->key_state.as<uint32_t>(), c->main.stream);
  CK(cudaStreamSynchronize(c->main.stream));
  return AS_OK;
}

template <typename T>
as_status d2h_vec(as_ctx* c, Lane* ln, std::vector<T>& v, const void* src, uint64_t n) {
  v.resize(n);
  if (n) CK(cudaMemcpyAsync(v.data(), src, n * sizeof(T), cudaMemcpyDeviceToHost, ln->stream));
  return AS_OK;
}

// The inputs of a call on the device: *d_bytes / *d_off are the caller's
// device arrays, or the lane's copies of its host arrays (checked here: the
// offsets start at 0 and never decrease). *N_out = total bytes (< 4 GiB).
as_status stage_records(as_ctx* c, Lane* ln, const as_records* rec, const uint8_t** d_bytes_out,
                        const uint64_t** d_off_out, uint64_t* N_out) {
  cudaStream_t st = ln->stream;
  const uint64_t n = rec->n_records;
  if (n > 0 && !rec->offsets) return fail(c, AS_ERR_ARG, "offsets is NULL");
  uint64_t N = 0;
  const uint8_t* d_bytes;
  const uint64_t* d_off;
  if (n > 0) {
    if (rec->on_device) {
      CK(cudaMemcpyAsync(&N, rec->offsets + n, 8, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
    } else {
      N = rec->offsets[n];
      if (rec->offsets[0] != 0) return fail(c, AS_ERR_ARG, "offsets[0] must be 0");
      for (uint64_t r = 0; r < n; ++r)
        if (rec->offsets[r + 1] < rec->offsets[r]) return fail(c, AS_ERR_ARG, "offsets must be non-decreasing");
    }
  }
  if (N >= (1ull << 32) - 64) return fail(c, AS_ERR_ARG, "a call takes less than 4 GiB of text");
  if (N > 0 && !rec->bytes) return fail(c, AS_ERR_ARG, "bytes is NULL");
  CKS(grow(ln->in_off, (n + 1) * 8));
  if (rec->on_device) {
    d_bytes = rec->bytes;
    d_off = rec->offsets;
  } else {
    CKS(grow(ln->in_bytes, N + 16));
    if (N) CK(cudaMemcpyAsync(ln->in_bytes.p, rec->bytes, N, cudaMemcpyHostToDevice, st));
    uint64_t zero = 0;
    if (n) CK(cudaMemcpyAsync(ln->in_off.p, rec->offsets, (n + 1) * 8, cudaMemcpyHostToDevice, st));
    else CK(cudaMemcpyAsync(ln->in_off.p, &zero, 8, cudaMemcpyHostToDevice, st));
    d_bytes = ln->in_bytes.as<uint8_t>();
    d_off = ln->in_off.as<uint64_t>();
  }
  if (n == 0) {
    static const uint64_t zero_off = 0;
    CK(cudaMemcpyAsync(ln->in_off.p, &zero_off, 8, cudaMemcpyHostToDevice, st));
    d_off = ln->in_off.as<uint64_t>();
  }
  *d_bytes_out = d_bytes;
  *d_off_out = d_off;
  *N_out = N;
  return AS_OK;
}

// Type names on the device: names = concatenation, name_off[t] .. name_off[t+1]
// = type t's bytes (t = 1..n_types), name_len[t] their length.
as_status upload_names(as_ctx* c, Lane* ln, const as_schema* sch) {
  cudaStream_t st = ln->stream;
  std::vector<uint32_t> noff(sch->n_types + 2, 0), nlen(sch->n_types + 1, 0);
  std::string all;
  for (uint32_t t = 1; t <= sch->n_types; ++t) {
    noff[t] = (uint32_t)all.size();
    all += sch->type_names[t - 1];
    noff[t + 1] = (uint32_t)all.size();
    nlen[t] = noff[t + 1] - noff[t];
  }
  CKS(grow(ln->names, all.size() + 16));
  CKS(grow(ln->name_off, noff.size() * 4));
  CKS(grow(ln->name_len, nlen.size() * 4));
  CK(cudaMemcpyAsync(ln->names.p, all.data(), all.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ln->name_off.p, noff.data(), noff.size() * 4, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ln->name_len.p, nlen.data(), nlen.size() * 4, cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));  // the host vectors above go out of scope
  return AS_OK;
}

// calibrate = true: run the tokenizer and the BF16 encoder only, recording
// the amax of every FP8 GEMM input, and set the static activation scales.
as_status anonymize_impl(as_ctx* c, Lane* ln, const as_records* rec, const as_schema* sch, const uint8_t* key,
                         size_t key_len, as_output** out, bool calibrate = false, int64_t rec_base = -1,
                         const FieldJob* fj = nullptr) {
  const as_config& g = c->cfg;
  cudaStream_t st = ln->stream;
  if (!rec || (!out && !calibrate)) return fail(c, AS_ERR_ARG, "records / out is NULL");
  if (out) *out = nullptr;
  CKI(validate_schema(c, sch));
  if (calibrate && g.precision != AS_FP8) return fail(c, AS_ERR_STATE, "calibration is for AS_FP8 contexts");
  if (!calibrate && g.precision == AS_FP8 && c->act_scale.empty())
    return fail(c, AS_ERR_STATE, "FP8 context without activation scales: call as_calibrate or as_set_scales first");
  if (!calibrate && rec_base < 0) CKI(set_key(c, key, key_len));  // serving sets the key once at start
  c->slug_len = sch->slug_hex_len;
  uint64_t n = rec->n_records;
  if (n > 0 && (!rec->offsets)) return fail(c, AS_ERR_ARG, "offsets is NULL");
  // ---- inputs
  uint64_t N = 0;
  const uint8_t* d_bytes = nullptr;
  const uint64_t* d_off = nullptr;
  CKI(stage_records(c, ln, rec, &d_bytes, &d_off, &N));
  uint32_t N32 = (uint32_t)N;
  const uint64_t launches0 = t_launches, replays0 = ln->graph_replays;
  const uint32_t call_id = ++c->call_id;
  // ---- tokenizer + recognizers
  CKS(grow(ln->counters, 64));
  uint32_t* cnt = ln->counters.as<uint32_t>();  // 0 T, 1 n_rx, 2 n_ner, 3 n_nerk, 4 n_rxk, 5 n_fin
  CK(cudaMemsetAsync(cnt, 0, 64, st));
  CKS(grow(ln->rs_bits, ((size_t)N / 32 + 1) * 4));
  CKS(grow(ln->tok_at, N * 2));
  CKS(grow(ln->scan_tiles, (scan_tiles_needed(std::max<uint64_t>(N + 1, 1) * 2) + 16) * 8));
  CKS(grow(ln->tok_ids, N * 4));
  CKS(grow(ln->tok_off, N * 4));
  CKS(grow(ln->tok_len, N * 4));
  CKS(grow(ln->rec_tok, (n + 1) * 8));
  VocabTable vt{c->vocab_slots.as<uint4>(), c->vocab_mask, c->vocab_lenmask.as<uint16_t>()};
  ProfScope ps_text(ln, kProfText, 0);
  launch_mark_record_starts(d_off, n, N32, ln->rs_bits.as<uint32_t>(), st);
  // the mark kernels count each tile's tokens / candidates into scan_tiles,
  // so the compactions skip their counting pass
  const size_t text_tiles = scan_tiles_needed(N32);
  CK(cudaMemsetAsync(ln->scan_tiles.p, 0, std::max<size_t>(1, text_tiles) * 4, st));
  launch_tokenize_mark(d_bytes, N32, ln->rs_bits.as<uint32_t>(), vt, ln->tok_at.as<uint16_t>(), st,
                       ln->scan_tiles.as<uint32_t>());
  launch_tokenize_table(ln->tok_at.as<uint16_t>(), N32, ln->tok_ids.as<int32_t>(), ln->tok_off.as<uint32_t>(),
                        ln->tok_len.as<uint32_t>(), cnt + 0, ln->scan_tiles.as<uint32_t>(), st);
  launch_record_token_starts(d_off, n, ln->tok_off.as<uint32_t>(), cnt + 0, N32, ln->rec_tok.as<uint64_t>(), st);
  // recognizers
  CKS(grow(ln->rx_len_b, N * 4));
  CKS(grow(ln->rx_type_b, N + 16));
  const RxTypes rxt = recognizer_table(sch);
  // with a multi-word kind on, the resolve pass may drop candidates: the
  // compaction then counts them itself
  const bool rx_long = rx_any_long(rxt);
  if (!rx_long) CK(cudaMemsetAsync(ln->scan_tiles.p, 0, std::max<size_t>(1, text_tiles) * 4, st));
  launch_recognize_mark(d_bytes, N32, ln->rs_bits.as<uint32_t>(), rxt, ln->rx_len_b.as<uint32_t>(),
                        ln->rx_type_b.as<uint8_t>(), st, rx_long ? nullptr : ln->scan_tiles.as<uint32_t>());
  if (rx_long)
    launch_recognize_resolve(d_off, n, ln->rx_len_b.as<uint32_t>(), ln->rx_type_b.as<uint8_t>(), st);
  CKS(grow(ln->rx_s, (N / 2 + 2) * 4));
  CKS(grow(ln->rx_l, (N / 2 + 2) * 4));
  CKS(grow(ln->rx_t, N / 2 + 2));
  launch_recognize_compact(ln->rx_len_b.as<uint32_t>(), ln->rx_type_b.as<uint8_t>(), N32, ln->rx_s.as<uint32_t>(),
                           ln->rx_l.as<uint32_t>(), ln->rx_t.as<uint8_t>(), cnt + 1, ln->scan_tiles.as<uint32_t>(), st,
                           !rx_long);
  CK(cudaGetLastError());  // a text-stage launch that was refused (its marks would be stale)
  ps_text.end();
  // ---- sync 1: token counts
  uint32_t h_cnt[2] = {0, 0};
  CK(cudaMemcpyAsync(h_cnt, cnt, 8, cudaMemcpyDeviceToHost, st));
  std::vector<uint64_t>& rt = ln->h_rec_tok;
  rt.resize(n + 1);
  CK(cudaMemcpyAsync(rt.data(), ln->rec_tok.p, (n + 1) * 8, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const uint64_t T = h_cnt[0], n_rx = h_cnt[1];
  // ---- sequences (windows) and encoder batches
  const uint32_t W = sch->window, S = sch->stride;
  std::vector<SeqDesc> seqs;
  seqs.reserve(n);
  uint64_t enc_tokens = 0;
  for (uint64_t r = 0; r < n; ++r) {
    const uint64_t a = rt[r], L = rt[r + 1] - rt[r];
    if (L == 0) continue;
    if (W == 0 || L <= W) {
      if (L > g.max_pos)
        return fail(c, AS_ERR_TOO_LONG, "record " + std::to_string(r) + " has " + std::to_string(L) +
                                            " tokens, more than max_pos without windows");
      seqs.push_back(SeqDesc{(uint32_t)a, (uint32_t)L, 0, 0, (uint16_t)L});
      enc_tokens += L;
      continue;
    }
    const uint32_t half = (W - S) / 2;
    std::vector<uint64_t> starts{0};
    while (starts.back() + W < L) starts.push_back(starts.back() + S);
    for (size_t w = 0; w < starts.size(); ++w) {
      const uint64_t s0 = starts[w];
      const uint32_t len = (uint32_t)std::min<uint64_t>(W, L - s0);
      const uint16_t lo = w == 0 ? 0 : (uint16_t)half;
      const uint16_t hi = w + 1 == starts.size() ? (uint16_t)len : (uint16_t)(S + half);
      seqs.push_back(SeqDesc{(uint32_t)(a + s0), len, 0, lo, hi});
      enc_tokens += len;
    }
  }
  // batches: whole sequences up to max_chunk_tokens rows (PACKED), or all
  // windows of one record (PER_RECORD: one record per launch sequence)
  std::vector<Chunk> chunks;
  if (g.mode == AS_MODE_PER_RECORD) {
    uint64_t i = 0;
    for (uint64_t r = 0; r < n && i < seqs.size(); ++r) {
      const uint64_t a = rt[r], b = rt[r + 1];
      if (a == b) continue;
      Chunk ch{i, i, 0, 0, 0};
      while (i < seqs.size() && seqs[i].src_tok >= a && seqs[i].src_tok < b) {
        seqs[i].row = (uint32_t)((ch.rows + 7) & ~7ull);
        ch.rows = seqs[i].row + seqs[i].len;
        ch.tokens += seqs[i].len;
        ch.max_len = std::max(ch.max_len, seqs[i].len);
        ch.s1 = ++i;
      }
      chunks.push_back(ch);
    }
  } else {
    // every sequence starts on a row that is a multiple of 8 (the padding rows
    // in between belong to no sequence and are never written out)
    // the lane's row cap (serving: from the activation budget), else the ctx's
    const uint64_t cap = ln->row_cap ? ln->row_cap : g.max_chunk_tokens ? g.max_chunk_tokens : (1ull << 19);
    Chunk cur{0, 0, 0, 0, 0};
    for (uint64_t i = 0; i < seqs.size(); ++i) {
      const uint64_t start = (cur.rows + 7) & ~7ull;
      if (cur.rows > 0 && start + seqs[i].len > cap) {
        chunks.push_back(cur);
        cur = Chunk{i, i, 0, 0, 0};
      }
      seqs[i].row = (uint32_t)((cur.rows + 7) & ~7ull);
      cur.s1 = i + 1;
      cur.rows = seqs[i].row + seqs[i].len;
      cur.tokens += seqs[i].len;
      cur.max_len = std::max(cur.max_len, seqs[i].len);
    }
    if (cur.rows) chunks.push_back(cur);
  }
  uint64_t max_rows = 0, max_seqs = 0;
  for (auto& ch : chunks) {
    max_rows = std::max(max_rows, encoder_rows(g, ch.rows));
    max_seqs = std::max<uint64_t>(max_seqs, ch.s1 - ch.s0);
  }
  CKS(grow(ln->seqs, std::max<size_t>(1, seqs.size()) * sizeof(SeqDesc)));
  if (!seqs.empty()) CK(cudaMemcpyAsync(ln->seqs.p, seqs.data(), seqs.size() * sizeof(SeqDesc), cudaMemcpyHostToDevice, st));
  CKI(ensure_encoder_buffers(c, ln, std::max<uint64_t>(max_rows, 1), max_seqs + 1));  // + the empty sequence
  const bool want_logits = g.keep_trace != 0;
  CKS(grow(ln->labels, T + 16));
  if (want_logits) CKS(grow(ln->logits, (T + 1) * g.n_labels * 4));
  CK(cudaMemsetAsync(ln->labels.p, 0, T + 16, st));
  if (calibrate) {
    c->calibrating = true;
    CK(cudaMemsetAsync(c->amax_dev.p, 0, (size_t)kActPerLayer * g.n_layers * 4, st));
  }
  // tcgen05 attention work items (one per 128-query tile, two int32 each),
  // all chunks in one upload
  std::vector<int32_t> items;
  std::vector<size_t> item_off{0};
  const bool tc_attn = g.attention == AS_ATTN_TCGEN05 && g.precision != AS_FP32;
  if (tc_attn) {
    std::vector<int32_t> lens, starts;
    for (const Chunk& ch : chunks) {
      lens.clear();
      starts.clear();
      for (uint64_t i = ch.s0; i < ch.s1; ++i) {
        lens.push_back((int32_t)seqs[i].len);
        starts.push_back((int32_t)seqs[i].row);
      }
      attention_items(starts.data(), lens.data(), (int32_t)lens.size(), items);
      if (graphable(g)) {
        // pad to the graph bucket with padding items (L = 0)
        const size_t n = (items.size() - item_off.back()) / 2;
        items.resize(item_off.back() + 2 * graph_bucket(n, 16), 0);
      }
      item_off.push_back(items.size());
    }
    CKS(grow(ln->attn_items, std::max<size_t>(items.size(), 1) * 4));
    if (!items.empty())
      CK(cudaMemcpyAsync(ln->attn_items.p, items.data(), items.size() * 4, cudaMemcpyHostToDevice, st));
  }
  for (size_t ci = 0; ci < chunks.size(); ++ci) {
    NvtxRange nvtx_batch("as.encoder_batch");
    const Chunk& ch = chunks[ci];
    double af = 0;  // attention FLOPs of the batch: QK^T and PV, 2 * 2 * L^2 * d per sequence
    for (uint64_t i = ch.s0; i < ch.s1; ++i) af += 4.0 * (double)seqs[i].len * seqs[i].len * g.d_model;
    as_status es = run_encoder_chunk(c, ln, ch, ln->seqs.as<SeqDesc>(), af, want_logits,
                                     tc_attn ? ln->attn_items.as<int32_t>() + item_off[ci] : nullptr,
                                     tc_attn ? (int32_t)((item_off[ci + 1] - item_off[ci]) / 2) : 0);
    if (es != AS_OK) {
      c->calibrating = false;
      return es;
    }
    if (ln->prof && ln->ev_used > 4096) {  // bound the event pool
      CK(cudaStreamSynchronize(st));
      prof_collect(ln);
    }
  }
  if (calibrate) {
    // static per-tensor activation scales: amax over the calibration set / 448
    c->calibrating = false;
    std::vector<unsigned int> bits((size_t)kActPerLayer * g.n_layers);
    CK(cudaMemcpyAsync(bits.data(), c->amax_dev.p, bits.size() * 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CKI(check_dev_error(c, ln));
    c->act_scale.resize(bits.size());
    for (size_t i = 0; i < bits.size(); ++i) {
      float a;
      memcpy(&a, &bits[i], 4);
      c->act_scale[i] = a > 0.f ? a / 448.0f : 1.0f;
    }
    return AS_OK;
  }
  // ---- BIO decode
  ProfScope ps_spans(ln, kProfSpans, 0);
  CKS(grow(ln->tok_flags, T + 16));
  CK(cudaMemsetAsync(ln->tok_flags.p, 0, T + 1, st));
  launch_token_flags(ln->rec_tok.as<uint64_t>(), n, ln->tok_flags.as<uint8_t>(), st);
  CKS(grow(ln->bio_start, T + 16));
  CKS(grow(ln->bio_end, T + 16));
  CKS(grow(ln->pos_t, (T + 1) * 4));
  launch_bio_mark(ln->labels.as<uint8_t>(), ln->tok_flags.as<uint8_t>(), (uint32_t)T, ln->bio_start.as<uint8_t>(),
                  ln->bio_end.as<uint8_t>(), st);
  exclusive_scan<uint32_t>(NonZeroU8{ln->bio_start.as<uint8_t>()}, T, ln->pos_t.as<uint32_t>(), cnt + 2,
                           ln->scan_tiles.as<uint32_t>(), st);
  CKS(grow(ln->ner_s, (T + 1) * 4));
  CKS(grow(ln->ner_l, (T + 1) * 4));
  CKS(grow(ln->ner_t, T + 16));
  launch_bio_emit(ln->labels.as<uint8_t>(), ln->bio_start.as<uint8_t>(), ln->bio_end.as<uint8_t>(), ln->pos_t.as<uint32_t>(),
                  (uint32_t)T, ln->tok_off.as<uint32_t>(), ln->tok_len.as<uint32_t>(), d_bytes, ln->ner_s.as<uint32_t>(),
                  ln->ner_l.as<uint32_t>(), ln->ner_t.as<uint8_t>(), st);
  launch_bio_to_bytes(ln->ner_s.as<uint32_t>(), ln->ner_l.as<uint32_t>(), cnt + 2, (uint32_t)T, ln->tok_off.as<uint32_t>(),
                      ln->tok_len.as<uint32_t>(), d_bytes, st);
  // ---- overlap rule + preserve
  const uint32_t ner_cap = (uint32_t)T, rx_cap = (uint32_t)n_rx;
  CKS(grow(ln->pos_k, (T + n_rx + 2) * 4));
  DBuf& keep = ln->keep;
  CKS(grow(keep, T + n_rx + 16));
  launch_ner_keep(ln->ner_s.as<uint32_t>(), ln->ner_l.as<uint32_t>(), ln->ner_t.as<uint8_t>(), cnt + 2, ner_cap,
                  ln->rx_s.as<uint32_t>(), ln->rx_l.as<uint32_t>(), cnt + 1, sch->preserve_mask, keep.as<uint8_t>(), st);
  exclusive_scan<uint32_t>(NonZeroU8{keep.as<uint8_t>()}, ner_cap, ln->pos_k.as<uint32_t>(), cnt + 3,
                           ln->scan_tiles.as<uint32_t>(), st, cnt + 2);  // over the NER spans found
  CKS(grow(ln->nk_s, (T + 1) * 4));
  CKS(grow(ln->nk_l, (T + 1) * 4));
  CKS(grow(ln->nk_t, T + 16));
  launch_compact_spans(ln->ner_s.as<uint32_t>(), ln->ner_l.as<uint32_t>(), ln->ner_t.as<uint8_t>(), keep.as<uint8_t>(),
                       ln->pos_k.as<uint32_t>(), cnt + 2, ner_cap, ln->nk_s.as<uint32_t>(), ln->nk_l.as<uint32_t>(),
                       ln->nk_t.as<uint8_t>(), st);
  launch_rx_keep(ln->rx_t.as<uint8_t>(), cnt + 1, rx_cap, sch->preserve_mask, keep.as<uint8_t>(), st);
  exclusive_scan<uint32_t>(NonZeroU8{keep.as<uint8_t>()}, rx_cap, ln->pos_k.as<uint32_t>(), cnt + 4,
                           ln->scan_tiles.as<uint32_t>(), st);
  CKS(grow(ln->rk_s, (n_rx + 1) * 4));
  CKS(grow(ln->rk_l, (n_rx + 1) * 4));
  CKS(grow(ln->rk_t, n_rx + 16));
  launch_compact_spans(ln->rx_s.as<uint32_t>(), ln->rx_l.as<uint32_t>(), ln->rx_t.as<uint8_t>(), keep.as<uint8_t>(),
                       ln->pos_k.as<uint32_t>(), cnt + 1, rx_cap, ln->rk_s.as<uint32_t>(), ln->rk_l.as<uint32_t>(),
                       ln->rk_t.as<uint8_t>(), st);
  const uint32_t fin_cap = ner_cap + rx_cap;
  CKS(grow(ln->fin_s, (fin_cap + 1) * 4));
  CKS(grow(ln->fin_l, (fin_cap + 1) * 4));
  CKS(grow(ln->fin_t, fin_cap + 16));
  launch_merge_spans(ln->rk_s.as<uint32_t>(), ln->rk_l.as<uint32_t>(), ln->rk_t.as<uint8_t>(), cnt + 4, rx_cap,
                     ln->nk_s.as<uint32_t>(), ln->nk_l.as<uint32_t>(), ln->nk_t.as<uint8_t>(), cnt + 3, ner_cap,
                     ln->fin_s.as<uint32_t>(), ln->fin_l.as<uint32_t>(), ln->fin_t.as<uint8_t>(), st);
  // the HMAC / map / substitution kernels read the final span count from cnt[5]
  sum_kept_kernel<<<1, 32, 0, st>>>(cnt);
  count_launch();
  ps_spans.end();
  uint32_t fin_total = fin_cap;
  const uint64_t n_detect = n;  // records the detection steps saw (sub-records with a field policy)
  if (fj) {
    // spans of the detected fields -> record coordinates, merged with the forced fields
    launch_field_translate(ln->fin_s.as<uint32_t>(), cnt + 5, fin_cap, fj->sub_off, fj->nf, fj->field_start, st);
    fin_total = fin_cap + fj->force_cap;
    CKS(grow(ln->ff_s, ((size_t)fin_total + 1) * 4));
    CKS(grow(ln->ff_l, ((size_t)fin_total + 1) * 4));
    CKS(grow(ln->ff_t, (size_t)fin_total + 16));
    launch_merge_spans(ln->fin_s.as<uint32_t>(), ln->fin_l.as<uint32_t>(), ln->fin_t.as<uint8_t>(), cnt + 5, fin_cap,
                       fj->fs_s, fj->fs_l, fj->fs_t, fj->n_force_dev, fj->force_cap, ln->ff_s.as<uint32_t>(),
                       ln->ff_l.as<uint32_t>(), ln->ff_t.as<uint8_t>(), st);
    launch_add_count(cnt + 5, fj->n_force_dev, st);
    std::swap(ln->fin_s, ln->ff_s);
    std::swap(ln->fin_l, ln->ff_l);
    std::swap(ln->fin_t, ln->ff_t);
    // the rest of the path works on the original records
    d_bytes = fj->bytes;
    d_off = fj->offsets;
    n = fj->n;
    N = fj->N;
    N32 = (uint32_t)N;
  }
  // ---- HMAC + map
  CKS(grow(ln->digests, (size_t)(fin_total + 1) * 32));
  ProfScope ps_hash(ln, kProfHash, 0);
  launch_hmac_spans(d_bytes, ln->fin_s.as<uint32_t>(), ln->fin_l.as<uint32_t>(), cnt + 5, fin_total,
                    c->key_state.as<uint32_t>(), ln->digests.as<uint32_t>(), st);
  launch_map_insert_spans(map_view(c), d_bytes, ln->fin_s.as<uint32_t>(), ln->fin_l.as<uint32_t>(),
                          ln->fin_t.as<uint8_t>(), ln->digests.as<uint32_t>(), cnt + 5, fin_total, d_off, n,
                          rec_base >= 0 ? (uint64_t)rec_base : c->records_done, call_id, ln->dev_err.as<DevError>(),
                          st);
  ps_hash.end();
  // ---- substitution
  CKI(upload_names(c, ln, sch));
  CKS(grow(ln->delta, (size_t)(fin_total + 1) * 8));
  CKS(grow(ln->shift, (size_t)(fin_total + 1) * 8));
  CKS(grow(ln->delta_total, 16));
  ProfScope ps_sub1(ln, kProfSubst, 0);
  launch_sub_delta(ln->fin_l.as<uint32_t>(), ln->fin_t.as<uint8_t>(), cnt + 5, fin_total + 1, ln->name_len.as<uint32_t>(),
                   sch->slug_hex_len, ln->delta.as<int64_t>(), st);
  exclusive_scan<int64_t>(LoadI64{ln->delta.as<int64_t>()}, fin_total + 1, ln->shift.as<int64_t>(),
                          ln->delta_total.as<int64_t>(), reinterpret_cast<int64_t*>(ln->scan_tiles.p), st, cnt + 5,
                          1);  // over the final spans + 1 (shift[n] = total)
  ps_sub1.end();
  // ---- sync 2: output size and counts
  CK(cudaGetLastError());  // a refused launch of the encoder or span stages
  int64_t total_delta = 0;
  uint32_t h_cnt2[6];
  CK(cudaMemcpyAsync(&total_delta, ln->delta_total.p, 8, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(h_cnt2, cnt, 24, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const uint64_t out_size = (uint64_t)((int64_t)N + total_delta);
  as_output* o = new as_output();
  o->ctx = c;
  o->device = c->device;
  o->call_id = call_id;
  const bool out_dev = fj ? fj->on_device : rec->on_device != 0;
  o->on_device = out_dev ? 1u : 0u;
  o->n = n;
  void* d_out = nullptr;
  uint64_t* d_out_off = nullptr;
  if (cudaMallocAsync(&d_out, out_size + 16, st) != cudaSuccess ||
      cudaMallocAsync(reinterpret_cast<void**>(&d_out_off), (n + 1) * 8, st) != cudaSuccess) {
    cudaGetLastError();
    if (d_out) cudaFreeAsync(d_out, st);
    delete o;
    return fail(c, AS_ERR_OOM, "output allocation failed");
  }
  ProfScope ps_sub2(ln, kProfSubst, 0);
  launch_sub_copy(d_bytes, N32, ln->fin_s.as<uint32_t>(), ln->fin_l.as<uint32_t>(), cnt + 5, ln->shift.as<int64_t>(),
                  reinterpret_cast<uint8_t*>(d_out), st);
  launch_sub_replace(ln->fin_s.as<uint32_t>(), ln->fin_t.as<uint8_t>(), cnt + 5, fin_total, ln->shift.as<int64_t>(),
                     ln->digests.as<uint32_t>(), ln->names.as<char>(), ln->name_off.as<uint32_t>(), sch->slug_hex_len,
                     reinterpret_cast<uint8_t*>(d_out), st);
  launch_sub_offsets(d_off, n, ln->fin_s.as<uint32_t>(), cnt + 5, ln->shift.as<int64_t>(), d_out_off, st);
  ps_sub2.end();
  if (out_dev) {
    o->d_bytes = d_out;
    o->d_off = d_out_off;
  } else {
    o->h_bytes.resize(out_size);
    o->h_off.resize(n + 1);
    cudaMemcpyAsync(o->h_bytes.data(), d_out, out_size, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(o->h_off.data(), d_out_off, (n + 1) * 8, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(d_out, st);
    cudaFreeAsync(d_out_off, st);
  }
  // ---- trace for as_debug_trace
  ln->last_n = n_detect;
  ln->last_T = T;
  ln->last_nrx = n_rx;
  ln->last_nfin = h_cnt2[5];
  ln->last_logits = want_logits;
  if (g.keep_trace) {
    CKS(d2h_vec(c, ln, ln->h_tok_ids, ln->tok_ids.p, T));
    CKS(d2h_vec(c, ln, ln->h_tok_off, ln->tok_off.p, T));
    CKS(d2h_vec(c, ln, ln->h_tok_len, ln->tok_len.p, T));
    CKS(d2h_vec(c, ln, ln->h_rx_s, ln->rx_s.p, n_rx));
    CKS(d2h_vec(c, ln, ln->h_rx_l, ln->rx_l.p, n_rx));
    CKS(d2h_vec(c, ln, ln->h_rx_t, ln->rx_t.p, n_rx));
    CKS(d2h_vec(c, ln, ln->h_labels, ln->labels.p, T));
    CKS(d2h_vec(c, ln, ln->h_logits, ln->logits.p, T * g.n_labels));
    CKS(d2h_vec(c, ln, ln->h_fin_s, ln->fin_s.p, h_cnt2[5]));
    CKS(d2h_vec(c, ln, ln->h_fin_l, ln->fin_l.p, h_cnt2[5]));
    CKS(d2h_vec(c, ln, ln->h_fin_t, ln->fin_t.p, h_cnt2[5]));
  }
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    as_output_free(o);
    return fail(c, AS_ERR_CUDA, std::string("stream: ") + cudaGetErrorString(e));
  }
  if (ln->prof) prof_collect(ln);
  as_status ds = check_dev_error(c, ln);
  if (ds != AS_OK) {
    as_output_free(o);
    return ds;
  }
  uint64_t n_entries = 0;
  if (cudaMemcpyAsync(&n_entries, c->map_ctr.as<unsigned long long>() + 1, 8, cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    as_output_free(o);
    return fail(c, AS_ERR_CUDA, "map counter read failed");
  }
  as_stats& s = o->stats;
  s.n_records = n;
  s.n_bytes = N;
  s.n_tokens = T;
  s.n_encoded_tokens = enc_tokens;
  s.n_sequences = seqs.size();
  s.n_regex_spans = n_rx;
  s.n_ner_spans = h_cnt2[2];
  s.n_final_spans = h_cnt2[5];
  s.n_out_bytes = out_size;
  s.n_map_entries = n_entries;
  // the largest map size any call has reported so far, raised atomically:
  // calls on other lanes read the counter and report in any order, and a
  // plain exchange could move it back and count entries twice
  uint64_t seen = c->n_entries_seen.load();
  while (seen < n_entries && !c->n_entries_seen.compare_exchange_weak(seen, n_entries)) {
  }
  s.n_new_entries = n_entries > seen ? n_entries - seen : 0;
  s.kernel_launches = t_launches - launches0;
  s.graph_replays = ln->graph_replays - replays0;
  if (rec_base < 0) c->records_done += n;
  *out = o;
  return AS_OK;
}

as_status map_collect(as_ctx* c, uint32_t call_lo, uint32_t call_hi, std::vector<as_entity>& ents,
                      std::vector<uint8_t>& orig) {
  cudaStream_t st = c->main.stream;
  const uint64_t slots = c->map_mask + 1;
  DBuf keep, pos, idx, tiles, total;
  auto cleanup = [&]() { release(keep); release(pos); release(idx); release(tiles); release(total); };
  if (grow(keep, slots) || grow(pos, slots * 4) || grow(tiles, (scan_tiles_needed(slots) + 4) * 4) ||
      grow(total, 16)) {
    cleanup();
    return fail(c, AS_ERR_OOM, "map export scratch");
  }
  MapView m = map_view(c);
  launch_map_select(m, call_lo, call_hi, keep.as<uint8_t>(), st);
  exclusive_scan<uint32_t>(NonZeroU8{keep.as<uint8_t>()}, slots, pos.as<uint32_t>(), total.as<uint32_t>(),
                           tiles.as<uint32_t>(), st);
  uint32_t cnt = 0;
  cudaMemcpyAsync(&cnt, total.p, 4, cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  if (grow(idx, (size_t)(cnt + 1) * 4)) { cleanup(); return fail(c, AS_ERR_OOM, "map export scratch"); }
  launch_map_gather(m, keep.as<uint8_t>(), pos.as<uint32_t>(), idx.as<uint32_t>(), st);
  uint64_t used = 0;
  cudaMemcpyAsync(&used, c->map_ctr.p, 8, cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  std::vector<MapSlot> hs(cnt);
  DBuf gathered;
  if (grow(gathered, (size_t)(cnt + 1) * sizeof(MapSlot))) { cleanup(); return fail(c, AS_ERR_OOM, "map export scratch"); }
  launch_map_gather_slots(m, idx.as<uint32_t>(), cnt, gathered.as<MapSlot>(), st);
  if (cnt) cudaMemcpyAsync(hs.data(), gathered.p, cnt * sizeof(MapSlot), cudaMemcpyDeviceToHost, st);
  std::vector<uint8_t> arena(used);
  if (used) cudaMemcpyAsync(arena.data(), c->map_arena.p, used, cudaMemcpyDeviceToHost, st);
  cudaError_t e = cudaStreamSynchronize(st);
  cleanup();
  release(gathered);
  if (e != cudaSuccess) return fail(c, AS_ERR_CUDA, std::string("map export: ") + cudaGetErrorString(e));
  std::vector<uint32_t> order(cnt);
  for (uint32_t i = 0; i < cnt; ++i) order[i] = i;
  auto bytes_of = [&](const MapSlot& s) { return arena.data() + s.arena_off; };
  std::sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) {
    const MapSlot &x = hs[a], &y = hs[b];
    if (x.type != y.type) return x.type < y.type;
    int r = memcmp(bytes_of(x), bytes_of(y), std::min(x.len, y.len));
    if (r != 0) return r < 0;
    return x.len < y.len;
  });
  uint64_t total_len = 0;
  for (auto& s : hs) total_len += s.len;
  orig.resize(total_len + 1);
  ents.resize(cnt);
  uint64_t p = 0;
  static const char* hex = "0123456789abcdef";
  for (uint32_t i = 0; i < cnt; ++i) {
    const MapSlot& s = hs[order[i]];
    as_entity& en = ents[i];
    memset(&en, 0, sizeof(en));
    en.type = s.type;
    en.original_len = s.len;
    if (s.arena_off != ~0ull) memcpy(orig.data() + p, bytes_of(s), s.len);
    en.original = nullptr;
    for (int k = 0; k < 64; ++k) en.full_hash[k] = hex[(s.digest[k >> 3] >> (28 - 4 * (k & 7))) & 15];
    en.full_hash[64] = 0;
    memcpy(en.slug, en.full_hash, c->slug_len);
    en.slug[c->slug_len] = 0;
    en.first_seen = s.first_seen;
    en.last_seen = s.last_seen;
    en.count = s.count;
    reinterpret_cast<uint64_t&>(en.original) = p;  // fixed up by the caller
    p += s.len;
  }
  return AS_OK;
}

}  // namespace

namespace as {
// Vocabulary table and device of a ctx, for entry points defined in other files.
bool ctx_vocab(const as_ctx* ctx, VocabTable* vt, int* device) {
  if (!ctx || !ctx->vocab_slots.p) return false;
  vt->slots = ctx->vocab_slots.as<uint4>();
  vt->mask = ctx->vocab_mask;
  vt->lenmask = ctx->vocab_lenmask.as<uint16_t>();
  *device = ctx->device;
  return true;
}
}  // namespace as

// ------------------------------------------------------------------ serving

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct ServeRequest {
  uint64_t id = 0;
  std::vector<uint8_t> bytes;
  int64_t t_submit = 0, t_done = 0;
  bool discard = false, done = false;
  as_status status = AS_OK;
  std::vector<uint8_t> out;
  uint64_t tokens = 0;
};

}  // namespace

// Continuous batching: admitted requests wait in FIFO order; every worker
// owns a lane (stream + buffers) and, whenever it is free, takes the oldest
// requests up to the batch byte budget and runs the whole path on them. With
// two or more lanes a batch is admitted while others are still on the GPU and
// their kernels overlap. Record index of a request = its id, so results and
// map sightings do not depend on which batch a request joined.
struct Server {
  as_ctx* c = nullptr;
  std::vector<std::string> names;
  std::vector<const char*> name_ptrs;
  uint8_t rx_types[AS_RX_KINDS] = {};
  as_schema schema{};
  uint64_t batch_bytes = 0;
  uint32_t max_batch = 0;
  uint64_t max_pending = 0;
  uint64_t act_budget = 0, row_cap = 0, act_peak = 0;
  uint32_t max_pos = 0;
  std::vector<std::unique_ptr<Lane>> lanes;
  std::vector<std::thread> workers;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<ServeRequest*> queue;
  std::unordered_map<uint64_t, ServeRequest*> live;
  uint64_t next_id = 0;
  bool stop = false;
  // statistics since start or the last reset
  std::vector<double> lat_ms;
  uint64_t completed = 0, rejected = 0, batches = 0, tokens = 0, failed = 0;
  int64_t t_stats0 = 0;

  void worker(Lane* ln);
  // encoder rows a record of b bytes can occupy at most (<= b tokens; windows
  // and the 8-row alignment of every sequence added)
  uint64_t bound_rows(uint64_t b) const {
    const uint64_t W = schema.window, S = schema.stride;
    if (b == 0) return 0;
    if (W == 0 || b <= W) return (std::min<uint64_t>(b, max_pos) + 7) & ~7ull;
    const uint64_t nw = 1 + (b - W + S - 1) / S;
    return b + (nw - 1) * (W - S) + 8 * nw;
  }
};

void Server::worker(Lane* ln) {
  cudaSetDevice(c->device);
  std::vector<ServeRequest*> batch;
  std::vector<uint8_t> arena;
  std::vector<uint64_t> offs;
  while (true) {
    batch.clear();
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_work.wait(lk, [&] { return stop || !queue.empty(); });
      if (queue.empty()) break;  // stop requested and nothing left
      // admission by device memory: the rows the batch can occupy stay within
      // the lane's row cap (the first request always goes in)
      uint64_t bytes = 0, rows = 0;
      while (!queue.empty() && batch.size() < max_batch) {
        const uint64_t b = queue.front()->bytes.size(), r = bound_rows(b);
        if (!batch.empty() && (bytes + b > batch_bytes || rows + r > row_cap)) break;
        bytes += b;
        rows += r;
        batch.push_back(queue.front());
        queue.pop_front();
      }
    }
    arena.clear();
    offs.assign(1, 0);
    for (ServeRequest* r : batch) {
      arena.insert(arena.end(), r->bytes.begin(), r->bytes.end());
      offs.push_back(arena.size());
    }
    as_records rec{arena.empty() ? nullptr : arena.data(), offs.data(), (uint64_t)batch.size(), 0};
    as_output* o = nullptr;
    // ids of one batch are consecutive (FIFO admission), so the first is the base
    const as_status st = anonymize_impl(c, ln, &rec, &schema, nullptr, 0, &o, false, (int64_t)batch[0]->id);
    const int64_t t = now_ns();
    std::vector<uint64_t> rec_tokens(batch.size(), 0);
    if (st == AS_OK && !ln->h_rec_tok.empty() && ln->h_rec_tok.size() == batch.size() + 1)
      for (size_t i = 0; i < batch.size(); ++i) rec_tokens[i] = ln->h_rec_tok[i + 1] - ln->h_rec_tok[i];
    uint64_t held = 0;
    for (auto& l : lanes) held += l->act_bytes.load();
    {
      std::lock_guard<std::mutex> lk(mu);
      act_peak = std::max(act_peak, held);
      ++batches;
      if (st == AS_OK) tokens += o->stats.n_encoded_tokens;
      for (size_t i = 0; i < batch.size(); ++i) {
        ServeRequest* r = batch[i];
        r->status = st;
        r->t_done = t;
        r->tokens = rec_tokens[i];
        if (st == AS_OK) {
          r->out.assign(o->h_bytes.begin() + o->h_off[i], o->h_bytes.begin() + o->h_off[i + 1]);
          ++completed;
          lat_ms.push_back((t - r->t_submit) * 1e-6);
        } else {
          ++failed;
        }
        r->done = true;
        if (r->discard) {
          live.erase(r->id);
          delete r;
        }
      }
    }
    cv_done.notify_all();
    if (o) as_output_free(o);
  }
}

// ------------------------------------------------------------------ C ABI

extern "C" {

const char* as_k_last_error(void) { return as::t_k_error.c_str(); }

const char* as_version(void) { return "anonshield-b300 0.1 (sm_103a)"; }

const char* as_last_error(const as_ctx*) { return t_err.c_str(); }

void as_free(void* p) { free(p); }

as_status as_create(const as_config* cfg, as_ctx** out) {
  if (!cfg || !out) return AS_ERR_ARG;
  *out = nullptr;
  as_ctx* c = new as_ctx();
  c->cfg = *cfg;
  const as_config& g = c->cfg;
  auto bail = [&](as_status s) {
    std::string m = t_err;
    as_destroy(c);
    set_k_error(m);
    return s;
  };
  if (g.vocab < 258 || g.n_vocab_words != g.vocab - 257 || !g.vocab_bytes || !g.vocab_offsets) {
    t_err = "vocab must be > 257 with vocab - 257 strings";
    return bail(AS_ERR_ARG);
  }
  if (g.d_model == 0 || g.n_heads == 0 || g.d_model != g.n_heads * 64) {
    t_err = "head dim must be 64 (d_model = 64 * n_heads)";
    return bail(AS_ERR_UNSUPPORTED);
  }
  if (g.d_model % 128 || g.d_model > 1024 || g.d_ffn % 128 || g.d_ffn == 0 || g.n_layers == 0 || g.n_labels < 9 ||
      g.n_labels > 32 || g.max_pos == 0 || g.max_pos > 4096) {
    t_err = "unsupported dimensions (d_model multiple of 128 up to 1024, d_ffn multiple of 128, 9..32 labels)";
    return bail(AS_ERR_UNSUPPORTED);
  }
  if (g.precision != AS_FP32 && g.precision != AS_BF16 && g.precision != AS_FP8) {
    t_err = "precision must be AS_FP32, AS_BF16 or AS_FP8";
    return bail(AS_ERR_UNSUPPORTED);
  }
  if (g.attention != AS_ATTN_MMA_SYNC && g.attention != AS_ATTN_TCGEN05) {
    t_err = "attention must be AS_ATTN_MMA_SYNC or AS_ATTN_TCGEN05";
    return bail(AS_ERR_ARG);
  }
  if (g.mode != AS_MODE_PACKED && g.mode != AS_MODE_PER_RECORD) {
    t_err = "mode must be AS_MODE_PACKED or AS_MODE_PER_RECORD";
    return bail(AS_ERR_ARG);
  }
  if (!g.weights || g.weights_len != expected_weights(g)) {
    t_err = "weights_len " + std::to_string(g.weights_len) + " != expected " + std::to_string(expected_weights(g));
    return bail(AS_ERR_ARG);
  }
  c->device = g.device;
  if (cudaSetDevice(g.device) != cudaSuccess) {
    cudaGetLastError();
    t_err = "cudaSetDevice failed";
    return bail(AS_ERR_CUDA);
  }
  if (cudaStreamCreateWithFlags(&c->main.stream, cudaStreamNonBlocking) != cudaSuccess) {
    t_err = "stream creation failed";
    return bail(AS_ERR_CUDA);
  }
  sha256_init_constants();
  as_status s;
  if ((s = build_vocab(c)) != AS_OK) return bail(s);
  if ((s = load_weights(c)) != AS_OK) return bail(s);
  uint64_t cap = g.map_capacity ? pow2_at_least(g.map_capacity) : (1ull << 22);
  uint64_t arena = g.map_arena_bytes ? g.map_arena_bytes : (256ull << 20);
  if (grow(c->map_slots, cap * sizeof(MapSlot)) || grow(c->map_arena, arena) || grow(c->map_ctr, 16) ||
      grow(c->main.dev_err, sizeof(DevError))) {
    t_err = "map allocation failed";
    return bail(AS_ERR_OOM);
  }
  c->map_arena.cap = arena;
  c->map_mask = cap - 1;
  cudaMemsetAsync(c->main.dev_err.p, 0, sizeof(DevError), c->main.stream);
  launch_map_init(map_view(c), c->main.stream);
  if (cudaStreamSynchronize(c->main.stream) != cudaSuccess) {
    t_err = std::string("init: ") + cudaGetErrorString(cudaGetLastError());
    return bail(AS_ERR_CUDA);
  }
  *out = c;
  return AS_OK;
}

void as_destroy(as_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  as_serve_stop(c);
  if (c->main.stream) cudaStreamSynchronize(c->main.stream);
  DBuf* all[] = {&c->w32, &c->w16, &c->w8, &c->amax_dev, &c->vocab_slots, &c->vocab_lenmask, &c->map_slots, &c->map_arena, &c->map_ctr,
                 &c->key_dev, &c->key_state};
  for (DBuf* b : all) release(*b);
  c->main.release_all();
  if (c->main.stream) cudaStreamDestroy(c->main.stream);
  for (auto& ln : c->stream_lanes) {
    cudaStreamSynchronize(ln->stream);
    ln->release_all();
    cudaStreamDestroy(ln->stream);
  }
  delete c;
}

as_status as_anonymize(as_ctx* ctx, const as_records* records, const as_schema* schema, const uint8_t* key,
                       size_t key_len, as_output** out) {
  if (!ctx) return AS_ERR_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, AS_ERR_CUDA, "cudaSetDevice failed");
  if (ctx->server) return fail(ctx, AS_ERR_STATE, "the ctx is serving: use as_submit / as_poll or stop serving");
  as_status s = anonymize_impl(ctx, &ctx->main, records, schema, key, key_len, out);
  if (s == AS_ERR_CUDA) cudaGetLastError();
  return s;
}

namespace {

as_status grow_pinned(void** p, size_t* cap, size_t need) {
  if (*cap >= need) return AS_OK;
  if (*p) cudaFreeHost(*p);
  *p = nullptr;
  *cap = 0;
  need = std::max<size_t>(need, 4096);
  if (cudaHostAlloc(p, need, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return AS_ERR_OOM;
  }
  *cap = need;
  return AS_OK;
}

}  // namespace

as_status as_anonymize_stream(as_ctx* c, const as_records* rec, const as_schema* sch, const uint8_t* key,
                              size_t key_len, const as_stream_config* scfg, as_output** out) {
  if (!c || !rec || !out) return AS_ERR_ARG;
  *out = nullptr;
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, AS_ERR_CUDA, "cudaSetDevice failed");
  if (c->server) return fail(c, AS_ERR_STATE, "the ctx is serving: use as_submit / as_poll or stop serving");
  if (rec->on_device) return fail(c, AS_ERR_ARG, "streaming takes host records (on_device = 0)");
  const uint64_t n = rec->n_records;
  if (!rec->offsets) return fail(c, AS_ERR_ARG, "offsets is NULL");
  if (rec->offsets[0] != 0) return fail(c, AS_ERR_ARG, "offsets[0] must be 0");
  for (uint64_t r = 0; r < n; ++r)
    if (rec->offsets[r + 1] < rec->offsets[r]) return fail(c, AS_ERR_ARG, "offsets must be non-decreasing");
  if (rec->offsets[n] && !rec->bytes) return fail(c, AS_ERR_ARG, "bytes is NULL");
  CKI(validate_schema(c, sch));
  if (c->cfg.precision == AS_FP8 && c->act_scale.empty())
    return fail(c, AS_ERR_STATE, "FP8 context without activation scales");
  CKI(set_key(c, key, key_len));
  const uint64_t budget = scfg && scfg->batch_bytes ? scfg->batch_bytes : (16ull << 20);
  if (budget >= (1ull << 32) - 64) return fail(c, AS_ERR_ARG, "batch_bytes must be below 4 GiB");
  const uint32_t n_lanes = scfg && scfg->lanes ? std::min<uint32_t>(scfg->lanes, 8) : 2;
  // batches: consecutive records, at most `budget` bytes each (a longer record alone)
  std::vector<uint64_t> cut{0};
  for (uint64_t r = 0; r < n; ++r)
    if (r > cut.back() && rec->offsets[r + 1] - rec->offsets[cut.back()] > budget) cut.push_back(r);
  if (n) cut.push_back(n);
  const size_t n_batches = cut.size() - 1;
  while (c->stream_lanes.size() < n_lanes) {
    auto ln = std::make_unique<Lane>();
    if (cudaStreamCreateWithFlags(&ln->stream, cudaStreamNonBlocking) != cudaSuccess ||
        grow(ln->dev_err, sizeof(DevError)) != AS_OK ||
        cudaMemsetAsync(ln->dev_err.p, 0, sizeof(DevError), ln->stream) != cudaSuccess) {
      if (ln->stream) cudaStreamDestroy(ln->stream);
      ln->release_all();
      return fail(c, AS_ERR_CUDA, "streaming lane set-up failed");
    }
    c->stream_lanes.push_back(std::move(ln));
  }
  const uint64_t base = c->records_done;
  const uint32_t call_lo = c->call_id.load() + 1;
  std::vector<as_output*> part(n_batches, nullptr);
  std::atomic<size_t> next{0};
  std::atomic<bool> failed{false};
  std::mutex err_mu;
  as_status first_err = AS_OK;
  std::string first_msg;
  auto worker = [&](Lane* ln) {
    cudaSetDevice(c->device);
    while (!failed.load()) {
      const size_t b = next.fetch_add(1);
      if (b >= n_batches) break;
      const uint64_t r0 = cut[b], r1 = cut[b + 1], m = r1 - r0;
      const uint64_t o0 = rec->offsets[r0], nb = rec->offsets[r1] - o0;
      as_status s = AS_OK;
      // the previous batch's H2D from this staging buffer has completed:
      // anonymize_impl synchronizes its stream before returning
      if (grow_pinned(reinterpret_cast<void**>(&ln->h_in), &ln->h_in_cap, nb + 16) != AS_OK ||
          grow_pinned(reinterpret_cast<void**>(&ln->h_in_off), &ln->h_in_off_cap, (m + 1) * 8) != AS_OK) {
        s = AS_ERR_OOM;
        t_err = "pinned staging allocation failed";
      } else {
        if (nb) memcpy(ln->h_in, rec->bytes + o0, nb);
        for (uint64_t i = 0; i <= m; ++i) ln->h_in_off[i] = rec->offsets[r0 + i] - o0;
        as_records part_rec{ln->h_in, ln->h_in_off, m, 0};
        s = anonymize_impl(c, ln, &part_rec, sch, nullptr, 0, &part[b], false, (int64_t)(base + r0));
        if (s == AS_ERR_CUDA) cudaGetLastError();
      }
      if (s != AS_OK) {
        std::lock_guard<std::mutex> lk(err_mu);
        if (first_err == AS_OK) {
          first_err = s;
          first_msg = "batch " + std::to_string(b) + " (records " + std::to_string(r0) + ".." +
                      std::to_string(r1 - 1) + "): " + t_err;
        }
        failed.store(true);
      }
    }
  };
  std::vector<std::thread> th;
  const uint32_t used = (uint32_t)std::min<size_t>(n_lanes, std::max<size_t>(n_batches, 1));
  for (uint32_t i = 0; i < used; ++i) th.emplace_back(worker, c->stream_lanes[i].get());
  for (auto& t : th) t.join();
  if (first_err != AS_OK) {
    for (as_output* p : part) as_output_free(p);
    return fail(c, first_err, first_msg);
  }
  // one host output in record order
  as_output* o = new as_output();
  o->ctx = c;
  o->device = c->device;
  o->on_device = 0;
  o->n = n;
  o->call_lo = call_lo;
  o->call_id = c->call_id.load();
  uint64_t total = 0;
  for (as_output* p : part) total += p->h_bytes.size();
  o->h_bytes.resize(total);
  o->h_off.resize(n + 1);
  o->h_off[0] = 0;
  uint64_t pos = 0, r = 0;
  for (as_output* p : part) {
    if (!p->h_bytes.empty()) memcpy(o->h_bytes.data() + pos, p->h_bytes.data(), p->h_bytes.size());
    for (uint64_t i = 1; i <= p->n; ++i) o->h_off[r + i] = pos + p->h_off[i];
    pos += p->h_bytes.size();
    r += p->n;
    const as_stats& ps = p->stats;
    as_stats& s = o->stats;
    s.n_records += ps.n_records;
    s.n_bytes += ps.n_bytes;
    s.n_tokens += ps.n_tokens;
    s.n_encoded_tokens += ps.n_encoded_tokens;
    s.n_sequences += ps.n_sequences;
    s.n_regex_spans += ps.n_regex_spans;
    s.n_ner_spans += ps.n_ner_spans;
    s.n_final_spans += ps.n_final_spans;
    s.n_out_bytes += ps.n_out_bytes;
    s.n_new_entries += ps.n_new_entries;
    s.n_map_entries = std::max(s.n_map_entries, ps.n_map_entries);
    s.kernel_launches += ps.kernel_launches;
    s.graph_replays += ps.graph_replays;
    as_output_free(p);
  }
  c->records_done += n;
  *out = o;
  return AS_OK;
}

as_status as_output_records(const as_output* o, const uint8_t** bytes, const uint64_t** offsets, uint64_t* n,
                            uint32_t* on_device) {
  if (!o || !bytes || !offsets || !n) return AS_ERR_ARG;
  if (o->on_device) {
    *bytes = reinterpret_cast<const uint8_t*>(o->d_bytes);
    *offsets = o->d_off;
  } else {
    *bytes = o->h_bytes.data();
    *offsets = o->h_off.data();
  }
  *n = o->n;
  if (on_device) *on_device = o->on_device;
  return AS_OK;
}

as_status as_output_stats(const as_output* o, as_stats* s) {
  if (!o || !s) return AS_ERR_ARG;
  *s = o->stats;
  return AS_OK;
}

as_status as_output_map(as_output* o, const as_entity** entries, uint64_t* n) {
  if (!o || !entries || !n) return AS_ERR_ARG;
  if (!o->map_loaded) {
    as_ctx* c = o->ctx;
    cudaSetDevice(c->device);
    as_status s = map_collect(c, o->call_lo ? o->call_lo : o->call_id, o->call_id, o->map, o->map_orig);
    if (s != AS_OK) return s;
    for (auto& e : o->map) e.original = o->map_orig.data() + reinterpret_cast<uint64_t&>(e.original);
    o->map_loaded = true;
  }
  *entries = o->map.data();
  *n = o->map.size();
  return AS_OK;
}

void as_output_free(as_output* o) {
  if (!o) return;
  if (o->d_bytes || o->d_off) {
    // cudaFree waits for the work in flight: valid after the ctx is gone too
    cudaSetDevice(o->device);
    if (o->d_bytes) cudaFree(o->d_bytes);
    if (o->d_off) cudaFree(o->d_off);
  }
  delete o;
}

as_status as_reidentify(as_ctx* c, const as_records* rec, const as_schema* sch, const uint8_t* key, size_t key_len,
                        as_output** out) {
  if (!c || !rec || !out) return AS_ERR_ARG;
  *out = nullptr;
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, AS_ERR_CUDA, "cudaSetDevice failed");
  if (c->server) return fail(c, AS_ERR_STATE, "re-identification while serving (the map is changing)");
  CKI(validate_schema(c, sch));
  const uint32_t L = sch->slug_hex_len;
  if (L == 0) return fail(c, AS_ERR_ARG, "slug_hex_len 0: the replacements carry no hash to re-identify");
  for (uint32_t t = 0; t < sch->n_types; ++t)
    if (std::strpbrk(sch->type_names[t], "[]")) return fail(c, AS_ERR_ARG, "type names must not contain brackets");
  CKI(set_key(c, key, key_len));
  Lane* ln = &c->main;
  cudaStream_t st = ln->stream;
  const uint64_t launches0 = t_launches;
  const uint64_t n = rec->n_records;
  uint64_t N = 0;
  const uint8_t* d_bytes = nullptr;
  const uint64_t* d_off = nullptr;
  CKI(stage_records(c, ln, rec, &d_bytes, &d_off, &N));
  const uint32_t N32 = (uint32_t)N;
  CKI(upload_names(c, ln, sch));
  // entries verified under the key, indexed by (type, slug prefix)
  const MapView m = map_view(c);
  const uint64_t slots = c->map_mask + 1;
  if (slots >= kReidAmbiguous) return fail(c, AS_ERR_CAPACITY, "map too large to index");
  CKS(grow(ln->rid_ok, slots));
  CKS(grow(ln->rid_tk, slots * 8));
  CKS(grow(ln->rid_tv, slots * 4));
  CK(cudaMemsetAsync(ln->rid_tk.p, 0, slots * 8, st));
  CK(cudaMemsetAsync(ln->rid_tv.p, 0xFF, slots * 4, st));
  const ReidTab tab{ln->rid_tk.as<unsigned long long>(), ln->rid_tv.as<uint32_t>(), slots - 1};
  launch_hmac_verify_slots(m, c->key_state.as<uint32_t>(), ln->rid_ok.as<uint8_t>(), st);
  launch_reid_index(m, 4 * std::min<uint32_t>(L, 14), tab, st);
  // pseudonyms
  CKS(grow(ln->counters, 64));
  CK(cudaMemsetAsync(ln->counters.p, 0, 64, st));
  unsigned long long* ctr = ln->counters.as<unsigned long long>();  // [0..3] stats, [4] low word = span count
  uint32_t* n_sp_dev = reinterpret_cast<uint32_t*>(ctr + 4);
  CKS(grow(ln->rs_bits, ((size_t)N / 32 + 1) * 4));
  CKS(grow(ln->rid_len, N * 4 + 4));
  CKS(grow(ln->rid_slot, N * 4 + 4));
  CKS(grow(ln->rid_flag, N + 16));
  CKS(grow(ln->rid_pos, (N + 1) * 4));
  CKS(grow(ln->scan_tiles, (scan_tiles_needed(std::max<uint64_t>(N + 1, 1) * 2) + 16) * 8));
  launch_mark_record_starts(d_off, n, N32, ln->rs_bits.as<uint32_t>(), st);
  launch_reid_mark(d_bytes, N32, ln->rs_bits.as<uint32_t>(), ln->names.as<char>(), ln->name_off.as<uint32_t>(),
                   sch->n_types, L, tab, m, ln->rid_ok.as<uint8_t>(), ln->rid_len.as<uint32_t>(),
                   ln->rid_slot.as<uint32_t>(), ln->rid_flag.as<uint8_t>(), ctr, st);
  exclusive_scan<uint32_t>(NonZeroU8{ln->rid_flag.as<uint8_t>()}, N, ln->rid_pos.as<uint32_t>(), n_sp_dev,
                           ln->scan_tiles.as<uint32_t>(), st);
  unsigned long long h_ctr[5] = {0, 0, 0, 0, 0};
  CK(cudaMemcpyAsync(h_ctr, ctr, sizeof(h_ctr), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const uint32_t n_sp = (uint32_t)(h_ctr[4] & 0xffffffffull);
  CKS(grow(ln->rid_s, (n_sp + 1) * 4));
  CKS(grow(ln->rid_l, (n_sp + 1) * 4));
  CKS(grow(ln->rid_k, (n_sp + 1) * 4));
  launch_reid_emit(ln->rid_len.as<uint32_t>(), ln->rid_slot.as<uint32_t>(), ln->rid_flag.as<uint8_t>(),
                   ln->rid_pos.as<uint32_t>(), N32, ln->rid_s.as<uint32_t>(), ln->rid_l.as<uint32_t>(),
                   ln->rid_k.as<uint32_t>(), st);
  CKS(grow(ln->delta, (size_t)(n_sp + 1) * 8));
  CKS(grow(ln->shift, (size_t)(n_sp + 1) * 8));
  CKS(grow(ln->delta_total, 16));
  launch_reid_delta(ln->rid_l.as<uint32_t>(), ln->rid_k.as<uint32_t>(), n_sp, m, ln->delta.as<int64_t>(), n_sp + 1, st);
  exclusive_scan<int64_t>(LoadI64{ln->delta.as<int64_t>()}, n_sp + 1, ln->shift.as<int64_t>(),
                          ln->delta_total.as<int64_t>(), reinterpret_cast<int64_t*>(ln->scan_tiles.p), st);
  int64_t total_delta = 0;
  CK(cudaMemcpyAsync(&total_delta, ln->delta_total.p, 8, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const uint64_t out_size = (uint64_t)((int64_t)N + total_delta);
  as_output* o = new as_output();
  o->ctx = c;
  o->device = c->device;
  o->map_loaded = true;  // re-identification adds no map entries
  o->on_device = rec->on_device ? 1u : 0u;
  o->n = n;
  void* d_out = nullptr;
  uint64_t* d_out_off = nullptr;
  if (cudaMallocAsync(&d_out, out_size + 16, st) != cudaSuccess ||
      cudaMallocAsync(reinterpret_cast<void**>(&d_out_off), (n + 1) * 8, st) != cudaSuccess) {
    cudaGetLastError();
    if (d_out) cudaFreeAsync(d_out, st);
    delete o;
    return fail(c, AS_ERR_OOM, "output allocation failed");
  }
  launch_sub_copy(d_bytes, N32, ln->rid_s.as<uint32_t>(), ln->rid_l.as<uint32_t>(), n_sp_dev, ln->shift.as<int64_t>(),
                  reinterpret_cast<uint8_t*>(d_out), st);
  launch_reid_replace(ln->rid_s.as<uint32_t>(), ln->rid_k.as<uint32_t>(), n_sp, ln->shift.as<int64_t>(), m,
                      reinterpret_cast<uint8_t*>(d_out), st);
  launch_sub_offsets(d_off, n, ln->rid_s.as<uint32_t>(), n_sp_dev, ln->shift.as<int64_t>(), d_out_off, st);
  if (o->on_device) {
    o->d_bytes = d_out;
    o->d_off = d_out_off;
  } else {
    o->h_bytes.resize(out_size);
    o->h_off.resize(n + 1);
    cudaMemcpyAsync(o->h_bytes.data(), d_out, out_size, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(o->h_off.data(), d_out_off, (n + 1) * 8, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(d_out, st);
    cudaFreeAsync(d_out_off, st);
  }
  const cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    as_output_free(o);
    return fail(c, AS_ERR_CUDA, std::string("stream: ") + cudaGetErrorString(e));
  }
  as_stats& s = o->stats;
  s.n_records = n;
  s.n_bytes = N;
  s.n_out_bytes = out_size;
  s.n_pseudonyms = h_ctr[0];
  s.n_reidentified = h_ctr[1];
  s.n_ambiguous = h_ctr[2];
  s.n_unverified = h_ctr[3];
  s.kernel_launches = t_launches - launches0;
  *out = o;
  return AS_OK;
}

as_status as_map_export(as_ctx* c, as_entity** entries, uint64_t* n) {
  if (!c || !entries || !n) return AS_ERR_ARG;
  cudaSetDevice(c->device);
  std::vector<as_entity> ents;
  std::vector<uint8_t> orig;
  as_status s = map_collect(c, 0, 0, ents, orig);
  if (s != AS_OK) return s;
  size_t bytes = ents.size() * sizeof(as_entity) + orig.size() + 1;
  uint8_t* blob = static_cast<uint8_t*>(malloc(bytes));
  if (!blob) return fail(c, AS_ERR_OOM, "host allocation");
  as_entity* e = reinterpret_cast<as_entity*>(blob);
  uint8_t* o = blob + ents.size() * sizeof(as_entity);
  if (!orig.empty()) memcpy(o, orig.data(), orig.size());
  for (size_t i = 0; i < ents.size(); ++i) {
    e[i] = ents[i];
    e[i].original = o + reinterpret_cast<uint64_t&>(ents[i].original);
  }
  *entries = e;
  *n = ents.size();
  return AS_OK;
}

as_status as_map_merge(const as_entity* const* shards, const uint64_t* n, const uint64_t* record_offset,
                       uint32_t n_shards, as_entity** out, uint64_t* n_out) {
  if (!out || !n_out || (n_shards && (!shards || !n))) return AS_ERR_ARG;
  struct Acc {
    const as_entity* first;  // type, bytes, hash and slug come from here
    uint64_t first_seen, last_seen, count;
  };
  // key: type byte then the original bytes; std::string orders bytes as
  // unsigned char with a prefix first, the order of as_map_export
  std::map<std::string, Acc> acc;
  uint64_t total_len = 0;
  for (uint32_t s = 0; s < n_shards; ++s) {
    if (n[s] && !shards[s]) return fail(nullptr, AS_ERR_ARG, "shard " + std::to_string(s) + " is NULL");
    const uint64_t off = record_offset ? record_offset[s] : 0;
    for (uint64_t i = 0; i < n[s]; ++i) {
      const as_entity& e = shards[s][i];
      if (e.type > 255 || (e.original_len && !e.original)) return fail(nullptr, AS_ERR_ARG, "malformed entry");
      std::string k(1, (char)e.type);
      k.append(reinterpret_cast<const char*>(e.original), e.original_len);
      auto it = acc.find(k);
      if (it == acc.end()) {
        acc.emplace(std::move(k), Acc{&e, e.first_seen + off, e.last_seen + off, e.count});
        total_len += e.original_len;
        continue;
      }
      Acc& a = it->second;
      if (memcmp(a.first->full_hash, e.full_hash, 64) != 0)
        return fail(nullptr, AS_ERR_STATE, "shards disagree on an entity's HMAC: maps made under different keys");
      a.first_seen = std::min(a.first_seen, e.first_seen + off);
      a.last_seen = std::max(a.last_seen, e.last_seen + off);
      a.count += e.count;
    }
  }
  const size_t bytes = acc.size() * sizeof(as_entity) + total_len + 1;
  uint8_t* blob = static_cast<uint8_t*>(malloc(bytes));
  if (!blob) return fail(nullptr, AS_ERR_OOM, "host allocation");
  as_entity* e = reinterpret_cast<as_entity*>(blob);
  uint8_t* o = blob + acc.size() * sizeof(as_entity);
  size_t i = 0;
  for (auto& kv : acc) {
    const Acc& a = kv.second;
    e[i] = *a.first;
    e[i].original = o;
    if (a.first->original_len) memcpy(o, a.first->original, a.first->original_len);
    o += a.first->original_len;
    e[i].first_seen = a.first_seen;
    e[i].last_seen = a.last_seen;
    e[i].count = a.count;
    ++i;
  }
  *out = e;
  *n_out = acc.size();
  return AS_OK;
}

as_status as_map_import(as_ctx* c, const uint8_t* key, size_t key_len, const as_entity* entries, uint64_t n) {
  if (!c || (n && !entries)) return AS_ERR_ARG;
  cudaSetDevice(c->device);
  as_status ks = set_key(c, key, key_len);
  if (ks != AS_OK) return ks;
  if (n == 0) return AS_OK;
  std::vector<uint8_t> orig;
  std::vector<uint64_t> off(n), first(n), last(n), count(n);
  std::vector<uint32_t> len(n), type(n), dig(n * 8);
  for (uint64_t i = 0; i < n; ++i) {
    const as_entity& e = entries[i];
    off[i] = orig.size();
    orig.insert(orig.end(), e.original, e.original + e.original_len);
    len[i] = e.original_len;
    type[i] = e.type;
    first[i] = e.first_seen;
    last[i] = e.last_seen;
    count[i] = e.count;
    for (int k = 0; k < 8; ++k) {
      uint32_t v = 0;
      for (int j = 0; j < 8; ++j) {
        char ch = e.full_hash[k * 8 + j];
        uint32_t nib = (ch >= '0' && ch <= '9') ? ch - '0' : (ch >= 'a' && ch <= 'f') ? ch - 'a' + 10 : 99;
        if (nib > 15) return fail(c, AS_ERR_ARG, "full_hash must be 64 lower-case hex characters");
        v = (v << 4) | nib;
      }
      dig[i * 8 + k] = v;
    }
  }
  DBuf b_orig, b_off, b_len, b_type, b_dig, b_first, b_last, b_count;
  DBuf* bs[] = {&b_orig, &b_off, &b_len, &b_type, &b_dig, &b_first, &b_last, &b_count};
  auto cleanup = [&]() { for (DBuf* b : bs) release(*b); };
  if (grow(b_orig, orig.size() + 1) || grow(b_off, n * 8) || grow(b_len, n * 4) || grow(b_type, n * 4) ||
      grow(b_dig, n * 32) || grow(b_first, n * 8) || grow(b_last, n * 8) || grow(b_count, n * 8)) {
    cleanup();
    return fail(c, AS_ERR_OOM, "import staging");
  }
  cudaStream_t st = c->main.stream;
  if (!orig.empty()) cudaMemcpyAsync(b_orig.p, orig.data(), orig.size(), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(b_off.p, off.data(), n * 8, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(b_len.p, len.data(), n * 4, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(b_type.p, type.data(), n * 4, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(b_dig.p, dig.data(), n * 32, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(b_first.p, first.data(), n * 8, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(b_last.p, last.data(), n * 8, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(b_count.p, count.data(), n * 8, cudaMemcpyHostToDevice, st);
  const uint32_t import_id = ++c->call_id;
  launch_map_import(map_view(c), b_orig.as<uint8_t>(), b_off.as<uint64_t>(), b_len.as<uint32_t>(),
                    b_type.as<uint32_t>(), b_dig.as<uint32_t>(), b_first.as<uint64_t>(), b_last.as<uint64_t>(),
                    b_count.as<uint64_t>(), n, import_id, c->main.dev_err.as<DevError>(), st);
  cudaError_t e = cudaStreamSynchronize(st);
  cleanup();
  if (e != cudaSuccess) return fail(c, AS_ERR_CUDA, std::string("import: ") + cudaGetErrorString(e));
  return check_dev_error(c, &c->main);
}

as_status as_map_clear(as_ctx* c) {
  if (!c) return AS_ERR_ARG;
  cudaSetDevice(c->device);
  launch_map_init(map_view(c), c->main.stream);
  c->n_entries_seen = 0;
  c->key_set = false;
  c->key.clear();
  if (cudaStreamSynchronize(c->main.stream) != cudaSuccess) return fail(c, AS_ERR_CUDA, "map clear");
  return AS_OK;
}

as_status as_calibrate(as_ctx* c, const as_records* records, const as_schema* schema) {
  if (!c) return AS_ERR_ARG;
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, AS_ERR_CUDA, "cudaSetDevice failed");
  if (c->server) return fail(c, AS_ERR_STATE, "the ctx is serving");
  as_status s = anonymize_impl(c, &c->main, records, schema, nullptr, 0, nullptr, true);
  if (s == AS_ERR_CUDA) cudaGetLastError();
  return s;
}

as_status as_get_scales(as_ctx* c, float* scales, uint64_t n) {
  if (!c || !scales) return AS_ERR_ARG;
  const uint64_t need = (uint64_t)kActPerLayer * c->cfg.n_layers;
  if (c->act_scale.size() != need) return fail(c, AS_ERR_STATE, "no activation scales yet");
  if (n < need) return fail(c, AS_ERR_ARG, "need room for 4 scales per layer");
  memcpy(scales, c->act_scale.data(), need * 4);
  return AS_OK;
}

as_status as_set_scales(as_ctx* c, const float* scales, uint64_t n) {
  if (!c || !scales) return AS_ERR_ARG;
  if (c->cfg.precision != AS_FP8) return fail(c, AS_ERR_STATE, "scales are for AS_FP8 contexts");
  const uint64_t need = (uint64_t)kActPerLayer * c->cfg.n_layers;
  if (n != need) return fail(c, AS_ERR_ARG, "expected 4 scales per layer");
  for (uint64_t i = 0; i < n; ++i)
    if (!(scales[i] > 0.f) || !std::isfinite(scales[i])) return fail(c, AS_ERR_ARG, "scales must be finite and > 0");
  c->act_scale.assign(scales, scales + n);
  return AS_OK;
}

as_status as_serve_start(as_ctx* c, const as_schema* schema, const uint8_t* key, size_t key_len,
                         const as_serve_config* cfg) {
  if (!c || !cfg) return AS_ERR_ARG;
  if (c->server) return fail(c, AS_ERR_STATE, "already serving");
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, AS_ERR_CUDA, "cudaSetDevice failed");
  CKI(validate_schema(c, schema));
  if (c->cfg.precision == AS_FP8 && c->act_scale.empty())
    return fail(c, AS_ERR_STATE, "FP8 context without activation scales");
  CKI(set_key(c, key, key_len));
  Server* sv = new Server();
  sv->c = c;
  for (uint32_t t = 0; t < schema->n_types; ++t) sv->names.emplace_back(schema->type_names[t]);
  for (auto& n : sv->names) sv->name_ptrs.push_back(n.c_str());
  sv->schema = *schema;
  sv->schema.type_names = sv->name_ptrs.data();
  if (schema->recognizer_types) {
    std::copy(schema->recognizer_types, schema->recognizer_types + AS_RX_KINDS, sv->rx_types);
    sv->schema.recognizer_types = sv->rx_types;
  }
  sv->batch_bytes = cfg->max_batch_bytes ? cfg->max_batch_bytes : UINT64_MAX;
  sv->max_batch = cfg->max_batch_records ? cfg->max_batch_records : 65536;
  sv->max_pending = cfg->max_pending ? cfg->max_pending : (1ull << 20);
  sv->next_id = c->records_done;
  sv->t_stats0 = now_ns();
  sv->max_pos = c->cfg.max_pos;
  const uint32_t n_lanes = cfg->lanes ? std::min<uint32_t>(cfg->lanes, 8) : 2;
  // admission by device memory: each lane's share of the activation budget
  // gives its row cap (largest multiple of 8 whose bucketed rows fit)
  sv->act_budget = cfg->activation_budget_bytes ? cfg->activation_budget_bytes : (40ull << 30);
  {
    const uint64_t share = sv->act_budget / n_lanes, per_row = encoder_held_bytes(c->cfg, 1);
    uint64_t lo = 0, hi = std::min<uint64_t>(share / per_row, 1ull << 31) / 8;  // in units of 8 rows
    while (lo < hi) {
      const uint64_t mid = (lo + hi + 1) / 2;
      if (encoder_held_bytes(c->cfg, encoder_rows(c->cfg, mid * 8)) <= share) lo = mid; else hi = mid - 1;
    }
    sv->row_cap = lo * 8;
    const uint64_t one_seq = ((uint64_t)c->cfg.max_pos + 7) & ~7ull;
    if (sv->row_cap < one_seq) {
      delete sv;
      return fail(c, AS_ERR_ARG, "activation budget of " + std::to_string(cfg->activation_budget_bytes) +
                                     " bytes cannot hold one full sequence per lane (" + std::to_string(one_seq) +
                                     " rows of " + std::to_string(per_row) + " bytes)");
    }
  }
  for (uint32_t i = 0; i < n_lanes; ++i) {
    auto ln = std::make_unique<Lane>();
    if (cudaStreamCreateWithFlags(&ln->stream, cudaStreamNonBlocking) != cudaSuccess ||
        grow(ln->dev_err, sizeof(DevError)) != AS_OK ||
        cudaMemsetAsync(ln->dev_err.p, 0, sizeof(DevError), ln->stream) != cudaSuccess) {
      for (auto& l : sv->lanes) {
        l->release_all();
        cudaStreamDestroy(l->stream);
      }
      if (ln->stream) cudaStreamDestroy(ln->stream);
      delete sv;
      return fail(c, AS_ERR_CUDA, "serving lane set-up failed");
    }
    ln->row_cap = sv->row_cap;
    sv->lanes.push_back(std::move(ln));
  }
  c->server = sv;
  for (auto& ln : sv->lanes) sv->workers.emplace_back(&Server::worker, sv, ln.get());
  return AS_OK;
}

as_status as_submit(as_ctx* c, const uint8_t* rec, uint64_t len, uint32_t flags, uint64_t* request_id) {
  if (!c || (!rec && len) || !request_id) return AS_ERR_ARG;
  Server* sv = c->server;
  if (!sv) return fail(c, AS_ERR_STATE, "not serving: call as_serve_start");
  auto* r = new ServeRequest();
  r->bytes.assign(rec, rec + len);
  r->discard = (flags & AS_SUBMIT_DISCARD) != 0;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) {
      delete r;
      return fail(c, AS_ERR_STATE, "serving is stopping");
    }
    if (sv->queue.size() >= sv->max_pending) {
      ++sv->rejected;
      delete r;
      return fail(c, AS_ERR_AGAIN, "admission queue full");
    }
    r->id = sv->next_id++;
    r->t_submit = now_ns();
    sv->queue.push_back(r);
    sv->live[r->id] = r;
    *request_id = r->id;
  }
  sv->cv_work.notify_one();
  return AS_OK;
}

as_status as_poll(as_ctx* c, uint64_t request_id, as_output** out, int64_t timeout_us) {
  if (!c || !out) return AS_ERR_ARG;
  *out = nullptr;
  Server* sv = c->server;
  if (!sv) return fail(c, AS_ERR_STATE, "not serving");
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->live.find(request_id);
  if (it == sv->live.end()) return fail(c, AS_ERR_ARG, "unknown request id (or submitted with AS_SUBMIT_DISCARD)");
  ServeRequest* r = it->second;
  if (r->discard) return fail(c, AS_ERR_ARG, "request was submitted with AS_SUBMIT_DISCARD");
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(timeout_us < 0 ? 0 : timeout_us);
  if (!sv->cv_done.wait_until(lk, deadline, [&] { return r->done; }))
    return fail(c, AS_ERR_TIMEOUT, "request not finished within the timeout");
  sv->live.erase(it);
  lk.unlock();
  const as_status st = r->status;
  if (st == AS_OK) {
    as_output* o = new as_output();
    o->ctx = c;
    o->device = c->device;
    o->on_device = 0;
    o->n = 1;
    o->h_bytes = std::move(r->out);
    o->h_off = {0, (uint64_t)o->h_bytes.size()};
    o->stats.n_records = 1;
    o->stats.n_bytes = r->bytes.size();
    o->stats.n_tokens = r->tokens;
    o->stats.n_out_bytes = o->h_bytes.size();
    o->map_loaded = true;  // per-request map views are not kept; use as_map_export
    *out = o;
  }
  delete r;
  return st == AS_OK ? AS_OK : fail(c, st, "the batch of this request failed");
}

as_status as_serve_stats(as_ctx* c, as_serve_stats_t* s, uint32_t reset) {
  if (!c || !s) return AS_ERR_ARG;
  Server* sv = c->server;
  if (!sv) return fail(c, AS_ERR_STATE, "not serving");
  std::lock_guard<std::mutex> lk(sv->mu);
  memset(s, 0, sizeof(*s));
  s->completed = sv->completed;
  s->rejected = sv->rejected;
  s->failed = sv->failed;
  s->batches = sv->batches;
  s->tokens = sv->tokens;
  s->pending = sv->queue.size();
  s->seconds = (now_ns() - sv->t_stats0) * 1e-9;
  s->activation_budget = sv->act_budget;
  s->row_cap = sv->row_cap;
  for (auto& l : sv->lanes) s->activation_bytes += l->act_bytes.load();
  s->activation_peak = std::max(sv->act_peak, s->activation_bytes);
  if (!sv->lat_ms.empty()) {
    std::vector<double> v = sv->lat_ms;
    auto pct = [&](double q) {
      size_t k = std::min(v.size() - 1, (size_t)(q * (v.size() - 1) + 0.5));
      std::nth_element(v.begin(), v.begin() + k, v.end());
      return v[k];
    };
    s->p50_ms = pct(0.50);
    s->p99_ms = pct(0.99);
    s->max_ms = *std::max_element(v.begin(), v.end());
  }
  if (reset) {
    sv->lat_ms.clear();
    sv->completed = sv->rejected = sv->batches = sv->tokens = sv->failed = 0;
    sv->t_stats0 = now_ns();
  }
  return AS_OK;
}

as_status as_serve_stop(as_ctx* c) {
  if (!c) return AS_ERR_ARG;
  Server* sv = c->server;
  if (!sv) return AS_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  for (auto& t : sv->workers) t.join();  // workers drain the queue first
  for (auto& kv : sv->live) delete kv.second;
  for (auto& ln : sv->lanes) {
    cudaStreamSynchronize(ln->stream);
    ln->release_all();
    cudaStreamDestroy(ln->stream);
  }
  c->records_done = std::max(c->records_done, sv->next_id);
  delete sv;
  c->server = nullptr;
  return AS_OK;
}

as_status as_autotune(as_ctx* c, uint64_t rows, as_tune_entry* entries) {
  if (!c || !entries) return AS_ERR_ARG;
  if (c->server) return fail(c, AS_ERR_STATE, "the ctx is serving");
  const as_config& g = c->cfg;
  if (g.precision == AS_FP32) return fail(c, AS_ERR_UNSUPPORTED, "FP32 contexts use the CUDA-core GEMM: nothing to tune");
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, AS_ERR_CUDA, "cudaSetDevice failed");
  if (rows == 0) rows = g.max_chunk_tokens ? g.max_chunk_tokens : (1ull << 19);
  if (rows > (1ull << 21)) return fail(c, AS_ERR_ARG, "rows above 2^21");
  const bool f8 = g.precision == AS_FP8;
  const uint64_t d = g.d_model, f = g.d_ffn, es = f8 ? 1 : 2;
  const LayerW& L = c->layers[0];
  struct Role {
    int epi;
    bool out8;
    uint64_t n, k;
    const void* w;
    const float* b;
  } roles[AS_TUNE_ROLES] = {
      {AS_EPI_BIAS, false, 3 * d, d, f8 ? (const void*)L.w_qkv8 : (const void*)L.w_qkv16, L.b_qkv},
      {AS_EPI_BIAS_RESID, false, d, d, f8 ? (const void*)L.w_o8 : (const void*)L.w_o16, L.b_o},
      {AS_EPI_BIAS_GELU, f8, f, d, f8 ? (const void*)L.w_1_8 : (const void*)L.w_1_16, L.b_1},
      {AS_EPI_BIAS_RESID, false, d, f, f8 ? (const void*)L.w_2_8 : (const void*)L.w_2_16, L.b_2}};
  // scratch operands (values do not change the timing): A, output, residual
  DBuf A, O, Rz;
  auto cleanup = [&]() { release(A); release(O); release(Rz); };
  cudaStream_t st = c->main.stream;
  if (grow(A, rows * std::max(d, f) * es) || grow(O, rows * std::max(3 * d, f) * 4) || grow(Rz, rows * d * 4)) {
    cleanup();
    return fail(c, AS_ERR_OOM, "autotune scratch");
  }
  if (cudaMemsetAsync(A.p, 0x3C, rows * std::max(d, f) * es, st) != cudaSuccess ||
      cudaMemsetAsync(Rz.p, 0, rows * d * 4, st) != cudaSuccess) {
    cleanup();
    return fail(c, AS_ERR_CUDA, "autotune scratch init");
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  DevError* err = c->main.dev_err.as<DevError>();
  as_status status = AS_OK;
  static_assert(kGemmCfgs <= AS_TUNE_CONFIGS, "one timing slot per tile configuration");
  for (int r = 0; r < AS_TUNE_ROLES && status == AS_OK; ++r) {
    const Role& ro = roles[r];
    as_tune_entry& en = entries[r];
    en.role = (uint32_t)r;
    en.m = rows;
    en.n = ro.n;
    en.k = ro.k;
    float best = 0.f;
    int best_cfg = -1;
    // a fused post-LN block has four choices: single-CTA tiles (cfg 0) or 2-SM
    // pairs (cfg 4), each with the long or the short main-loop ring (cfg | 2)
    const int block = r == 1 ? 0 : (r == 3 ? 1 : -1);
    const bool fused = block >= 0 && ln_fused(g, block);
    for (int cfg = 0; cfg < kGemmCfgs && status == AS_OK; ++cfg) {
      en.ms[cfg] = -1.f;
      if (fused ? (cfg & 1) != 0 : !gemm_tcgen05_cfg_valid(cfg, (int64_t)ro.n)) continue;
      auto launch = [&]() {
        if (fused)
          return gemm_tcgen05_resid_ln(f8, (int64_t)rows, (int64_t)ro.n, (int64_t)ro.k, A.p, ro.w, ro.b, Rz.as<float>(),
                                       block == 0 ? L.ln1_g : L.ln2_g, block == 0 ? L.ln1_b : L.ln2_b,
                                       f8 ? nullptr : O.as<__nv_bfloat16>(), f8 ? O.as<uint8_t>() : nullptr, 1.0f,
                                       1.0f, err, st, (cfg & 4) != 0, (cfg & 2) != 0);
        return gemm_tcgen05_ex(ro.epi, f8, ro.out8, (int64_t)rows, (int64_t)ro.n, (int64_t)ro.k, A.p, ro.w, ro.b,
                               ro.epi == AS_EPI_BIAS_RESID ? Rz.as<float>() : nullptr, O.p, 1.0f, 1.0f, err, st, cfg);
      };
      status = launch();  // warm-up (also sets the kernel's shared-memory attribute)
      if (status != AS_OK) break;
      cudaEventRecord(e0, st);
      for (int i = 0; i < 3 && status == AS_OK; ++i) status = launch();
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) status = AS_ERR_CUDA;
      if (status != AS_OK) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      en.ms[cfg] = ms / 3.f;
      if (best_cfg < 0 || en.ms[cfg] < best) {
        best = en.ms[cfg];
        best_cfg = cfg;
      }
    }
    en.chosen = best_cfg;
    if (status == AS_OK) c->gemm_cfg[r] = best_cfg;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaError_t e = cudaStreamSynchronize(st);
  cleanup();
  if (status != AS_OK) return fail(c, status, std::string("autotune: ") + as_k_last_error());
  if (e != cudaSuccess) return fail(c, AS_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
  return check_dev_error(c, &c->main);
}

as_status as_set_tiles(as_ctx* c, const int32_t* cfg) {
  if (!c || !cfg) return AS_ERR_ARG;
  if (c->server) return fail(c, AS_ERR_STATE, "the ctx is serving");
  const uint64_t d = c->cfg.d_model, f = c->cfg.d_ffn;
  const uint64_t n[AS_TUNE_ROLES] = {3 * d, d, f, d};
  for (int r = 0; r < AS_TUNE_ROLES; ++r)
    if (cfg[r] != -1 && !gemm_tcgen05_cfg_valid(cfg[r], (int64_t)n[r]))
      return fail(c, AS_ERR_ARG, "tile configuration " + std::to_string(cfg[r]) + " is not valid for projection " +
                                     std::to_string(r));
  for (int r = 0; r < AS_TUNE_ROLES; ++r) c->gemm_cfg[r] = cfg[r];
  return AS_OK;
}

as_status as_get_tiles(as_ctx* c, int32_t* cfg) {
  if (!c || !cfg) return AS_ERR_ARG;
  for (int r = 0; r < AS_TUNE_ROLES; ++r) cfg[r] = c->gemm_cfg[r];
  return AS_OK;
}

// staged: host records already copied to ln->f_bytes / ln->f_off (JSONL ingest)
as_status fields_impl(as_ctx* c, const as_records* rec, const as_fields* fl, const as_field_policy* pol,
                      const as_schema* sch, const uint8_t* key, size_t key_len, as_output** out, bool staged) {
  Lane* ln = &c->main;
  cudaStream_t st = ln->stream;
  const uint64_t n = rec->n_records, nf = fl->n_fields;
  if (n > 0 && !rec->offsets) return fail(c, AS_ERR_ARG, "offsets is NULL");
  if (nf > 0 && (!fl->start || !fl->len || !fl->id)) return fail(c, AS_ERR_ARG, "field arrays are NULL");
  if (pol->n_ids > 0 && (!pol->action || !pol->force_type)) return fail(c, AS_ERR_ARG, "policy arrays are NULL");
  if (pol->default_action != AS_FIELD_DETECT && pol->default_action != AS_FIELD_EXCLUDE)
    return fail(c, AS_ERR_ARG, "default_action must be AS_FIELD_DETECT or AS_FIELD_EXCLUDE");
  // record offsets on the host (validation, field -> record)
  std::vector<uint64_t> off(n + 1, 0);
  if (n > 0) {
    if (rec->on_device) {
      CK(cudaMemcpyAsync(off.data(), rec->offsets, (n + 1) * 8, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
    } else {
      memcpy(off.data(), rec->offsets, (n + 1) * 8);
    }
    if (off[0] != 0) return fail(c, AS_ERR_ARG, "offsets[0] must be 0");
    for (uint64_t r = 0; r < n; ++r)
      if (off[r + 1] < off[r]) return fail(c, AS_ERR_ARG, "offsets must be non-decreasing");
  }
  const uint64_t N = off[n];
  if (N >= (1ull << 32) - 64) return fail(c, AS_ERR_ARG, "a call takes less than 4 GiB of text");
  if (N > 0 && !rec->bytes) return fail(c, AS_ERR_ARG, "bytes is NULL");
  // fields: sorted, disjoint, each inside one record; actions from the policy
  std::vector<uint32_t> f_start(nf);
  std::vector<uint64_t> sub_off(nf + 1, 0);
  std::vector<uint32_t> fr_s, fr_l;
  std::vector<uint8_t> fr_t;
  uint64_t prev_end = 0, r = 0;
  for (uint64_t k = 0; k < nf; ++k) {
    const uint64_t a = fl->start[k], b = a + fl->len[k];
    if (a < prev_end || b > N)
      return fail(c, AS_ERR_ARG, "field " + std::to_string(k) + ": fields must be sorted, disjoint and inside the bytes");
    while (r < n && off[r + 1] <= a) ++r;  // the record holding byte a (empty fields at a record end: the next one)
    if (fl->len[k] > 0 && (r >= n || b > off[r + 1]))
      return fail(c, AS_ERR_ARG, "field " + std::to_string(k) + " crosses a record boundary");
    prev_end = b;
    const uint32_t id = fl->id[k];
    const uint8_t act = id < pol->n_ids ? pol->action[id] : pol->default_action;
    f_start[k] = (uint32_t)a;
    uint64_t detect_len = 0;
    if (act == AS_FIELD_DETECT) {
      detect_len = fl->len[k];
    } else if (act == AS_FIELD_FORCE) {
      const uint8_t t = pol->force_type[id];
      if (t < 1 || t > sch->n_types)
        return fail(c, AS_ERR_ARG, "field id " + std::to_string(id) + ": force_type must be 1..n_types");
      if (fl->len[k] > 0) {
        fr_s.push_back((uint32_t)a);
        fr_l.push_back(fl->len[k]);
        fr_t.push_back(t);
      }
    } else if (act != AS_FIELD_EXCLUDE) {
      return fail(c, AS_ERR_ARG, "field id " + std::to_string(id) + ": unknown action");
    }
    sub_off[k + 1] = sub_off[k] + detect_len;
  }
  const uint64_t n_sub_bytes = sub_off[nf];
  const uint32_t nforce = (uint32_t)fr_s.size();
  // device inputs: the original records, the field starts, the sub-record offsets, the forced spans
  const uint8_t* d_bytes;
  const uint64_t* d_off;
  if (rec->on_device) {
    d_bytes = rec->bytes;
    d_off = rec->offsets;
  } else {
    if (!staged) {
      CKS(grow(ln->f_bytes, N + 16));
      CKS(grow(ln->f_off, (n + 1) * 8));
      if (N) CK(cudaMemcpyAsync(ln->f_bytes.p, rec->bytes, N, cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync(ln->f_off.p, off.data(), (n + 1) * 8, cudaMemcpyHostToDevice, st));
    }
    d_bytes = ln->f_bytes.as<uint8_t>();
    d_off = ln->f_off.as<uint64_t>();
  }
  CKS(grow(ln->f_start, (nf + 1) * 4));
  CKS(grow(ln->f_sub_off, (nf + 1) * 8));
  CKS(grow(ln->f_sub, n_sub_bytes + 16));
  CKS(grow(ln->fr_s, ((size_t)nforce + 1) * 4));
  CKS(grow(ln->fr_l, ((size_t)nforce + 1) * 4));
  CKS(grow(ln->fr_t, (size_t)nforce + 16));
  CKS(grow(ln->fs_s, ((size_t)nforce + 1) * 4));
  CKS(grow(ln->fs_l, ((size_t)nforce + 1) * 4));
  CKS(grow(ln->fs_t, (size_t)nforce + 16));
  CKS(grow(ln->f_keep, (size_t)nforce + 16));
  CKS(grow(ln->f_pos, ((size_t)nforce + 1) * 4));
  CKS(grow(ln->f_cnt, 16));
  CKS(grow(ln->scan_tiles, (scan_tiles_needed(std::max<uint64_t>(nforce + 1, 1) * 2) + 16) * 8));
  if (nf) CK(cudaMemcpyAsync(ln->f_start.p, f_start.data(), nf * 4, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ln->f_sub_off.p, sub_off.data(), (nf + 1) * 8, cudaMemcpyHostToDevice, st));
  const uint32_t counts[2] = {0, nforce};  // [0]: forced spans kept, [1]: forced spans given
  CK(cudaMemcpyAsync(ln->f_cnt.p, counts, 8, cudaMemcpyHostToDevice, st));
  if (nforce) {
    CK(cudaMemcpyAsync(ln->fr_s.p, fr_s.data(), nforce * 4, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ln->fr_l.p, fr_l.data(), nforce * 4, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ln->fr_t.p, fr_t.data(), nforce, cudaMemcpyHostToDevice, st));
  }
  launch_field_gather(d_bytes, ln->f_start.as<uint32_t>(), ln->f_sub_off.as<uint64_t>(), nf, ln->f_sub.as<uint8_t>(),
                      st);
  if (nforce) {
    launch_field_force_trim(d_bytes, ln->fr_s.as<uint32_t>(), ln->fr_l.as<uint32_t>(), ln->f_keep.as<uint8_t>(), nforce,
                            st);
    exclusive_scan<uint32_t>(NonZeroU8{ln->f_keep.as<uint8_t>()}, nforce, ln->f_pos.as<uint32_t>(),
                             ln->f_cnt.as<uint32_t>(), ln->scan_tiles.as<uint32_t>(), st);
    launch_compact_spans(ln->fr_s.as<uint32_t>(), ln->fr_l.as<uint32_t>(), ln->fr_t.as<uint8_t>(),
                         ln->f_keep.as<uint8_t>(), ln->f_pos.as<uint32_t>(), ln->f_cnt.as<uint32_t>() + 1, nforce,
                         ln->fs_s.as<uint32_t>(), ln->fs_l.as<uint32_t>(), ln->fs_t.as<uint8_t>(), st);
  }
  // the host vectors above are read by the copies: finish them before they go out of scope
  CK(cudaStreamSynchronize(st));
  FieldJob fj{d_bytes, d_off, n, N, ln->f_start.as<uint32_t>(), ln->f_sub_off.as<uint64_t>(), nf,
              ln->fs_s.as<uint32_t>(), ln->fs_l.as<uint32_t>(), ln->fs_t.as<uint8_t>(), ln->f_cnt.as<uint32_t>(),
              nforce, rec->on_device != 0};
  as_records sub{ln->f_sub.as<uint8_t>(), ln->f_sub_off.as<uint64_t>(), nf, 1};
  as_status s = anonymize_impl(c, ln, &sub, sch, key, key_len, out, false, -1, &fj);
  if (s == AS_ERR_CUDA) cudaGetLastError();
  return s;
}

as_status as_anonymize_fields(as_ctx* c, const as_records* rec, const as_fields* fl, const as_field_policy* pol,
                              const as_schema* sch, const uint8_t* key, size_t key_len, as_output** out) {
  if (!c || !rec || !fl || !pol || !out) return AS_ERR_ARG;
  *out = nullptr;
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, AS_ERR_CUDA, "cudaSetDevice failed");
  if (c->server) return fail(c, AS_ERR_STATE, "the ctx is serving: use as_submit / as_poll or stop serving");
  CKI(validate_schema(c, sch));
  return fields_impl(c, rec, fl, pol, sch, key, key_len, out, false);
}

as_status as_anonymize_jsonl(as_ctx* c, const as_records* rec, const as_jsonl_policy* jp, const as_schema* sch,
                             const uint8_t* key, size_t key_len, as_output** out) {
  if (!c || !rec || !jp || !out) return AS_ERR_ARG;
  *out = nullptr;
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, AS_ERR_CUDA, "cudaSetDevice failed");
  if (c->server) return fail(c, AS_ERR_STATE, "the ctx is serving: use as_submit / as_poll or stop serving");
  CKI(validate_schema(c, sch));
  const uint32_t nk = jp->n_keys;
  if (nk > 0 && (!jp->key_names || !jp->action || !jp->force_type))
    return fail(c, AS_ERR_ARG, "policy arrays are NULL");
  if (nk > (1u << 20)) return fail(c, AS_ERR_ARG, "at most 2^20 key names");
  Lane* ln = &c->main;
  cudaStream_t st = ln->stream;
  const uint64_t n = rec->n_records;
  if (n > 0 && !rec->offsets) return fail(c, AS_ERR_ARG, "offsets is NULL");
  // the lines on the device: the caller's arrays, or copies in the lane's field staging buffers
  std::vector<uint64_t> off(n + 1, 0);
  if (n > 0) {
    if (rec->on_device) {
      CK(cudaMemcpyAsync(off.data(), rec->offsets, (n + 1) * 8, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
    } else {
      memcpy(off.data(), rec->offsets, (n + 1) * 8);
    }
    if (off[0] != 0) return fail(c, AS_ERR_ARG, "offsets[0] must be 0");
    for (uint64_t r = 0; r < n; ++r)
      if (off[r + 1] < off[r]) return fail(c, AS_ERR_ARG, "offsets must be non-decreasing");
  }
  const uint64_t N = off[n];
  if (N >= (1ull << 32) - 64) return fail(c, AS_ERR_ARG, "a call takes less than 4 GiB of text");
  if (N > 0 && !rec->bytes) return fail(c, AS_ERR_ARG, "bytes is NULL");
  const uint8_t* d_bytes;
  const uint64_t* d_off;
  if (rec->on_device) {
    d_bytes = rec->bytes;
    d_off = rec->offsets;
  } else {
    CKS(grow(ln->f_bytes, N + 16));
    CKS(grow(ln->f_off, (n + 1) * 8));
    if (N) CK(cudaMemcpyAsync(ln->f_bytes.p, rec->bytes, N, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ln->f_off.p, off.data(), (n + 1) * 8, cudaMemcpyHostToDevice, st));
    d_bytes = ln->f_bytes.as<uint8_t>();
    d_off = ln->f_off.as<uint64_t>();
  }
  // key names on the device
  std::vector<uint32_t> koff(nk + 1, 0);
  std::string kall;
  for (uint32_t t = 0; t < nk; ++t) {
    if (!jp->key_names[t]) return fail(c, AS_ERR_ARG, "key name is NULL");
    kall += jp->key_names[t];
    koff[t + 1] = (uint32_t)kall.size();
  }
  CKS(grow(ln->j_names, kall.size() + 16));
  CKS(grow(ln->j_koff, (nk + 1) * 4));
  if (!kall.empty()) CK(cudaMemcpyAsync(ln->j_names.p, kall.data(), kall.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ln->j_koff.p, koff.data(), (nk + 1) * 4, cudaMemcpyHostToDevice, st));
  const JsonKeys K{ln->j_names.as<char>(), ln->j_koff.as<uint32_t>(), nk};
  const uint64_t launches0 = t_launches;
  // fields: count per line, prefix sum, emit; then to the host for the per-field call
  CKS(grow(ln->j_cnt, (n + 1) * 4));
  CKS(grow(ln->j_bad, n + 16));
  CKS(grow(ln->j_pos, (n + 1) * 4));
  CKS(grow(ln->counters, 64));
  CKS(grow(ln->scan_tiles, (scan_tiles_needed(std::max<uint64_t>(n + 1, 1) * 2) + 16) * 8));
  CK(cudaMemsetAsync(ln->counters.p, 0, 64, st));
  unsigned long long* n_bad_dev = ln->counters.as<unsigned long long>();
  uint32_t* n_fields_dev = reinterpret_cast<uint32_t*>(n_bad_dev + 1);
  launch_jsonl_count(d_bytes, d_off, n, K, ln->j_cnt.as<uint32_t>(), ln->j_bad.as<uint8_t>(), n_bad_dev, st);
  exclusive_scan<uint32_t>(LoadU32{ln->j_cnt.as<uint32_t>()}, n, ln->j_pos.as<uint32_t>(), n_fields_dev,
                           ln->scan_tiles.as<uint32_t>(), st);
  unsigned long long h_cnt[2] = {0, 0};
  CK(cudaMemcpyAsync(h_cnt, ln->counters.p, 16, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const uint64_t n_bad = h_cnt[0], nf = (uint32_t)(h_cnt[1] & 0xffffffffull);
  CKS(grow(ln->j_fs, (nf + 1) * 8));
  CKS(grow(ln->j_fl, (nf + 1) * 4));
  CKS(grow(ln->j_fid, (nf + 1) * 4));
  launch_jsonl_emit(d_bytes, d_off, n, K, ln->j_pos.as<uint32_t>(), ln->j_bad.as<uint8_t>(), ln->j_fs.as<uint64_t>(),
                    ln->j_fl.as<uint32_t>(), ln->j_fid.as<uint32_t>(), st);
  std::vector<uint64_t> fs(nf);
  std::vector<uint32_t> fln(nf), fid(nf);
  if (nf) {
    CK(cudaMemcpyAsync(fs.data(), ln->j_fs.p, nf * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(fln.data(), ln->j_fl.p, nf * 4, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(fid.data(), ln->j_fid.p, nf * 4, cudaMemcpyDeviceToHost, st));
  }
  CK(cudaStreamSynchronize(st));
  // policy over ids: the listed keys, then "other keys" (default), then malformed lines (detect)
  std::vector<uint8_t> act(nk + 2), ft(nk + 2, 0);
  for (uint32_t t = 0; t < nk; ++t) {
    act[t] = jp->action[t];
    ft[t] = jp->force_type[t];
  }
  act[nk] = jp->default_action;
  act[nk + 1] = AS_FIELD_DETECT;
  const as_fields fields{fs.data(), fln.data(), fid.data(), nf};
  const as_field_policy pol{nk + 2, act.data(), ft.data(), jp->default_action};
  as_status s = fields_impl(c, rec, &fields, &pol, sch, key, key_len, out, !rec->on_device);
  if (s == AS_OK && *out) {
    (*out)->stats.n_fields = nf;
    (*out)->stats.n_malformed = n_bad;
    (*out)->stats.kernel_launches = t_launches - launches0;  // the scan's launches and the per-field call's
  }
  return s;
}

as_status as_get_stream(as_ctx* c, void** stream) {
  if (!c || !stream) return AS_ERR_ARG;
  *stream = reinterpret_cast<void*>(c->main.stream);
  return AS_OK;
}

as_status as_profile(as_ctx* c, uint32_t enable) {
  if (!c) return AS_ERR_ARG;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->main.stream);
  c->main.ev_pending.clear();
  c->main.ev_used = 0;
  c->main.prof_acc = as_profile_stats{};
  c->main.prof = enable != 0;
  return AS_OK;
}

as_status as_profile_read(as_ctx* c, as_profile_stats* s) {
  if (!c || !s) return AS_ERR_ARG;
  *s = c->main.prof_acc;
  return AS_OK;
}

as_status as_debug_trace(as_ctx* c, as_trace* t) {
  if (!c || !t) return AS_ERR_ARG;
  if (!c->cfg.keep_trace) return fail(c, AS_ERR_STATE, "create the context with keep_trace = 1");
  t->n_records = c->main.last_n;
  t->n_tokens = c->main.last_T;
  t->n_regex = c->main.last_nrx;
  t->n_final = c->main.last_nfin;
  t->rec_tok = c->main.h_rec_tok.data();
  t->tok_ids = c->main.h_tok_ids.data();
  t->tok_off = c->main.h_tok_off.data();
  t->tok_len = c->main.h_tok_len.data();
  t->regex_start = c->main.h_rx_s.data();
  t->regex_len = c->main.h_rx_l.data();
  t->regex_type = c->main.h_rx_t.data();
  t->logits = c->main.last_logits ? c->main.h_logits.data() : nullptr;
  t->labels = c->main.h_labels.data();
  t->final_start = c->main.h_fin_s.data();
  t->final_len = c->main.h_fin_l.data();
  t->final_type = c->main.h_fin_t.data();
  return AS_OK;
}

}  // extern "C"
