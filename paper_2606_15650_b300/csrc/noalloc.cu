// Tokenizer entry point that allocates no memory (as_tokenize_static).
//
// Some callers cannot call cudaMalloc: hosts whose device memory is owned by
// their own allocator (a framework that reserved the GPU's memory up front and
// hands out pieces of it itself), and latency-bound loops where an allocation
// would synchronize the device and stall work already queued on it.
// This entry point runs the same tokenizer kernels as as_anonymize, but its
// scratch memory (record-start bitmap, per-byte token ids, per-byte prefix
// sums, scan tile sums) lives in one file-scope __device__ array of fixed
// size, so a call allocates nothing: the caller passes the inputs and the
// output arrays, all on the device.
//
// Limits and rules:
//   - at most kStaticMaxBytes (1 MiB) of text per call; larger calls are
//     rejected with AS_ERR_ARG;
//   - every GPU that loads the library holds the array (about 6.4 MB) until
//     the process exits;
//   - the first call on a device looks the array's address up with
//     cudaGetSymbolAddress (host code cannot use the symbol itself); make
//     that first call before any stream capture;
//   - all calls share the one array and it keeps the last call's contents:
//     what must start at zero is cleared on every call, but two calls that
//     overlap on the GPU (different streams or host threads) race;
//   - the call makes the ctx's device current while it runs and restores the
//     caller's current device before it returns.
#include <mutex>

#include "scan.cuh"
#include "stages.cuh"

namespace as {

// Looks up the ctx's vocabulary table and device (defined in runtime.cu).
bool ctx_vocab(const as_ctx* ctx, VocabTable* vt, int* device);

namespace {

constexpr uint32_t kStaticMaxBytes = AS_STATIC_MAX_BYTES;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffRs = 0;
constexpr size_t kOffTokAt = align256(kOffRs + ((size_t)kStaticMaxBytes / 32 + 1) * 4);
constexpr size_t kOffPos = align256(kOffTokAt + (size_t)kStaticMaxBytes * 2);
constexpr size_t kOffTiles = align256(kOffPos + ((size_t)kStaticMaxBytes + 1) * 4);
constexpr size_t kScratchBytes =
    align256(kOffTiles + ((size_t)kStaticMaxBytes + kScanTile - 1) / kScanTile * 4 + 4);

}  // namespace

static __device__ __align__(256) uint8_t g_tokenize_scratch[kScratchBytes];

namespace {

std::mutex g_mu;
void* g_scratch_addr[64] = {};

// Device address of the scratch array on `device` (current), looked up once.
void* scratch_address(int device, cudaError_t* err) {
  std::lock_guard<std::mutex> lk(g_mu);
  *err = cudaSuccess;
  if (device < 0 || device >= 64) {
    *err = cudaErrorInvalidDevice;
    return nullptr;
  }
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    *err = cudaGetSymbolAddress(&p, g_tokenize_scratch);
    if (*err != cudaSuccess) return nullptr;
    g_scratch_addr[device] = p;
  }
  return g_scratch_addr[device];
}

// Restores the caller's current device when the entry point returns.
struct DeviceRestore {
  int saved = -1;
  DeviceRestore() {
    if (cudaGetDevice(&saved) != cudaSuccess) saved = -1;
  }
  ~DeviceRestore() {
    if (saved >= 0) cudaSetDevice(saved);
  }
};

struct NonZeroTok {
  const uint16_t* p;
  __device__ uint32_t operator()(uint64_t i) const { return p[i] != 0; }
};

// Token lengths with the token count read on the device (no host sync).
__global__ void static_token_lengths_kernel(const uint32_t* __restrict__ off, const uint32_t* n_dev, uint32_t N,
                                            uint32_t* __restrict__ len) {
  const uint32_t T = *n_dev;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x)
    len[t] = (t + 1 < T ? off[t + 1] : N) - off[t];
}

}  // namespace
}  // namespace as

using namespace as;

extern "C" as_status as_tokenize_static(as_ctx* ctx, const uint8_t* bytes, const uint64_t* offsets,
                                        uint64_t n_records, uint64_t n_bytes, int32_t* tok_ids, uint32_t* tok_off,
                                        uint32_t* tok_len, uint64_t* rec_tok, uint32_t* n_tokens, void* stream) {
  VocabTable vt{};
  int device = 0;
  if (!ctx || !ctx_vocab(ctx, &vt, &device)) {
    set_k_error("as_tokenize_static: invalid context");
    return AS_ERR_ARG;
  }
  if (n_bytes > kStaticMaxBytes) {
    set_k_error("as_tokenize_static: " + std::to_string(n_bytes) + " bytes exceed the static limit of " +
                std::to_string(kStaticMaxBytes) + " bytes per call");
    return AS_ERR_ARG;
  }
  if (!offsets || !rec_tok || !n_tokens || (n_bytes && (!bytes || !tok_ids || !tok_off || !tok_len))) {
    set_k_error("as_tokenize_static: NULL input or output pointer");
    return AS_ERR_ARG;
  }
  DeviceRestore restore;
  AS_CUDA_OK(cudaSetDevice(device));
  cudaError_t e;
  uint8_t* base = static_cast<uint8_t*>(scratch_address(device, &e));
  if (!base) {
    set_k_error(std::string("as_tokenize_static: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
    return AS_ERR_CUDA;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const uint32_t N = (uint32_t)n_bytes;
  uint32_t* rs = reinterpret_cast<uint32_t*>(base + kOffRs);
  uint16_t* tok_at = reinterpret_cast<uint16_t*>(base + kOffTokAt);
  uint32_t* pos = reinterpret_cast<uint32_t*>(base + kOffPos);
  uint32_t* tiles = reinterpret_cast<uint32_t*>(base + kOffTiles);
  // the bitmap must start at zero: the launcher clears it before marking
  launch_mark_record_starts(offsets, n_records, N, rs, st);
  launch_tokenize_mark(bytes, N, rs, vt, tok_at, st);
  exclusive_scan<uint32_t>(NonZeroTok{tok_at}, N, pos, n_tokens, tiles, st);
  launch_tokenize_emit(tok_at, pos, N, tok_ids, tok_off, st);
  if (N) {
    static_token_lengths_kernel<<<grid_1d(N, 256, 148 * 64), 256, 0, st>>>(tok_off, n_tokens, N, tok_len);
    count_launch();
  }
  launch_record_token_offsets(offsets, n_records, pos, N, n_tokens, rec_tok, st);
  AS_CUDA_OK(cudaGetLastError());
  return AS_OK;
}
