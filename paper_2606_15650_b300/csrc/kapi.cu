// Kernel-level entry points (include/anonshield_kernels.h): the encoder's
// building blocks on caller-owned device buffers, for unit checks.
#include <vector>

#include "encoder.cuh"

using namespace as;

extern "C" {

uint64_t as_k_launch_count(void) { return g_launches.load(); }

as_status as_k_gemm(int precision, int engine, int epilogue, int64_t M, int64_t N, int64_t K, const void* A,
                    const void* B, const float* bias, const float* resid, void* out, void* stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (epilogue < AS_EPI_BIAS || epilogue > AS_EPI_BIAS_RESID) {
    set_k_error("as_k_gemm: bad epilogue");
    return AS_ERR_ARG;
  }
  if (epilogue == AS_EPI_BIAS_RESID && !resid) {
    set_k_error("as_k_gemm: residual epilogue needs resid");
    return AS_ERR_ARG;
  }
  if (precision == AS_BF16) {
    if (engine != AS_GEMM_AUTO && engine != AS_GEMM_TCGEN05) {
      set_k_error("as_k_gemm: BF16 runs on the tcgen05 engine");
      return AS_ERR_UNSUPPORTED;
    }
    return gemm_tcgen05(epilogue, M, N, K, A, B, bias, resid, out, nullptr, st);
  }
  if (precision == AS_FP32) {
    if (engine != AS_GEMM_AUTO && engine != AS_GEMM_SIMT) {
      set_k_error("as_k_gemm: FP32 runs on the SIMT engine");
      return AS_ERR_UNSUPPORTED;
    }
    return gemm_simt_f32(epilogue, M, N, K, static_cast<const float*>(A), static_cast<const float*>(B), bias, resid,
                         static_cast<float*>(out), st);
  }
  set_k_error("as_k_gemm: precision must be AS_FP32 or AS_BF16");
  return AS_ERR_ARG;
}

as_status as_k_gemm_resid_ln(int in_e4m3, int64_t M, int64_t N, int64_t K, const void* A, const void* B,
                             const float* bias, float* x32, const float* ln_g, const float* ln_b, void* out16,
                             void* out8, float out8_scale, float alpha, int pair, void* stream) {
  return gemm_tcgen05_resid_ln(in_e4m3 != 0, M, N, K, A, B, bias, x32, ln_g, ln_b,
                               static_cast<__nv_bfloat16*>(out16), static_cast<uint8_t*>(out8), out8_scale, alpha,
                               nullptr, reinterpret_cast<cudaStream_t>(stream), (pair & 1) != 0, (pair & 2) != 0);
}

as_status as_k_gemm_fp8(int epilogue, int out_e4m3, int64_t M, int64_t N, int64_t K, const void* A8, const void* B8,
                        float alpha, float out_scale, const float* bias, const float* resid, void* out, void* stream) {
  if (epilogue == AS_EPI_BIAS_RESID && !resid) {
    set_k_error("as_k_gemm_fp8: residual epilogue needs resid");
    return AS_ERR_ARG;
  }
  return gemm_tcgen05_ex(epilogue, true, out_e4m3 != 0, M, N, K, A8, B8, bias, resid, out, alpha, out_scale, nullptr,
                         reinterpret_cast<cudaStream_t>(stream));
}

as_status as_k_attention(int precision, const void* qkv, void* out, const int32_t* seq_start, const int32_t* seq_len,
                         int32_t n_seq, int64_t rows, int32_t d_model, int32_t n_heads, void* stream) {
  (void)rows;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // the kernel needs the longest sequence for its grid: read it from the host copy
  std::vector<int32_t> lens(n_seq > 0 ? n_seq : 0);
  if (n_seq > 0) {
    AS_CUDA_OK(cudaMemcpyAsync(lens.data(), seq_len, n_seq * 4, cudaMemcpyDeviceToHost, st));
    AS_CUDA_OK(cudaStreamSynchronize(st));
  }
  int32_t mx = 0;
  for (int32_t v : lens) mx = v > mx ? v : mx;
  if (precision == AS_BF16)
    return attention_bf16(static_cast<const __nv_bfloat16*>(qkv), static_cast<__nv_bfloat16*>(out), seq_start,
                          seq_len, n_seq, mx, d_model, n_heads, st);
  if (precision == AS_FP32)
    return attention_f32(static_cast<const float*>(qkv), static_cast<float*>(out), seq_start, seq_len, n_seq, mx,
                         d_model, n_heads, st);
  set_k_error("as_k_attention: precision must be AS_FP32 or AS_BF16");
  return AS_ERR_ARG;
}

}  // extern "C"

namespace {
// Work items from the host copies of the sequence table, then one tcgen05
// attention launch (BF16 output, or E4M3 of value / out_scale when out8).
as_status attention_tc_entry(const char* name, bool out8, const void* qkv, void* out, float out_scale,
                             const int32_t* seq_start, const int32_t* seq_len, int32_t n_seq, int64_t rows,
                             int32_t d_model, int32_t n_heads, void* stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  std::vector<int32_t> lens(n_seq > 0 ? n_seq : 0), starts(n_seq > 0 ? n_seq : 0);
  if (n_seq > 0) {
    AS_CUDA_OK(cudaMemcpyAsync(lens.data(), seq_len, n_seq * 4, cudaMemcpyDeviceToHost, st));
    AS_CUDA_OK(cudaMemcpyAsync(starts.data(), seq_start, n_seq * 4, cudaMemcpyDeviceToHost, st));
    AS_CUDA_OK(cudaStreamSynchronize(st));
  }
  int32_t mx = 0;
  for (int32_t i = 0; i < n_seq; ++i) {
    if (starts[i] < 0 || lens[i] < 0 || (int64_t)starts[i] + lens[i] > rows) {
      set_k_error(std::string(name) + ": every sequence must lie inside the rows");
      return AS_ERR_ARG;
    }
    mx = lens[i] > mx ? lens[i] : mx;
  }
  std::vector<int32_t> items;
  attention_items(starts.data(), lens.data(), n_seq, items);
  if (items.empty()) return AS_OK;
  int32_t* d_items = nullptr;
  AS_CUDA_OK(cudaMallocAsync(reinterpret_cast<void**>(&d_items), items.size() * 4, st));
  cudaError_t e = cudaMemcpyAsync(d_items, items.data(), items.size() * 4, cudaMemcpyHostToDevice, st);
  as_status s = e == cudaSuccess ? AS_OK : AS_ERR_CUDA;
  if (s == AS_OK) {
    const auto* q = static_cast<const __nv_bfloat16*>(qkv);
    const int32_t n_items = (int32_t)(items.size() / 2);
    s = out8 ? attention_tcgen05_e4m3(q, static_cast<uint8_t*>(out), out_scale, d_items, n_items, mx, rows, d_model,
                                      n_heads, nullptr, st)
             : attention_tcgen05(q, static_cast<__nv_bfloat16*>(out), d_items, n_items, mx, rows, d_model, n_heads,
                                 nullptr, st);
  }
  cudaFreeAsync(d_items, st);
  if (e != cudaSuccess) set_k_error(std::string(name) + ": " + cudaGetErrorString(e));
  return s;
}
}  // namespace

extern "C" {

as_status as_k_attention_tc(const void* qkv, void* out, const int32_t* seq_start,
                            const int32_t* seq_len, int32_t n_seq, int64_t rows, int32_t d_model, int32_t n_heads,
                            void* stream) {
  return attention_tc_entry("as_k_attention_tc", false, qkv, out, 1.0f, seq_start, seq_len, n_seq, rows, d_model,
                            n_heads, stream);
}

as_status as_k_attention_tc_e4m3(const void* qkv, void* out8, float out_scale, const int32_t* seq_start,
                                 const int32_t* seq_len, int32_t n_seq, int64_t rows, int32_t d_model,
                                 int32_t n_heads, void* stream) {
  return attention_tc_entry("as_k_attention_tc_e4m3", true, qkv, out8, out_scale, seq_start, seq_len, n_seq, rows,
                            d_model, n_heads, stream);
}

as_status as_k_layernorm(const float* in, const float* g, const float* b, float* out_f32, void* out_bf16, int64_t rows,
                         int32_t d, void* stream) {
  return layernorm_rows(in, g, b, out_f32, static_cast<__nv_bfloat16*>(out_bf16), rows, d,
                        reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
