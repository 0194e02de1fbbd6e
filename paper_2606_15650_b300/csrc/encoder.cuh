// Encoder kernels of the token classifier (AnonShield §2 stage (2)).
#pragma once

#include <vector>

#include "../../include/anonshield_kernels.h"
#include "common.cuh"

namespace as {

// C = epi(A . B^T) on tcgen05 (BF16 in, FP32 accumulate). See gemm_tc.cu.
as_status gemm_tcgen05(int epi, int64_t M, int64_t N, int64_t K, const void* A, const void* B, const float* bias,
                       const float* resid, void* out, DevError* err, cudaStream_t st);
// General form: A and B in BF16 or E4M3 (in_e4m3), output BF16 / FP32 (by
// epilogue) or E4M3 (out_e4m3, GELU epilogue only, value / out_scale with
// saturation); out = epi(alpha * (A . B^T)). cfg: tile configuration
// 0..kGemmCfgs-1 (bit 0: tile order along M instead of N; bit 1: 128-column
// tiles, 6 stages, instead of 256-column tiles, 4 stages; bit 2: 2-SM
// cta_group::2 pairs on a 256-row tile, each CTA loading its own A rows and
// half of the weight tile, no multicast), -1 = the default (256-column tiles
// when N allows, order along N, no pairs).
constexpr int kGemmCfgs = 8;
bool gemm_tcgen05_cfg_valid(int cfg, int64_t N);
// Post-LN residual block in one kernel: x32 <- LN(x32 + alpha (A . B^T) + bias)
// with gain ln_g and bias ln_b (eps 1e-5, biased variance), in place, plus a
// BF16 copy (out16) or an E4M3 copy of value / out8_scale (out8) when
// non-null (not both). A row of N columns is one cluster of gemm_resid_ln_cluster(N) CTAs
// (0: N not supported, use the residual GEMM and layernorm_rows instead); pair:
// 2-SM MMA pairs along M as well (a cluster of twice that many CTAs); deep: a
// shorter main-loop ring for four residual / output buffers per epilogue warp
// (for K = d, where the epilogue's bytes bound the kernel).
int gemm_resid_ln_cluster(int64_t N);
as_status gemm_tcgen05_resid_ln(bool in_e4m3, int64_t M, int64_t N, int64_t K, const void* A, const void* B,
                                const float* bias, float* x32, const float* ln_g, const float* ln_b,
                                __nv_bfloat16* out16, uint8_t* out8, float out8_scale, float alpha, DevError* err,
                                cudaStream_t st, bool pair = false, bool deep = false);
as_status gemm_tcgen05_ex(int epi, bool in_e4m3, bool out_e4m3, int64_t M, int64_t N, int64_t K, const void* A,
                          const void* B, const float* bias, const float* resid, void* out, float alpha,
                          float out_scale, DevError* err, cudaStream_t st, int cfg = -1);
// Same contract in FP32 on CUDA cores.
as_status gemm_simt_f32(int epi, int64_t M, int64_t N, int64_t K, const float* A, const float* B, const float* bias,
                        const float* resid, float* out, cudaStream_t st);

// Self-attention over packed sequences (see anonshield_kernels.h).
as_status attention_f32(const float* qkv, float* out, const int32_t* seq_start, const int32_t* seq_len, int32_t n_seq,
                        int32_t max_len, int32_t d_model, int32_t n_heads, cudaStream_t st);
as_status attention_bf16(const __nv_bfloat16* qkv, __nv_bfloat16* out, const int32_t* seq_start,
                         const int32_t* seq_len, int32_t n_seq, int32_t max_len, int32_t d_model, int32_t n_heads,
                         cudaStream_t st);

// Self-attention on tcgen05 (see attn_tc.cu), persistent over work items:
// attention_items appends one item per 128-query tile of each sequence, two
// int32 each (the sequence's first row; L | (q0 << 16)), longest sequences
// first; rows of each sequence inside [0, rows). An item with L = 0 is
// padding. n_items counts items (pairs); the array is 8-byte aligned.
void attention_items(const int32_t* seq_start, const int32_t* seq_len, int32_t n_seq, std::vector<int32_t>& items);
as_status attention_tcgen05(const __nv_bfloat16* qkv, __nv_bfloat16* out, const int32_t* items, int32_t n_items,
                            int32_t max_len, int64_t rows, int32_t d_model, int32_t n_heads, DevError* err,
                            cudaStream_t st);
// The same writing E4M3 (value / out_scale, saturating), for FP8 contexts.
as_status attention_tcgen05_e4m3(const __nv_bfloat16* qkv, uint8_t* out, float out_scale, const int32_t* items,
                                 int32_t n_items, int32_t max_len, int64_t rows, int32_t d_model, int32_t n_heads,
                                 DevError* err, cudaStream_t st);

// Row LayerNorm; writes FP32 and (optionally) BF16 copies.
as_status layernorm_rows(const float* in, const float* g, const float* b, float* out_f32, __nv_bfloat16* out_bf16,
                         int64_t rows, int32_t d, cudaStream_t st);

// X = LN(E[ids[row_tok[r]]] + P[row_pos[r]]) for each encoder row.
as_status embed_ln(const int32_t* tok_ids, const int32_t* row_tok, const int32_t* row_pos, const float* tok_emb,
                   const float* pos_emb, const float* g, const float* b, float* out_f32, __nv_bfloat16* out_bf16,
                   int64_t rows, int32_t d, cudaStream_t st);

// Last LayerNorm fused with the classifier: logits = LN(in) . Wc^T + bc, argmax
// (lowest label wins ties). A row whose own flag is set writes its logits and
// label to token row_tok[r] (window merge). C <= 32.
as_status layernorm_classify(const float* in, const float* g, const float* b, const float* cls_w, const float* cls_b,
                             int32_t C, const int32_t* row_tok, const uint8_t* row_own, float* logits,
                             uint8_t* labels, int64_t rows, int32_t d, cudaStream_t st);

// Same with the second copy in E4M3 (value / e4m3_scale, saturating) when
// out_e4m3 is not NULL.
as_status layernorm_rows_ex(const float* in, const float* g, const float* b, float* out_f32, __nv_bfloat16* out_bf16,
                            uint8_t* out_e4m3, float e4m3_scale, int64_t rows, int32_t d, cudaStream_t st);
as_status embed_ln_ex(const int32_t* tok_ids, const int32_t* row_tok, const int32_t* row_pos, const float* tok_emb,
                      const float* pos_emb, const float* g, const float* b, float* out_f32, __nv_bfloat16* out_bf16,
                      uint8_t* out_e4m3, float e4m3_scale, int64_t rows, int32_t d, cudaStream_t st);
// BF16 attention writing E4M3 (value / out_scale, saturating).
as_status attention_bf16_e4m3(const __nv_bfloat16* qkv, uint8_t* out, float out_scale, const int32_t* seq_start,
                              const int32_t* seq_len, int32_t n_seq, int32_t max_len, int32_t d_model,
                              int32_t n_heads, cudaStream_t st);
// amax (as float bits, atomicMax) and E4M3 quantization (n even).
void amax_f32(const float* x, uint64_t n, unsigned int* amax_bits, cudaStream_t st);
void amax_bf16(const __nv_bfloat16* x, uint64_t n, unsigned int* amax_bits, cudaStream_t st);
void quantize_e4m3(const float* x, uint8_t* y, uint64_t n, float scale, cudaStream_t st);

// FP32 -> BF16 copy (round to nearest even).
void convert_f32_bf16(const float* in, __nv_bfloat16* out, uint64_t n, cudaStream_t st);

}  // namespace as
