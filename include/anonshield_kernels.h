/*
 * anonshield_kernels.h — kernel-level entry points on device buffers.
 *
 * These expose the encoder's building blocks (AnonShield §2 stage (2): the
 * transformer token classifier) one at a time so that each kernel can be
 * checked against a plain reference of the same operation. All pointers are
 * device pointers on the current device; `stream` is a cudaStream_t (NULL =
 * legacy default stream). Calls are asynchronous on `stream` unless stated.
 * Return AS_OK or a negative as_status; as_k_last_error() gives the message
 * of the last failure on the calling thread.
 */
#ifndef ANONSHIELD_KERNELS_H
#define ANONSHIELD_KERNELS_H

#include "anonshield.h"

#ifdef __cplusplus
extern "C" {
#endif

/* GEMM epilogues: out = epi(A[M,K] . B[N,K]^T). */
#define AS_EPI_BIAS       0  /* out = acc + bias[n]                (act type)  */
#define AS_EPI_BIAS_GELU  1  /* out = gelu_erf(acc + bias[n])      (act type)  */
#define AS_EPI_BIAS_RESID 2  /* out = acc + bias[n] + resid[m,n]   (FP32 out)  */

/* GEMM engines. */
#define AS_GEMM_AUTO     0   /* BF16 -> tcgen05, FP32 -> SIMT                   */
#define AS_GEMM_TCGEN05  1   /* BF16 only: TMA + tcgen05.mma + TMEM, sm_103a    */
#define AS_GEMM_SIMT     2   /* FP32 only: CUDA-core FP32                       */

/* C = epi(A . B^T). Row-major A[M][K] and B[N][K] (B is an nn.Linear weight
 * [out][in]); precision AS_FP32: A, B float, act type float; AS_BF16: A, B
 * __nv_bfloat16, act type __nv_bfloat16, FP32 accumulation. bias: float[N]
 * (may be NULL = 0). resid/out for AS_EPI_BIAS_RESID: float[M][N].
 * Constraints: M >= 1; N % 128 == 0; K % 64 == 0 (BF16) or K % 8 == 0
 * (FP32); 16-byte aligned base pointers. AS_ERR_ARG otherwise. */
as_status as_k_gemm(int precision, int engine, int epilogue, int64_t M, int64_t N, int64_t K,
                    const void* A, const void* B, const float* bias, const float* resid, void* out,
                    void* stream);

/* E4M3 GEMM on tcgen05 (kind::f8f6f4): out = epi(alpha * (A8 . B8^T)), A8
 * [M][K] and B8 [N][K] E4M3 bytes, FP32 accumulation. Outputs as for
 * AS_EPI_* in BF16 (FP32 for AS_EPI_BIAS_RESID); with out_e4m3 = 1
 * (AS_EPI_BIAS_GELU only) the output is E4M3 of value / out_scale, rounded
 * to nearest even and saturated to +-448. K % 128 == 0, N % 128 == 0. */
as_status as_k_gemm_fp8(int epilogue, int out_e4m3, int64_t M, int64_t N, int64_t K, const void* A8, const void* B8,
                        float alpha, float out_scale, const float* bias, const float* resid, void* out, void* stream);

/* Post-LN residual block of the encoder in one kernel (AnonShield §2 stage
 * (2) encoder, post-LN form): x32 <- LN(x32 + alpha (A . B^T) + bias) with
 * gain ln_g[N] and bias ln_b[N], eps 1e-5, biased variance, in place
 * (float[M][N]); out16 (bf16[M][N]) or out8 (E4M3 bytes of value /
 * out8_scale, saturated) receives a copy when not NULL (at most one). A, B BF16 (in_e4m3 =
 * 0, K % 64 == 0) or E4M3 (in_e4m3 = 1, K % 128 == 0). Each 128-row block
 * runs on a cluster of CTAs that split the row: N must be 128, 256, 384,
 * 512, 768 or 1024. pair: bit 0 adds 2-SM MMA pairs along M (256-row blocks
 * on twice as many CTAs); bit 1 trades main-loop stages for four residual /
 * output buffers per epilogue warp (results identical in every mode).
 * 16-byte aligned pointers. AS_ERR_ARG otherwise. */
as_status as_k_gemm_resid_ln(int in_e4m3, int64_t M, int64_t N, int64_t K, const void* A, const void* B,
                             const float* bias, float* x32, const float* ln_g, const float* ln_b, void* out16,
                             void* out8, float out8_scale, float alpha, int pair, void* stream);

/* Multi-head self-attention over packed variable-length sequences.
 * qkv: [rows][3*d] (Q | K | V column blocks; head j owns columns j*64..j*64+63
 * of each), act type of `precision`; out: [rows][d] act type. Sequence s
 * covers rows seq_start[s] .. seq_start[s]+seq_len[s]-1 (int32, device);
 * tokens attend within their sequence only, scale 1/sqrt(64). Head dim 64,
 * seq_len <= 4096. */
as_status as_k_attention(int precision, const void* qkv, void* out, const int32_t* seq_start,
                         const int32_t* seq_len, int32_t n_seq, int64_t rows, int32_t d_model,
                         int32_t n_heads, void* stream);

/* The same attention (BF16) on the tcgen05 tensor cores: S = Q K^T and
 * O = P V in TMEM, softmax in four warps, Q, K and V read by TMA straight
 * from the qkv rows. Every sequence must lie inside [0, rows) (AS_ERR_ARG
 * otherwise; checked on the host, which reads seq_start / seq_len back). */
as_status as_k_attention_tc(const void* qkv, void* out, const int32_t* seq_start,
                            const int32_t* seq_len, int32_t n_seq, int64_t rows, int32_t d_model, int32_t n_heads,
                            void* stream);

/* The tcgen05 attention with E4M3 output, as the FP8 encoder uses it: out8
 * [rows][d] bytes, the E4M3 code (round to nearest even, saturating at +-448)
 * of each output value divided by out_scale (> 0; AS_ERR_ARG otherwise).
 * Rows outside every sequence are not written. Same inputs and checks as
 * as_k_attention_tc. */
as_status as_k_attention_tc_e4m3(const void* qkv, void* out8, float out_scale, const int32_t* seq_start,
                                 const int32_t* seq_len, int32_t n_seq, int64_t rows, int32_t d_model,
                                 int32_t n_heads, void* stream);

/* Row LayerNorm (biased variance, eps 1e-5): out_f32 = LN(in) * g + b, and
 * a BF16 copy in out_bf16 when it is not NULL. in/out_f32 may alias. */
as_status as_k_layernorm(const float* in, const float* g, const float* b, float* out_f32, void* out_bf16,
                         int64_t rows, int32_t d, void* stream);

/* Device count of kernel launches made by this library since load. */
uint64_t as_k_launch_count(void);
const char* as_k_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* ANONSHIELD_KERNELS_H */
