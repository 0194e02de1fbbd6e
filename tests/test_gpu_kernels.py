"""Encoder kernels against plain PyTorch references of the same operation.

GEMM (tcgen05 BF16 and SIMT FP32) against torch matmul in FP32 on the same
(BF16-rounded) operands; attention against a per-sequence softmax(QK^T/8)V
in FP32; LayerNorm against torch.nn.functional.layer_norm. Shapes cover
several tiles, ragged M tails, both N tile widths and all epilogues.
"""
import math

import pytest
import torch

import paper_2606_15650_b300.api as api

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _ref_gemm(A, B, bias, resid, epi):
    y = A.float() @ B.float().T
    if bias is not None:
        y = y + bias
    if epi == "bias_gelu":
        y = torch.nn.functional.gelu(y, approximate="none")
    if epi == "bias_resid":
        y = y + resid
    return y


@pytest.mark.parametrize("M,N,K", [(1, 128, 64), (128, 256, 64), (200, 384, 128), (1000, 768, 768),
                                   (4096, 2304, 768), (777, 768, 3072), (300, 3072, 768), (129, 128, 512)])
@pytest.mark.parametrize("epi", ["bias", "bias_gelu", "bias_resid"])
def test_gemm_tcgen05_bf16(M, N, K, epi):
    g = torch.Generator(device=DEV).manual_seed(M * 7 + N + K)
    A = torch.randn(M, K, device=DEV, generator=g).to(torch.bfloat16)
    B = (0.05 * torch.randn(N, K, device=DEV, generator=g)).to(torch.bfloat16)
    bias = torch.randn(N, device=DEV, generator=g)
    resid = torch.randn(M, N, device=DEV, generator=g) if epi == "bias_resid" else None
    out = torch.empty(M, N, device=DEV, dtype=torch.float32 if epi == "bias_resid" else torch.bfloat16)
    api.gemm("bf16", epi, A, B, bias, resid, out, engine="tcgen05")
    torch.cuda.synchronize()
    ref = _ref_gemm(A, B, bias, resid, epi)
    tol = 2e-3 * math.sqrt(K) * 0.05 * 4 + (8e-3 * ref.abs() if out.dtype == torch.bfloat16 else 0)
    err = (out.float() - ref).abs()
    assert bool((err <= tol + 1e-4).all()), f"max err {err.max().item()} at {divmod(int(err.argmax()), N)}"


def _e4m3(x, scale):
    return (x / scale).clamp(-448, 448).to(torch.float8_e4m3fn)


@pytest.mark.parametrize("M,N,K", [(1, 128, 128), (128, 256, 128), (200, 384, 256), (1000, 768, 768),
                                   (4096, 2304, 768), (777, 768, 3072), (300, 3072, 768)])
@pytest.mark.parametrize("epi,out8", [("bias", False), ("bias_gelu", False), ("bias_gelu", True), ("bias_resid", False)])
def test_gemm_tcgen05_fp8(M, N, K, epi, out8):
    """E4M3 GEMM against FP32 matmul of the dequantized operands."""
    g = torch.Generator(device=DEV).manual_seed(M + 3 * N + K)
    A = torch.randn(M, K, device=DEV, generator=g)
    B = 0.05 * torch.randn(N, K, device=DEV, generator=g)
    sa, sb = A.abs().max().item() / 448, B.abs().max().item() / 448
    A8, B8 = _e4m3(A, sa), _e4m3(B, sb)
    bias = torch.randn(N, device=DEV, generator=g)
    resid = torch.randn(M, N, device=DEV, generator=g) if epi == "bias_resid" else None
    if out8:
        out = torch.empty(M, N, device=DEV, dtype=torch.float8_e4m3fn)
    else:
        out = torch.empty(M, N, device=DEV, dtype=torch.float32 if epi == "bias_resid" else torch.bfloat16)
    ref = _ref_gemm(A8.float() * sa, B8.float() * sb, bias, resid, epi)
    so = ref.abs().max().item() / 448 if out8 else 0.0
    api.gemm_fp8(epi, A8, B8, sa * sb, bias, resid, out, out_scale=so)
    torch.cuda.synchronize()
    if out8:
        got = out.float() * so
        exp = (ref / so).clamp(-448, 448).to(torch.float8_e4m3fn).float() * so
        # accumulation order (and the GELU approximation, |err| <= 1.5e-7) may move a value across an
        # E4M3 rounding boundary: at most one step, 2^-3 of the larger magnitude (or one subnormal step)
        step = torch.maximum(exp.abs(), got.abs()) * 0.125 + 2e-3 * so
        assert ((got - exp).abs() <= step).all()
        assert (got == exp).float().mean().item() > 0.99
    else:
        tol = 2e-3 * math.sqrt(K) * 0.05 * 4 + (8e-3 * ref.abs() if out.dtype == torch.bfloat16 else 0)
        err = (out.float() - ref).abs()
        assert bool((err <= tol + 1e-4).all()), f"max err {err.max().item()}"


@pytest.mark.parametrize("M,N,K", [(1, 128, 8), (130, 256, 64), (300, 384, 128), (517, 768, 768)])
@pytest.mark.parametrize("epi", ["bias", "bias_gelu", "bias_resid"])
def test_gemm_simt_fp32(M, N, K, epi):
    g = torch.Generator(device=DEV).manual_seed(M + N + K)
    A = torch.randn(M, K, device=DEV, generator=g)
    B = 0.05 * torch.randn(N, K, device=DEV, generator=g)
    bias = torch.randn(N, device=DEV, generator=g)
    resid = torch.randn(M, N, device=DEV, generator=g) if epi == "bias_resid" else None
    out = torch.empty(M, N, device=DEV)
    api.gemm("fp32", epi, A, B, bias, resid, out, engine="simt")
    torch.cuda.synchronize()
    ref = _ref_gemm(A.double(), B.double(), bias.double(), None if resid is None else resid.double(), epi)
    assert torch.allclose(out.double(), ref, atol=1e-4, rtol=1e-5)


def _ref_attention(qkv, starts, lens, d, h):
    out = torch.zeros(qkv.shape[0], d, device=qkv.device, dtype=torch.float32)
    for s, L in zip(starts.tolist(), lens.tolist()):
        x = qkv[s:s + L].float()
        q = x[:, :d].view(L, h, 64).transpose(0, 1)
        k = x[:, d:2 * d].view(L, h, 64).transpose(0, 1)
        v = x[:, 2 * d:].view(L, h, 64).transpose(0, 1)
        p = torch.softmax(q @ k.transpose(1, 2) / 8.0, dim=-1)
        out[s:s + L] = (p @ v).transpose(0, 1).reshape(L, d)
    return out


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
@pytest.mark.parametrize("d,h", [(128, 2), (768, 12)])
def test_attention(prec, d, h):
    g = torch.Generator(device="cpu").manual_seed(d)
    lens = torch.tensor([1, 5, 64, 65, 300, 512, 17, 128], dtype=torch.int32)
    starts = torch.zeros_like(lens)
    starts[1:] = torch.cumsum(lens, 0)[:-1]
    rows = int(lens.sum())
    dt = torch.bfloat16 if prec == "bf16" else torch.float32
    qkv = torch.randn(rows, 3 * d, generator=g).to(DEV).to(dt)
    out = torch.full((rows, d), float("nan"), device=DEV, dtype=dt)
    api.attention(prec, qkv, out, starts.to(DEV), lens.to(DEV), d, h)
    torch.cuda.synchronize()
    ref = _ref_attention(qkv, starts, lens, d, h)
    tol = 2.5e-2 if prec == "bf16" else 1e-5
    assert torch.isfinite(out.float()).all()
    assert (out.float() - ref).abs().max().item() < tol


@pytest.mark.parametrize("d,h", [(128, 2), (768, 12), (1024, 16)])
@pytest.mark.parametrize("lens", [[1, 5, 64, 65, 300, 512, 17, 128], [127, 128, 129, 255, 256, 257, 1000, 8, 2048],
                                  [63, 64, 65, 191, 192, 193, 33, 4096]])
@pytest.mark.parametrize("gap", [0, 3])
def test_attention_tcgen05(d, h, lens, gap):
    """tcgen05 attention against the per-sequence softmax reference; packed (gap 0) and
    with unused rows between sequences (gap 3: starts on any row)."""
    g = torch.Generator(device="cpu").manual_seed(d + len(lens) + gap)
    lens = torch.tensor(lens, dtype=torch.int32)
    starts = torch.zeros_like(lens)
    for i in range(1, len(lens)):
        starts[i] = int(starts[i - 1]) + int(lens[i - 1]) + gap * (i % 3)
    rows = int(starts[-1] + lens[-1]) + 5
    qkv = torch.randn(rows, 3 * d, generator=g).to(DEV).to(torch.bfloat16)
    out = torch.full((rows, d), float("nan"), device=DEV, dtype=torch.bfloat16)
    api.attention_tc(qkv, out, starts.to(DEV), lens.to(DEV), d, h)
    torch.cuda.synchronize()
    ref = _ref_attention(qkv, starts, lens, d, h)
    for s0, L in zip(starts.tolist(), lens.tolist()):
        got = out[s0:s0 + L].float()
        assert torch.isfinite(got).all()
        assert (got - ref[s0:s0 + L]).abs().max().item() < 2.5e-2
    # rows outside every sequence are not written
    written = torch.zeros(rows, dtype=torch.bool)
    for s0, L in zip(starts.tolist(), lens.tolist()):
        written[s0:s0 + L] = True
    assert torch.isnan(out[~written.to(DEV)].float()).all()


@pytest.mark.parametrize("engine", ["tcgen05", "mma_sync"])
@pytest.mark.parametrize("lens", [[300, 200, 57], [1, 2, 3, 130], [64, 65, 63]])
def test_attention_ignores_rows_outside_sequences(engine, lens):
    """Rows between and after the sequences hold NaN: keys past a sequence end (masked,
    P = 0) must contribute exactly nothing, whatever their V rows contain."""
    d, h, gap = 128, 2, 5
    g = torch.Generator(device="cpu").manual_seed(len(lens))
    starts, acc = [], 0
    for L in lens:
        starts.append(acc)
        acc += L + gap
    rows = acc - gap
    qkv = torch.full((rows + 256, 3 * d), float("nan"), dtype=torch.bfloat16)
    for s0, L in zip(starts, lens):
        qkv[s0:s0 + L] = torch.randn(L, 3 * d, generator=g).to(torch.bfloat16)
    qkv = qkv.to(DEV)
    out = torch.zeros(rows, d, device=DEV, dtype=torch.bfloat16)
    st = torch.tensor(starts, dtype=torch.int32)
    ln = torch.tensor(lens, dtype=torch.int32)
    if engine == "tcgen05":
        api.attention_tc(qkv[:rows], out, st.to(DEV), ln.to(DEV), d, h)
    else:
        api.attention("bf16", qkv[:rows], out, st.to(DEV), ln.to(DEV), d, h)
    torch.cuda.synchronize()
    ref = _ref_attention(qkv[:rows], st, ln, d, h)
    for s0, L in zip(starts, lens):
        got = out[s0:s0 + L].float()
        assert torch.isfinite(got).all()
        assert (got - ref[s0:s0 + L]).abs().max().item() < 2.5e-2


@pytest.mark.parametrize("lens", [[1, 5, 64, 65, 300, 512, 17, 128], [63, 64, 65, 191, 192, 193, 33, 1000]])
def test_attention_tcgen05_e4m3_output(lens):
    """E4M3 output of the tcgen05 attention (the FP8 encoder's form): each code is
    the value / out_scale rounded to E4M3, so the decoded value times out_scale
    is the attention within one E4M3 rounding (relative 2^-4) plus the BF16
    attention error. Rows between sequences keep their sentinel bytes."""
    d, h, gap = 768, 12, 3
    g = torch.Generator(device="cpu").manual_seed(len(lens) + 11)
    starts, acc = [], 0
    for L in lens:
        starts.append(acc)
        acc += L + gap
    rows = acc
    qkv = torch.randn(rows, 3 * d, generator=g).to(DEV).to(torch.bfloat16)
    out8 = torch.full((rows, d), 0x5A, device=DEV, dtype=torch.uint8)
    st = torch.tensor(starts, dtype=torch.int32)
    ln = torch.tensor(lens, dtype=torch.int32)
    scale = 0.02   # |value| / scale stays far below the E4M3 maximum of 448
    api.attention_tc_e4m3(qkv, out8, scale, st.to(DEV), ln.to(DEV), d, h)
    torch.cuda.synchronize()
    ref = _ref_attention(qkv, st, ln, d, h)
    got = out8.view(torch.float8_e4m3fn).float() * scale
    written = torch.zeros(rows, dtype=torch.bool, device=DEV)
    for s0, L in zip(starts, lens):
        written[s0:s0 + L] = True
        err = (got[s0:s0 + L] - ref[s0:s0 + L]).abs()
        assert torch.isfinite(got[s0:s0 + L]).all()
        # E4M3 rounding (half a spacing: 2^-4 relative) of a value within 2.5e-2 of ref
        assert (err <= ref[s0:s0 + L].abs() * 2.0 ** -4 + 3e-2).all(), err.max().item()
    assert (out8[~written] == 0x5A).all()
    with pytest.raises(api.AnonShieldError):
        api.attention_tc_e4m3(qkv, out8, 0.0, st.to(DEV), ln.to(DEV), d, h)


def test_attention_tcgen05_large_logits():
    """Scores far apart (raises of the running maximum by more than 2^8) stay exact."""
    d, h, L = 128, 2, 700
    g = torch.Generator(device="cpu").manual_seed(5)
    qkv = torch.randn(L, 3 * d, generator=g)
    qkv[:, :d] *= 6.0          # |S| up to several hundred: exp2 range far beyond 2^8
    qkv[:, d:2 * d] *= 6.0
    qkv = qkv.to(DEV).to(torch.bfloat16)
    out = torch.empty(L, d, device=DEV, dtype=torch.bfloat16)
    st = torch.tensor([0], dtype=torch.int32)
    ln = torch.tensor([L], dtype=torch.int32)
    api.attention_tc(qkv, out, st.to(DEV), ln.to(DEV), d, h)
    torch.cuda.synchronize()
    ref = _ref_attention(qkv, st, ln, d, h)
    assert (out.float() - ref).abs().max().item() < 5e-2


def test_attention_tcgen05_rejects_out_of_range():
    qkv = torch.zeros(64, 3 * 128, device=DEV, dtype=torch.bfloat16)
    out = torch.zeros(64, 128, device=DEV, dtype=torch.bfloat16)
    with pytest.raises(api.AnonShieldError):
        api.attention_tc(qkv, out, torch.tensor([0, 50], dtype=torch.int32, device=DEV),
                         torch.tensor([10, 20], dtype=torch.int32, device=DEV), 128, 2)


@pytest.mark.parametrize("d", [128, 768, 1024])
def test_layernorm(d):
    g = torch.Generator(device=DEV).manual_seed(d)
    x = 3 * torch.randn(1000, d, device=DEV, generator=g) + 1
    gam = 1 + 0.1 * torch.randn(d, device=DEV, generator=g)
    bet = 0.1 * torch.randn(d, device=DEV, generator=g)
    out = torch.empty_like(x)
    out16 = torch.empty(1000, d, device=DEV, dtype=torch.bfloat16)
    api.layernorm(x, gam, bet, out, out16)
    torch.cuda.synchronize()
    ref = torch.nn.functional.layer_norm(x.double(), (d,), gam.double(), bet.double(), eps=1e-5)
    assert (out.double() - ref).abs().max().item() < 2e-5
    assert torch.equal(out16, out.to(torch.bfloat16))


def test_attention_tcgen05_ragged_query_tiles_stress():
    """Many sequences whose last 128-query tile is mostly empty: softmax warps
    with no valid query row compute nothing but must keep the pipeline's
    barrier phases in step. Several persistent units per CTA and repeated
    launches give those warps every chance to run ahead. The result equals the
    mma.sync engine's (same BF16 inputs) within BF16 rounding of P, on every
    launch, and every launch completes (no bounded wait runs out)."""
    d, h = 768, 12
    g = torch.Generator(device="cpu").manual_seed(99)
    base = torch.tensor([129, 130, 140, 159, 257, 260, 288, 385, 390, 400, 1, 2, 31, 33], dtype=torch.int32)
    lens = base.repeat(120)[torch.randperm(14 * 120, generator=g)]
    starts = torch.zeros_like(lens)
    starts[1:] = torch.cumsum(lens, 0)[:-1]
    rows = int(lens.sum())
    qkv = torch.randn(rows, 3 * d, generator=g).to(DEV).to(torch.bfloat16)
    ref = torch.empty(rows, d, device=DEV, dtype=torch.bfloat16)
    api.attention("bf16", qkv, ref, starts.to(DEV), lens.to(DEV), d, h)
    for _ in range(5):
        out = torch.empty(rows, d, device=DEV, dtype=torch.bfloat16)
        api.attention_tc(qkv, out, starts.to(DEV), lens.to(DEV), d, h)
        torch.cuda.synchronize()
        assert torch.isfinite(out.float()).all()
        assert (out.float() - ref.float()).abs().max().item() < 2.5e-2
