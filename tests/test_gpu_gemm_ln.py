"""Fused residual + LayerNorm GEMM (clustered tcgen05 kernel) against PyTorch.

x32 <- LN(x32 + alpha A.B^T + bias) with a row split over a cluster of CTAs:
compared with a plain FP32 PyTorch composition (matmul, add, layer_norm) and
with this library's two-kernel path (residual GEMM, then the LayerNorm
kernel), whose GEMM accumulates in the same order. Shapes span every
supported width (cluster of 1 to 4 CTAs, or 2 to 8 with 2-SM pairs along
M, whose results must equal the single-CTA tiles'), a single row, ragged row counts
and both projection depths (K = d and K = 4d); E4M3 operands too. The BF16
copy is the FP32 result rounded; the E4M3 copy that of value / scale.
"""
import pytest
import torch

import paper_2606_15650_b300.api as api

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _inputs(M, N, K, seed, e4m3=False):
    g = torch.Generator(device=DEV).manual_seed(seed)
    A = torch.randn(M, K, device=DEV, generator=g)
    B = torch.randn(N, K, device=DEV, generator=g) * (1.0 / K ** 0.5)
    if e4m3:
        A8 = A.clamp(-8, 8).to(torch.float8_e4m3fn)
        B8 = (B * 16).clamp(-8, 8).to(torch.float8_e4m3fn)
        A, B = A8, B8
    else:
        A, B = A.to(torch.bfloat16), B.to(torch.bfloat16)
    bias = torch.randn(N, device=DEV, generator=g) * 0.1
    x = torch.randn(M, N, device=DEV, generator=g)
    gam = 1.0 + 0.1 * torch.randn(N, device=DEV, generator=g)
    bet = 0.1 * torch.randn(N, device=DEV, generator=g)
    return A, B, bias, x, gam, bet


def _torch_ref(A, B, bias, x, gam, bet, alpha):
    y = alpha * (A.float() @ B.float().T) + bias + x
    return torch.nn.functional.layer_norm(y, (y.shape[1],), gam, bet, eps=1e-5)


@pytest.mark.parametrize("pair,deep", [(False, False), (True, False), (False, True), (True, True)])
@pytest.mark.parametrize("M,N,K", [(1, 768, 768), (200, 768, 3072), (4096, 768, 768), (300, 128, 512),
                                   (1000, 384, 384), (513, 512, 512), (777, 1024, 1024), (256, 256, 1024)])
def test_bf16_against_torch_and_two_kernels(M, N, K, pair, deep):
    A, B, bias, x, gam, bet = _inputs(M, N, K, seed=M + N + K)
    ref = _torch_ref(A, B, bias, x, gam, bet, 1.0)
    x_fused = x.clone()
    out16 = torch.empty(M, N, device=DEV, dtype=torch.bfloat16)
    api.gemm_resid_ln(A, B, bias, x_fused, gam, bet, out16=out16, pair=pair, deep=deep)
    torch.cuda.synchronize()
    err = (x_fused - ref).abs().max().item()
    assert err < 2e-3, err
    assert torch.equal(out16, x_fused.to(torch.bfloat16))
    if N not in (128, 256, 512, 768, 1024):
        return  # widths the row LayerNorm kernel takes
    # the two-kernel path: the same GEMM accumulation, LayerNorm by the row kernel
    y = torch.empty(M, N, device=DEV, dtype=torch.float32)
    api.gemm("bf16", "bias_resid", A, B, bias, x, y)
    two = torch.empty_like(y)
    api.layernorm(y, gam, bet, two)
    torch.cuda.synchronize()
    assert (x_fused - two).abs().max().item() < 2e-5


@pytest.mark.parametrize("pair,deep", [(False, False), (True, False), (False, True), (True, True)])
@pytest.mark.parametrize("M,N,K", [(1000, 768, 768), (130, 768, 3072), (64, 1024, 1024)])
def test_e4m3_operands_and_copy(M, N, K, pair, deep):
    A8, B8, bias, x, gam, bet = _inputs(M, N, K, seed=7 * M + N, e4m3=True)
    alpha = 1.0 / 16
    ref = _torch_ref(A8, B8, bias, x, gam, bet, alpha)
    x_fused = x.clone()
    out8 = torch.empty(M, N, device=DEV, dtype=torch.uint8)
    scale = 0.0625
    api.gemm_resid_ln(A8, B8, bias, x_fused, gam, bet, out8=out8, out8_scale=scale, alpha=alpha, pair=pair,
                      deep=deep)
    torch.cuda.synchronize()
    assert (x_fused - ref).abs().max().item() < 2e-3
    want = (x_fused / scale).clamp(-448, 448).to(torch.float8_e4m3fn).view(torch.uint8)
    assert torch.equal(out8, want)


def test_unsupported_width_is_refused():
    A, B, bias, x, gam, bet = _inputs(64, 640, 128, seed=1)
    with pytest.raises(api.AnonShieldError):
        api.gemm_resid_ln(A, B, bias, x, gam, bet)


@pytest.mark.parametrize("M,N,K", [(1, 768, 768), (1000, 768, 3072), (513, 128, 512), (777, 1024, 1024)])
def test_pairs_bit_identical(M, N, K):
    """2-SM pairs and the staging depth change which SM multiplies and when bytes
    move, not the accumulation order."""
    A, B, bias, x, gam, bet = _inputs(M, N, K, seed=3 * M + K)
    outs = []
    for pair in (False, True):
        for deep in (False, True):
            y = x.clone()
            api.gemm_resid_ln(A, B, bias, y, gam, bet, pair=pair, deep=deep)
            outs.append(y)
    torch.cuda.synchronize()
    assert all(torch.equal(outs[0], y) for y in outs[1:])
