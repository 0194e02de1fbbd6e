"""Pins for the oracle's reduced-precision arithmetic (oracle/lowp.py and the
rounding points of oracle/encoder.py).

The paper states no arithmetic precision for its GPU NER (§2 stage (2)); the
BF16 and FP8 E4M3 modes are readings of the workload specification. The
roundings are written in the oracle from the formats' definitions (frexp and
round-half-even on the spacing). They are checked here against things other
than themselves:

* the 256 E4M3 codes decoded from their bit layout agree with PyTorch's own
  float8_e4m3fn decoding, and the known landmarks (448, 2^-6, 2^-9, the two
  NaN codes) hold;
* every representable value rounds to itself, every midpoint between two
  neighbours rounds to the neighbour with the even code, and points just off
  a midpoint round to the nearer neighbour;
* a sweep of float32 values over the whole E4M3 range (saturation included)
  and the BF16 range agrees with PyTorch's dtype conversions;
* the encoder's rounding points: with both rounding functions replaced by the
  identity the reduced-precision encoder equals the FP64 one, and a one-token
  one-layer model (where attention is exactly V) computed by hand with
  PyTorch's float8 / bfloat16 conversions equals the oracle's FP8 and BF16
  logits.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import synth
from oracle import encoder as E
from oracle import lowp


# ---------------------------------------------------------------- formats

def test_e4m3_code_table_matches_torch():
    ours = lowp.e4m3_code_values()
    theirs = torch.arange(256, dtype=torch.int32).to(torch.uint8).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(np.isnan(ours), np.isnan(theirs))
    fin = ~np.isnan(ours)
    assert np.array_equal(ours[fin], theirs[fin])
    assert np.isnan(ours[0x7F]) and np.isnan(ours[0xFF]) and int(np.isnan(ours).sum()) == 2
    assert np.nanmax(ours) == 448.0 and ours[0x08] == 2.0 ** -6 and ours[0x01] == 2.0 ** -9


def _positive_e4m3():
    v = lowp.e4m3_code_values()[:0x7F]           # codes 0x00..0x7E: 0 and the positive finite values
    return v                                     # increasing with the code


def test_e4m3_fixed_points_and_ties_to_even():
    v = _positive_e4m3()
    assert np.all(np.diff(v) > 0)
    assert np.array_equal(lowp.round_e4m3(v), v) and np.array_equal(lowp.round_e4m3(-v), -v)
    lo, hi = v[:-1], v[1:]
    mid = (lo + hi) / 2
    even_is_lo = (np.arange(len(lo)) % 2) == 0    # code i even <=> mantissa LSB 0
    want = np.where(even_is_lo, lo, hi)
    assert np.array_equal(lowp.round_e4m3(mid), want)
    eps = (hi - lo) * 1e-6
    assert np.array_equal(lowp.round_e4m3(mid - eps), lo)
    assert np.array_equal(lowp.round_e4m3(mid + eps), hi)
    # saturation: everything beyond the largest finite value becomes +-448
    assert np.array_equal(lowp.round_e4m3(np.array([449.0, 500.0, 1e30, -1e30])), [448.0, 448.0, 448.0, -448.0])


def test_e4m3_sweep_matches_torch():
    rng = np.random.default_rng(7)
    x = np.concatenate([rng.standard_normal(200000) * 10.0 ** rng.uniform(-4, 2.8, 200000),
                        rng.uniform(-600, 600, 20000), [0.0, -0.0, 2.0 ** -10, 2.0 ** -9 * 1.5]]).astype(np.float32)
    t = torch.from_numpy(x).clamp(-448.0, 448.0).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(lowp.round_e4m3(x.astype(np.float64)), t)


def test_bf16_sweep_matches_torch_and_ties():
    rng = np.random.default_rng(8)
    x = (rng.standard_normal(300000) * 10.0 ** rng.uniform(-30, 30, 300000)).astype(np.float32)
    x = np.concatenate([x, np.array([1e-40, -3e-39, 0.0], np.float32)])   # subnormals
    t = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(lowp.round_bf16(x.astype(np.float64)), t)
    # ties between neighbours 2^-7 apart near 1 go to the even one
    assert lowp.round_bf16(np.array([1 + 2.0 ** -8]))[0] == 1.0
    assert lowp.round_bf16(np.array([1 + 3 * 2.0 ** -8]))[0] == 1 + 2.0 ** -6


def test_tensor_scale_maps_amax_to_448():
    x = np.array([0.3, -1.7, 0.02])
    s = lowp.tensor_scale(x)
    assert s == 1.7 / 448
    assert abs(lowp.quantize_e4m3(np.array([-1.7]), s)[0] + 1.7) < 1e-15
    assert lowp.tensor_scale(np.zeros(3)) == 1.0


# ---------------------------------------------------------------- encoder rounding points

def _tiny(n_layers=1, seed=5):
    d = synth.ModelDims(vocab=300, d_model=16, n_heads=2, d_ffn=32, n_layers=n_layers, n_labels=5, max_pos=8)
    return d, synth.make_weights(d, seed=seed, random_affine=True)


def test_identity_rounding_reduces_to_fp64(monkeypatch):
    d, w = _tiny(n_layers=2)
    ids = [3, 200, 7, 299, 42]
    ref = E.Encoder(d, w).logits(ids)
    monkeypatch.setattr(lowp, "round_bf16", lambda x: np.asarray(x, np.float64))
    monkeypatch.setattr(lowp, "round_e4m3", lambda x: np.asarray(x, np.float64))
    for prec in ("bf16", "fp8"):
        enc = E.Encoder(d, w, precision=prec, act_scales=[0.01 * (i + 1) for i in range(8)])
        assert np.allclose(enc.logits(ids), ref, rtol=0, atol=1e-12), prec


def _by_hand_one_token(d, w, tok, prec, scales):
    """One token, one layer: attention is exactly V. Rounding with torch's dtype conversions."""
    f64 = torch.float64

    def bf(x):
        return torch.as_tensor(x, dtype=f64).to(torch.float32).to(torch.bfloat16).to(f64)

    def f8(x, s):
        y = (torch.as_tensor(x, dtype=f64) / s).to(torch.float32).clamp(-448, 448)
        return y.to(torch.float8_e4m3fn).to(f64) * s

    def inp(x, slot):
        return bf(x) if prec == "bf16" else f8(x, scales[slot])

    def wt(name):
        W = torch.as_tensor(w[name], dtype=f64)
        return bf(W) if prec == "bf16" else f8(W, float(W.abs().max()) / 448.0)

    def ln(x, g, b):
        x = torch.as_tensor(x, dtype=f64)
        mu = x.mean()
        return (x - mu) / torch.sqrt(((x - mu) ** 2).mean() + 1e-5) * torch.as_tensor(g, dtype=f64) + \
            torch.as_tensor(b, dtype=f64)

    T = lambda k: torch.as_tensor(w[k], dtype=f64)
    m = d.d_model
    x = ln(T("tok_emb")[tok] + T("pos_emb")[0], w["emb_ln_g"], w["emb_ln_b"])
    qkv = bf(inp(x, 0) @ wt("l0.w_qkv").T + T("l0.b_qkv"))
    a = qkv[2 * m:]                                      # softmax over one key = 1; bf16(1) = 1
    x = ln(x + inp(a, 1) @ wt("l0.w_o").T + T("l0.b_o"), w["l0.ln1_g"], w["l0.ln1_b"])
    h = inp(x, 2) @ wt("l0.w_1").T + T("l0.b_1")
    h = 0.5 * h * (1 + torch.erf(h / np.sqrt(2.0)))
    x = ln(x + inp(h, 3) @ wt("l0.w_2").T + T("l0.b_2"), w["l0.ln2_g"], w["l0.ln2_b"])
    return (x @ T("cls_w").T + T("cls_b")).numpy()


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_one_token_layer_by_hand(prec):
    d, w = _tiny(n_layers=1)
    scales = [0.013, 0.011, 0.017, 0.007]
    for tok in (1, 77, 299):
        enc = E.Encoder(d, w, precision=prec, act_scales=scales)
        got = enc.logits([tok])[0]
        want = _by_hand_one_token(d, w, tok, prec, scales)
        assert np.allclose(got, want, rtol=0, atol=1e-12), (prec, tok, got - want)


def test_calibrate_is_amax_over_448():
    d, w = _tiny(n_layers=1)
    seqs = [[5, 6, 7], [250]]
    sc = E.calibrate(E.Encoder(d, w), seqs)
    # the QKV input of layer 0 is the embedding LayerNorm: its amax is computable directly
    x = np.concatenate([E.layer_norm(np.asarray(w["tok_emb"], np.float64)[s] +
                                     np.asarray(w["pos_emb"], np.float64)[:len(s)], w["emb_ln_g"], w["emb_ln_b"])
                        for s in seqs])
    assert sc[0] == pytest.approx(np.abs(x).max() / 448.0, rel=1e-15)
    assert len(sc) == 4 and all(s > 0 for s in sc)


def test_reduced_precision_error_ordering_c1():
    """Sanity on the c1 model: BF16 rounding moves the logits a little, E4M3 more."""
    dims = synth.C1.dims
    w = synth.make_weights(dims, seed=9, random_affine=True)
    rng = np.random.default_rng(3)
    seqs = [rng.integers(1, dims.vocab, size=n).tolist() for n in (40, 90, 7)]
    ref = [E.Encoder(dims, w).logits(s) for s in seqs]
    sc = E.calibrate(E.Encoder(dims, w), seqs)
    eb = max(np.abs(E.Encoder(dims, w, "bf16").logits(s) - r).max() for s, r in zip(seqs, ref))
    e8 = max(np.abs(E.Encoder(dims, w, "fp8", sc).logits(s) - r).max() for s, r in zip(seqs, ref))
    assert 0 < eb < 2e-2 and eb < e8 < 1e-1
