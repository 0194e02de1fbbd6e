"""Thin Python binding of the C ABI (include/anonshield.h, anonshield_kernels.h).

Argument marshalling only: every step of the pseudonymization path runs in
the CUDA library. PyTorch tensors may be passed wherever the C ABI takes a
device pointer (their data_ptr() is used); nothing here computes any part of
the method. If the compiled library is missing, importing fails loudly.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libanonshield.so")

AS_OK = 0
STATUS = {0: "AS_OK", -1: "AS_ERR_ARG", -2: "AS_ERR_OOM", -3: "AS_ERR_CUDA", -4: "AS_ERR_TOO_LONG",
          -5: "AS_ERR_TIMEOUT", -6: "AS_ERR_STATE", -7: "AS_ERR_UNSUPPORTED", -8: "AS_ERR_CAPACITY",
          -9: "AS_ERR_AGAIN"}
PRECISION = {"fp32": 0, "bf16": 1, "fp8": 2}
MODE = {"packed": 0, "per_record": 1}
EPI = {"bias": 0, "bias_gelu": 1, "bias_resid": 2}
ENGINE = {"auto": 0, "tcgen05": 1, "simt": 2}
ATTENTION = {"tcgen05": 0, "mma_sync": 1}
RX_KIND = {"mac": 0, "ipv6": 1, "ipv4": 2, "cve": 3, "hostname": 4, "url": 5, "hash": 6, "uuid": 7, "cpe": 8,
           "oid": 9, "cert_fp": 10, "pem": 11}
RX_KINDS = 12


def recognizer_table(types: dict[str, int]) -> tuple[int, ...]:
    """Kind -> entity type table for Schema.recognizers from {kind name: type} (others off)."""
    t = [0] * RX_KINDS
    for k, v in types.items():
        t[RX_KIND[k]] = v
    return tuple(t)


class AnonShieldError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Config(C.Structure):
    _fields_ = [("vocab", C.c_uint32), ("d_model", C.c_uint32), ("n_heads", C.c_uint32), ("d_ffn", C.c_uint32),
                ("n_layers", C.c_uint32), ("n_labels", C.c_uint32), ("max_pos", C.c_uint32),
                ("precision", C.c_uint32), ("mode", C.c_uint32),
                ("weights", C.POINTER(C.c_float)), ("weights_len", C.c_uint64),
                ("vocab_bytes", C.POINTER(C.c_uint8)), ("vocab_offsets", C.POINTER(C.c_uint32)),
                ("n_vocab_words", C.c_uint32), ("max_chunk_tokens", C.c_uint64), ("map_capacity", C.c_uint64),
                ("map_arena_bytes", C.c_uint64), ("device", C.c_int32), ("keep_trace", C.c_uint32),
                ("no_graphs", C.c_uint32), ("attention", C.c_uint32), ("no_fused_ln", C.c_uint32)]


class _Records(C.Structure):
    _fields_ = [("bytes", C.c_void_p), ("offsets", C.c_void_p), ("n_records", C.c_uint64), ("on_device", C.c_uint32)]


class _Schema(C.Structure):
    _fields_ = [("n_types", C.c_uint32), ("type_names", C.POINTER(C.c_char_p)), ("preserve_mask", C.c_uint64),
                ("slug_hex_len", C.c_uint32), ("window", C.c_uint32), ("stride", C.c_uint32),
                ("recognizer_types", C.POINTER(C.c_uint8))]


class _JsonlPolicy(C.Structure):
    _fields_ = [("n_keys", C.c_uint32), ("key_names", C.POINTER(C.c_char_p)), ("action", C.POINTER(C.c_uint8)),
                ("force_type", C.POINTER(C.c_uint8)), ("default_action", C.c_uint8)]


class _Entity(C.Structure):
    _fields_ = [("type", C.c_uint32), ("original_len", C.c_uint32), ("original", C.POINTER(C.c_uint8)),
                ("full_hash", C.c_char * 65), ("slug", C.c_char * 65),
                ("first_seen", C.c_uint64), ("last_seen", C.c_uint64), ("count", C.c_uint64)]


class _Stats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("n_records", "n_bytes", "n_tokens", "n_encoded_tokens", "n_sequences",
                                          "n_regex_spans", "n_ner_spans", "n_final_spans", "n_out_bytes",
                                          "n_map_entries", "n_new_entries", "kernel_launches",
                                          "graph_replays", "n_pseudonyms", "n_reidentified", "n_ambiguous",
                                          "n_unverified", "n_fields", "n_malformed")]


class _Trace(C.Structure):
    _fields_ = [("n_records", C.c_uint64), ("n_tokens", C.c_uint64), ("n_regex", C.c_uint64), ("n_final", C.c_uint64),
                ("rec_tok", C.POINTER(C.c_uint64)), ("tok_ids", C.POINTER(C.c_int32)),
                ("tok_off", C.POINTER(C.c_uint32)), ("tok_len", C.POINTER(C.c_uint32)),
                ("regex_start", C.POINTER(C.c_uint32)), ("regex_len", C.POINTER(C.c_uint32)),
                ("regex_type", C.POINTER(C.c_uint8)), ("logits", C.POINTER(C.c_float)),
                ("labels", C.POINTER(C.c_uint8)), ("final_start", C.POINTER(C.c_uint32)),
                ("final_len", C.POINTER(C.c_uint32)), ("final_type", C.POINTER(C.c_uint8))]


class _ServeConfig(C.Structure):
    _fields_ = [("lanes", C.c_uint32), ("max_batch_bytes", C.c_uint64), ("max_batch_records", C.c_uint32),
                ("max_pending", C.c_uint64), ("activation_budget_bytes", C.c_uint64)]


class _ServeStats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("completed", "rejected", "failed", "batches", "tokens", "pending")] + \
               [(n, C.c_double) for n in ("seconds", "p50_ms", "p99_ms", "max_ms")] + \
               [(n, C.c_uint64) for n in ("activation_budget", "row_cap", "activation_bytes", "activation_peak")]


class _Fields(C.Structure):
    _fields_ = [("start", C.c_void_p), ("len", C.c_void_p), ("id", C.c_void_p), ("n_fields", C.c_uint64)]


class _FieldPolicy(C.Structure):
    _fields_ = [("n_ids", C.c_uint32), ("action", C.c_void_p), ("force_type", C.c_void_p),
                ("default_action", C.c_uint8)]


FIELD_ACTION = {"detect": 0, "exclude": 1, "force": 2}


class _StreamConfig(C.Structure):
    _fields_ = [("batch_bytes", C.c_uint64), ("lanes", C.c_uint32)]


class _TuneEntry(C.Structure):
    _fields_ = [("role", C.c_uint32), ("m", C.c_uint64), ("n", C.c_uint64), ("k", C.c_uint64),
                ("chosen", C.c_int32), ("ms", C.c_float * 8)]


TUNE_ROLES = ("qkv", "attn_out", "ffn1", "ffn2")


class _Profile(C.Structure):
    _fields_ = [("gemm_launches", C.c_uint64), ("gemm_ms", C.c_double), ("gemm_flops", C.c_double),
                ("attn_launches", C.c_uint64), ("attn_ms", C.c_double), ("attn_flops", C.c_double),
                ("stage_calls", C.c_uint64), ("stage_ms", C.c_double * 4)]

# order of _Profile.stage_ms (as_profile_stats.stage_ms)
PROFILE_STAGES = ("text", "spans", "hash_map", "substitution")


EXPORTED = ["as_create", "as_destroy", "as_anonymize", "as_output_records", "as_output_stats", "as_output_map",
            "as_output_free", "as_map_export", "as_map_import", "as_map_merge", "as_map_clear", "as_debug_trace", "as_last_error",
            "as_free", "as_version", "as_get_stream", "as_profile", "as_profile_read", "as_tokenize_static", "as_calibrate",
            "as_get_scales", "as_set_scales", "as_anonymize_stream", "as_anonymize_fields", "as_anonymize_jsonl", "as_reidentify", "as_autotune", "as_set_tiles", "as_get_tiles", "as_serve_start", "as_submit", "as_poll", "as_serve_stats",
            "as_serve_stop", "as_k_gemm", "as_k_gemm_fp8", "as_k_attention", "as_k_attention_tc", "as_k_attention_tc_e4m3", "as_k_layernorm", "as_k_launch_count",
            "as_k_last_error"]

_lib = None


def load() -> C.CDLL:
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                          "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(LIB_PATH)
    P = C.c_void_p
    lib.as_create.argtypes = [C.POINTER(_Config), C.POINTER(P)]
    lib.as_destroy.argtypes = [P]
    lib.as_destroy.restype = None
    lib.as_anonymize.argtypes = [P, C.POINTER(_Records), C.POINTER(_Schema), C.c_char_p, C.c_size_t, C.POINTER(P)]
    lib.as_output_records.argtypes = [P, C.POINTER(P), C.POINTER(P), C.POINTER(C.c_uint64), C.POINTER(C.c_uint32)]
    lib.as_output_stats.argtypes = [P, C.POINTER(_Stats)]
    lib.as_output_map.argtypes = [P, C.POINTER(C.POINTER(_Entity)), C.POINTER(C.c_uint64)]
    lib.as_output_free.argtypes = [P]
    lib.as_output_free.restype = None
    lib.as_map_export.argtypes = [P, C.POINTER(C.POINTER(_Entity)), C.POINTER(C.c_uint64)]
    lib.as_map_import.argtypes = [P, C.c_char_p, C.c_size_t, C.POINTER(_Entity), C.c_uint64]
    lib.as_map_merge.argtypes = [C.POINTER(C.POINTER(_Entity)), C.POINTER(C.c_uint64), C.POINTER(C.c_uint64),
                                 C.c_uint32, C.POINTER(C.POINTER(_Entity)), C.POINTER(C.c_uint64)]
    lib.as_map_clear.argtypes = [P]
    lib.as_debug_trace.argtypes = [P, C.POINTER(_Trace)]
    lib.as_last_error.argtypes = [P]
    lib.as_last_error.restype = C.c_char_p
    lib.as_free.argtypes = [P]
    lib.as_free.restype = None
    lib.as_version.restype = C.c_char_p
    lib.as_get_stream.argtypes = [P, C.POINTER(P)]
    lib.as_calibrate.argtypes = [P, C.POINTER(_Records), C.POINTER(_Schema)]
    lib.as_get_scales.argtypes = [P, P, C.c_uint64]
    lib.as_set_scales.argtypes = [P, P, C.c_uint64]
    lib.as_autotune.argtypes = [P, C.c_uint64, C.POINTER(_TuneEntry)]
    lib.as_set_tiles.argtypes = [P, C.POINTER(C.c_int32)]
    lib.as_get_tiles.argtypes = [P, C.POINTER(C.c_int32)]
    lib.as_anonymize_fields.argtypes = [P, C.POINTER(_Records), C.POINTER(_Fields), C.POINTER(_FieldPolicy),
                                        C.POINTER(_Schema), C.c_char_p, C.c_size_t, C.POINTER(P)]
    lib.as_reidentify.argtypes = [P, C.POINTER(_Records), C.POINTER(_Schema), C.c_char_p, C.c_size_t, C.POINTER(P)]
    lib.as_anonymize_jsonl.argtypes = [P, C.POINTER(_Records), C.POINTER(_JsonlPolicy), C.POINTER(_Schema), C.c_char_p,
                                       C.c_size_t, C.POINTER(P)]
    lib.as_anonymize_stream.argtypes = [P, C.POINTER(_Records), C.POINTER(_Schema), C.c_char_p, C.c_size_t,
                                        C.POINTER(_StreamConfig), C.POINTER(P)]
    lib.as_serve_start.argtypes = [P, C.POINTER(_Schema), C.c_char_p, C.c_size_t, C.POINTER(_ServeConfig)]
    lib.as_submit.argtypes = [P, P, C.c_uint64, C.c_uint32, C.POINTER(C.c_uint64)]
    lib.as_poll.argtypes = [P, C.c_uint64, C.POINTER(P), C.c_int64]
    lib.as_serve_stats.argtypes = [P, C.POINTER(_ServeStats), C.c_uint32]
    lib.as_serve_stop.argtypes = [P]
    lib.as_profile.argtypes = [P, C.c_uint32]
    lib.as_profile_read.argtypes = [P, C.POINTER(_Profile)]
    lib.as_tokenize_static.argtypes = [P, P, P, C.c_uint64, C.c_uint64, P, P, P, P, P, P]
    lib.as_k_gemm.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int64, C.c_int64, C.c_int64, P, P, P, P, P, P]
    lib.as_k_gemm_fp8.argtypes = [C.c_int, C.c_int, C.c_int64, C.c_int64, C.c_int64, P, P, C.c_float, C.c_float,
                                  P, P, P, P]
    lib.as_k_gemm_resid_ln.argtypes = [C.c_int, C.c_int64, C.c_int64, C.c_int64, P, P, P, P, P, P, P, P, C.c_float,
                                       C.c_float, C.c_int, P]
    lib.as_k_attention.argtypes = [C.c_int, P, P, P, P, C.c_int32, C.c_int64, C.c_int32, C.c_int32, P]
    lib.as_k_attention_tc.argtypes = [P, P, P, P, C.c_int32, C.c_int64, C.c_int32, C.c_int32, P]
    lib.as_k_attention_tc_e4m3.argtypes = [P, P, C.c_float, P, P, C.c_int32, C.c_int64, C.c_int32, C.c_int32, P]
    lib.as_k_layernorm.argtypes = [P, P, P, P, P, C.c_int64, C.c_int32, P]
    lib.as_k_launch_count.restype = C.c_uint64
    lib.as_k_last_error.restype = C.c_char_p
    _lib = lib
    return lib


def _ptr(x) -> int | None:
    """Device pointer of a torch tensor, or None."""
    if x is None:
        return None
    return x.data_ptr()


_rt = None


def _cudart():
    """The CUDA runtime the library links (for plain device-to-host copies)."""
    global _rt
    if _rt is None:
        _rt = C.CDLL("libcudart.so.13")
    return _rt


def _check_rt(err: int):
    if err != 0:
        raise AnonShieldError(-3, f"cudaMemcpy failed with error {err}")


def _check_k(status: int):
    if status != AS_OK:
        raise AnonShieldError(status, (load().as_k_last_error() or b"").decode())


# ------------------------------------------------------------ kernel level

def gemm(precision: str, epilogue: str, A, B, bias=None, resid=None, out=None, engine: str = "auto", stream=None):
    """out = epi(A @ B^T) on device tensors (A [M,K], B [N,K]); returns out."""
    M, K = A.shape
    N = B.shape[0]
    _check_k(load().as_k_gemm(PRECISION[precision], ENGINE[engine], EPI[epilogue], M, N, K, _ptr(A), _ptr(B),
                              _ptr(bias), _ptr(resid), _ptr(out), stream))
    return out


def gemm_fp8(epilogue: str, A8, B8, alpha: float, bias=None, resid=None, out=None, out_scale: float = 0.0,
             stream=None):
    """out = epi(alpha * A8 @ B8^T) with E4M3 operands (torch.float8_e4m3fn or uint8 tensors)."""
    M, K = A8.shape
    N = B8.shape[0]
    out_e4m3 = 1 if out_scale > 0 else 0
    _check_k(load().as_k_gemm_fp8(EPI[epilogue], out_e4m3, M, N, K, _ptr(A8), _ptr(B8), alpha, out_scale or 1.0,
                                  _ptr(bias), _ptr(resid), _ptr(out), stream))
    return out


def gemm_resid_ln(A, B, bias, x32, ln_g, ln_b, out16=None, out8=None, out8_scale: float = 1.0, alpha: float = 1.0,
                  pair: bool = False, deep: bool = False, stream=None):
    """x32 <- LayerNorm(x32 + alpha * A @ B^T + bias) in place (BF16 or E4M3 operands), plus copies."""
    M, K = A.shape
    N = B.shape[0]
    in8 = 1 if A.element_size() == 1 else 0
    _check_k(load().as_k_gemm_resid_ln(in8, M, N, K, _ptr(A), _ptr(B), _ptr(bias), _ptr(x32), _ptr(ln_g),
                                       _ptr(ln_b), _ptr(out16), _ptr(out8), out8_scale, alpha,
                                       (1 if pair else 0) | (2 if deep else 0), stream))
    return x32


def attention(precision: str, qkv, out, seq_start, seq_len, d_model: int, n_heads: int, stream=None):
    _check_k(load().as_k_attention(PRECISION[precision], _ptr(qkv), _ptr(out), _ptr(seq_start), _ptr(seq_len),
                                   int(seq_len.numel()), int(qkv.shape[0]), d_model, n_heads, stream))
    return out


def attention_tc(qkv, out, seq_start, seq_len, d_model: int, n_heads: int, stream=None):
    """tcgen05 attention (BF16) over packed sequences."""
    _check_k(load().as_k_attention_tc(_ptr(qkv), _ptr(out), _ptr(seq_start), _ptr(seq_len),
                                      int(seq_len.numel()), int(qkv.shape[0]), d_model, n_heads, stream))
    return out


def attention_tc_e4m3(qkv, out8, out_scale: float, seq_start, seq_len, d_model: int, n_heads: int, stream=None):
    """tcgen05 attention with E4M3 output (codes of value / out_scale) over packed sequences."""
    _check_k(load().as_k_attention_tc_e4m3(_ptr(qkv), _ptr(out8), float(out_scale), _ptr(seq_start), _ptr(seq_len),
                                           int(seq_len.numel()), int(qkv.shape[0]), d_model, n_heads, stream))
    return out8


def layernorm(x, g, b, out_f32, out_bf16=None, stream=None):
    rows, d = x.shape
    _check_k(load().as_k_layernorm(_ptr(x), _ptr(g), _ptr(b), _ptr(out_f32), _ptr(out_bf16), rows, d, stream))
    return out_f32


def launch_count() -> int:
    return int(load().as_k_launch_count())


# ------------------------------------------------------------ batch API

@dataclass
class Schema:
    type_names: tuple[str, ...]
    preserve_mask: int = 0
    slug_hex_len: int = 10
    window: int = 0
    stride: int = 0
    # entity type per recognizer kind (RX_KIND order, 0 = off); None = the
    # five address/CVE recognizers to types 1..4 (see recognizer_table)
    recognizers: tuple[int, ...] | None = None


@dataclass
class Entity:
    type: int
    original: bytes
    full_hash: str
    slug: str
    first_seen: int
    last_seen: int
    count: int


def _entities(ptr, n) -> list[Entity]:
    out = []
    for i in range(n):
        e = ptr[i]
        out.append(Entity(int(e.type), C.string_at(e.original, e.original_len) if e.original_len else b"",
                          e.full_hash.decode(), e.slug.decode(), int(e.first_seen), int(e.last_seen), int(e.count)))
    return out


def _entity_array(entries: list[Entity]):
    """ctypes array of as_entity for `entries` (plus the buffers it points into)."""
    arr = (_Entity * max(len(entries), 1))()
    bufs = []
    for i, e in enumerate(entries):
        b = (C.c_uint8 * max(len(e.original), 1)).from_buffer_copy(e.original + b"\0")
        bufs.append(b)
        arr[i].type = e.type
        arr[i].original_len = len(e.original)
        arr[i].original = C.cast(b, C.POINTER(C.c_uint8))
        arr[i].full_hash = e.full_hash.encode()
        arr[i].slug = e.slug.encode()
        arr[i].first_seen = e.first_seen
        arr[i].last_seen = e.last_seen
        arr[i].count = e.count
    return arr, bufs


def map_merge(shards: list[list[Entity]], record_offsets: list[int] | None = None) -> list[Entity]:
    """Host-side union of replica maps (as_map_merge); runs without a GPU."""
    lib = load()
    arrs = [_entity_array(s) for s in shards]
    ptrs = (C.POINTER(_Entity) * max(len(shards), 1))(*[C.cast(a, C.POINTER(_Entity)) for a, _ in arrs])
    ns = (C.c_uint64 * max(len(shards), 1))(*[len(s) for s in shards])
    offs = (C.c_uint64 * max(len(shards), 1))(*(record_offsets or [0] * len(shards)))
    p, n = C.POINTER(_Entity)(), C.c_uint64()
    st = lib.as_map_merge(ptrs, ns, offs, len(shards), C.byref(p), C.byref(n))
    if st != AS_OK:
        raise AnonShieldError(st, (lib.as_last_error(None) or b"").decode())
    try:
        return _entities(p, n.value)
    finally:
        lib.as_free(C.cast(p, C.c_void_p))


class Output:
    """Result of one anonymize call (owns the library's as_output)."""

    def __init__(self, ctx: "Context", handle: int):
        self._ctx = ctx
        self._h = C.c_void_p(handle)

    def _records(self):
        b, o, n, dev = C.c_void_p(), C.c_void_p(), C.c_uint64(), C.c_uint32()
        st = load().as_output_records(self._h, C.byref(b), C.byref(o), C.byref(n), C.byref(dev))
        self._ctx._check(st)
        return b.value, o.value, n.value, dev.value

    def arrays(self) -> tuple[np.ndarray, np.ndarray]:
        """(bytes uint8, offsets uint64) on the host (copied from the device if needed)."""
        b, o, n, dev = self._records()
        if dev:
            raise ValueError("output lives on the device: use device_pointers()")
        offs = np.ctypeslib.as_array(C.cast(o, C.POINTER(C.c_uint64)), shape=(n + 1,)).copy()
        size = int(offs[-1])
        if size == 0 or not b:
            return np.zeros(0, np.uint8), offs
        data = np.ctypeslib.as_array(C.cast(b, C.POINTER(C.c_uint8)), shape=(size,)).copy()
        return data, offs

    def device_pointers(self) -> tuple[int, int, int]:
        b, o, n, dev = self._records()
        if not dev:
            raise ValueError("output lives on the host")
        return b, o, n

    def copy_to_host(self) -> list[bytes]:
        """Records of a device-resident output, copied to the host (cudaMemcpy)."""
        b, o, n = self.device_pointers()
        rt = _cudart()
        offs = np.empty(n + 1, np.uint64)
        _check_rt(rt.cudaMemcpy(C.c_void_p(offs.ctypes.data), C.c_void_p(o), C.c_size_t((n + 1) * 8), 2))
        size = int(offs[-1])
        data = np.empty(max(size, 1), np.uint8)
        if size:
            _check_rt(rt.cudaMemcpy(C.c_void_p(data.ctypes.data), C.c_void_p(b), C.c_size_t(size), 2))
        return [data[offs[i]:offs[i + 1]].tobytes() for i in range(n)]

    def records(self) -> list[bytes]:
        data, offs = self.arrays()
        return [data[offs[i]:offs[i + 1]].tobytes() for i in range(len(offs) - 1)]

    def stats(self) -> dict:
        s = _Stats()
        self._ctx._check(load().as_output_stats(self._h, C.byref(s)))
        return {k: int(getattr(s, k)) for k, _ in _Stats._fields_}

    def map(self) -> list[Entity]:
        if getattr(self._ctx, "_h", None) is None:
            raise AnonShieldError(-6, "the output's context is closed: its map cannot be read")
        p, n = C.POINTER(_Entity)(), C.c_uint64()
        self._ctx._check(load().as_output_map(self._h, C.byref(p), C.byref(n)))
        return _entities(p, n.value)

    def free(self):
        if self._h:
            load().as_output_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Context:
    """One as_ctx: model weights, vocabulary and entity map on one GPU."""

    def __init__(self, dims, weights_blob: np.ndarray, vocab_words: list[bytes], precision: str = "bf16",
                 mode: str = "packed", max_chunk_tokens: int = 0, map_capacity: int = 0, map_arena_bytes: int = 0,
                 keep_trace: bool = False, device: int = 0, attention: str = "tcgen05", graphs: bool = True,
                 fused_ln: bool | str = True):
        """fused_ln: True (both post-LN blocks as one kernel each), False, "attn" or "ffn" (that block only)."""
        lib = load()
        self.dims = dims
        self.device = device
        self._w = np.ascontiguousarray(weights_blob, dtype=np.float32)
        vb = b"".join(vocab_words)
        self._vb = np.frombuffer(vb, dtype=np.uint8).copy() if vb else np.zeros(1, np.uint8)
        offs = np.zeros(len(vocab_words) + 1, dtype=np.uint32)
        offs[1:] = np.cumsum([len(w) for w in vocab_words])
        self._vo = offs
        cfg = _Config(vocab=dims.vocab, d_model=dims.d_model, n_heads=dims.n_heads, d_ffn=dims.d_ffn,
                      n_layers=dims.n_layers, n_labels=dims.n_labels, max_pos=dims.max_pos,
                      precision=PRECISION[precision], mode=MODE[mode],
                      weights=self._w.ctypes.data_as(C.POINTER(C.c_float)), weights_len=self._w.size,
                      vocab_bytes=self._vb.ctypes.data_as(C.POINTER(C.c_uint8)),
                      vocab_offsets=self._vo.ctypes.data_as(C.POINTER(C.c_uint32)),
                      n_vocab_words=len(vocab_words), max_chunk_tokens=max_chunk_tokens,
                      map_capacity=map_capacity, map_arena_bytes=map_arena_bytes, device=device,
                      keep_trace=1 if keep_trace else 0, no_graphs=0 if graphs else 1,
                      attention=ATTENTION[attention],
                      no_fused_ln={True: 0, False: 3, "attn": 2, "ffn": 1}[fused_ln])
        h = C.c_void_p()
        st = lib.as_create(C.byref(cfg), C.byref(h))
        if st != AS_OK:
            raise AnonShieldError(st, (lib.as_k_last_error() or b"").decode())
        self._h = h
        self.precision = precision

    def _check(self, st: int):
        if st != AS_OK:
            raise AnonShieldError(st, (load().as_last_error(self._h) or b"").decode())

    @staticmethod
    def _schema(s: Schema):
        names = (C.c_char_p * len(s.type_names))(*[n.encode() for n in s.type_names])
        sc = _Schema(n_types=len(s.type_names), type_names=names, preserve_mask=s.preserve_mask,
                     slug_hex_len=s.slug_hex_len, window=s.window, stride=s.stride)
        if s.recognizers is not None:
            if len(s.recognizers) != RX_KINDS:
                raise ValueError(f"recognizers needs {RX_KINDS} entries (one per recognizer kind)")
            table = (C.c_uint8 * RX_KINDS)(*s.recognizers)
            sc.recognizer_types = C.cast(table, C.POINTER(C.c_uint8))
            return sc, (names, table)
        return sc, names

    def anonymize(self, data, offsets, schema: Schema, key: bytes) -> Output:
        """data/offsets: numpy (host) or torch CUDA tensors (device, read in place)."""
        on_dev = hasattr(data, "is_cuda") and data.is_cuda
        if on_dev:
            rec = _Records(bytes=data.data_ptr(), offsets=offsets.data_ptr(), n_records=offsets.numel() - 1,
                           on_device=1)
            keep = (data, offsets)
        else:
            d = np.ascontiguousarray(data, dtype=np.uint8)
            o = np.ascontiguousarray(offsets, dtype=np.uint64)
            rec = _Records(bytes=d.ctypes.data if d.size else None, offsets=o.ctypes.data, n_records=o.size - 1,
                           on_device=0)
            keep = (d, o)
        sc, names = self._schema(schema)
        out = C.c_void_p()
        st = load().as_anonymize(self._h, C.byref(rec), C.byref(sc), key, len(key), C.byref(out))
        del keep, names
        self._check(st)
        return Output(self, out.value)

    @staticmethod
    def _records(data, offsets):
        """(as_records, objects to keep alive) for numpy host arrays or torch CUDA tensors."""
        if hasattr(data, "is_cuda") and data.is_cuda:
            rec = _Records(bytes=data.data_ptr(), offsets=offsets.data_ptr(), n_records=offsets.numel() - 1,
                           on_device=1)
            return rec, (data, offsets)
        d = np.ascontiguousarray(data, dtype=np.uint8)
        o = np.ascontiguousarray(offsets, dtype=np.uint64)
        rec = _Records(bytes=d.ctypes.data if d.size else None, offsets=o.ctypes.data, n_records=o.size - 1,
                       on_device=0)
        return rec, (d, o)

    def anonymize_jsonl(self, data, offsets, key_names, policy: dict, schema: Schema, key: bytes,
                        default: str = "detect") -> Output:
        """JSON Lines (as_anonymize_jsonl): one JSON line per record. policy maps a key name
        to "detect", "exclude" or ("force", entity_type); other keys take ``default``."""
        rec, keep = self._records(data, offsets)
        names = [k.encode() if isinstance(k, str) else bytes(k) for k in key_names]
        nk = len(names)
        acts = np.zeros(max(nk, 1), np.uint8)
        ftyp = np.zeros(max(nk, 1), np.uint8)
        for i, k in enumerate(key_names):
            a = policy.get(k, default)
            if isinstance(a, tuple):
                acts[i], ftyp[i] = FIELD_ACTION[a[0]], a[1]
            else:
                acts[i] = FIELD_ACTION[a]
        cnames = (C.c_char_p * max(nk, 1))(*names)
        jp = _JsonlPolicy(n_keys=nk, key_names=cnames, action=acts.ctypes.data_as(C.POINTER(C.c_uint8)),
                          force_type=ftyp.ctypes.data_as(C.POINTER(C.c_uint8)), default_action=FIELD_ACTION[default])
        sc, snames = self._schema(schema)
        out = C.c_void_p()
        st = load().as_anonymize_jsonl(self._h, C.byref(rec), C.byref(jp), C.byref(sc), key, len(key), C.byref(out))
        del keep, snames, cnames, acts, ftyp
        self._check(st)
        return Output(self, out.value)

    def reidentify(self, data, offsets, schema: Schema, key: bytes) -> Output:
        """Controlled re-identification (as_reidentify) against this context's entity map."""
        rec, keep = self._records(data, offsets)
        sc, names = self._schema(schema)
        out = C.c_void_p()
        st = load().as_reidentify(self._h, C.byref(rec), C.byref(sc), key, len(key), C.byref(out))
        del keep, names
        self._check(st)
        return Output(self, out.value)

    def anonymize_fields(self, data, offsets, field_start, field_len, field_id, policy: dict, schema: Schema,
                         key: bytes, default: str = "detect") -> Output:
        """Per-field policy (as_anonymize_fields). policy maps a field id to "detect", "exclude"
        or ("force", entity_type); other ids take ``default`` ("detect" or "exclude")."""
        on_dev = hasattr(data, "is_cuda") and data.is_cuda
        if on_dev:
            rec = _Records(bytes=data.data_ptr(), offsets=offsets.data_ptr(), n_records=offsets.numel() - 1,
                           on_device=1)
            keep = (data, offsets)
        else:
            d = np.ascontiguousarray(data, dtype=np.uint8)
            o = np.ascontiguousarray(offsets, dtype=np.uint64)
            rec = _Records(bytes=d.ctypes.data if d.size else None, offsets=o.ctypes.data, n_records=o.size - 1,
                           on_device=0)
            keep = (d, o)
        fs = np.ascontiguousarray(field_start, dtype=np.uint64)
        fl = np.ascontiguousarray(field_len, dtype=np.uint32)
        fi = np.ascontiguousarray(field_id, dtype=np.uint32)
        n_ids = (max(policy) + 1) if policy else 0
        act = np.full(max(n_ids, 1), FIELD_ACTION[default], np.uint8)
        ftype = np.zeros(max(n_ids, 1), np.uint8)
        for fid, a in policy.items():
            if isinstance(a, tuple):
                act[fid], ftype[fid] = FIELD_ACTION[a[0]], a[1]
            else:
                act[fid] = FIELD_ACTION[a]
        flds = _Fields(start=fs.ctypes.data, len=fl.ctypes.data, id=fi.ctypes.data, n_fields=fs.size)
        pol = _FieldPolicy(n_ids=n_ids, action=act.ctypes.data, force_type=ftype.ctypes.data,
                           default_action=FIELD_ACTION[default])
        sc, names = self._schema(schema)
        out = C.c_void_p()
        st = load().as_anonymize_fields(self._h, C.byref(rec), C.byref(flds), C.byref(pol), C.byref(sc), key,
                                        len(key), C.byref(out))
        del keep, names
        self._check(st)
        return Output(self, out.value)

    def anonymize_stream(self, data, offsets, schema: Schema, key: bytes, batch_bytes: int = 0,
                         lanes: int = 0) -> Output:
        """Host records in overlapping batches (as_anonymize_stream); output on the host."""
        d = np.ascontiguousarray(data, dtype=np.uint8)
        o = np.ascontiguousarray(offsets, dtype=np.uint64)
        rec = _Records(bytes=d.ctypes.data if d.size else None, offsets=o.ctypes.data, n_records=o.size - 1,
                       on_device=0)
        sc, names = self._schema(schema)
        cfg = _StreamConfig(batch_bytes=batch_bytes, lanes=lanes)
        out = C.c_void_p()
        st = load().as_anonymize_stream(self._h, C.byref(rec), C.byref(sc), key, len(key), C.byref(cfg),
                                        C.byref(out))
        del names
        self._check(st)
        return Output(self, out.value)

    def autotune(self, rows: int = 0) -> list[dict]:
        """Time every tile configuration of the four projection GEMMs; keep the fastest."""
        ent = (_TuneEntry * 4)()
        self._check(load().as_autotune(self._h, rows, ent))
        return [{"role": TUNE_ROLES[e.role], "m": e.m, "n": e.n, "k": e.k, "chosen": e.chosen,
                 "ms": [float(x) for x in e.ms]} for e in ent]

    def set_tiles(self, cfg: list[int]):
        arr = (C.c_int32 * 4)(*cfg)
        self._check(load().as_set_tiles(self._h, arr))

    def tiles(self) -> list[int]:
        arr = (C.c_int32 * 4)()
        self._check(load().as_get_tiles(self._h, arr))
        return list(arr)

    def calibrate(self, data, offsets, schema: Schema):
        """FP8: set static activation scales from calibration records (host arrays)."""
        d = np.ascontiguousarray(data, dtype=np.uint8)
        o = np.ascontiguousarray(offsets, dtype=np.uint64)
        rec = _Records(bytes=d.ctypes.data if d.size else None, offsets=o.ctypes.data, n_records=o.size - 1,
                       on_device=0)
        sc, names = self._schema(schema)
        self._check(load().as_calibrate(self._h, C.byref(rec), C.byref(sc)))
        del names

    def scales(self) -> np.ndarray:
        out = np.zeros(4 * self.dims.n_layers, np.float32)
        self._check(load().as_get_scales(self._h, out.ctypes.data, out.size))
        return out

    def set_scales(self, scales: np.ndarray):
        sc = np.ascontiguousarray(scales, dtype=np.float32)
        self._check(load().as_set_scales(self._h, sc.ctypes.data, sc.size))

    def map_export(self) -> list[Entity]:
        p, n = C.POINTER(_Entity)(), C.c_uint64()
        self._check(load().as_map_export(self._h, C.byref(p), C.byref(n)))
        try:
            return _entities(p, n.value)
        finally:
            load().as_free(C.cast(p, C.c_void_p))

    def map_import(self, key: bytes, entries: list[Entity]):
        arr, bufs = _entity_array(entries)
        self._check(load().as_map_import(self._h, key, len(key), arr, len(entries)))

    # ---- serving loop (continuous batching)
    def serve_start(self, schema: Schema, key: bytes, lanes: int = 2, max_batch_bytes: int = 0,
                    max_batch_records: int = 0, max_pending: int = 0, activation_budget: int = 0):
        """activation_budget: bytes of encoder activations over all lanes (0 = 40 GiB)."""
        sc, names = self._schema(schema)
        cfg = _ServeConfig(lanes=lanes, max_batch_bytes=max_batch_bytes, max_batch_records=max_batch_records,
                           max_pending=max_pending, activation_budget_bytes=activation_budget)
        self._check(load().as_serve_start(self._h, C.byref(sc), key, len(key), C.byref(cfg)))
        del names

    def submit(self, record: bytes, discard: bool = False) -> int | None:
        """Queue one record; returns its request id, or None when the queue is full."""
        rid = C.c_uint64()
        st = load().as_submit(self._h, bytes(record) if record else None, len(record), 1 if discard else 0,
                              C.byref(rid))
        if st == -9:
            return None
        self._check(st)
        return rid.value

    def poll(self, request_id: int, timeout_s: float = 10.0) -> bytes | None:
        """The anonymized record, or None if it is not ready within the timeout."""
        out = C.c_void_p()
        st = load().as_poll(self._h, request_id, C.byref(out), int(timeout_s * 1e6))
        if st == -5:
            return None
        self._check(st)
        return Output(self, out.value).records()[0]

    def serve_stats(self, reset: bool = False) -> dict:
        s = _ServeStats()
        self._check(load().as_serve_stats(self._h, C.byref(s), 1 if reset else 0))
        return {k: getattr(s, k) for k, _ in _ServeStats._fields_}

    def serve_stop(self):
        self._check(load().as_serve_stop(self._h))

    def stream(self) -> int:
        """The ctx's cudaStream_t (as an int), for torch.cuda.ExternalStream."""
        p = C.c_void_p()
        self._check(load().as_get_stream(self._h, C.byref(p)))
        return p.value or 0

    def profile(self, enable: bool):
        self._check(load().as_profile(self._h, 1 if enable else 0))

    def profile_read(self) -> dict:
        s = _Profile()
        self._check(load().as_profile_read(self._h, C.byref(s)))
        d = {k: getattr(s, k) for k, _ in _Profile._fields_ if k != "stage_ms"}
        d["stage_ms"] = dict(zip(PROFILE_STAGES, list(s.stage_ms)))
        return d

    def map_clear(self):
        self._check(load().as_map_clear(self._h))

    def trace(self) -> dict:
        t = _Trace()
        self._check(load().as_debug_trace(self._h, C.byref(t)))
        T, nr, nf, n = t.n_tokens, t.n_regex, t.n_final, t.n_records

        def arr(p, k, dt):
            if k == 0 or not p:
                return np.zeros(0, dt)
            return np.ctypeslib.as_array(p, shape=(k,)).astype(dt, copy=True)

        C_ = self.dims.n_labels
        logits = arr(t.logits, T * C_, np.float32).reshape(T, C_) if t.logits else None
        return {"rec_tok": arr(t.rec_tok, n + 1, np.uint64), "tok_ids": arr(t.tok_ids, T, np.int32),
                "tok_off": arr(t.tok_off, T, np.uint32), "tok_len": arr(t.tok_len, T, np.uint32),
                "regex_start": arr(t.regex_start, nr, np.uint32), "regex_len": arr(t.regex_len, nr, np.uint32),
                "regex_type": arr(t.regex_type, nr, np.uint8), "logits": logits,
                "labels": arr(t.labels, T, np.uint8), "final_start": arr(t.final_start, nf, np.uint32),
                "final_len": arr(t.final_len, nf, np.uint32), "final_type": arr(t.final_type, nf, np.uint8)}

    def close(self):
        if getattr(self, "_h", None):
            load().as_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


STATIC_MAX_BYTES = 1 << 20


def _require_device_tensor(t, name: str, dtypes: tuple, device: int):
    """Refuse anything the kernels cannot read in place: a host tensor, another GPU's
    memory, a strided view or the wrong element type would hand the device a pointer it
    cannot use (a fault) or bytes it misreads (wrong tokens)."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise AnonShieldError(-1, f"{name} must be a torch CUDA tensor, got {type(t).__name__}")
    if not t.is_cuda or t.device.index != device:
        raise AnonShieldError(-1, f"{name} must be on cuda:{device} (the context's device), got {t.device}")
    if not t.is_contiguous():
        raise AnonShieldError(-1, f"{name} must be contiguous")
    if t.dtype not in dtypes:
        raise AnonShieldError(-1, f"{name} has dtype {t.dtype}, expected one of {', '.join(map(str, dtypes))}")


def tokenize_static(ctx: "Context", data, offsets, stream=None) -> dict:
    """Tokenize device-resident records without any allocation inside the call.

    data (uint8) and offsets (int64/uint64, n+1) are contiguous CUDA tensors
    on the context's device; anything else is refused with AS_ERR_ARG before
    the library is called. The output tensors are allocated here, by the
    caller side, before the call; the library call itself allocates nothing.
    Returns the outputs as tensors."""
    import torch
    _require_device_tensor(data, "data", (torch.uint8,), ctx.device)
    _require_device_tensor(offsets, "offsets", (torch.int64, torch.uint64), ctx.device)
    if offsets.dim() != 1 or offsets.numel() < 1:
        raise AnonShieldError(-1, "offsets must be a 1-D tensor of n_records + 1 entries")
    n = offsets.numel() - 1
    n_bytes = int(data.numel())
    dev = data.device
    out = {"tok_ids": torch.empty(max(n_bytes, 1), dtype=torch.int32, device=dev),
           "tok_off": torch.empty(max(n_bytes, 1), dtype=torch.int32, device=dev),
           "tok_len": torch.empty(max(n_bytes, 1), dtype=torch.int32, device=dev),
           "rec_tok": torch.empty(n + 1, dtype=torch.int64, device=dev),
           "n_tokens": torch.zeros(1, dtype=torch.int32, device=dev)}
    st = load().as_tokenize_static(ctx._h, _ptr(data), _ptr(offsets), n, n_bytes, _ptr(out["tok_ids"]),
                                   _ptr(out["tok_off"]), _ptr(out["tok_len"]), _ptr(out["rec_tok"]),
                                   _ptr(out["n_tokens"]), stream)
    _check_k(st)
    return out


def version() -> str:
    return load().as_version().decode()
