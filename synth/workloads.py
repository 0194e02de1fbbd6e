"""The five seeded workloads: record-shape parameters and encoder dimensions.

c1  small:     256 records, token lengths uniform 32..512, 2-layer d=128 encoder, FP32.
c2  dataset:   70,951 records, lognormal(median 300, sigma 0.6) clipped 32..512,
               12-layer d=768 encoder, FP32 baseline vs BF16.
c3  packed:    lognormal(median 600, sigma 1.0) clipped 16..4096, windows 512/384,
               Zipf(1.1) entity reuse over 50k distinct entities, 12-layer d=768, FP8.
c4  serving:   lognormal(median 300, sigma 0.6) clipped 32..4096, Poisson arrivals.
c5  streaming: 1,000,000 records, lognormal(median 1500, sigma 0.8) clipped 16..4096,
               24-layer d=1024 encoder, 17 labels; URLs, hashes and CPE names planted
               besides the address/CVE kinds (the 8-type schema's recognizer types).
c1x            c1's shape with every recognizer kind planted, 23-label encoder.

Entity density is ~8 entities per 300 tokens (26.7 per 1k tokens) unless a
workload sets it. Seeds: records 1001, weights 2002, key 3003, arrivals 4004,
calibration 5005.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

SEED_RECORDS = 1001
SEED_WEIGHTS = 2002
SEED_KEY = 3003
SEED_ARRIVALS = 4004
SEED_CALIB = 5005


@dataclass(frozen=True)
class ModelDims:
    vocab: int = 8192
    d_model: int = 768
    n_heads: int = 12
    d_ffn: int = 3072
    n_layers: int = 12
    n_labels: int = 9
    max_pos: int = 512

    @property
    def d_head(self) -> int:
        return self.d_model // self.n_heads

    @property
    def n_types(self) -> int:
        return (self.n_labels - 1) // 2


@dataclass(frozen=True)
class RecordShape:
    n_records: int
    length_dist: str              # "uniform" or "lognormal"
    lo: int
    hi: int
    median: float = 300.0
    sigma: float = 0.6
    entities_per_1k: float = 8000.0 / 300.0
    zipf_distinct: int = 0        # >0: entities drawn Zipf(zipf_s) from this many distinct
    zipf_s: float = 1.1
    # extra entity kinds planted besides the five address/CVE kinds, from
    # EXTRA_KINDS; a share EXTRA_SHARE of fresh entities is drawn from them
    extra_kinds: tuple[str, ...] = ()


EXTRA_KINDS = ("url", "hash", "cpe", "uuid", "oid", "cert_fp", "pem")
EXTRA_SHARE = 0.35


@dataclass(frozen=True)
class Workload:
    name: str
    records: RecordShape
    dims: ModelDims
    window: int = 0               # 0: no sliding windows (records must fit max_pos)
    stride: int = 0
    note: str = ""
    extra: dict = field(default_factory=dict)


TYPE_NAMES_4 = ("IP_ADDRESS", "HOSTNAME", "CVE_ID", "MAC_ADDRESS")
TYPE_NAMES_8 = TYPE_NAMES_4 + ("URL", "HASH", "CPE", "ORGANIZATION")
TYPE_NAMES_11 = TYPE_NAMES_8 + ("UUID", "OID", "CERTIFICATE")
# recognizer kind -> entity type for TYPE_NAMES_8 (kind order MAC, IPv6, IPv4, CVE,
# host name, URL, hash, UUID, CPE, OID, certificate fingerprint, PEM; 0 = off)
RECOGNIZERS_8 = (4, 1, 1, 3, 2, 5, 6, 0, 7, 0, 0, 0)
RECOGNIZERS_11 = (4, 1, 1, 3, 2, 5, 6, 9, 7, 10, 11, 11)
# entity type (1-based index into TYPE_NAMES_11) of each planted extra kind
EXTRA_KIND_TYPE = {"url": 5, "hash": 6, "cpe": 7, "uuid": 9, "oid": 10, "cert_fp": 11, "pem": 11}

C1 = Workload(
    "c1-small-fp32",
    RecordShape(256, "uniform", 32, 512),
    ModelDims(vocab=8192, d_model=128, n_heads=2, d_ffn=512, n_layers=2, n_labels=9),
    note="256 scan records, 2L d128 encoder, one record per launch",
)
C2 = Workload(
    "c2-dataset-bf16",
    RecordShape(70951, "lognormal", 32, 512, median=300.0, sigma=0.6),
    ModelDims(),
    note="70,951 scan records, 12L d768 encoder",
)
C3 = Workload(
    "c3-packed-fp8",
    RecordShape(70951, "lognormal", 16, 4096, median=600.0, sigma=1.0, zipf_distinct=50000),
    ModelDims(),
    window=512, stride=384,
    note="windows 512/384, Zipf(1.1) reuse over 50k entities",
)
C4 = Workload(
    "c4-serving-bf16",
    RecordShape(70951, "lognormal", 32, 4096, median=300.0, sigma=0.6),
    ModelDims(),
    window=512, stride=384,
    note="Poisson arrivals at 1k/5k/20k/50k records/s",
)
C5 = Workload(
    "c5-streaming-fp8",
    RecordShape(1_000_000, "lognormal", 16, 4096, median=1500.0, sigma=0.8, extra_kinds=("url", "hash", "cpe")),
    ModelDims(vocab=8192, d_model=1024, n_heads=16, d_ffn=4096, n_layers=24, n_labels=17),
    window=512, stride=384,
    note="1M records, 24L d1024 encoder, 17 labels",
)

# c1 with every recognizer kind planted and a 23-label (11-type) encoder
C1X = Workload(
    "c1x-small-recognizers",
    RecordShape(256, "uniform", 32, 512, extra_kinds=EXTRA_KINDS),
    ModelDims(vocab=8192, d_model=128, n_heads=2, d_ffn=512, n_layers=2, n_labels=23),
    note="c1 records with URLs, hashes, CPE names, UUIDs, OIDs and certificates planted",
)

WORKLOADS = {w.name.split("-")[0]: w for w in (C1, C2, C3, C4, C5, C1X)}


def scaled(w: Workload, n_records: int) -> Workload:
    """Same workload with a different record count (for bounded samples)."""
    return replace(w, records=replace(w.records, n_records=n_records))
