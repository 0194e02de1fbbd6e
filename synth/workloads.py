"""The five seeded workloads: record-shape parameters and encoder dimensions.

c1  small:     256 records, token lengths uniform 32..512, 2-layer d=128 encoder, FP32.
c2  dataset:   70,951 records, lognormal(median 300, sigma 0.6) clipped 32..512,
               12-layer d=768 encoder, FP32 baseline vs BF16.
c3  packed:    lognormal(median 600, sigma 1.0) clipped 16..4096, windows 512/384,
               Zipf(1.1) entity reuse over 50k distinct entities, 12-layer d=768, FP8.
c4  serving:   lognormal(median 300, sigma 0.6) clipped 32..4096, Poisson arrivals.
c5  streaming: 1,000,000 records, lognormal(median 1500, sigma 0.8) clipped 16..4096,
               24-layer d=1024 encoder, 17 labels.

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
    RecordShape(1_000_000, "lognormal", 16, 4096, median=1500.0, sigma=0.8),
    ModelDims(vocab=8192, d_model=1024, n_heads=16, d_ffn=4096, n_layers=24, n_labels=17),
    window=512, stride=384,
    note="1M records, 24L d1024 encoder, 17 labels",
)

WORKLOADS = {w.name.split("-")[0]: w for w in (C1, C2, C3, C4, C5)}


def scaled(w: Workload, n_records: int) -> Workload:
    """Same workload with a different record count (for bounded samples)."""
    return replace(w, records=replace(w.records, n_records=n_records))
