"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package only draws inputs: records, the subword vocabulary, encoder
weights and the HMAC key. It holds none of the method's arithmetic (no
tokenizer, recognizer, encoder, decoder or hash), so a mistake in either
implementation cannot hide in shared code.
"""
from .workloads import (C1, C2, C3, C4, C5, C1X, WORKLOADS, ModelDims, RecordShape, Workload,
                        TYPE_NAMES_4, TYPE_NAMES_8, TYPE_NAMES_11, RECOGNIZERS_8, RECOGNIZERS_11, EXTRA_KINDS, EXTRA_KIND_TYPE, SEED_RECORDS, SEED_WEIGHTS, SEED_KEY,
                        SEED_ARRIVALS, SEED_CALIB, scaled)
from .vocab import make_vocab, vocab_arrays, FIRST_WORD_ID
from .records import RecordSet, make_records, records_from_list
from .fielded import COLUMNS, JSONL_KEYS, FieldedRecords, make_fielded_records, make_jsonl_records
from .model import make_weights, pack_blob, blob_layout, blob_size, make_key

__all__ = ["COLUMNS", "JSONL_KEYS", "FieldedRecords", "make_fielded_records", "make_jsonl_records",
    "C1", "C2", "C3", "C4", "C5", "C1X", "WORKLOADS", "ModelDims", "RecordShape", "Workload",
    "TYPE_NAMES_4", "TYPE_NAMES_8", "TYPE_NAMES_11", "RECOGNIZERS_8", "RECOGNIZERS_11", "EXTRA_KINDS", "EXTRA_KIND_TYPE", "SEED_RECORDS", "SEED_WEIGHTS", "SEED_KEY",
    "SEED_ARRIVALS", "SEED_CALIB", "scaled", "make_vocab", "vocab_arrays", "FIRST_WORD_ID",
    "RecordSet", "make_records", "records_from_list", "make_weights", "pack_blob",
    "blob_layout", "blob_size", "make_key",
]
