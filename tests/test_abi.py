"""The C ABI library loads and exports every symbol the headers declare (no GPU calls)."""
import os
import re

import pytest

import paper_2606_15650_b300.api as api

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols() -> set[str]:
    names = set()
    for h in ("anonshield.h", "anonshield_kernels.h"):
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(as_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_library_exports_declared_symbols():
    lib = api.load()
    names = declared_symbols()
    assert len(names) >= 20
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"
    assert set(api.EXPORTED) <= names


def test_version_string():
    assert "sm_103a" in api.version()


def test_structs_match_header_sizes():
    # ctypes layouts follow the C structs field by field; spot-check sizes
    import ctypes as C
    assert C.sizeof(api._Records) == 32
    assert C.sizeof(api._Entity) == 4 + 4 + 8 + 65 + 65 + 6 + 24


def test_tokenize_static_refuses_unusable_tensors():
    """The no-allocation tokenizer's binding refuses, before any library call, tensors the
    kernels could not read in place: host memory, wrong dtypes, strided views."""
    import torch

    class FakeCtx:
        device = 0
        _h = None

    good_offs = torch.tensor([0, 4], dtype=torch.int64)
    cases = [
        (torch.zeros(4, dtype=torch.uint8), good_offs, "cuda:0"),            # host tensor
        (b"abcd", good_offs, "torch CUDA tensor"),                            # not a tensor
    ]
    for data, offs, msg in cases:
        with pytest.raises(api.AnonShieldError) as e:
            api.tokenize_static(FakeCtx(), data, offs)
        assert e.value.status == -1 and msg in str(e.value)
