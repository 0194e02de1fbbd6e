"""The C ABI library loads and exports every symbol the headers declare (no GPU calls)."""
import os
import re

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
