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


# C struct of the header -> the binding's ctypes mirror
_MIRRORS = {"as_config": "_Config", "as_records": "_Records", "as_schema": "_Schema", "as_entity": "_Entity",
            "as_stats": "_Stats", "as_trace": "_Trace", "as_fields": "_Fields", "as_field_policy": "_FieldPolicy",
            "as_jsonl_policy": "_JsonlPolicy", "as_stream_config": "_StreamConfig",
            "as_serve_config": "_ServeConfig", "as_serve_stats_t": "_ServeStats", "as_tune_entry": "_TuneEntry",
            "as_profile_stats": "_Profile"}


def test_c_program_builds_against_headers_and_layouts_match(tmp_path):
    """The boundary is plain C: a C99 program including both headers compiles, links against
    the library and calls an entry point that needs no GPU; every struct's size and every
    field's offset, as the C compiler lays them out, equal the binding's ctypes mirror."""
    import ctypes as C
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "anonshield.h"', '#include "anonshield_kernels.h"',
             'int main(void) {', '  printf("version %s\\n", as_version());']
    for cname, pyname in _MIRRORS.items():
        lines.append(f'  printf("size {cname} %zu\\n", sizeof({cname}));')
        for field, _ in getattr(api, pyname)._fields_:
            lines.append(f'  printf("off {cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ['  return 0;', '}']
    src = tmp_path / "abi.c"
    src.write_text("\n".join(lines) + "\n")
    lib_dir = os.path.dirname(api.LIB_PATH)
    exe = tmp_path / "abi"
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                        "-L", lib_dir, "-lanonshield", f"-Wl,-rpath,{lib_dir}", "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    got = {}
    for line in out.stdout.splitlines():
        parts = line.split()
        if parts[0] == "size":
            got[("size", parts[1])] = int(parts[2])
        elif parts[0] == "off":
            got[("off", parts[1], parts[2])] = int(parts[3])
    assert "sm_103a" in out.stdout
    for cname, pyname in _MIRRORS.items():
        st = getattr(api, pyname)
        assert got[("size", cname)] == C.sizeof(st), cname
        for field, _ in st._fields_:
            assert got[("off", cname, field)] == getattr(st, field).offset, (cname, field)
