"""CPU checks of the C ABI: the library builds, loads, exports every symbol
declared in include/sph.h, and the ctypes structs match the C layout.
No compute call is made (no GPU here)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sph.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sph_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1909_07439_gb300 import build, native
    build.build()
    return native.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (sph_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(lib, n)


def test_binding_covers_header():
    from paper_1909_07439_gb300 import native
    assert set(declared_functions()) == set(native.EXPORTS)


def test_struct_layout_matches_c(tmp_path):
    import ctypes
    from paper_1909_07439_gb300 import native
    src = tmp_path / "sz.c"
    src.write_text('#include "sph.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu\\n", sizeof(sph_params),'
                   ' sizeof(sph_state), sizeof(sph_stats), offsetof(sph_state, keys),'
                   ' offsetof(sph_params, box_len));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True,
                                       check=True).stdout.split()))
    assert got == [ctypes.sizeof(native.sph_params), ctypes.sizeof(native.sph_state),
                   ctypes.sizeof(native.sph_stats), native.sph_state.keys.offset,
                   native.sph_params.box_len.offset]


def test_params_default_are_the_papers(lib):
    from paper_1909_07439_gb300 import native
    p = native.sph_params_default()
    assert abs(p.gamma - 5 / 3) < 1e-7 and p.alpha_av == 1 and p.beta_av == 2
    assert p.alpha_u == 1 and abs(p.c_cour - 0.3) < 1e-7 and p.kernel == 0
    assert p.n_leaf == 16 and p.n_group == 8 and abs(p.hfact - 1.2) < 1e-7


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1909_07439_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), f
                assert "sph_oracle" not in text and "liboracle" not in text, f


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_1909_07439_gb300 import native
    monkeypatch.setattr(native, "_lib", None)
    monkeypatch.setattr(native, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(native.NativeLibraryMissing):
        native.load()
