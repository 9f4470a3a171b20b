"""CPU-side checks of the C ABI: the library builds, loads, and exports exactly
what include/qt.h declares.  No compute call is made (no GPU here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qt.h")


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^QT_API\s+[\w\s\*]+?\b(qt_\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def libqt():
    from paper_1101_3228_gb300 import build
    path = build.build()
    return ctypes.CDLL(path), path


def test_header_declares_the_boundary():
    names = _declared()
    for need in ("qt_build_grids", "qt_transitions", "qt_backward", "qt_price", "qt_counts_from_samples"):
        assert need in names


def test_library_exports_every_declared_symbol(libqt):
    lib, path = libqt
    for name in _declared():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = sorted({ln.split()[-1] for ln in out.splitlines() if " T " in ln and ln.split()[-1].startswith("qt_")})
    assert exported == _declared()


def test_binding_lists_the_same_symbols():
    from paper_1101_3228_gb300 import binding
    assert sorted(binding.EXPORTS) == _declared()


def test_status_strings_without_gpu(libqt):
    lib, _ = libqt
    lib.qt_status_string.restype = ctypes.c_char_p
    assert lib.qt_status_string(0) == b"ok"
    assert lib.qt_status_string(4) == b"device wait timed out"


def test_create_without_gpu_fails_cleanly(libqt):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib, _ = libqt
    h = ctypes.c_void_p()
    st = lib.qt_create(ctypes.byref(h), 0)
    assert st != 0 and not h.value


def test_struct_layouts_match_header():
    """The ctypes mirrors of the ABI structs have the sizes the C compiler gives them."""
    from paper_1101_3228_gb300 import binding as B
    src = r"""
#include <stdio.h>
#include "qt.h"
int main(void){printf("%zu %zu %zu %zu\n", sizeof(qt_model), sizeof(qt_options), sizeof(qt_dump), sizeof(qt_stats));return 0;}
"""
    import tempfile
    with tempfile.TemporaryDirectory() as td:
        c = os.path.join(td, "s.c")
        exe = os.path.join(td, "s")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        sizes = list(map(int, subprocess.run([exe], capture_output=True, text=True).stdout.split()))
    assert sizes == [ctypes.sizeof(B.QtModel), ctypes.sizeof(B.QtOptions), ctypes.sizeof(B.QtDump),
                     ctypes.sizeof(B.QtStats)]


def test_product_path_has_no_oracle_or_cpu_fallback():
    """The package never imports the oracle, and the binding refuses to run without a GPU."""
    pkg = os.path.join(ROOT, "paper_1101_3228_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "qt_oracle" not in txt, f
