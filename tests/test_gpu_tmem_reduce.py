"""The tensor-core screen takes its 16-column chunk minima straight from the
tensor-memory loads (tcgen05.ld.red ... .min.f32).  This test pins what that
instruction returns on this GPU: the exact per-thread minimum (and maximum) of the
loaded columns, with the loaded values intact, for known contents."""
import os
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.gpu
def test_tmem_load_reduction_is_the_exact_min():
    from paper_1101_3228_gb300.build import _nvcc
    nvcc = _nvcc()            # NVCC, PATH, then the toolkit's standard location
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "tmem_ld_red")
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2",
                        os.path.join(HERE, "cuda", "tmem_ld_red.cu"), "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=120).stdout
    line = next(l for l in out.splitlines() if l.startswith("ld.red probe:"))
    assert line == ("ld.red probe: min16@0 bad 0, min16@16 bad 0, max32 bad 0, "
                    "loaded values bad 0 (of 128 rows)"), out
