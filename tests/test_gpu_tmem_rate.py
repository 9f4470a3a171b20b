"""Measured rates of the two steps of the tensor-core screen's accumulator
round trip (tests/cuda/tmem_ld_rate.cu): reading a 256-column accumulator with
the epilogue's reduction loads, and one 128 x 256 x 32 FP16 MMA tile from
issue to its mbarrier, also with two tiles (both accumulators) per commit.  The screen's rate is limited by how many accumulator
columns it can turn around per unit time (its 512 columns over the round
trip); this test prints the ceilings of both steps and checks that they are
of a sane order."""
import os
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.gpu
def test_tmem_read_and_mma_round_trip_rates():
    from paper_1101_3228_gb300.build import _nvcc
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "tmem_ld_rate")
        subprocess.run([_nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O2",
                        os.path.join(HERE, "cuda", "tmem_ld_rate.cu"), "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=120).stdout
    print(out)
    reads, tiles = {}, {}
    for ln in out.splitlines():
        p = ln.split()
        if p[:2] == ["tmem_ld_rate", "warps"]:
            reads[int(p[2])] = float(p[4])
        elif p[:2] == ["tmem_ld_rate", "mma_tile"]:
            tiles[(int(p[3]), int(p[5]))] = (float(p[7]), float(p[9]), int(p[11]))
    assert set(reads) == {4, 8, 16} and set(tiles) == {(1, 1), (2, 1), (1, 2)}
    assert all(v > 0 for v in reads.values())
    for cyc, tflops, timeouts in tiles.values():
        assert timeouts == 0 and cyc > 0 and 0 < tflops < 2600.0
