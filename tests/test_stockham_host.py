"""The shared-memory Stockham transform of the CUDA path (csrc/fft.cuh, the stages of cta_fft that
the plane passes and the generic z pass run) on the host: the header is compiled with g++ and
every supported length (4 ... 1024, radices 8, 4, 2, 3, 5) is transformed forward and inverse on
seeded Gaussian inputs, in FP32, in FP64 and in double-float pairs (the FP64 residual's passes),
against the DFT of the same input summed in long double.

Bound: an FFT's normwise error grows like log2(N) roundings, so it is taken as log2(1024) u with
u the unit roundoff (2^-24 FP32, 2^-53 FP64, 2^-48 for the pairs).

The per-stage twiddle tables of the FP32 plane passes (build_stw: each Stockham stage's twiddles in rows of R - 1
consecutive entries) must give bitwise the outputs of the plain table, since they hold the same
values and the stage multiplies by them in the same order; every power-of-two length must fit
its per-stage table in the plain table's space."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2606_25541_b300", "csrc")
CUDA_INC = "/usr/local/cuda/include"


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("g++ or the CUDA headers are missing")
    exe = str(tmp_path_factory.mktemp("stockham") / "stockham_host_check")
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-w", f"-I{CSRC}", f"-I{CUDA_INC}",
                    os.path.join(HERE, "stockham_host_check.cpp"), "-o", exe], check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=300).stdout
    return {k: float(v) for k, v in (line.split() for line in out.strip().splitlines())}


def test_every_supported_length_matches_the_dft(results):
    assert results["lengths"] == 16
    assert results["stockham_fp32"] <= 10 * 2.0 ** -24
    assert results["stockham_fp64"] <= 10 * 2.0 ** -53
    assert results["stockham_dfloat"] <= 10 * 2.0 ** -48
    # and the FP32 run really is FP32, the pairs really more than FP32
    assert results["stockham_fp32"] > 1e-9
    assert results["stockham_dfloat"] < 1e-12


def test_per_stage_twiddle_tables_are_bitwise_the_plain_table(results):
    # nine power-of-two lengths x 3 inputs x (FP32, FP64) x (forward, inverse)
    assert results["stw_checked"] == 9 * 3 * 4
    assert results["stw_mismatch"] == 0
    assert results["pow2_not_fitting"] == 0
