"""The double-float primitives of the CUDA path's FP64 residual (csrc/dfloat.cuh) on the host:
the header is compiled with g++ (no floating-point contraction, as the device code forbids it
through round-to-nearest intrinsics) and checked against long double on a million seeded
operand pairs, a quarter of them near cancellation.

Bounds (u = 2^-48, the format's precision): TwoSum and the FMA TwoProduct exact; conversion
from FP64 within u |x|; the sloppy sum within 4 u (|a| + |b|); the product within 6 u |a b|;
every result normalised (|lo| <= 2^-24 |hi|); a double literal folded at compile time within u.
The integer-path conversions between FP64 and double-float that the device uses (exponent
rebias and round-to-nearest-even by integer operations, one exact FP64 addition) give bitwise
the values of the plain conversions on three million seeded doubles and the rounding edge cases.
The register four-step transform of the z pass (fft.cuh, 16 x nf/16) is run on the host in
double-float and in FP64 against a long-double DFT (lengths 64 and 128, forward on the
half-filled input and inverse): double-float within 2e-14 normwise, FP64 within 1e-15."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2606_25541_b300", "csrc")
CUDA_INC = "/usr/local/cuda/include"
U = 2.0 ** -48


def _run(tmp_path_factory, name):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("g++ or the CUDA headers are missing")
    exe = str(tmp_path_factory.mktemp("dfloat") / name)
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-w", f"-I{CSRC}", f"-I{CUDA_INC}",
                    os.path.join(HERE, name + ".cpp"), "-o", exe], check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=300).stdout
    return {k: float(v) for k, v in (line.split() for line in out.strip().splitlines())}


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    return _run(tmp_path_factory, "dfloat_check")


def test_error_free_transformations_are_exact(results):
    assert results["two_sum_inexact"] == 0
    assert results["two_prod_inexact"] == 0


def test_double_float_error_bounds(results):
    assert results["conv"] <= U
    assert results["add"] <= 4 * U
    assert results["mul"] <= 6 * U
    assert results["constant"] <= U
    # and the format is really about 48 bits, not FP32 with extra steps
    assert results["add"] > 0 and results["mul"] < 2.0 ** -40


def test_results_are_normalised(results):
    assert results["unnormalised"] == 0


def test_register_transform_in_double_float(tmp_path_factory):
    r = _run(tmp_path_factory, "dfloat_fft_check")
    assert r["fft_dfloat"] < 2e-14
    assert r["fft_fp64"] < 1e-15


def test_integer_path_conversions_are_bitwise_the_plain_ones(tmp_path_factory):
    r = _run(tmp_path_factory, "dfloat_conv_check")
    assert r["checked"] > 3e6 and r["int_path"] > 0.5 * r["checked"]
    assert r["to_dfr_mismatch"] == 0
    assert r["to_d_mismatch"] == 0
