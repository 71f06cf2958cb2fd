"""Pins of the oracle's own discrete Fourier transform (``oracle/fft.py``) against the
definition X[k] = sum_n x[n] exp(-2 pi i n k / N) summed term by term, for every length
the operator uses (the FFT lengths of the z columns and planes, 4 .. 1024, with factors 2,
3 and 5) and the odd and prime lengths of the small test grids. The discrete operator of
Sec. 3, Eq. (18) is built from these transforms, so a wrong twiddle sign, a transposed
index split or a missing 1/N would show here first."""
import numpy as np
import pytest

from oracle import fft as offt

LENGTHS = [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 15, 16, 30, 32, 36, 37, 60, 64, 96, 128, 160, 192,
           256, 320, 384, 512, 640, 768, 1024]


@pytest.mark.parametrize("n", LENGTHS)
def test_fft_matches_the_direct_sum(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((3, n)) + 1j * rng.standard_normal((3, n))
    ref = offt.dft_direct(x)
    got = offt.fft(x)
    assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref), n
    back = offt.ifft(got)
    assert np.linalg.norm(back - offt.dft_direct(got, inverse=True)) <= 1e-13 * np.linalg.norm(x), n
    assert np.linalg.norm(back - x) <= 1e-13 * np.linalg.norm(x), n


@pytest.mark.parametrize("n", [8, 12, 128, 160])
def test_single_tones_and_parseval(n):
    """The DFT of exp(2 pi i m j / n) is n at bin m and zero elsewhere; sum |X|^2 = n sum |x|^2."""
    j = np.arange(n)
    for m in (0, 1, n // 2, n - 1, 3 % n):
        X = offt.fft(np.exp(2j * np.pi * m * j / n))
        ref = np.zeros(n, complex)
        ref[m] = n
        assert np.max(np.abs(X - ref)) < 1e-12 * n, (n, m)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    X = offt.fft(x)
    assert abs(np.sum(np.abs(X) ** 2) - n * np.sum(np.abs(x) ** 2)) < 1e-12 * n * np.sum(np.abs(x) ** 2)


def test_fft_shift_theorem_fixes_the_sign_convention():
    """A circular shift by s multiplies bin k by exp(-2 pi i k s / n) (forward sign negative)."""
    n, s = 96, 5
    rng = np.random.default_rng(4)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    k = np.arange(n)
    got = offt.fft(np.roll(x, s))
    assert np.allclose(got, offt.fft(x) * np.exp(-2j * np.pi * k * s / n), atol=1e-12, rtol=0)


def test_multi_axis_transforms_and_library_agreement():
    """fftn transforms along each listed axis and nothing else; it also agrees with numpy's
    transform (an independent library implementation) to rounding."""
    rng = np.random.default_rng(5)
    x = rng.standard_normal((3, 10, 12, 8)) + 1j * rng.standard_normal((3, 10, 12, 8))
    got = offt.fftn(x, axes=(1, 2, 3))
    ref = offt.dft_direct(offt.dft_direct(offt.dft_direct(x, axis=1), axis=2), axis=3)
    assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)
    assert np.linalg.norm(got - np.fft.fftn(x, axes=(1, 2, 3))) <= 1e-13 * np.linalg.norm(ref)
    two = offt.ifft2(got[:, 0], axes=(1, 2))
    assert np.linalg.norm(two - np.fft.ifft2(got[:, 0], axes=(1, 2))) <= 1e-13 * np.linalg.norm(two)


@pytest.mark.parametrize("n", [1, 2, 7, 8, 9, 128])
def test_fftfreq_ordering(n):
    """Bin k carries frequency k for k < ceil(n/2) and k - n above (Nyquist negative)."""
    f = offt.fftfreq(n, 0.5)
    for k in range(n):
        want = k if k < (n + 1) // 2 else k - n
        assert f[k] * n * 0.5 == pytest.approx(want, abs=1e-12)
