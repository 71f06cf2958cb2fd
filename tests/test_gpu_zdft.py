"""The z pass's forward transform (K2 at nf = 128) on the CUDA cores and on the tensor cores
(split-BF16 dense DFT products, psfd_zdft_measure) against the FP64 DFT of the zero-padded
columns (the unnormalised transform of Sec. 3, Eq. (18)). Bounds: 2e-6 normwise for the FP32
register transform (FP32 roundoff times the transform depth) and 5e-5 for three BF16
products (each operand carried to 16 bits: about 2^-16 per product term)."""
import numpy as np
import pytest

from paper_2606_25541_b300 import layouts

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def psfd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_25541_b300 import psfd as m
    m.load()
    return m


def _reference(x):
    """FP64 DFT along z of the columns zero padded to 128 (plane p at index p + 1)."""
    ns, nslab, ny, nx = x.shape
    full = np.zeros((ns, 128, ny, nx), np.complex128)
    full[:, 1:nslab + 1] = x
    return np.fft.fft(full, axis=1)


@pytest.mark.parametrize("nslab,nx,ny", [(60, 256, 4), (7, 128, 3), (63, 384, 2)])
def test_forward_z_transform_on_both_units(psfd, nslab, nx, ny):
    x = layouts.random_field((3, nslab, ny, nx), seed=nslab).astype(np.complex64)
    # a dynamic range like the spectra K2 sees: columns scaled over six decades
    x *= np.logspace(-3, 3, nx)[None, None, None, :].astype(np.float32)
    ref = _reference(x.astype(np.complex128))
    xd = torch.tensor(x, device="cuda")
    for method, tol in ((0, 2e-6), (1, 5e-5)):
        out = torch.full((3, 128, ny, nx), float("nan"), dtype=torch.complex64, device="cuda")
        psfd.zdft_measure(method, xd, out)
        torch.cuda.synchronize()
        assert psfd.zdft_status() == 0
        got = out.cpu().numpy().astype(np.complex128)
        # per column, relative to the column's norm (the columns span six decades)
        err = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert np.max(err) < tol, (method, float(np.max(err)))
