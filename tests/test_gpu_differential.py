"""GPU parity of the differential PSFD operator (psfd_apply_differential: curl curl E - k0^2 eps E
with spectral, PML-stretched derivatives, Sec. 3, Eqs. (4)-(7)) against the FP64 oracle
(oracle/differential_oracle.apply_differential) on the same seeded inputs. Both sides compute
in FP64; the bar is 1e-12 of max |out| (the FFT rounding of a few transforms of length <= 128,
amplified by the k^2 of the second derivative, stays near 1e-14)."""
import numpy as np
import pytest

from oracle import differential_oracle as dif
from paper_2606_25541_b300 import layouts

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

LAM = 13.5
TOL = 1e-12

# (n, nz, n_pml, dx, dz, theta, phi): every supported transverse and column length, a column
# without PML, oblique incidence in both planes and a ragged clip height inside the column
CASES = [
    (8, 32, 6, 4.0, 2.0, 6.0, 0.0),
    (16, 64, 12, 2.0, 1.0, 6.0, 20.0),
    (32, 128, 24, 2.0, 1.0, 9.0, 45.0),
    (64, 32, 0, 1.0, 2.0, 0.0, 0.0),
    (64, 128, 30, 1.0, 0.5, 6.0, 90.0),
]


@pytest.fixture(scope="module")
def psfd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_25541_b300 import psfd as m
    m.load()
    return m


def _problem(n, nz, n_pml, dx, dz, theta, phi, seed):
    """A seeded line/space clip of 0.7 nz - 2 n_pml planes (at least one) in the middle of the column."""
    nslab = max(1, int(0.7 * (nz - 2 * n_pml)) - 3)
    clip = layouts.small_clip(nx=n, ny=n, nslab=nslab, dx=dx, dz=dz, seed=seed, stack=layouts.empty_stack(),
                              theta=(theta,), pol=(0,))
    eps = np.ones((nz, n, n), np.complex128)
    z0 = (nz - nslab) // 2
    eps[z0:z0 + nslab] = clip.eps
    return dif.DiffProblem(nx=n, ny=n, nz=nz, dx=dx, dy=dx, dz=dz, wavelength=LAM, eps_bg=1.0, eps=eps,
                           n_pml=n_pml, theta=theta, phi=phi)


def _field(p, seed):
    rng = np.random.default_rng(seed)
    shape = (3, p.nz, p.ny, p.nx)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _gpu_apply(psfd, p, E):
    dev = torch.device("cuda:0")
    eps = torch.from_numpy(np.ascontiguousarray(p.eps)).to(dev)
    e = torch.from_numpy(np.ascontiguousarray(E)).to(dev)
    out = torch.full_like(e, float("nan"))
    work = torch.full_like(e, float("nan"))
    st = psfd.apply_differential(p.nx, p.nz, p.n_pml, p.dx, p.dz, p.wavelength, p.eps_bg, p.theta, p.phi, eps, e,
                                 out, work)
    torch.cuda.synchronize()
    assert st == 0, psfd.strerror(st)
    return out.cpu().numpy()


@pytest.mark.parametrize("case", CASES, ids=[f"n{c[0]}_nz{c[1]}_pml{c[2]}" for c in CASES])
def test_differential_apply_matches_oracle(psfd, case):
    p = _problem(*case, seed=11)
    E = _field(p, 5)
    ref = dif.apply_differential(p, E)
    got = _gpu_apply(psfd, p, E)
    assert np.all(np.isfinite(got))
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert err < TOL, err


def test_differential_apply_of_the_rhs_and_linearity(psfd):
    """The operator on the structured right-hand side of Eq. (3) (smooth in z, zero outside the
    clip) and on a linear combination: A(a E1 + b E2) = a A E1 + b A E2 to rounding."""
    p = _problem(16, 64, 10, 2.0, 1.0, 6.0, 30.0, seed=4)
    b = dif.differential_rhs(p)
    got = _gpu_apply(psfd, p, b)
    ref = dif.apply_differential(p, b)
    assert np.max(np.abs(got - ref)) < TOL * np.max(np.abs(ref))
    E1, E2 = _field(p, 1), _field(p, 2)
    a, c = 0.3 - 1.1j, -2.0 + 0.5j
    lhs = _gpu_apply(psfd, p, a * E1 + c * E2)
    rhs = a * _gpu_apply(psfd, p, E1) + c * _gpu_apply(psfd, p, E2)
    assert np.max(np.abs(lhs - rhs)) < TOL * np.max(np.abs(lhs))


def test_differential_apply_rejects_unsupported_sizes(psfd):
    """Unsupported lengths and a PML that fills the column are rejected before any device work."""
    p = _problem(16, 64, 10, 2.0, 1.0, 6.0, 0.0, seed=4)
    dev = torch.device("cuda:0")
    e = torch.zeros((3, 64, 16, 16), dtype=torch.complex128, device=dev)
    eps = torch.ones((64, 16, 16), dtype=torch.complex128, device=dev)
    bad = [
        (12, 64, 10, 2.0, 1.0),   # transverse length
        (16, 48, 10, 2.0, 1.0),   # column length
        (16, 64, 32, 2.0, 1.0),   # PML fills the column
        (16, 64, 10, 0.0, 1.0),   # spacing
    ]
    for n, nz, npml, dx, dz in bad:
        st = psfd.apply_differential(n, nz, npml, dx, dz, p.wavelength, 1.0, 6.0, 0.0, eps, e, e.clone(), e.clone())
        assert st == -1, (n, nz, npml, dx, dz, st)


@pytest.mark.parametrize("precond", [0, 1])
def test_differential_gmres_on_the_device_matches_the_oracle(psfd, precond):
    """GMRES(20) on the device (psfd_solve_differential) against the oracle's GMRES(20) on the
    same system and preconditioner (Sec. 3's comparison): the solutions agree to the solve
    tolerance's scale and the device's residual is at most rtol. The operator counts (thousands
    of restarted steps without a preconditioner) agree within a factor 1.4: the two
    orthogonalise differently (classical twice on the device, modified on the host), so their
    rounding, and with it the restart history, differs."""
    p = _problem(8, 32, 6, 4.0, 2.0, 6.0, 0.0, seed=3)
    b = dif.differential_rhs(p)
    g = dif._geometry(p)
    if precond:
        x_ref, mv_ref, _ = dif.gmres_restarted(lambda v: dif.spectral_damping(p, dif.apply_differential(p, v, g), g),
                                               dif.spectral_damping(p, b, g), 1e-10, 20, 20000)
    else:
        x_ref, mv_ref, _ = dif.gmres_restarted(lambda v: dif.apply_differential(p, v, g), b, 1e-10, 20, 20000)
    dev = torch.device("cuda:0")
    eps = torch.from_numpy(np.ascontiguousarray(p.eps)).to(dev)
    bd = torch.from_numpy(np.ascontiguousarray(b)).to(dev)
    x = torch.full_like(bd, float("nan"))
    st, mv, rel = psfd.solve_differential(p.nx, p.nz, p.n_pml, p.dx, p.dz, p.wavelength, p.eps_bg, p.theta, p.phi,
                                          eps, bd, x, precond=precond, restart=20, max_matvecs=20000, rtol=1e-10)
    torch.cuda.synchronize()
    assert st == 0, psfd.strerror(st)
    assert rel <= 1e-10
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - x_ref) <= 1e-6 * np.linalg.norm(x_ref)
    # the device solution solves the system: ||b - A x|| small against ||b|| (unpreconditioned check)
    r = b - dif.apply_differential(p, xg, g)
    assert np.linalg.norm(r) <= 1e-6 * np.linalg.norm(b)
    assert mv_ref / 1.4 <= mv <= 1.4 * mv_ref, (mv, mv_ref)
