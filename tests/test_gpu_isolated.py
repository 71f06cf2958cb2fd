"""GPU parity of the isolated clip (psfd_set_green with the spherically windowed dyadic Green's
function, Sec. 3, Eqs. (13)-(18)) against the FP64 oracle of the same Bloch-envelope problem.
Tolerances as in test_gpu_parity.py: 1e-12 (FP64) and 3e-5 (FP32) for one application."""
import math

import numpy as np
import pytest

from oracle import isolated_oracle as iso
from paper_2606_25541_b300 import layouts

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N, D, NSLAB, NF = 32, 2.0, 6, 32
R = 31.0  # above the block's diameter (20 x 20 x 12 nm), with 64 >= 20 + R and NF dz >= NSLAB dz + R
THETA, PHI, POL = [6.0, 0.0], [20.0, 0.0], [0, 1]


@pytest.fixture(scope="module")
def psfd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_25541_b300 import psfd as m
    m.load()
    return m


def _eps_slab():
    e = np.ones((NSLAB, N, N), np.complex128)
    e[:, 11:21, 11:21] = (0.94 + 0.04j) ** 2
    return e


def _solver(psfd, precision):
    g = psfd.make_grid(N, N, NSLAB, NF, D, D, D, 13.5)
    s = psfd.Solver(g, precision, 2)
    s.set_stack(np.zeros(0, np.complex128), np.zeros(0), 1.0)
    s.set_green(psfd.GREEN_SPHERICAL, R)
    s.set_potential(_eps_slab())
    s.set_illumination(THETA, PHI, POL)
    return s


def _oracle_problem(i):
    eb = np.ones((NF, N, N), np.complex128)
    eb[1:NSLAB + 1] = _eps_slab()  # slab plane p sits at z index p + 1 of the padded column
    return iso.IsolatedProblem(nx=N, ny=N, nz=NF, dx=D, dy=D, dz=D, wavelength=13.5, eps_bg=1.0, eps=eb, R=R,
                               theta=THETA[i], phi=PHI[i], pol=POL[i], bloch=True)


def _oracle_apply_slab(i, u_slab):
    p = _oracle_problem(i)
    ub = np.zeros((3, NF, N, N), np.complex128)
    ub[:, 1:NSLAB + 1] = u_slab
    return iso.apply_isolated(p, ub)[:, 1:NSLAB + 1]


@pytest.mark.parametrize("fp64", [True, False])
def test_isolated_apply_matches_oracle(psfd, fp64):
    s = _solver(psfd, psfd.FP64 if fp64 else psfd.FP32_REFINED)
    u = layouts.random_field((2, 3, NSLAB, N, N), seed=5)
    dt = torch.complex128 if fp64 else torch.complex64
    ud = torch.tensor(u, dtype=dt, device="cuda")
    out = torch.empty_like(ud)
    s.apply(ud, out)
    got = out.cpu().numpy()
    u_used = u if fp64 else u.astype(np.complex64).astype(np.complex128)
    for i in range(2):
        ref = _oracle_apply_slab(i, u_used[i])
        tol = 1e-12 if fp64 else 3e-5
        assert np.linalg.norm(got[i] - ref) < tol * np.linalg.norm(ref), i
        w_got, w_ref = u_used[i] - got[i], u_used[i] - ref
        assert np.linalg.norm(w_got - w_ref) < tol * np.linalg.norm(w_ref), i
    s.close()


def test_isolated_solve_matches_oracle(psfd):
    """The FP32 + refinement solve of the isolated clip against oracle GMRES on the same
    right-hand side (the incident envelope on the slab planes)."""
    s = _solver(psfd, psfd.FP32_REFINED)
    rep = s.solve(tol=1e-9, inner_tol=1e-4, max_iter=300, max_outer=10)
    assert rep["relres"] <= 1e-9
    for i in range(2):
        b = s.get_rhs(i)
        x, its, res = iso.gmres(lambda v: _oracle_apply_slab(i, v), b, rtol=1e-12)
        got = s.get_solution(i)
        assert np.linalg.norm(got - x) < 1e-7 * np.linalg.norm(x), i
        assert np.linalg.norm(x - b) > 1e-3 * np.linalg.norm(b)  # the block scatters
    s.close()


def test_set_green_rejects_a_window_the_padding_cannot_hold(psfd):
    g = psfd.make_grid(N, N, NSLAB, NF, D, D, D, 13.5)
    s = psfd.Solver(g, psfd.FP64, 1)
    with pytest.raises(psfd.PsfdError):
        s.set_green(psfd.GREEN_SPHERICAL, 60.0)  # nf dz = 64 < 12 + 60
    with pytest.raises(psfd.PsfdError):
        s.set_green(psfd.GREEN_SPHERICAL, -1.0)
    s.close()
