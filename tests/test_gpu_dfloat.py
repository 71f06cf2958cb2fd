"""The FP64 residual with its z pass (and the column passes of split planes) in double-float (PSFD_RESID_DFLOAT, psfd_apply with
PSFD_FP64_DF) against the FP64 oracle and the all-FP64 path.

Double-float carries about 48 significant bits; the sloppy sum and the FMA product each err
by a few 2^-48 relative to their operands, and a length-128 transform stacks seven levels of
them, so the z pass stays near 1e-14 normwise. The bar is the FP64 operator's (1e-12
normwise, on A u and on the scattered part u - A u), and a refined solve with the
double-float residual must still reach a 1e-11 target."""
import numpy as np
import pytest

import oracle
from paper_2606_25541_b300 import layouts

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module")
def psfd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_25541_b300 import psfd as m
    m.load()
    return m


# (nx, ny, nslab, nz_min): nf = 64 and 128 run the double-float z pass (full tiles, fewer
# x-modes than a tile, the thickest slab nf = 128 allows); split FP64 planes with ny = 128 or
# 256 run the double-float column passes (128 x 128 both, 256 x 256 at a short nf the column
# passes alone); the other cases keep every FP64 pass
DF_CASES = [
    (16, 16, 12, 64),
    (32, 16, 20, 128),
    (4, 32, 20, 128),
    (8, 8, 62, 128),
    (128, 128, 9, 128),
    (256, 256, 4, 0),
    (8, 8, 4, 0),
    (16, 8, 30, 160),
    (16, 32, 9, 256),
]


def _apply(psfd, s, u, precision):
    ud = torch.tensor(u, dtype=torch.complex128, device="cuda")
    out = torch.full_like(ud, float("nan"))
    s.apply(ud, out, precision=precision)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("nx,ny,nslab,nz", DF_CASES)
def test_double_float_apply_matches_oracle(psfd, nx, ny, nslab, nz):
    prob = layouts.small_clip(nx=nx, ny=ny, nslab=nslab, dx=2.0, dz=1.5, seed=nx + ny + nslab, nz_min=nz,
                              stack=layouts.ru_mosi_stack(10))
    prob = prob.with_illumination([6.0, 8.0], [0.0, 30.0], [0, 1])
    s = psfd.Solver.from_problem(prob, precision=psfd.FP32_REFINED)
    u = layouts.random_field((prob.n_rhs, 3, nslab, ny, nx), seed=11)
    got = _apply(psfd, s, u, psfd.FP64_DF)
    f64 = _apply(psfd, s, u, psfd.FP64)
    nf = s.grid.nf
    s.close()
    for i in range(prob.n_rhs):
        ref = oracle.apply_operator(oracle.setup_rhs(prob, i), u[i])
        assert _rel(got[i], ref) < 1e-12, i
        assert _rel(u[i] - got[i], u[i] - ref) < 1e-12, i
    fused = nx == ny and nx <= 64
    if nf in (64, 128) or (not fused and ny in (128, 256) and nx % 8 == 0):
        # a double-float pass ran: close to the FP64 one, but not bit for bit
        assert _rel(u - got, u - f64) < 1e-12
        assert not np.array_equal(got, f64)
    else:
        assert np.array_equal(got, f64)


def test_double_float_apply_full_line_space_clip(psfd):
    """The 128 x 128 x 60 line/space clip (nf = 128) at full size, two illuminations."""
    prob = layouts.line_space_clip()
    prob = prob.with_illumination(prob.theta_deg[[5, 16]], prob.phi_deg[[5, 16]], prob.pol[[5, 16]])
    u = layouts.random_field((2, 3, prob.nslab, prob.ny, prob.nx), seed=5)
    s = psfd.Solver.from_problem(prob, precision=psfd.FP32_REFINED)
    got = _apply(psfd, s, u, psfd.FP64_DF)
    s.close()
    for i in range(2):
        ref = oracle.apply_operator(oracle.setup_rhs(prob, i), u[i])
        assert _rel(u[i] - got[i], u[i] - ref) < 1e-12, i


def test_isolated_clip_keeps_the_fp64_pass(psfd):
    """The spherical kernel has no double-float pass: FP64_DF equals FP64 bit for bit."""
    n, nslab, nf = 32, 6, 32
    eps = np.ones((nslab, n, n), np.complex128)
    eps[:, 11:21, 11:21] = (0.94 + 0.04j) ** 2
    g = psfd.make_grid(n, n, nslab, nf, 2.0, 2.0, 2.0, 13.5)
    s = psfd.Solver(g, psfd.FP32_REFINED, 1)
    s.set_stack(np.zeros(0, np.complex128), np.zeros(0), 1.0)
    s.set_green(psfd.GREEN_SPHERICAL, 31.0)
    s.set_potential(eps)
    s.set_illumination([6.0], [20.0], [0])
    u = layouts.random_field((1, 3, nslab, n, n), seed=3)
    assert np.array_equal(_apply(psfd, s, u, psfd.FP64_DF), _apply(psfd, s, u, psfd.FP64))
    s.close()


@pytest.fixture(scope="module")
def contact_hole_reference():
    prob = layouts.contact_hole_clip()
    orders, x, info = oracle.solve(prob, 0, rtol=1e-13)
    return prob, orders, x


def _orders_err(got, ref):
    key = {(m, n): k for k, (m, n) in enumerate(zip(ref["m"], ref["n"]))}
    idx = [key[(m, n)] for m, n in zip(got["m"], got["n"])]
    return _rel(got["amp"], ref["amp"][idx])


@pytest.mark.parametrize("tol,order_tol", [(1e-8, 1e-6), (1e-11, 1e-9)])
def test_refined_solve_with_double_float_residual(psfd, contact_hole_reference, tol, order_tol):
    """The contact-hole clip (nf = 64) refined to tol with either residual arithmetic: both
    certify the target, match the oracle's orders, and agree with each other."""
    prob, ref, xref = contact_hole_reference
    out = {}
    for kind in (psfd.RESID_DFLOAT, psfd.RESID_FP64):
        s = psfd.Solver.from_problem(prob, precision=psfd.FP32_REFINED)
        s.set_residual_arith(kind)
        rep = s.solve(tol=tol, inner_tol=1e-4, max_iter=200, max_outer=12)
        assert rep["status"] == 0 and rep["relres"] <= tol, (kind, rep)
        got = s.diffraction_orders(0)
        assert _orders_err(got, ref) < order_tol, kind
        out[kind] = s.get_solution(0)
        s.close()
    # the solution errs by at most the condition number (below 1e3 here) times the residual
    assert _rel(out[psfd.RESID_DFLOAT], xref) < 2e3 * tol
    assert _rel(out[psfd.RESID_DFLOAT], out[psfd.RESID_FP64]) < 2e3 * tol


def test_residual_arith_rejects_unknown_kinds(psfd, contact_hole_reference):
    prob = contact_hole_reference[0]
    s = psfd.Solver.from_problem(prob, precision=psfd.FP32_REFINED)
    with pytest.raises(psfd.PsfdError):
        s.set_residual_arith(2)
    s.close()
