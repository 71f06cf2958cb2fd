"""The autotuner (psfd_autotune, psfd_tune_set): every tile shape it may choose gives bitwise the
same operator output and solve as the built-in shape, on a fused-plane grid, the half-plane
line/space grid, a split-plane grid and a Stockham z length, and the tuner's report is
consistent with what it stored."""
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
    yield m
    m.tune_reset()


def _grid(psfd, p):
    return psfd.make_grid(p.nx, p.ny, p.nslab, p.nf, p.dx, p.dy, p.dz, p.wavelength, p.eps_bg)


CASES = [
    ("fused 64^2, nf 64", lambda: layouts.small_clip(nx=64, ny=64, nslab=20, dx=2.0, dz=2.0, seed=3,
                                                      stack=layouts.ru_mosi_stack(40),
                                                      theta=(6.0, 4.0), phi=(0.0, 45.0), pol=(0, 1))),
    ("half-plane 128^2, nf 128", lambda: layouts.line_space_clip().with_illumination([8.0, 0.0], [45.0, 0.0],
                                                                                      [1, 0])),
    ("split 256^2, nf 96", lambda: layouts.small_clip(nx=256, ny=256, nslab=12, dx=1.0, dz=1.0, seed=5,
                                                       stack=layouts.ru_mosi_stack(40), nz_min=96,
                                                       theta=(6.0,), phi=(20.0,), pol=(1,))),
]


def _shapes(psfd, g, precision):
    """Every shape psfd_tune_set accepts for the grid, one tunable at a time."""
    out = []
    for zx in (1, 2, 4, 8, 16):
        out.append((zx, 0, 0))
    for rb in (1, 2, 4, 8, 16, 32):
        out.append((0, rb, 0))
    for cx in (1, 2, 4, 8, 16, 32):
        out.append((0, 0, cx))
    for pf in (148, 296, 592):
        out.append((0, 0, 0, pf))
    ok = []
    for t in out:
        try:
            psfd.tune_set(g, precision, *t)
            ok.append(t)
        except psfd.PsfdError:
            pass
    psfd.tune_reset()
    return ok


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("precision", [0, 1])
def test_every_tile_shape_gives_bitwise_the_same_apply(psfd, name, make, precision):
    prob = make()
    g = _grid(psfd, prob)
    dt = torch.complex128 if precision == 0 else torch.complex64
    u = torch.tensor(layouts.random_field((prob.n_rhs, 3, prob.nslab, prob.ny, prob.nx), seed=11), dtype=dt,
                     device="cuda")
    psfd.tune_reset()
    s = psfd.Solver.from_problem(prob, precision)
    ref = torch.empty_like(u)
    s.apply(u, ref)
    shapes = _shapes(psfd, g, precision)
    assert len(shapes) >= 3, shapes
    for t in shapes:
        psfd.tune_set(g, precision, *t)
        out = torch.full_like(u, float("nan"))
        s.apply(u, out)
        torch.cuda.synchronize()
        assert torch.equal(out, ref), (name, t)
    psfd.tune_reset()
    s.close()


def test_autotuned_solve_is_bitwise_the_built_in_one(psfd):
    prob = CASES[2][1]()
    psfd.tune_reset()
    s = psfd.Solver.from_problem(prob, psfd.FP32_REFINED)
    rep0 = s.solve(tol=1e-8, inner_tol=1e-4, max_iter=300)
    x0 = s.get_solution(0)
    o0 = s.diffraction_orders(0)["amp"]
    r = s.autotune(force=True)
    assert r["candidates"] >= 3 and r["default_ms"] > 0 and 0 < r["tuned_ms"] <= r["default_ms"], r
    assert s.autotune()["candidates"] == 0  # the grid is in the table now
    rep1 = s.solve(tol=1e-8, inner_tol=1e-4, max_iter=300)
    assert (rep1["iterations"], rep1["outer"], rep1["relres"]) == (rep0["iterations"], rep0["outer"], rep0["relres"])
    assert np.array_equal(s.get_solution(0), x0)
    assert np.array_equal(s.diffraction_orders(0)["amp"], o0)
    s.close()
    psfd.tune_reset()
