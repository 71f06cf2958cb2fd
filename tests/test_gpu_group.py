"""psfd_solve_group: several contexts solved at once, each on its own stream and host thread.

A batch of illuminations split over two contexts and solved together must give, context by
context, bitwise the solutions and diffraction orders of solving each context alone (a
context's arithmetic does not depend on the other's); a repeated context is rejected.
"""
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


def _halves(prob):
    h = prob.n_rhs // 2
    return [prob.with_illumination(prob.theta_deg[sl], prob.phi_deg[sl], prob.pol[sl])
            for sl in (slice(0, h), slice(h, prob.n_rhs))]


def _results(s, n):
    return [(s.get_solution(i), s.diffraction_orders(i)["amp"]) for i in range(n)]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_group_solve_is_bitwise_the_solves_alone(psfd, precision):
    prec = psfd.FP32_REFINED if precision == "fp32" else psfd.FP64
    prob = layouts.small_clip(nx=32, ny=32, nslab=7, dx=2.0, dz=1.5, seed=11, stack=layouts.ru_mosi_stack(40),
                              theta=(6.0, 6.0, 3.0, 3.0), phi=(0.0, 0.0, 45.0, 45.0), pol=(0, 1, 0, 1))
    kw = dict(tol=1e-9, inner_tol=1e-4, max_iter=400, max_outer=10)
    parts = _halves(prob)
    streams = [torch.cuda.Stream() for _ in parts]
    solvers = [psfd.Solver.from_problem(p, prec, stream=st) for p, st in zip(parts, streams)]
    alone = []
    for s, p in zip(solvers, parts):
        s.solve(**kw)
        torch.cuda.synchronize()
        alone.append(_results(s, p.n_rhs))
    reps = psfd.solve_group(solvers, **kw)
    torch.cuda.synchronize()
    assert len(reps) == 2 and all(r["relres"] <= 1e-9 for r in reps)
    for s, p, ref in zip(solvers, parts, alone):
        for (x, a), (x0, a0) in zip(_results(s, p.n_rhs), ref):
            assert np.array_equal(x, x0)
            assert np.array_equal(a, a0)
    for s in solvers:
        s.close()


def test_group_solve_rejects_a_repeated_context(psfd):
    prob = layouts.small_clip(nx=16, ny=16, nslab=5, dx=4.0, dz=2.0, seed=1)
    s = psfd.Solver.from_problem(prob, psfd.FP32_REFINED)
    with pytest.raises(psfd.PsfdError) as e:
        psfd.solve_group([s, s], tol=1e-8)
    assert e.value.status == psfd.E_ARG
    s.close()
