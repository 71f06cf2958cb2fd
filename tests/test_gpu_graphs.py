"""CUDA-graph replay of the Krylov step (psfd_set_graphs): bitwise the same results and the
same kernel count as launching the kernels one by one."""
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


def _run(psfd, prob, precision, graphs, **kw):
    s = psfd.Solver.from_problem(prob, precision)
    s.set_graphs(graphs)
    reps, sols = [], []
    for _ in range(2):  # the second solve replays what the first captured
        s.set_illumination(prob.theta_deg, prob.phi_deg, prob.pol)
        torch.cuda.synchronize()
        n0 = psfd.launch_count()
        rep = s.solve(**kw)
        torch.cuda.synchronize()
        reps.append((rep["iterations"], rep["outer"], rep["relres"], psfd.launch_count() - n0))
        sols.append([s.get_solution(i) for i in range(prob.n_rhs)])
    s.close()
    return reps, sols


@pytest.mark.parametrize("precision,krylov", [(0, 0), (1, 0), (1, 1)])
def test_graph_replay_is_bitwise_the_same(psfd, precision, krylov):
    prob = layouts.small_clip(nx=32, ny=32, nslab=6, dx=2.0, dz=2.0, seed=8, stack=layouts.ru_mosi_stack(40),
                              theta=(6.0, 8.0, 4.0), phi=(0.0, 45.0, 90.0), pol=(0, 1, 0))
    kw = dict(tol=1e-10 if precision == 0 else 1e-8, inner_tol=1e-4, max_iter=300, max_outer=10,
              check_every=3, krylov=krylov, restart=8 if krylov else 0)
    reps_on, sols_on = _run(psfd, prob, precision, True, **kw)
    reps_off, sols_off = _run(psfd, prob, precision, False, **kw)
    assert reps_on == reps_off, (reps_on, reps_off)
    for a, b in zip(sols_on, sols_off):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
