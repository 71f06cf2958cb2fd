"""CUDA-graph replay of the Krylov step (psfd_set_graphs) and the device-side sweep loop
(psfd_set_device_loop): bitwise the same results, iteration counts and residual history, and
the same kernel count, as launching the kernels one by one."""
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


def _run(psfd, prob, precision, graphs, loop=True, **kw):
    s = psfd.Solver.from_problem(prob, precision)
    s.set_graphs(graphs)
    s.set_device_loop(loop)
    reps, sols, hists = [], [], []
    for _ in range(2):  # the second solve replays what the first captured
        s.set_illumination(prob.theta_deg, prob.phi_deg, prob.pol)
        torch.cuda.synchronize()
        n0 = psfd.launch_count()
        rep = s.solve(**kw)
        torch.cuda.synchronize()
        reps.append((rep["iterations"], rep["outer"], rep["relres"], psfd.launch_count() - n0))
        sols.append([s.get_solution(i) for i in range(prob.n_rhs)])
        hists.append([s.residual_history(i) for i in range(prob.n_rhs)])
    s.close()
    return reps, sols, hists


@pytest.mark.parametrize("precision,krylov", [(0, 0), (1, 0), (1, 1)])
def test_graph_replay_is_bitwise_the_same(psfd, precision, krylov):
    prob = layouts.small_clip(nx=32, ny=32, nslab=6, dx=2.0, dz=2.0, seed=8, stack=layouts.ru_mosi_stack(40),
                              theta=(6.0, 8.0, 4.0), phi=(0.0, 45.0, 90.0), pol=(0, 1, 0))
    kw = dict(tol=1e-10 if precision == 0 else 1e-8, inner_tol=1e-4, max_iter=300, max_outer=10,
              check_every=3, krylov=krylov, restart=8 if krylov else 0)
    runs = {name: _run(psfd, prob, precision, graphs, loop, **kw)
            for name, graphs, loop in (("loop", True, True), ("ticks", True, False), ("plain", False, False))}
    reps0, sols0, hists0 = runs["plain"]
    for name in ("loop", "ticks"):
        reps, sols, hists = runs[name]
        if name == "ticks":
            assert reps == reps0, (name, reps, reps0)
        else:  # the loop also runs one small condition kernel per tick
            assert [r[:3] for r in reps] == [r[:3] for r in reps0], (name, reps, reps0)
            assert all(a[3] > b[3] for a, b in zip(reps, reps0)), (reps, reps0)
        for a, b in zip(sols, sols0):
            for x, y in zip(a, b):
                assert np.array_equal(x, y), name
        for a, b in zip(hists, hists0):
            for x, y in zip(a, b):
                assert all(np.array_equal(x[k], y[k]) for k in x), name
