"""Serving loop: continuous batching of mask-clip requests through psfd_server_*.

A request's diffraction orders must be identical (bitwise) whether it is solved alone or
admitted into a bucket where other requests are already mid-solve, and must match the
oracle within the FP32-with-FP64-refinement tolerance (1e-6).
"""
import numpy as np
import pytest

import oracle
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


def _clips():
    st = layouts.ru_mosi_stack(40)
    a = layouts.small_clip(nx=16, ny=16, nslab=5, seed=1, stack=st, theta=(6.0, 2.0), phi=(0.0, 30.0), pol=(0, 1))
    b = layouts.small_clip(nx=16, ny=16, nslab=5, seed=2, stack=st, theta=(4.0,), phi=(45.0,), pol=(1,))
    c = layouts.small_clip(nx=8, ny=8, nslab=4, seed=3, stack=layouts.ru_mosi_stack(5), theta=(6.0, 6.0),
                           phi=(0.0, 0.0), pol=(0, 1))
    d = layouts.small_clip(nx=16, ny=16, nslab=5, seed=4, stack=st, theta=(0.0, 3.0, 8.0), phi=(0.0, 90.0, 10.0),
                           pol=(1, 0, 1))
    return [a, b, c, d]


def _solve_alone(psfd, prob, precision):
    srv = psfd.Server(precision, slots_per_context=6, tol=1e-9)
    t = srv.submit(prob)
    srv.run_until_done()
    state, status = srv.status(t)
    assert state == 2 and status == psfd.OK
    out = [srv.orders(t, i) for i in range(prob.n_rhs)]
    srv.close()
    return out


@pytest.mark.parametrize("precision,rounds", [(1, 0), (0, 0), (1, 3)])
def test_results_are_identical_alone_and_in_the_mix(psfd, precision, rounds):
    """rounds > 0: fused rounds, one graph launch advancing both buckets (two grids) per round."""
    clips = _clips()
    alone = [_solve_alone(psfd, p, precision) for p in clips]

    srv = psfd.Server(precision, slots_per_context=6, tol=1e-9)
    srv.set_rounds(rounds)
    t0 = srv.submit(clips[0])
    t1 = srv.submit(clips[1])
    for _ in range(3):
        srv.progress()
    assert srv.status(t0)[0] == 1 and srv.status(t1)[0] == 1
    # late arrivals: admitted next to the running requests (same grid) or into a new bucket
    t2 = srv.submit(clips[2])
    t3 = srv.submit(clips[3])
    # t3 joins t0's bucket between two of its engine steps (a bucket is never changed while
    # a step of it is on the device), t2 gets a bucket of its own at once
    for _ in range(200):
        srv.progress()
        if srv.status(t3)[0] >= 1:
            break
    assert srv.status(t3)[0] >= 1 and srv.status(t2)[0] >= 1
    assert srv.status(t0)[0] == 1, "the late request should overlap the running ones"
    used, n_ctx = srv.memory()
    assert n_ctx == 2 and used > 0
    srv.run_until_done()
    for t, p, ref in zip((t0, t1, t2, t3), clips, alone):
        state, status = srv.status(t)
        assert state == 2 and status == psfd.OK
        for i in range(p.n_rhs):
            got = srv.orders(t, i)
            np.testing.assert_array_equal(got["m"], ref[i]["m"])
            np.testing.assert_array_equal(got["amp"], ref[i]["amp"])
        srv.release(t)
    srv.close()


def test_served_orders_match_the_oracle(psfd):
    p = _clips()[3]
    srv = psfd.Server(psfd.FP32_REFINED, slots_per_context=4, tol=1e-9)
    t = srv.submit(p)
    srv.run_until_done()
    for i in range(p.n_rhs):
        got = srv.orders(t, i)
        ref, _, _ = oracle.solve(p, i, rtol=1e-13)
        key = {(m, n): k for k, (m, n) in enumerate(zip(ref["m"], ref["n"]))}
        idx = [key[(m, n)] for m, n in zip(got["m"], got["n"])]
        err = np.linalg.norm(got["amp"] - ref["amp"][idx]) / np.linalg.norm(ref["amp"])
        assert err < 1e-6, (i, err)
    srv.close()


def test_budget_admits_one_bucket_at_a_time(psfd):
    clips = _clips()
    probe = psfd.Server(psfd.FP32_REFINED, slots_per_context=4, tol=1e-9)
    probe.submit(clips[0])
    probe.progress()
    one_bucket, _ = probe.memory()
    probe.close()
    srv = psfd.Server(psfd.FP32_REFINED, hbm_budget=int(one_bucket * 1.05), slots_per_context=4, tol=1e-9)
    ta = srv.submit(clips[0])
    tc = srv.submit(clips[2])  # other grid: waits for the first bucket to drain
    srv.progress()
    assert srv.status(ta)[0] == 1 and srv.status(tc)[0] == 0
    assert srv.memory()[1] == 1
    srv.run_until_done()
    assert srv.status(ta)[0] == 2 and srv.status(tc)[0] == 2
    ref = _solve_alone(psfd, clips[2], psfd.FP32_REFINED)
    np.testing.assert_array_equal(srv.orders(tc, 1)["amp"], ref[1]["amp"])
    srv.close()


def test_request_over_the_budget_is_rejected_and_queued_one_cancelled(psfd):
    """A request whose bucket alone exceeds the HBM budget finishes at admission with
    PSFD_E_BUDGET (it would otherwise wait forever); a queued request can be cancelled; the
    others are served as usual."""
    clips = _clips()
    probe = psfd.Server(psfd.FP32_REFINED, slots_per_context=2, tol=1e-9)
    probe.submit(clips[2])
    probe.progress()
    small_bucket, _ = probe.memory()
    probe.close()
    srv = psfd.Server(psfd.FP32_REFINED, hbm_budget=int(small_bucket * 1.05), slots_per_context=2, tol=1e-9)
    tc = srv.submit(clips[2])   # 8 x 8 grid, 2 illuminations: fills its bucket
    ta = srv.submit(clips[0])   # 16 x 16 grid: its bucket alone is over the budget
    tb = srv.submit(clips[2])   # same grid as tc: waits for its slots, then is cancelled
    srv.progress()
    assert srv.status(ta) == (2, psfd.E_BUDGET)
    assert srv.status(tc)[0] == 1 and srv.status(tb)[0] == 0
    srv.release(tb)
    with pytest.raises(psfd.PsfdError):
        srv.status(tb)
    with pytest.raises(psfd.PsfdError) as e:
        srv.release(tc)  # running
    assert e.value.status == psfd.E_STATE
    srv.run_until_done()
    assert srv.status(tc) == (2, psfd.OK)
    ref = _solve_alone(psfd, clips[2], psfd.FP32_REFINED)
    np.testing.assert_array_equal(srv.orders(tc, 0)["amp"], ref[0]["amp"])
    srv.close()


@pytest.mark.parametrize("cap", [1, 2])
def test_requests_in_flight_are_capped_and_results_unchanged(psfd, cap):
    """psfd_server_set_max_running: never more than cap requests running after a progress()
    call, admission still in arrival order, and every request's orders bitwise those of its
    solve alone."""
    clips = _clips()
    alone = [_solve_alone(psfd, p, 1) for p in clips]
    srv = psfd.Server(1, slots_per_context=6, tol=1e-9)
    srv.set_max_running(cap)
    tickets = [srv.submit(p) for p in clips]
    first_running = []
    for _ in range(100000):
        srv.progress()
        states = [srv.status(t)[0] for t in tickets]
        assert sum(s == 1 for s in states) <= cap
        for i, s in enumerate(states):
            if s >= 1 and i not in first_running:
                first_running.append(i)
        if all(s == 2 for s in states):
            break
    assert all(srv.status(t)[0] == 2 for t in tickets)
    assert first_running == sorted(first_running)  # admitted in arrival order
    for t, p, ref in zip(tickets, clips, alone):
        assert srv.status(t)[1] == psfd.OK
        for i in range(p.n_rhs):
            got = srv.orders(t, i)
            assert np.array_equal(got["amp"], ref[i]["amp"])
    srv.close()
