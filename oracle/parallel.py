"""Oracle solves timed on one core, or several at once in a process pool (test infrastructure).

Used by ``tests/`` and by the CPU-baseline leg of ``bench.py`` only. Each worker process runs
single-threaded (BLAS pinned to one thread: the oracle's transforms and GMRES projections are
matrix products) and is started with ``spawn``, never forked, so that a pool started after a
CUDA context exists in the parent does not inherit it.
"""
from __future__ import annotations

import contextlib
import multiprocessing as mp
import os
import time

from .psfd_oracle import solve

__all__ = ["solve_timed", "solve_many", "apply_many", "usable_processes"]


class _StampedHistory(list):
    """GMRES residual history that also records when each iteration finished."""

    def __init__(self):
        super().__init__()
        self.stamps = []

    def append(self, res):
        self.stamps.append(time.perf_counter())
        super().append(res)


def _one_thread():
    try:
        from threadpoolctl import threadpool_limits
        return threadpool_limits(1)
    except ImportError:
        return contextlib.nullcontext()


def solve_timed(prob, i: int, rtol: float, marks=(), maxiter: int = 400) -> dict:
    """Solve illumination i to rtol on one thread and time it.

    For every tolerance m in `marks` (looser than rtol) the result also holds the time an
    oracle solve stopped at m would take: the time until GMRES first reached m, plus the time
    this solve spent after its last iteration (forming the solution from the basis, a little
    longer for the longer basis of the tighter solve, and the orders)."""
    hist = _StampedHistory()
    with _one_thread():
        t0 = time.perf_counter()
        orders, _, info = solve(prob, i, rtol=rtol, maxiter=maxiter, history=hist)
        t1 = time.perf_counter()
    tail = t1 - (hist.stamps[-1] if hist.stamps else t0)
    at = {}
    for m in marks:
        k = next((j for j, r in enumerate(hist) if r <= m), None)
        if k is not None:
            at[m] = {"seconds": hist.stamps[k] - t0 + tail, "iterations": k + 1}
    info = {k: v for k, v in info.items() if k in ("iterations", "relres")}
    return {"i": i, "orders": orders, "seconds": t1 - t0, "at": at, **info}


def _worker(args):
    prob, i, rtol, marks = args
    return solve_timed(prob, i, rtol, marks)


def _apply_worker(args):
    """Seconds for `reps` oracle operator applications of illumination i on one thread."""
    from .psfd_oracle import apply_operator, rhs_vector, setup_rhs
    prob, i, reps = args
    with _one_thread():
        ctx = setup_rhs(prob, i)
        u = rhs_vector(ctx)
        t0 = time.perf_counter()
        for _ in range(reps):
            apply_operator(ctx, u)
        return time.perf_counter() - t0


def apply_many(prob, indices, reps: int, processes: int) -> tuple[list, float]:
    """`reps` operator applications of each illumination in `indices`, one single-threaded
    spawn worker each, all at once. Returns (seconds per worker, wall seconds of the pool)."""
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(processes=processes) as pool:
        out = pool.map(_apply_worker, [(prob, int(i), int(reps)) for i in indices], chunksize=1)
    return out, time.perf_counter() - t0


def usable_processes(limit: int, bytes_per_process: float) -> int:
    """At most `limit` workers, no more than the host's cores, and no more than the available
    memory holds at `bytes_per_process` each."""
    n = min(limit, os.cpu_count() or 1)
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    avail = float(line.split()[1]) * 1024.0
                    n = min(n, max(1, int(0.8 * avail // bytes_per_process)))
                    break
    except OSError:
        pass
    return max(1, n)


def solve_many(prob, indices, rtol: float, processes: int, marks=()) -> tuple[list, float]:
    """Solve the given illuminations in a spawn pool of `processes` single-threaded workers.
    Returns (results in the order of `indices`, wall seconds of the whole pool)."""
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(processes=processes) as pool:
        out = pool.map(_worker, [(prob, int(i), rtol, tuple(marks)) for i in indices], chunksize=1)
    return out, time.perf_counter() - t0
