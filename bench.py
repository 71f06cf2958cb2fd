#!/usr/bin/env python
"""Benchmark: solves/s of the LS-PSFD solver on the 128 x 128 x 60 line/space clip.

One step solves one batch: the 128 x 128 nm line/space clip at 1 nm (60 absorber
planes, nf = 128, Ru/40 x (Mo/Si) stack) under 18 illuminations (polar 0/4/8 deg x
azimuth 0/45/90 deg x s/p). A step runs the whole hot path on the GPU: potential,
per-mode stack tables and right-hand sides, the FP32 BiCGStab solves inside FP64
defect correction (every operator application, Krylov update and FP64 residual), and
the diffraction orders. A "solve" is one illumination solved to the FP64 relative
residual --tol (1e-8 by default, which keeps the reflected orders within 1e-6 of the
FP64 reference; the line reports the measured difference).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank solves its own seeded clip (independent replicas, weak
scaling); timing is bracketed by a barrier and device synchronisation, and the
maximum over ranks is reported. Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2606_25541_b300 import layouts  # noqa: E402

METRIC = "solves/s at 1e-6 order error, FP32+refine vs FP64; p50/p99 latency; HBM %"
UNIT = "solves/s"
WORKLOAD = "line_space_128x128x60_nf128_18rhs"
FP64_NOMINAL_TFLOPS = 1.25  # B300 FP64 vector rate, nominal
# The headline metric is quoted at 1e-6 order error. Solving to an FP64 relative residual of
# 3e-7, with FP32 sweeps asked for 2e-7, keeps the largest per-illumination order error against
# a tight (1e-11) FP64 solve near 3e-7 on the line/space batch, a factor ~3 inside the target;
# every run measures and reports that error. The other modes default to 1e-8 / 1e-4.
HEADLINE_TOL, HEADLINE_INNER_TOL = 3e-7, 2e-7
DEFAULT_TOL, DEFAULT_INNER_TOL = 1e-8, 1e-4


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--tol", type=float, default=None,
                    help="FP64 relative residual target (default 3e-7 for the headline, serving and reference "
                         "arms; 1e-8 for the other modes)")
    ap.add_argument("--inner-tol", type=float, default=None, help="FP32 sweep tolerance (default 2e-7 / 1e-4)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison run")
    ap.add_argument("--no-autotune", action="store_true", help="keep the built-in tile shapes")
    ap.add_argument("--groups", type=int, default=1,
                    help="headline: contexts the 18 illuminations are split over, solved side by side "
                         "(psfd_solve_group); 1 = one context")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the sampled precision sweep and large clip in the default run")
    ap.add_argument("--profile-only", action="store_true", help="one profiled step, for ncu launch lists")
    ap.add_argument("--plain-launches", action="store_true",
                    help="with --profile-only: launch every kernel on its own (no CUDA graphs)")
    ap.add_argument("--apply", action="store_true",
                    help="operator applications/s only (psfd_apply), for kernel captures")
    ap.add_argument("--rhs", type=int, default=18, help="illuminations used by --apply and --profile-only")
    ap.add_argument("--apply-clip", choices=["line_space", "split1024"], default="line_space",
                    help="--apply: the 128^2 line/space clip, or a 1024^2 x 8-plane clip whose planes take "
                         "the split row and column passes")
    ap.add_argument("--pf", type=str, default=None,
                    help="--apply: comma-separated L2 prefetch distances of the half-plane kernels to time")
    ap.add_argument("--precision", choices=["fp32", "fp64", "fp64df", "both", "all"], default="both",
                    help="--apply precision (fp64df: FP64 data with the residual's double-float passes; "
                         "both = fp32 + fp64, all = the three)")
    ap.add_argument("--krylov", choices=["bicgstab", "gmres"], default="bicgstab",
                    help="inner Krylov method of the refined solve")
    ap.add_argument("--restart", type=int, default=0, help="GMRES basis size per sweep (0 = maximum)")
    ap.add_argument("--sweep", action="store_true",
                    help="precision sweep on the 256 x 256 x 60 Manhattan clip (FP64 vs FP32 + FP64 refinement)")
    ap.add_argument("--crosscheck", action="store_true",
                    help="decomposition vs the 40-bilayer stack meshed into the domain, 256 x 256 crop")
    ap.add_argument("--bilayers", type=int, default=40, help="Mo/Si bilayers of the --crosscheck stack")
    ap.add_argument("--large", action="store_true",
                    help="1024 x 1024 x 60 curvilinear clip, 8 illuminations in memory-bounded batches")
    ap.add_argument("--layers", type=str, default=None,
                    help="layer-count study: comma-separated Mo/Si bilayer counts (decomposition, outer fixed "
                         "point and stack meshed into the domain on the 256 x 256 crop)")
    ap.add_argument("--mesh-max", type=int, default=10, help="largest bilayer count --layers meshes into the domain")
    ap.add_argument("--isolated", action="store_true",
                    help="an isolated clip with the spherically windowed kernel (block absorber, padded box)")
    ap.add_argument("--differential", action="store_true",
                    help="FP64 applications/s of the differential PSFD operator (PML column) and of the "
                         "Lippmann-Schwinger operator on the same 64 x 64 x 30 clip")
    ap.add_argument("--precond-study", action="store_true",
                    help="Sec. 3's preconditioner comparison on the GPU (differential none / spectral damping, LS)")
    ap.add_argument("--zdft", action="store_true",
                    help="z pass forward transform: CUDA-core register FFT vs split-BF16 tensor-core DFT")
    ap.add_argument("--autotune", action="store_true",
                    help="autotuner table: built-in vs tuned tile shapes per workload grid")
    ap.add_argument("--small", action="store_true",
                    help="the 32 x 32 x 30 contact-hole clip (one illumination): ms per solve, CUDA graphs on/off")
    ap.add_argument("--fixed-point", action="store_true",
                    help="the outer fixed-point loop of Eq. (8) against the folded solve, per stack size")
    ap.add_argument("--fp-bilayers", type=str, default="0,10,40", help="Mo/Si bilayers for --fixed-point")
    ap.add_argument("--serve", type=int, default=24,
                    help="requests in the serving-loop sample (0 = skip); --serve-only prints only that")
    ap.add_argument("--serve-only", action="store_true")
    ap.add_argument("--serve-sizes", type=str, default="64,128")
    ap.add_argument("--serve-rounds", type=int, default=4,
                    help="ticks per fused serving round (0 = independent buckets only)")
    ap.add_argument("--serve-slots", type=int, default=18, help="illumination slots per serving context")
    ap.add_argument("--serve-budget-gb", type=float, default=120.0, help="HBM budget of the server")
    ap.add_argument("--serve-fp64-sample", type=int, default=8, help="requests timed on the plain FP64 path")
    return ap.parse_args(argv)


def run_serving(n_req: int, sizes, tol: float, inner_tol: float, seed: int = 4, slots: int = 18,
                budget_gb: float = 120.0, rounds: int = 4, fp64_sample: int = 8):
    """Seeded Poisson stream of mixed-size Manhattan clips through the continuous-batching server.

    Every request is first solved alone (its isolated service time); the arrival rate is then set
    to 0.8 of the one-at-a-time capacity and the stream is replayed through psfd_server_*. The
    one-at-a-time latency under the same arrivals is the FIFO recursion over the isolated
    service times. Latency = completion - arrival, wall clock. At 0.8 load the stream's
    solves/s is its arrival rate; the capacity is the saturated run (all requests submitted
    at once). The stream and the saturated run are measured with fused rounds (one graph
    launch per round advances every bucket, `rounds` ticks) and with independent buckets on
    priority streams. The plain FP64 path is timed one request at a time on the first
    `fp64_sample` requests."""
    from paper_2606_25541_b300 import psfd
    reqs = layouts.serving_requests(n_req, seed=seed, sizes=sizes)
    kw = dict(hbm_budget=int(budget_gb * 2 ** 30), slots_per_context=slots, tol=tol, inner_tol=inner_tol)
    service = []
    srv = psfd.Server(psfd.FP32_REFINED, **kw)
    srv.submit(reqs[0])
    srv.run_until_done()  # warm-up
    for p in reqs:
        t0 = time.perf_counter()
        t = srv.submit(p)
        srv.run_until_done()
        service.append(time.perf_counter() - t0)
        srv.release(t)
    srv.close()
    rng = np.random.default_rng(seed + 1)
    rate = 0.8 / float(np.mean(service))
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
    fifo, done = [], 0.0
    for a, s in zip(arrivals, service):
        done = max(a, done) + s
        fifo.append(done - a)
    def served(ticks, max_running=0):
        srv = psfd.Server(psfd.FP32_REFINED, **kw)
        srv.set_rounds(ticks)
        srv.set_max_running(max_running)
        pending, lat, i, peak_ctx = {}, [], 0, 0
        start = time.perf_counter()
        while i < n_req or pending:
            now = time.perf_counter() - start
            while i < n_req and arrivals[i] <= now:
                pending[srv.submit(reqs[i])] = arrivals[i]
                i += 1
            if not pending:
                time.sleep(max(0.0, arrivals[i] - now))
                continue
            srv.progress()
            peak_ctx = max(peak_ctx, srv.memory()[1])
            now = time.perf_counter() - start
            for t in list(pending):
                state, status = srv.status(t)
                if state == 2:
                    if status != psfd.OK:
                        raise RuntimeError(f"request {t} failed: {psfd.strerror(status)}")
                    lat.append(now - pending.pop(t))
                    srv.release(t)
        makespan = time.perf_counter() - start
        # capacity: every request submitted at once (the server keeps the device full)
        t0 = time.perf_counter()
        tickets = [srv.submit(p) for p in reqs]
        srv.run_until_done()
        saturated = time.perf_counter() - t0
        for t in tickets:
            srv.release(t)
        srv.close()
        return {"p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                "solves_per_s": n_rhs / makespan, "saturated_solves_per_s": n_rhs / saturated,
                "peak_contexts": peak_ctx}

    n_rhs = int(sum(p.n_rhs for p in reqs))
    fused = served(rounds) if rounds > 0 else None
    independent = served(0)
    # at most two requests in flight: most of the overlap, the tail close to one at a time;
    # and one at a time through the same server loop (its polling and admission included)
    limited = served(0, max_running=2)
    single = served(0, max_running=1)
    # the plain FP64 path one request at a time, on a sample of the stream
    sample = reqs[:fp64_sample]
    srv = psfd.Server(psfd.FP64, **kw)
    t = srv.submit(sample[0])
    srv.run_until_done()
    srv.release(t)
    t0 = time.perf_counter()
    for p in sample:
        t = srv.submit(p)
        srv.run_until_done()
        srv.release(t)
    fp64_s = time.perf_counter() - t0
    srv.close()
    n_sample = int(sum(p.n_rhs for p in sample))
    return {"requests": n_req, "illuminations": n_rhs, "sizes_nm": list(sizes), "offered_load": 0.8,
            "mode": "independent buckets on priority streams, at most two requests in flight",
            **limited,
            "unlimited": independent,
            "fused_rounds": dict(fused, ticks_per_round=rounds) if fused else None,
            "one_in_flight_served": single,
            "one_at_a_time": {"what": "FIFO recursion over the isolated service times (no server overhead)",
                              "p50_ms": 1e3 * float(np.percentile(fifo, 50)),
                              "p99_ms": 1e3 * float(np.percentile(fifo, 99)),
                              "solves_per_s": n_rhs / float(np.sum(service))},
            "fp64_one_at_a_time": {"solves_per_s": n_sample / fp64_s,
                                   "fp32_refined_same_sample": n_sample / float(np.sum(service[:fp64_sample])),
                                   "sample": f"the first {fp64_sample} requests of the stream"},
            "stream": "seeded Poisson arrivals; 1-18 illuminations, 50-70 nm Manhattan absorber, "
                      "z from {64,96,128} nm, slab rounded up to 8 planes"}


def run_apply(args):
    """Operator applications per second on the line/space clip (one application = K1, K2,
    K3 over every illumination of the batch), with CUDA events on the current stream."""
    import torch
    from paper_2606_25541_b300 import psfd
    if args.apply_clip == "split1024":  # 1024^2 planes (split row and column passes), 8 planes
        prob = layouts.small_clip(nx=1024, ny=1024, nslab=8, dx=1.0, dz=1.0, seed=2, stack=layouts.ru_mosi_stack(40),
                                  theta=(6.0,), phi=(0.0,), pol=(0,))
        workload = f"small_clip_1024x1024x8_nf{prob.nf}_{args.rhs}rhs"
    else:
        prob = layouts.line_space_clip(seed=2)
        workload = WORKLOAD.replace("18rhs", f"{args.rhs}rhs")
    sel = np.arange(args.rhs) % prob.n_rhs
    prob = prob.with_illumination(prob.theta_deg[sel], prob.phi_deg[sel], prob.pol[sel])
    stream = torch.cuda.current_stream()
    out = {"mode": "apply", "workload": workload}
    precs = {"both": ["fp32", "fp64"], "all": ["fp32", "fp64", "fp64df"]}.get(args.precision, [args.precision])
    for name in precs:
        prec = psfd.FP64 if name == "fp64" else psfd.FP32_REFINED
        apply_prec = {"fp32": psfd.FP32_REFINED, "fp64": psfd.FP64, "fp64df": psfd.FP64_DF}[name]
        s = psfd.Solver.from_problem(prob, prec, stream=stream)
        dt = torch.complex64 if name == "fp32" else torch.complex128
        u = torch.tensor(layouts.random_field((args.rhs, 3, prob.nslab, prob.ny, prob.nx), seed=1), dtype=dt,
                         device="cuda")
        y = torch.empty_like(u)
        grid = psfd.make_grid(prob.nx, prob.ny, prob.nslab, prob.nf, prob.dx, prob.dy, prob.dz, prob.wavelength)
        for pf in ([int(v) for v in args.pf.split(",")] if args.pf else [None]):
            if pf is not None:  # the half-plane kernels' L2 prefetch distance (0: none)
                psfd.tune_set(grid, psfd.FP64 if name == "fp64" else psfd.FP32_REFINED, pf=pf)
            for _ in range(args.warmup):
                s.apply(u, y, precision=apply_prec)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                s.apply(u, y, precision=apply_prec)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / max(args.steps, 1)
            key = name if pf is None else f"{name}_pf{pf}"
            out[key] = {"ms_per_application": ms, "applications_per_s": 1e3 / ms,
                        "rhs_applications_per_s": args.rhs * 1e3 / ms}
        psfd.tune_reset()
        s.close()
    print(json.dumps(out), flush=True)
    return 0


def run_sweep(args):
    print(json.dumps({"mode": "precision_sweep", **precision_sweep(args.tol, args.inner_tol, args.steps,
                                                                   args.warmup)}), flush=True)
    return 0


def precision_sweep(tol: float, inner_tol: float, steps: int, warmup: int) -> dict:
    """Precision sweep on the 256 x 256 x 60 Manhattan clip (nf = 128, 6 deg s and p): the plain
    FP64 path and the FP32 path with FP64 defect correction, each timed over whole solves of
    both illuminations, with the order error of every variant against the FP64 solution; the
    split-BF16 tensor-core row is the z transform stage measured against the CUDA cores."""
    import torch
    from paper_2606_25541_b300 import psfd
    prob = layouts.manhattan_clip(256, seed=3)
    stream = torch.cuda.current_stream()
    eps_dev = torch.from_numpy(prob.eps).cuda()
    out = {"workload": f"manhattan_256x256x60_nf{prob.nf}_2rhs", "n_rhs": prob.n_rhs, "tol": tol}
    orders = {}
    for name, prec, kw in (("fp64", psfd.FP64, dict(tol=tol, max_iter=600)),
                           ("fp32_refined", psfd.FP32_REFINED,
                            dict(tol=tol, inner_tol=inner_tol, max_iter=400, max_outer=12))):
        s = psfd.Solver.from_problem(prob, prec, stream=stream)

        def step():
            s.set_potential(eps_dev)
            s.set_illumination(prob.theta_deg, prob.phi_deg, prob.pol)
            return s.solve(**kw)

        for _ in range(max(warmup, 1)):
            rep = step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            rep = step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        orders[name] = [s.diffraction_orders(i) for i in range(prob.n_rhs)]
        out[name] = {"solves_per_s": prob.n_rhs * 1e3 / ms, "ms_per_batch": ms, "iterations": rep["iterations"],
                     "outer": rep["outer"], "relres": rep["relres"]}
        s.close()

    def err(a, b):
        key = {(m, n): k for k, (m, n) in enumerate(zip(b["m"], b["n"]))}
        idx = [key[(m, n)] for m, n in zip(a["m"], a["n"])]
        return float(np.linalg.norm(a["amp"] - b["amp"][idx]) / np.linalg.norm(b["amp"]))

    out["fp32_refined"]["order_rel_err_vs_fp64"] = max(
        err(a, b) for a, b in zip(orders["fp32_refined"], orders["fp64"]))
    out["fp32_refined"]["speedup_vs_fp64"] = out["fp32_refined"]["solves_per_s"] / out["fp64"]["solves_per_s"]
    out["bf16x3_tensor_cores"] = {"status": "the z transform stage measured, not used in the solve "
                                            "(slower and less accurate than the CUDA-core transform)",
                                  **zdft_rows()}
    return out


def run_large(args):
    print(json.dumps({"mode": "large_clip", **large_clip(args.tol, args.inner_tol, args.warmup)}), flush=True)
    return 0


def large_clip(tol: float, inner_tol: float, warmup: int, n_rhs: int | None = None) -> dict:
    """Large curvilinear clip, 1024 x 1024 x 60 (nf = 160), 4 polar angles x s/p (or the first
    n_rhs of them), FP32 with FP64 defect correction and the memory-light layout (BiCGStab pool,
    FP32 spectra inside the FP64 ones): the illuminations run in the largest batches whose
    workspace fits a 180 GB budget."""
    import torch
    from paper_2606_25541_b300 import psfd
    prob = layouts.curvilinear_clip()
    if n_rhs:
        prob = prob.with_illumination(prob.theta_deg[:n_rhs], prob.phi_deg[:n_rhs], prob.pol[:n_rhs])
    budget = 180e9
    g = psfd.make_grid(prob.nx, prob.ny, prob.nslab, prob.nf, prob.dx, prob.dy, prob.dz, prob.wavelength,
                       prob.eps_bg)
    batch = max(b for b in range(1, prob.n_rhs + 1) if psfd.workspace_bytes(g, psfd.FP32_REFINED, b) <= budget)
    stream = torch.cuda.current_stream()
    s = psfd.Solver.from_problem(prob, psfd.FP32_REFINED, max_rhs=batch, hbm_budget=int(budget), stream=stream,
                                 set_inputs=False)
    s.set_stack(prob.n_layers, prob.d_layers, prob.n_sub)
    s.set_potential(prob.eps)
    kw = dict(tol=tol, inner_tol=inner_tol, max_iter=600, max_outer=12)
    groups = [list(range(i, min(i + batch, prob.n_rhs))) for i in range(0, prob.n_rhs, batch)]

    def run_all():
        reps, effs = [], []
        for grp in groups:
            s.set_illumination(prob.theta_deg[grp], prob.phi_deg[grp], prob.pol[grp])
            reps.append(s.solve(**kw))
            effs += [float(s.diffraction_orders(i)["eff"].sum()) for i in range(len(grp))]
        return reps, effs

    if warmup > 0:
        run_all()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    reps, effs = run_all()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    out = {"workload": f"curvilinear_1024x1024x60_nf{prob.nf}_{prob.n_rhs}rhs", "n_rhs": prob.n_rhs,
           "batch_rhs": batch, "workspace_gb": psfd.workspace_bytes(g, psfd.FP32_REFINED, batch) / 1e9,
           "budget_gb": budget / 1e9, "solves_per_s": prob.n_rhs * 1e3 / ms, "ms_total": ms,
           "iterations": [r["iterations"] for r in reps], "outer": [r["outer"] for r in reps],
           "relres": max(r["relres"] for r in reps), "reflected_efficiency": effs}
    s.close()
    return out


def run_crosscheck(args):
    """The decomposition against a conventional PSFD with the Ru + n x (Mo/Si) stack meshed into
    the domain (z extended by the stack's thickness, thickness-weighted permittivity per 1 nm
    cell, substrate-only reflection) on a 256 x 256 crop of the 1024 x 1024 curvilinear clip,
    6 deg s and p, both solved in FP32 with FP64 refinement (n = --bilayers). Reported: the
    reflected efficiency of every propagating order from both, their relative difference
    (phase-free), times, iterations and convergence. The difference is the meshed stack's
    discretisation error at 1 nm."""
    import dataclasses
    import torch
    from paper_2606_25541_b300 import psfd
    big = layouts.curvilinear_clip()
    crop = dataclasses.replace(big, nx=256, ny=256, eps=np.ascontiguousarray(big.eps[:, :256, :256]),
                               name="curvilinear_crop_256x256x60")
    crop = crop.with_illumination([6.0, 6.0], [0.0, 0.0], [0, 1])
    n_l, d_l, n_s = layouts.ru_mosi_stack(args.bilayers)
    crop = dataclasses.replace(crop, n_layers=n_l, d_layers=d_l, n_sub=n_s)
    full, depth = layouts.stack_in_domain(crop)
    stream = torch.cuda.current_stream()
    kw = dict(tol=args.tol, inner_tol=args.inner_tol, max_iter=1000, max_outer=12, raise_on_error=False)
    out = {"mode": "stack_in_domain_crosscheck", "workload": "curvilinear_crop_256x256x60",
           "bilayers": args.bilayers,
           "stack_in_domain": {"planes": full.nslab, "nf": full.nf, "depth_nm": depth}}
    effs = {}
    for name, prob in (("decomposition", crop), ("stack_in_domain", full)):
        s = psfd.Solver.from_problem(prob, psfd.FP32_REFINED, stream=stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rep = s.solve(**kw)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        orders = [s.diffraction_orders(i) for i in range(prob.n_rhs)]
        effs[name] = orders
        out[name] = {"seconds": dt, "iterations": rep["iterations"], "outer": rep["outer"], "relres": rep["relres"],
                     "status": psfd.strerror(rep["status"]),
                     "reflected_efficiency": [float(o["eff"].sum()) for o in orders]}
        s.close()
    diffs = []
    for a, b in zip(effs["stack_in_domain"], effs["decomposition"]):
        key = {(m, n): k for k, (m, n) in enumerate(zip(b["m"], b["n"]))}
        idx = [key[(m, n)] for m, n in zip(a["m"], a["n"])]
        diffs.append(float(np.linalg.norm(a["eff"] - b["eff"][idx]) / np.linalg.norm(b["eff"])))
    out["efficiency_rel_diff"] = diffs
    print(json.dumps(out), flush=True)
    return 0


def run_layers(args):
    """Cost against the number of stack layers (the paper's comparison of the background-field
    method with a full-domain PSFD, Sec. 4): for Ru + n x (Mo/Si), the 256 x 256 crop of the
    1024 x 1024 curvilinear clip (60 planes at 1 nm, 6 deg s and p) solved three ways in FP32
    with FP64 refinement to --tol: the decomposition with R folded into the operator, the
    paper's outer fixed point of Eq. (8), and the stack meshed into the domain (thickness-
    weighted permittivity per 1 nm cell, substrate-only reflection; up to --mesh-max bilayers).
    Reported per n: seconds, Krylov iterations, outer steps, status, and the relative
    difference of the reflected efficiencies of the meshed solve against the decomposition."""
    import dataclasses
    import torch
    from paper_2606_25541_b300 import psfd
    big = layouts.curvilinear_clip()
    crop = dataclasses.replace(big, nx=256, ny=256, eps=np.ascontiguousarray(big.eps[:, :256, :256]),
                               name="curvilinear_crop_256x256x60")
    crop = crop.with_illumination([6.0, 6.0], [0.0, 0.0], [0, 1])
    stream = torch.cuda.current_stream()
    kw = dict(tol=args.tol, inner_tol=args.inner_tol, max_iter=1000, max_outer=12, raise_on_error=False)
    out = {"mode": "layer_count_study", "workload": "curvilinear_crop_256x256x60_2rhs", "tol": args.tol, "rows": []}

    def timed(prob, fixed_point=False):
        s = psfd.Solver.from_problem(prob, psfd.FP32_REFINED, stream=stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rep = s.solve_fixed_point(max_steps=300, **kw) if fixed_point else s.solve(**kw)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        eff = [s.diffraction_orders(i) for i in range(prob.n_rhs)]
        s.close()
        return {"seconds": dt, "iterations": rep["iterations"], "outer": rep["outer"], "relres": rep["relres"],
                "status": psfd.strerror(rep["status"])}, eff

    for nb in (int(v) for v in args.layers.split(",")):
        n_l, d_l, n_s = layouts.ru_mosi_stack(nb)
        prob = dataclasses.replace(crop, n_layers=n_l, d_layers=d_l, n_sub=n_s)
        row = {"bilayers": nb, "layers": len(n_l)}
        row["decomposition"], eff_dec = timed(prob)
        row["fixed_point"], _ = timed(prob, fixed_point=True)
        if nb <= args.mesh_max:
            full, depth = layouts.stack_in_domain(prob)
            row["stack_in_domain"], eff_full = timed(full)
            row["stack_in_domain"].update({"planes": full.nslab, "nf": full.nf, "depth_nm": depth})
            diffs = []
            for a, b in zip(eff_full, eff_dec):
                key = {(m, n): k for k, (m, n) in enumerate(zip(b["m"], b["n"]))}
                idx = [key[(m, n)] for m, n in zip(a["m"], a["n"])]
                diffs.append(float(np.linalg.norm(a["eff"] - b["eff"][idx]) / np.linalg.norm(b["eff"])))
            row["efficiency_rel_diff"] = diffs
        out["rows"].append(row)
        print(json.dumps(row), flush=True)
    print(json.dumps(out), flush=True)
    return 0


def run_isolated(args):
    """An isolated clip (the paper's spherically windowed dyadic kernel, Sec. 3, Eqs. (13)-(18)):
    a 40 x 40 nm absorber block, 60 nm thick (n = 0.94 + 0.04i, 2 nm cells), in a 256 x 256 nm
    transverse period (128 x 128 cells, vacuum around the block) with a z column of 256 nm
    (nf = 128); R = 83 nm exceeds the block's diameter, and period and column exceed its extent
    plus R. Two illuminations (6 deg s, 0 deg p), FP32 with FP64 refinement to --tol, no stack.
    Reported: solves/s over --steps solves of the pair and operator applications/s."""
    import torch
    from paper_2606_25541_b300 import psfd
    n, d, nslab, nf = 128, 2.0, 30, 128
    R = 1.001 * d * math.sqrt(20 ** 2 + 20 ** 2 + 30 ** 2)
    eps = np.ones((nslab, n, n), np.complex128)
    eps[:, 54:74, 54:74] = (0.94 + 0.04j) ** 2
    g = psfd.make_grid(n, n, nslab, nf, d, d, d, 13.5)
    stream = torch.cuda.current_stream()
    s = psfd.Solver(g, psfd.FP32_REFINED, 2, stream=stream)
    s.set_stack(np.zeros(0, np.complex128), np.zeros(0), 1.0)
    s.set_green(psfd.GREEN_SPHERICAL, R)
    s.set_potential(eps)
    kw = dict(tol=args.tol, inner_tol=args.inner_tol, max_iter=400, max_outer=12)

    def step():
        s.set_illumination([6.0, 0.0], [0.0, 0.0], [0, 1])
        return s.solve(**kw)

    for _ in range(max(args.warmup, 1)):
        rep = step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        rep = step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    u = torch.tensor(layouts.random_field((2, 3, nslab, n, n), seed=1), dtype=torch.complex64, device="cuda")
    y = torch.empty_like(u)
    s.apply(u, y)
    torch.cuda.synchronize()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(20):
        s.apply(u, y)
    a1.record(stream)
    torch.cuda.synchronize()
    out = {"mode": "isolated_clip", "workload": "block_40x40x60nm_in_256x256x256nm_2rhs", "R_nm": R,
           "tol": args.tol, "solves_per_s": 2e3 / ms, "ms_per_pair": ms, "iterations": rep["iterations"],
           "outer": rep["outer"], "relres": rep["relres"],
           "fp32_applications_per_s": 20e3 / a0.elapsed_time(a1)}
    s.close()
    print(json.dumps(out), flush=True)
    return 0


def run_differential(args):
    """Per-application cost of the two formulations of Sec. 3 on one seeded 64 x 64 x 30 clip at
    2 nm (one illumination, 6 deg): the differential PSFD operator on its z column (30 nm PML,
    34 nm vacuum spacer above and below the clip: 128 planes) and the Lippmann-Schwinger operator
    on the clip's own planes (nf = 64, no stack), both in FP64. Reported: applications/s of each,
    their ratio, and the differential apply's effective HBM rate (E and eps read, out written
    once: 112 bytes per cell), so that the preconditioner study's operator counts convert to
    time."""
    import torch
    from paper_2606_25541_b300 import psfd
    n, d, nslab, nf, npml, nz = 64, 2.0, 30, 64, 15, 128
    prob = layouts.small_clip(nx=n, ny=n, nslab=nslab, dx=d, dz=d, seed=7, stack=layouts.empty_stack(),
                              theta=(6.0,), pol=(0,))
    eps_col = np.ones((nz, n, n), np.complex128)
    z0 = (nz - nslab) // 2
    eps_col[z0:z0 + nslab] = prob.eps
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream()
    reps = max(args.steps, 1) * 10

    def timed(fn):
        for _ in range(max(args.warmup, 3)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    eps_d = torch.from_numpy(eps_col).to(dev)
    E = torch.from_numpy(layouts.random_field((3, nz, n, n), seed=2)).to(dev)
    out, work = torch.empty_like(E), torch.empty_like(E)
    sp = stream.cuda_stream

    def diff_apply():
        st = psfd.apply_differential(n, nz, npml, d, d, 13.5, 1.0, 6.0, 0.0, eps_d, E, out, work, stream=sp)
        if st != 0:
            raise RuntimeError(psfd.strerror(st))

    ms_diff = timed(diff_apply)
    g = psfd.make_grid(n, n, nslab, nf, d, d, d, 13.5)
    s = psfd.Solver(g, psfd.FP64, 1, stream=stream)
    s.set_stack(np.zeros(0, np.complex128), np.zeros(0), 1.0)
    s.set_potential(prob.eps)
    s.set_illumination([6.0], [0.0], [0])
    u = torch.from_numpy(layouts.random_field((1, 3, nslab, n, n), seed=3)).to(dev)
    y = torch.empty_like(u)
    ms_ls = timed(lambda: s.apply(u, y, precision=psfd.FP64))
    s.close()
    cells = nz * n * n
    print(json.dumps({"mode": "differential_vs_ls_apply", "workload": "clip_64x64x30_2nm_column_128_planes",
                      "dtype": "c128", "differential_ms": ms_diff, "differential_applications_per_s": 1e3 / ms_diff,
                      "differential_gbs_112B_per_cell": 112.0 * cells / (ms_diff * 1e6),
                      "ls_ms": ms_ls, "ls_applications_per_s": 1e3 / ms_ls,
                      "ratio_ls_over_differential_ms": ms_ls / ms_diff, "reps": reps}), flush=True)
    return 0


def run_autotune(args):
    """The autotuner on the workload sizes: per grid and precision, one operator application
    with the built-in tile shapes against the tuned ones (psfd_autotune, forced)."""
    import torch
    from paper_2606_25541_b300 import psfd
    torch.cuda.set_device(0)
    serving = layouts.serving_requests(40, sizes=(64, 128, 256, 384, 512))
    by_size = {}
    for r in serving:
        by_size.setdefault((r.nx, r.ny, r.nslab, r.nf), r)
    cases = [("line_space_128x128x60_nf128_18rhs", layouts.line_space_clip(), (psfd.FP32_REFINED, psfd.FP64)),
             ("manhattan_256x256x60_nf128_2rhs", layouts.manhattan_clip(), (psfd.FP32_REFINED, psfd.FP64))]
    for key in sorted(by_size, key=lambda k: k[0] * k[1])[:: max(1, len(by_size) // 4)]:
        r = by_size[key]
        cases.append((f"serving_{key[0]}x{key[1]}x{key[2]}_nf{key[3]}_{r.n_rhs}rhs", r, (psfd.FP32_REFINED,)))
    big = layouts.curvilinear_clip()
    big = big.with_illumination(big.theta_deg[:2], big.phi_deg[:2], big.pol[:2])
    cases.append(("curvilinear_1024x1024x60_nf160_2rhs", big, (psfd.FP32_REFINED,)))
    rows = []
    for name, prob, precisions in cases:
        for prec in precisions:
            s = psfd.Solver.from_problem(prob, prec)
            rep = s.autotune(force=True)
            s.close()
            rows.append({"workload": name, "precision": "fp32" if prec == psfd.FP32_REFINED else "fp64", **rep,
                         "speedup": rep["default_ms"] / rep["tuned_ms"]})
            torch.cuda.empty_cache()
    print(json.dumps({"mode": "autotune", "rows": rows}), flush=True)
    return 0


def run_precond_study(args):
    """The preconditioner comparison of Sec. 3 on the GPU: one seeded Manhattan clip in free
    space (no stack), 6 deg s, solved to relative residual 1e-8 by GMRES(60) three ways:
    the differential PSFD with PMLs (psfd_solve_differential) without and with the spectral
    damping preconditioner, and the Lippmann-Schwinger form (the Green's function as
    preconditioner; psfd_solve, FP64 GMRES(24), the device's largest cycle). Reports operator
    applications and wall time, relative to the unpreconditioned solve (the paper's table
    reports both)."""
    import torch
    from paper_2606_25541_b300 import psfd
    torch.cuda.set_device(0)
    dev = torch.device("cuda:0")
    rows = {}
    for n, dx, dz, nslab, spacer, pml in ((32, 4.0, 2.0, 14, 20.0, 30.0), (64, 2.0, 2.0, 14, 20.0, 30.0)):
        prob = layouts.small_clip(nx=n, ny=n, nslab=nslab, dx=dx, dz=dz, seed=21, stack=layouts.empty_stack(),
                                  theta=(6.0,), phi=(0.0,), pol=(0,))
        # the differential column (input preparation): PML, spacer, slab, spacer, PML, and the
        # scattered-field source k0^2 (eps - eps_bg) E_inc with E_inc = s exp(-i beta z), s-polarised
        ns, npml = int(round(spacer / dz)), int(round(pml / dz))
        nz = 2 * npml + 2 * ns + nslab
        eps = np.full((nz, n, n), prob.eps_bg, np.complex128)
        eps[npml + ns:npml + ns + nslab] = prob.eps
        k0 = 2 * math.pi / prob.wavelength
        th = math.radians(6.0)
        beta = k0 * math.cos(th)
        inc = np.exp(-1j * beta * np.arange(nz) * dz)
        b = np.zeros((3, nz, n, n), np.complex128)
        b[1] = k0 * k0 * (eps - prob.eps_bg) * inc[:, None, None]  # s = (-sin 0, cos 0, 0)
        epsd = torch.from_numpy(eps).to(dev)
        bd = torch.from_numpy(b).to(dev)
        row = {"grid": [n, n, nz], "slab_planes": nslab, "dx_nm": dx, "dz_nm": dz}
        for name, pc in (("none", 0), ("spectral_damping", 1)):
            x = torch.zeros_like(bd)
            t0 = time.perf_counter()
            st, mv, rel = psfd.solve_differential(n, nz, npml, dx, dz, prob.wavelength, prob.eps_bg, 6.0, 0.0, epsd,
                                                  bd, x, precond=pc, restart=60, max_matvecs=40000, rtol=1e-8)
            torch.cuda.synchronize()
            row[name] = {"matvecs": mv, "relres": rel, "seconds": time.perf_counter() - t0, "status": st}
        s = psfd.Solver.from_problem(prob, psfd.FP64)
        s.solve(tol=1e-8, max_iter=2000, krylov=psfd.GMRES, restart=24)  # warm-up (graph capture)
        s.set_illumination(prob.theta_deg, prob.phi_deg, prob.pol)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rep = s.solve(tol=1e-8, max_iter=2000, krylov=psfd.GMRES, restart=24)
        torch.cuda.synchronize()
        row["lippmann_schwinger"] = {"matvecs": rep["iterations"], "relres": rep["relres"],
                                     "seconds": time.perf_counter() - t0}
        s.close()
        t_none = row["none"]["seconds"]
        for k in ("none", "spectral_damping", "lippmann_schwinger"):
            row[k]["relative_wall_time"] = row[k]["seconds"] / t_none
        rows[f"manhattan_{n}x{n}x{nslab}"] = row
    print(json.dumps({"mode": "precond_study", **rows}), flush=True)
    return 0


def run_zdft(args):
    print(json.dumps({"mode": "zdft", "workload": "manhattan_256x256x60_nf128_6columns_sets", **zdft_rows()}),
          flush=True)
    return 0


def zdft_rows() -> dict:
    """The z pass's forward transform on the 256 x 256 x 60 Manhattan clip's columns (3
    components x 2 illuminations): CUDA-core register transform vs split-BF16 tensor-core DFT
    products, time per launch (CUDA events, 20 launches after 3), algorithmic HBM rate (60
    planes read, 128 bins written, 8 B each), tensor-core rate of the products, and the error
    against an FP64 DFT of a sample of columns."""
    import torch
    from paper_2606_25541_b300 import psfd
    torch.cuda.set_device(0)
    n, nslab, nsets = 256, 60, 6
    x = torch.tensor(layouts.random_field((nsets, nslab, n, n), seed=12), dtype=torch.complex64, device="cuda")
    out = torch.empty((nsets, 128, n, n), dtype=torch.complex64, device="cuda")
    xs = x[:, :, :8].cpu().numpy().astype(np.complex128)
    full = np.zeros((nsets, 128, 8, n), np.complex128)
    full[:, 1:nslab + 1] = xs
    ref = np.fft.fft(full, axis=1)
    rows = {}
    cols = nsets * n * n
    for method, name in ((0, "cuda_cores_register_fft"), (1, "tensor_cores_split_bf16")):
        for _ in range(3):
            psfd.zdft_measure(method, x, out)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(20):
            psfd.zdft_measure(method, x, out)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 20
        got = out[:, :, :8].cpu().numpy().astype(np.complex128)
        err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        bytes_ = cols * (nslab + 128) * 8.0
        row = {"ms": ms, "algorithmic_GBps": bytes_ / (ms * 1e-3) / 1e9, "rel_err_vs_fp64": err,
               "status": psfd.zdft_status()}
        if method == 1:
            flops = 2 * 3 * 2.0 * 128 * 64 * 2 * cols  # 2 matrices x 3 products x 2 M K N
            row["tensor_TFLOPs"] = flops / (ms * 1e-3) / 1e12
        rows[name] = row
    return rows


def run_small(args):
    """The contact-hole clip (32 x 32 x 30 at 2 nm, nf = 64, one s-polarised plane wave at 6 deg)
    solved to relative residual 1e-10 in FP64 and in FP32 with FP64 refinement, with the
    Krylov step replayed as a CUDA graph and with its kernels launched one by one. A clip this
    small is L2-resident: launch overhead, not HBM, decides its speed. Wall time per solve
    (set_illumination + solve, host synchronised), mean over --steps solves after --warmup."""
    import torch
    from paper_2606_25541_b300 import psfd
    prob = layouts.contact_hole_clip()
    out = {"mode": "small_clip", "workload": "contact_hole_32x32x30_nf64_1rhs", "tol": 1e-10}
    steps = max(args.steps, 20)
    for name, prec in (("fp64", psfd.FP64), ("fp32_refined", psfd.FP32_REFINED)):
        for graphs in (True, False):
            s = psfd.Solver.from_problem(prob, prec)
            s.set_graphs(graphs)
            kw = dict(tol=1e-10, inner_tol=1e-4, max_iter=400, max_outer=12)
            for _ in range(max(args.warmup, 3)):
                s.set_illumination(prob.theta_deg, prob.phi_deg, prob.pol)
                s.solve(**kw)
            torch.cuda.synchronize()
            n0 = psfd.launch_count()
            t0 = time.perf_counter()
            for _ in range(steps):
                s.set_illumination(prob.theta_deg, prob.phi_deg, prob.pol)
                rep = s.solve(**kw)
            torch.cuda.synchronize()
            dt = (time.perf_counter() - t0) / steps
            out[f"{name}_{'graphs' if graphs else 'launches'}"] = {
                "ms_per_solve": dt * 1e3, "solves_per_s": 1.0 / dt, "iterations": rep["iterations"],
                "relres": rep["relres"], "kernels_per_solve": (psfd.launch_count() - n0) / steps}
            s.close()
    print(json.dumps(out), flush=True)
    return 0


def run_fixed_point(args):
    """The paper's outer fixed-point loop (Eq. (8): free-space solves with R rebuilt from the
    previous step's mask field) against the folded operator, on the 128 x 128 x 60 line/space
    clip with its 18 illuminations, FP32 with FP64 refinement, both to the same folded FP64
    residual (--tol), for Ru + n x Mo/Si stacks (--fp-bilayers; 0 = the Ru cap on Si alone).
    Reported per stack: seconds, Krylov iterations, outer steps of the loop, and the relative
    difference of the reflected orders between the two (normwise over all illuminations)."""
    import dataclasses
    import torch
    from paper_2606_25541_b300 import psfd
    base = layouts.line_space_clip(seed=2)
    stream = torch.cuda.current_stream()
    kw = dict(tol=args.tol, inner_tol=args.inner_tol, max_iter=400, max_outer=12, raise_on_error=False)
    out = {"mode": "fixed_point_vs_folded", "workload": WORKLOAD, "tol": args.tol, "stacks": []}
    for nb in (int(v) for v in args.fp_bilayers.split(",")):
        n_l, d_l, n_s = layouts.ru_mosi_stack(nb)
        prob = dataclasses.replace(base, n_layers=n_l, d_layers=d_l, n_sub=n_s)
        row = {"bilayers": nb}
        orders = {}
        for name in ("folded", "fixed_point"):
            s = psfd.Solver.from_problem(prob, psfd.FP32_REFINED, stream=stream)
            s.solve(**kw)  # warm-up: tables, pool and the first-call paths
            s.set_illumination(prob.theta_deg, prob.phi_deg, prob.pol)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rep = s.solve(**kw) if name == "folded" else s.solve_fixed_point(max_steps=200, **kw)
            torch.cuda.synchronize()
            row[name] = {"seconds": time.perf_counter() - t0, "iterations": rep["iterations"],
                         "outer": rep["outer"], "relres": rep["relres"], "status": psfd.strerror(rep["status"])}
            if name == "fixed_point":
                row[name]["outer_steps_per_rhs"] = [int(np.sum(s.residual_history(i)["kind"] == 2))
                                                    for i in range(prob.n_rhs)]
            orders[name] = orders_all(s, prob.n_rhs)
            s.close()
        row["orders_rel_diff"] = orders_rel_err(orders["fixed_point"], orders["folded"])
        out["stacks"].append(row)
        print(json.dumps(row), flush=True)
    print(json.dumps(out), flush=True)
    return 0


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def reduce_max(value: float, world: int, device=None) -> float:
    """Maximum of a float over all ranks (identity when world == 1)."""
    if world == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle sample (the baseline and the reference arm)
# ---------------------------------------------------------------------------
ORACLE_TIGHT = 1e-11      # the oracle solve the GPU orders are checked against
ORACLE_BYTES_PER_PROC = 3e9


def oracle_apply_seconds(prob, i: int, reps: int = 1) -> float:
    """Mean wall time of one oracle operator application (illumination i) on one thread."""
    import oracle
    from oracle.parallel import _one_thread
    with _one_thread():
        ctx = oracle.setup_rhs(prob, i)
        u = oracle.rhs_vector(ctx)
        t0 = time.perf_counter()
        for _ in range(reps):
            oracle.apply_operator(ctx, u)
        return (time.perf_counter() - t0) / reps


def cpu_model() -> str:
    """The host CPU's model name (from /proc/cpuinfo) and its logical core count."""
    name = "unknown"
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    name = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return f"{name}, {os.cpu_count()} logical cores on the host"


def orders_vs(got: dict, ref: dict) -> float:
    """Relative 2-norm difference of the order amplitudes of one illumination, matched by (m, n)."""
    key = {(int(m), int(n)): k for k, (m, n) in enumerate(zip(ref["m"], ref["n"]))}
    idx = [key[(int(m), int(n))] for m, n in zip(got["m"], got["n"])]
    assert len(idx) == len(ref["m"])
    return float(np.linalg.norm(got["amp"] - ref["amp"][idx]) / np.linalg.norm(ref["amp"]))


def cpu_baseline(prob, rtol: float, gpu_orders: list):
    """The oracle timed on the host: one illumination on one core (the baseline value), the same
    per operator application, and the batch on all usable cores; plus the GPU orders of that
    illumination checked against the oracle solved to 1e-11."""
    from oracle.parallel import apply_many, solve_timed, usable_processes
    i = 5
    r = solve_timed(prob, i, ORACLE_TIGHT, marks=(rtol,))
    t_tol = r["at"][rtol]["seconds"]
    n_app = r["at"][rtol]["iterations"] + 1  # GMRES applications + the one for the orders
    t_app = oracle_apply_seconds(prob, i)
    # all cores: concurrent applications (bounded), scaled to solves by the single-core ratio of
    # a solve's time to its applications' time (which carries GMRES's orthogonalisation)
    procs = usable_processes(prob.n_rhs, ORACLE_BYTES_PER_PROC)
    reps = 2
    per, wall = apply_many(prob, range(procs), reps, procs)
    app_rate = procs * reps / max(per)
    overhead = t_tol / (n_app * t_app)
    return {
        "value": 1.0 / t_tol, "unit": UNIT, "cores": 1, "kind": "oracle", "host": cpu_model(),
        "sample": f"illumination {i} of 18 (theta {prob.theta_deg[i]:g}, phi {prob.phi_deg[i]:g}, pol "
                  f"{int(prob.pol[i])}) solved by the FP64 oracle (its own FFT, GMRES) on one thread: "
                  f"{t_tol:.1f} s to relative residual {rtol:g} ({r['at'][rtol]['iterations']} iterations, "
                  f"orders included), timed within one solve to {ORACLE_TIGHT:g} ({r['iterations']} "
                  f"iterations, {r['seconds']:.1f} s)",
        "per_application": {"value": 1.0 / t_app, "unit": "operator applications/s", "cores": 1,
                            "seconds": t_app},
        "all_cores": {"value": app_rate / (n_app * overhead), "unit": UNIT, "cores": procs,
                      "per_application": {"value": app_rate, "unit": "operator applications/s"},
                      "sample": f"{reps} oracle operator applications of each of illuminations 0-{procs - 1} at "
                                f"once, one single-threaded process each (spawn pool; slowest {max(per):.1f} s, "
                                f"{wall:.1f} s wall with start-up); solves/s = applications/s / ({n_app} "
                                f"applications per solve x {overhead:.2f}, the single-core ratio of solve time "
                                f"to application time)"},
        "order_error_vs_oracle_1e-11": {"illumination": i,
                                        "rel_err": orders_vs(gpu_orders[i], r["orders"])},
    }


def run_reference(args):
    """The reference arm: the oracle on the host. One step is a bounded sample: one oracle
    operator application (one thread) on the next illumination; solves/s follow from the
    applications one oracle solve needs (GMRES iterations + 1 for the orders, measured by a full
    solve before the warm-up). GMRES's orthogonalisation is left out of the steps, so the value
    is an upper bound of the oracle's solves/s."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from oracle.parallel import solve_timed
    prob = layouts.line_space_clip(seed=2)
    rtol = args.tol
    full = solve_timed(prob, 5, rtol)
    n_app = full["iterations"] + 1
    for w in range(args.warmup):
        oracle_apply_seconds(prob, w % prob.n_rhs)
    times = [oracle_apply_seconds(prob, (args.warmup + k) % prob.n_rhs) for k in range(args.steps)]
    t_app = sum(times) / len(times)
    value = 1.0 / (n_app * t_app)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_app,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "reference_step": "one oracle operator application (one illumination, "
                                                           "one thread); solves/s = 1 / (applications per "
                                                           "solve x seconds per application)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "host": cpu_model(),
                         "sample": f"{args.steps} oracle operator applications on one thread, "
                                   f"{t_app:.2f} s each; one oracle solve to {rtol:g} takes {n_app} "
                                   f"applications (illumination 5: {full['seconds']:.1f} s in full)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
def orders_all(solver, n_rhs):
    return [solver.diffraction_orders(i) for i in range(n_rhs)]


class SolverGroup:
    """A batch of illuminations split over k contexts, each on its own stream, solved together
    through psfd_solve_group (k = 1: one context and psfd_solve). Each context's inputs are set on
    its own stream after the main stream's work; the main stream waits for every context's
    stream after a solve, so events on it bracket the whole batch."""

    def __init__(self, psfd, prob, precision, k, main_stream, dev):
        import torch
        self.psfd = psfd
        k = max(1, min(int(k), prob.n_rhs))
        cut = np.linspace(0, prob.n_rhs, k + 1).round().astype(int)
        self.parts = [prob.with_illumination(prob.theta_deg[a:b], prob.phi_deg[a:b], prob.pol[a:b])
                      for a, b in zip(cut[:-1], cut[1:])]
        self.main = main_stream
        self.streams = [main_stream] + [torch.cuda.Stream(dev) for _ in range(k - 1)]
        self.solvers = [psfd.Solver.from_problem(p, precision, stream=st) for p, st in zip(self.parts, self.streams)]

    def set_inputs(self, eps):
        for s, p, st in zip(self.solvers, self.parts, self.streams):
            st.wait_stream(self.main)
            s.set_potential(eps)
            s.set_illumination(p.theta_deg, p.phi_deg, p.pol)

    def solve(self, **kw):
        if len(self.solvers) == 1:
            reps = [self.solvers[0].solve(**kw)]
        else:
            reps = self.psfd.solve_group(self.solvers, **kw)
        for st in self.streams[1:]:
            self.main.wait_stream(st)
        return {"iterations": max(r["iterations"] for r in reps), "outer": max(r["outer"] for r in reps),
                "relres": max(r["relres"] for r in reps)}

    def orders(self):
        return [s.diffraction_orders(i) for s, p in zip(self.solvers, self.parts) for i in range(p.n_rhs)]

    def close(self):
        for s in self.solvers:
            s.close()


def orders_rel_err(a, b):
    num = sum(float(np.sum(np.abs(x["amp"] - y["amp"]) ** 2)) for x, y in zip(a, b))
    den = sum(float(np.sum(np.abs(y["amp"]) ** 2)) for y in b)
    return math.sqrt(num / den)


def run_ours(args):
    import torch
    from paper_2606_25541_b300 import psfd

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    prob = layouts.line_space_clip(seed=2 + rank)
    if args.profile_only and args.rhs < prob.n_rhs:  # a smaller batch for full ncu captures
        k = args.rhs
        prob = prob.with_illumination(prob.theta_deg[:k], prob.phi_deg[:k], prob.pol[:k])
    n_rhs = prob.n_rhs
    solve_kw = dict(tol=args.tol, inner_tol=args.inner_tol, max_iter=400, max_outer=12, check_every=4,
                    krylov=psfd.GMRES if args.krylov == "gmres" else psfd.BICGSTAB, restart=args.restart)

    eps_dev = torch.from_numpy(prob.eps).to(dev)
    th, ph, po = prob.theta_deg, prob.phi_deg, prob.pol

    def step_single(s, kw=solve_kw):
        s.set_potential(eps_dev)
        s.set_illumination(th, ph, po)
        return s.solve(**kw)

    if args.profile_only:
        solver = psfd.Solver.from_problem(prob, psfd.FP32_REFINED, stream=stream)
        if args.plain_launches:  # every kernel its own launch (ncu lists no kernels inside a graph's loop)
            solver.set_graphs(False)
        step_single(solver)
        torch.cuda.synchronize()
        return 0

    # the batch as args.groups contexts solved side by side, each on its own stream
    group = SolverGroup(psfd, prob, psfd.FP32_REFINED, args.groups, stream, dev)

    def step(g, kw=solve_kw, eps=None):
        g.set_inputs(eps_dev if eps is None else eps)
        return g.solve(**kw)

    for _ in range(args.warmup):
        rep = step(group)
    torch.cuda.synchronize()
    # first use of this grid: time the tile shapes once (bitwise the same results), untimed
    tuned = None if args.no_autotune else group.solvers[0].autotune()
    step(group)
    torch.cuda.synchronize()

    # reference orders for the order error the metric is quoted at: FP64 solve to 1e-11 (untimed)
    sref = psfd.Solver.from_problem(prob, psfd.FP64, stream=stream)
    sref.solve(tol=1e-11, max_iter=800)
    orders_ref = orders_all(sref, n_rhs)
    sref.close()

    def order_error(orders):
        return {"normwise": orders_rel_err(orders, orders_ref),
                "max_per_illumination": max(orders_rel_err([a], [b]) for a, b in zip(orders, orders_ref))}

    # ---- timed region: device-resident inputs ----
    clocks = ClockSampler(torch.cuda.current_device())
    if rank == 0:
        clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    n0 = psfd.launch_count()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    reps = []
    for k in range(args.steps):
        reps.append(step(group))
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = psfd.launch_count() - n0
    clk = clocks.stop() if rank == 0 else None
    per_step = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    t_ms = reduce_max(ev[0].elapsed_time(ev[-1]), world, dev)
    value = n_rhs * args.steps * world / (t_ms * 1e-3)

    # ---- per-kernel timing of the same workload: one context of the whole batch, launches one
    #      after another (CUDA events on its stream; per-pass records need sequential launches) ----
    psolver = psfd.Solver.from_problem(prob, psfd.FP32_REFINED, stream=stream)
    step_single(psolver)
    torch.cuda.synchronize()
    psfd.profile_enable(True)
    for _ in range(args.steps):
        step_single(psolver)
    torch.cuda.synchronize()
    psfd.profile_enable(False)
    prof = psfd.profile_read()
    total_prof_ms = sum(v["ms"] for v in prof.values())
    psolver.close()

    # ---- end to end through the C ABI with host buffers: eps copied once per step from pinned
    #      host memory (every context reads the device copy), the orders read back ----
    eps_host = torch.from_numpy(prob.eps).pin_memory()
    d2h = 0

    def e2e_step():
        nonlocal d2h
        eps_in = eps_host.to(dev, non_blocking=True)
        step(group, eps=eps_in)
        out = group.orders()
        d2h = sum(o["m"].nbytes + o["n"].nbytes + o["amp"].nbytes + o["a_s"].nbytes + o["a_p"].nbytes
                  + o["eff"].nbytes for o in out)
        return out

    e2e_step()
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        orders32 = e2e_step()
    torch.cuda.synchronize()
    barrier(world)
    t_e2e = reduce_max(time.perf_counter() - t0, world, dev)
    h2d = prob.eps.nbytes + th.nbytes + ph.nbytes + po.nbytes

    # ---- plain FP64 path on the same batch (grouped the same way), and the order difference ----
    fp64 = None
    if not args.no_fp64:
        s64 = SolverGroup(psfd, prob, psfd.FP64, args.groups, stream, dev)
        step(s64)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rep64 = step(s64)
        e1.record(stream)
        torch.cuda.synchronize()
        t64 = reduce_max(e0.elapsed_time(e1), world, dev)
        orders64 = s64.orders()
        fp64 = {"value": n_rhs * world / (t64 * 1e-3), "unit": UNIT, "ms_per_step": t64, "tol": args.tol,
                "iterations": rep64["iterations"], "relres": rep64["relres"],
                "order_error_vs_fp64_1e-11": order_error(orders64),
                "order_rel_err_fp32_refined_vs_fp64": orders_rel_err(orders32, orders64)}
        s64.close()

    # ---- the same FP32 + refinement step solved 30x tighter (FP64 residual 1e-8) ----
    tight_kw = dict(solve_kw, tol=DEFAULT_TOL, inner_tol=DEFAULT_INNER_TOL)

    step(group, tight_kw)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        rep_t = step(group, tight_kw)
    e1.record(stream)
    torch.cuda.synchronize()
    t_tight = reduce_max(e0.elapsed_time(e1), world, dev)
    tight = {"value": n_rhs * args.steps * world / (t_tight * 1e-3), "unit": UNIT, "tol": DEFAULT_TOL,
             "inner_tol": DEFAULT_INNER_TOL, "iterations": rep_t["iterations"], "outer": rep_t["outer"],
             "relres": rep_t["relres"], "order_error_vs_fp64_1e-11": order_error(group.orders())}

    # the other workloads, sampled: cfg 3's precision sweep (256^2 Manhattan, both paths and the
    # tensor-core stage) and cfg 5's large clip (1024^2, 2 of its 8 illuminations), at 1e-8
    extra = {}
    if world == 1 and not args.no_extra:
        group.close()
        torch.cuda.empty_cache()
        extra["precision_sweep_manhattan_256"] = precision_sweep(DEFAULT_TOL, DEFAULT_INNER_TOL, 1, 1)
        torch.cuda.empty_cache()
        extra["large_clip_curvilinear_1024_2rhs"] = large_clip(DEFAULT_TOL, DEFAULT_INNER_TOL, 1, n_rhs=2)
        torch.cuda.empty_cache()
        group = None

    serving = None
    if args.serve > 0 and world == 1:
        sizes = tuple(int(s) for s in args.serve_sizes.split(","))
        serving = run_serving(args.serve, sizes, args.tol, args.inner_tol, rounds=args.serve_rounds)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(prob, args.tol, orders32)

    if rank != 0:
        return 0

    hbm_peak, peak_kind = measured_peaks()
    kernels = {}
    for name, v in prof.items():
        if v["launches"] == 0:
            continue
        kernels[name] = {"launches": v["launches"], "ms": round(v["ms"], 4),
                         "share_of_profiled": round(v["ms"] / total_prof_ms, 4),
                         "GBps": round(v["bytes"] / (v["ms"] * 1e-3) / 1e9, 1),
                         "GFLOPs": round(v["flops"] / (v["ms"] * 1e-3) / 1e9, 1)}
    dom = max(prof, key=lambda k: prof[k]["ms"])
    d = prof[dom]
    if dom.endswith("fp64"):
        achieved = d["flops"] / (d["ms"] * 1e-3) / 1e12
        roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": FP64_NOMINAL_TFLOPS,
                    "unit": "TFLOP/s", "frac": achieved / FP64_NOMINAL_TFLOPS,
                    "traffic": ncu_traffic(dom, d["bytes"] / max(d["launches"], 1)),
                    "peak_kind": "nominal FP64 (148 SMs x 2 FP64 FMA/clk x 2.03 GHz class)"}
    else:
        achieved = d["bytes"] / (d["ms"] * 1e-3) / 1e9
        roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved / hbm_peak, "traffic": ncu_traffic(dom, d["bytes"] / max(d["launches"], 1)),
                    "peak_kind": peak_kind}
    lat = sorted(per_step)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": [prob.nx, prob.ny, prob.nslab, prob.nf], "dx_nm": prob.dx,
                   "n_rhs": n_rhs, "precision": f"FP32 {'GMRES' if args.krylov == 'gmres' else 'BiCGStab'} inside FP64 defect correction",
                   "tol": args.tol, "inner_tol": args.inner_tol, "parallelism": f"replicas x{world}",
                   "contexts": f"{len(group.solvers) if group else args.groups} contexts of the batch solved side by side on their own streams (psfd_solve_group)",
                   "l2": f"inputs larger than L2: {solver_bytes(prob) / 1e9:.1f} GB working set per step"},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "what": "per-step (18-illumination batch) device time"},
        "iterations": reps[-1]["iterations"], "outer": reps[-1]["outer"], "relres": reps[-1]["relres"],
        "order_error_vs_fp64_1e-11": order_error(orders32),
        "order_error_vs_oracle_1e-11": cpu["order_error_vs_oracle_1e-11"] if cpu else None,
        "roofline": roofline, "kernels": kernels, "autotune": tuned,
        "cpu_baseline": cpu,
        "e2e": {"value": n_rhs * args.steps * world / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "clocks": clk,
        "fp64_plain": fp64,
        "fp32_refined_at_tol_1e-8": tight,
        "serving": serving,
        **extra,
    }
    print(json.dumps(line), flush=True)
    if group is not None:
        group.close()
    return 0


def ncu_traffic(kernel: str, alg_bytes_per_launch: float):
    """DRAM bytes per launch of `kernel` from the committed ncu capture (profiles/ncu_traffic.json),
    scaled from the captured launch by algorithmic bytes; None if absent or if the kernel sources
    changed since the capture."""
    import hashlib
    here = os.path.dirname(os.path.abspath(__file__))
    path = os.path.join(here, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    h = hashlib.sha256()
    for src in rec["sources"]:
        with open(os.path.join(here, src), "rb") as f:
            h.update(f.read())
    k = rec["kernels"].get(kernel)
    if k is None or h.hexdigest()[:16] != rec["sources_sha256_16"]:
        return None
    return k["dram_bytes"] / k["algorithmic_bytes"] * alg_bytes_per_launch


def solver_bytes(prob) -> float:
    from paper_2606_25541_b300 import psfd
    g = psfd.make_grid(prob.nx, prob.ny, prob.nslab, prob.nf, prob.dx, prob.dy, prob.dz, prob.wavelength,
                       prob.eps_bg)
    return float(psfd.workspace_bytes(g, psfd.FP32_REFINED, prob.n_rhs))


def main(argv=None):
    args = parse_args(argv)
    headline = not (args.apply or args.sweep or args.large or args.crosscheck or args.fixed_point or args.small
                    or args.layers or args.isolated or args.differential or args.autotune or args.zdft
                    or args.precond_study)
    if args.tol is None:
        args.tol = HEADLINE_TOL if headline else DEFAULT_TOL
    if args.inner_tol is None:
        args.inner_tol = HEADLINE_INNER_TOL if headline else DEFAULT_INNER_TOL
    if args.impl == "reference":
        return run_reference(args)
    if args.apply:
        return run_apply(args)
    if args.sweep:
        return run_sweep(args)
    if args.large:
        return run_large(args)
    if args.crosscheck:
        return run_crosscheck(args)
    if args.fixed_point:
        return run_fixed_point(args)
    if args.small:
        return run_small(args)
    if args.autotune:
        return run_autotune(args)
    if args.zdft:
        return run_zdft(args)
    if args.precond_study:
        return run_precond_study(args)
    if args.layers:
        return run_layers(args)
    if args.isolated:
        return run_isolated(args)
    if args.differential:
        return run_differential(args)
    if args.serve_only:
        sizes = tuple(int(s) for s in args.serve_sizes.split(","))
        print(json.dumps({"mode": "serving", **run_serving(args.serve, sizes, args.tol, args.inner_tol,
                                                           slots=args.serve_slots, budget_gb=args.serve_budget_gb,
                                                           rounds=args.serve_rounds,
                                                           fp64_sample=args.serve_fp64_sample)}), flush=True)
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
