"""ctypes binding of ``libpsfd.so`` (C ABI in ``include/psfd.h``).

Argument marshalling only: every step of the solver runs in the library's CUDA
kernels. Host arrays are numpy complex128/float64/int32; device arrays are torch
CUDA tensors, passed by pointer. Loading fails loudly if the library is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpsfd.so")

OK = 0
E_ARG, E_NOMEM, E_BUDGET, E_CUDA, E_NOT_CONVERGED, E_BREAKDOWN, E_ANOMALY, E_TIMEOUT, E_STATE = \
    -1, -2, -3, -4, -5, -6, -7, -8, -9
FP64, FP32_REFINED = 0, 1
FP64_DF = 2  # apply only: FP64 data, z pass in double-float
RESID_FP64, RESID_DFLOAT = 0, 1
HOST, DEVICE = 0, 1


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nslab", ctypes.c_int), ("nf", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("wavelength", ctypes.c_double), ("eps_bg", ctypes.c_double)]


BICGSTAB, GMRES = 0, 1
GREEN_PERIODIC, GREEN_SPHERICAL = 0, 1


class SolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("max_outer", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("check_every", ctypes.c_int), ("krylov", ctypes.c_int),
                ("restart", ctypes.c_int), ("reserved", ctypes.c_int * 2)]


class Report(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("outer", ctypes.c_int), ("relres", ctypes.c_double),
                ("seconds", ctypes.c_double), ("status", ctypes.c_int), ("reserved", ctypes.c_int * 3)]


class Request(ctypes.Structure):
    _fields_ = [("grid", Grid), ("n_layers", ctypes.c_int), ("n_complex", ctypes.POINTER(ctypes.c_double)),
                ("thickness_nm", ctypes.POINTER(ctypes.c_double)), ("n_sub", ctypes.POINTER(ctypes.c_double)),
                ("eps", ctypes.POINTER(ctypes.c_double)), ("n_rhs", ctypes.c_int),
                ("theta_deg", ctypes.POINTER(ctypes.c_double)), ("phi_deg", ctypes.POINTER(ctypes.c_double)),
                ("pol", ctypes.POINTER(ctypes.c_int))]


class TuneReport(ctypes.Structure):
    _fields_ = [("default_ms", ctypes.c_double), ("tuned_ms", ctypes.c_double), ("zx", ctypes.c_int),
                ("rb", ctypes.c_int), ("cx", ctypes.c_int), ("candidates", ctypes.c_int), ("pf", ctypes.c_int)]


class PsfdError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"psfd status {status}: {msg}")
        self.status = status


_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)

_SIGS = {
    "psfd_strerror": (ctypes.c_char_p, [_I]),
    "psfd_last_error": (ctypes.c_char_p, [_P]),
    "psfd_supported_length": (_I, [_I]),
    "psfd_workspace_bytes": (_I, [ctypes.POINTER(Grid), _I, _I, ctypes.POINTER(ctypes.c_size_t)]),
    "psfd_create": (_I, [ctypes.POINTER(_P), ctypes.POINTER(Grid), _I, _I, ctypes.c_size_t, _P]),
    "psfd_destroy": (_I, [_P]),
    "psfd_set_stream": (_I, [_P, _P]),
    "psfd_set_stack": (_I, [_P, _I, _D, _D, _D]),
    "psfd_set_potential": (_I, [_P, _P, _I]),
    "psfd_set_illumination": (_I, [_P, _I, _D, _D, _IP]),
    "psfd_set_graphs": (_I, [_P, _I]),
    "psfd_set_device_loop": (_I, [_P, _I]),
    "psfd_set_residual_arith": (_I, [_P, _I]),
    "psfd_autotune": (_I, [_P, _I, ctypes.POINTER(TuneReport)]),
    "psfd_tune_set": (_I, [ctypes.POINTER(Grid), _I, _I, _I, _I, _I]),
    "psfd_tune_reset": (_I, []),
    "psfd_set_green": (_I, [_P, _I, ctypes.c_double]),
    "psfd_solve": (_I, [_P, ctypes.POINTER(SolveOpts), ctypes.POINTER(Report)]),
    "psfd_solve_group": (_I, [ctypes.POINTER(_P), _I, ctypes.POINTER(SolveOpts), ctypes.POINTER(Report)]),
    "psfd_solve_fixed_point": (_I, [_P, ctypes.POINTER(SolveOpts), _I, ctypes.c_double, ctypes.POINTER(Report)]),
    "psfd_num_orders": (_I, [_P, _I, _IP]),
    "psfd_diffraction_orders": (_I, [_P, _I, _I, _IP, _IP, _D, _D, _D]),
    "psfd_apply": (_I, [_P, _I, _I, _I, _P, _P]),
    "psfd_get_solution": (_I, [_P, _I, _P, _I]),
    "psfd_get_rhs": (_I, [_P, _I, _P, _I]),
    "psfd_set_initial_guess": (_I, [_P, _I, _P, _I]),
    "psfd_residual_history": (_I, [_P, _I, _I, _IP, _IP, _IP, _D]),
    "psfd_get_mode_tables": (_I, [_P, _I, _D, _D, _D]),
    "psfd_test_fft": (_I, [_I, _I, _I, _I, _P]),
    "psfd_zdft_measure": (_I, [_I, _I, _I, _I, _I, _P, _P, _P]),
    "psfd_zdft_status": (_I, [_IP]),
    "psfd_apply_fp32_static": (_I, [ctypes.POINTER(Grid), _I, _D, _D, _D, ctypes.c_double, ctypes.c_double, _P,
                                    _P, _P, _P]),
    "psfd_apply_differential": (_I, [_I, _I, _I, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double, _P, _P, _P, _P, _P]),
    "psfd_solve_differential": (_I, [_I, _I, _I, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double, _I, _P, _P, _P, _P, _I, _I,
                                     ctypes.c_double, _IP, _D, _P]),
    "psfd_solve_differential_work": (ctypes.c_size_t, [_I, _I, _I]),
    "psfd_server_create": (_I, [ctypes.POINTER(_P), _I, ctypes.c_size_t, _I, ctypes.POINTER(SolveOpts)]),
    "psfd_server_destroy": (_I, [_P]),
    "psfd_server_submit": (_I, [_P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_longlong)]),
    "psfd_server_progress": (_I, [_P, _IP]),
    "psfd_server_set_rounds": (_I, [_P, _I]),
    "psfd_server_set_max_running": (_I, [_P, _I]),
    "psfd_server_status": (_I, [_P, ctypes.c_longlong, _IP, _IP]),
    "psfd_server_orders": (_I, [_P, ctypes.c_longlong, _I, _I, _IP, _IP, _D, _D, _D]),
    "psfd_server_release": (_I, [_P, ctypes.c_longlong]),
    "psfd_server_memory": (_I, [_P, ctypes.POINTER(ctypes.c_size_t), _IP]),
    "psfd_launch_count": (_I, [ctypes.POINTER(ctypes.c_ulonglong)]),
    "psfd_profile_enable": (_I, [_I]),
    "psfd_profile_classes": (_I, []),
    "psfd_profile_get": (_I, [_I, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_ulonglong), _D, _D,
                              _D]),
}


def apply_fp32_static(grid: Grid, n_layers, thickness, n_sub, theta_deg, phi_deg, eps, u, out, stream=None):
    """out = A u through the allocation-free entry point (no context; the library's static
    device scratch holds every intermediate). eps: complex128 CUDA tensor (nslab, ny, nx);
    u, out: complex64 CUDA tensors (3, nslab, ny, nx). Returns the status code."""
    n = _c128(n_layers).reshape(-1)
    d = np.ascontiguousarray(thickness, dtype=np.float64).reshape(-1)
    ns = np.array([complex(n_sub).real, complex(n_sub).imag], dtype=np.float64)
    nn = n.view(np.float64) if n.size else np.zeros(2, np.float64)
    return load().psfd_apply_fp32_static(ctypes.byref(grid), int(n.size), _dptr(nn), _dptr(d if d.size else np.zeros(1)),
                                         _dptr(ns), float(theta_deg), float(phi_deg),
                                         ctypes.c_void_p(eps.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream))


def apply_differential(n, nz, n_pml, dx, dz, wavelength, eps_bg, theta_deg, phi_deg, eps, E, out, work,
                       stream=None):
    """out = curl curl E - k0^2 eps E (the differential PSFD operator, PML in z) on the GPU.
    eps: complex128 CUDA tensor (nz, n, n); E, out, work: complex128 CUDA tensors
    (3, nz, n, n), work being scratch. Returns the status code."""
    return load().psfd_apply_differential(int(n), int(nz), int(n_pml), float(dx), float(dz), float(wavelength),
                                          float(eps_bg), float(theta_deg), float(phi_deg),
                                          ctypes.c_void_p(eps.data_ptr()), ctypes.c_void_p(E.data_ptr()),
                                          ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(work.data_ptr()),
                                          _stream_ptr(stream))


def zdft_measure(method: int, x, out, stream=None):
    """Forward z transform of the z pass, x: complex64 CUDA tensor (nsets, nslab, ny, nx) ->
    out (nsets, 128, ny, nx); method 0 = CUDA cores, 1 = tensor cores (split BF16)."""
    ns, nslab, ny, nx = x.shape
    st = load().psfd_zdft_measure(int(method), int(nx), int(ny), int(ns), int(nslab), ctypes.c_void_p(x.data_ptr()),
                                  ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream))
    if st != OK:
        raise PsfdError(st, strerror(st))
    return out


def zdft_status() -> int:
    flag = ctypes.c_int(0)
    st = load().psfd_zdft_status(ctypes.byref(flag))
    if st != OK:
        raise PsfdError(st, strerror(st))
    return flag.value


def tune_set(grid: Grid, precision: int, zx: int = 0, rb: int = 0, cx: int = 0, pf: int = 0):
    """Store tile shapes for a grid and precision in the autotuner's table (0 = built-in)."""
    st = load().psfd_tune_set(ctypes.byref(grid), int(precision), int(zx), int(rb), int(cx), int(pf))
    if st != OK:
        raise PsfdError(st, strerror(st))


def tune_reset():
    """Empty the autotuner's table (every grid back to the built-in shapes)."""
    load().psfd_tune_reset()


def solve_differential(n, nz, n_pml, dx, dz, wavelength, eps_bg, theta_deg, phi_deg, eps, b, x, precond=0,
                       restart=60, max_matvecs=20000, rtol=1e-8, stream=None):
    """GMRES(restart) on the device for the differential system (psfd_solve_differential):
    eps, b, x complex128 CUDA tensors; precond 0 = none, 1 = spectral damping. Returns
    (status, matvecs, relres)."""
    import torch
    lib = load()
    need = int(lib.psfd_solve_differential_work(int(n), int(nz), int(restart)))
    work = torch.empty(need, dtype=torch.complex128, device=b.device)
    mv = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    st = lib.psfd_solve_differential(int(n), int(nz), int(n_pml), float(dx), float(dz), float(wavelength),
                                     float(eps_bg), float(theta_deg), float(phi_deg), int(precond),
                                     ctypes.c_void_p(eps.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                     ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(work.data_ptr()), int(restart),
                                     int(max_matvecs), float(rtol), ctypes.byref(mv), ctypes.byref(rel),
                                     _stream_ptr(stream))
    return st, mv.value, rel.value


def launch_count() -> int:
    """Kernels launched by the library since it was loaded."""
    n = ctypes.c_ulonglong(0)
    load().psfd_launch_count(ctypes.byref(n))
    return int(n.value)


def profile_enable(on: bool = True):
    load().psfd_profile_enable(int(bool(on)))


def profile_read():
    """Per-class totals since profile_enable(True): {name: {launches, ms, bytes, flops}}."""
    lib = load()
    out = {}
    for c in range(lib.psfd_profile_classes()):
        name = ctypes.c_char_p()
        n = ctypes.c_ulonglong(0)
        ms, by, fl = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_double(0)
        st = lib.psfd_profile_get(c, ctypes.byref(name), ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by),
                                  ctypes.byref(fl))
        if st != OK:
            raise PsfdError(st, strerror(st))
        out[name.value.decode()] = {"launches": int(n.value), "ms": ms.value, "bytes": by.value,
                                    "flops": fl.value}
    return out


def load(path: str = LIB_PATH):
    """Load the library (once). Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2606_25541_b300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def strerror(status: int) -> str:
    return load().psfd_strerror(status).decode()


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def supported_length(n: int) -> bool:
    return bool(load().psfd_supported_length(int(n)))


def make_grid(nx, ny, nslab, nf, dx, dy, dz, wavelength, eps_bg=1.0) -> Grid:
    return Grid(int(nx), int(ny), int(nslab), int(nf), float(dx), float(dy), float(dz), float(wavelength),
                float(eps_bg))


def workspace_bytes(grid: Grid, precision: int, max_rhs: int) -> int:
    out = ctypes.c_size_t(0)
    st = load().psfd_workspace_bytes(ctypes.byref(grid), int(precision), int(max_rhs), ctypes.byref(out))
    if st != OK:
        raise PsfdError(st, strerror(st))
    return int(out.value)


def solve_group(solvers, tol=1e-10, max_iter=500, max_outer=12, inner_tol=1e-4, check_every=4,
                raise_on_error=True, krylov=BICGSTAB, restart=0):
    """psfd_solve_group: solve several distinct Solvers at once, each on its own stream (its
    results are bitwise those of its own solve). Returns one report per solver."""
    n = len(solvers)
    lib = load()
    o = SolveOpts(float(tol), int(max_iter), int(max_outer), float(inner_tol), int(check_every), int(krylov),
                  int(restart))
    ctxs = (_P * n)(*[s.ctx for s in solvers])
    reps = (Report * n)()
    st = lib.psfd_solve_group(ctxs, n, ctypes.byref(o), reps)
    out = [{"iterations": r.iterations, "outer": r.outer, "relres": r.relres, "seconds": r.seconds, "status": st}
           for r in reps]
    if raise_on_error and st != OK:
        raise PsfdError(st, strerror(st))
    return out


class Solver:
    """One solver context (device state for one clip and up to max_rhs illuminations)."""

    def __init__(self, grid: Grid, precision: int = FP32_REFINED, max_rhs: int = 1, hbm_budget: int = 0,
                 stream=None):
        self.lib = load()
        self.grid = grid
        self.precision = precision
        self.max_rhs = max_rhs
        self.ctx = ctypes.c_void_p()
        st = self.lib.psfd_create(ctypes.byref(self.ctx), ctypes.byref(grid), int(precision), int(max_rhs),
                                  ctypes.c_size_t(int(hbm_budget)), _stream_ptr(stream))
        if st != OK:
            raise PsfdError(st, strerror(st))
        self.n_rhs = 0

    @classmethod
    def from_problem(cls, prob, precision=FP32_REFINED, max_rhs=None, hbm_budget=0, stream=None,
                     set_inputs=True):
        g = make_grid(prob.nx, prob.ny, prob.nslab, prob.nf, prob.dx, prob.dy, prob.dz, prob.wavelength,
                      prob.eps_bg)
        s = cls(g, precision, max_rhs or prob.n_rhs, hbm_budget, stream)
        if set_inputs:
            s.set_stack(prob.n_layers, prob.d_layers, prob.n_sub)
            s.set_potential(prob.eps)
            s.set_illumination(prob.theta_deg, prob.phi_deg, prob.pol)
        return s

    def _check(self, st):
        if st != OK:
            msg = self.lib.psfd_last_error(self.ctx).decode()
            raise PsfdError(st, f"{strerror(st)}: {msg}")
        return st

    def close(self):
        if self.ctx:
            self.lib.psfd_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        self._check(self.lib.psfd_set_stream(self.ctx, _stream_ptr(stream)))

    def set_stack(self, n_layers, thickness, n_sub):
        n = _c128(n_layers).reshape(-1)
        d = np.ascontiguousarray(thickness, dtype=np.float64).reshape(-1)
        ns = np.array([complex(n_sub).real, complex(n_sub).imag], dtype=np.float64)
        nn = n.view(np.float64) if n.size else np.zeros(2, np.float64)
        self._check(self.lib.psfd_set_stack(self.ctx, int(n.size), _dptr(nn),
                                            _dptr(d if d.size else np.zeros(1)), _dptr(ns)))

    def set_potential(self, eps):
        """eps: complex128 (nslab, ny, nx) as a numpy array or torch tensor (CPU, e.g. pinned, or CUDA)."""
        if hasattr(eps, "data_ptr"):
            self._keep_eps = eps
            where = DEVICE if eps.is_cuda else HOST
            self._check(self.lib.psfd_set_potential(self.ctx, ctypes.c_void_p(eps.data_ptr()), where))
        else:
            e = _c128(eps)
            self._keep_eps = e
            self._check(self.lib.psfd_set_potential(self.ctx, e.ctypes.data_as(ctypes.c_void_p), HOST))

    def set_green(self, kind: int, R: float = 0.0):
        """GREEN_PERIODIC (default) or GREEN_SPHERICAL with window radius R (isolated clip);
        call before set_illumination."""
        self._check(self.lib.psfd_set_green(self.ctx, int(kind), float(R)))

    def set_graphs(self, enable: bool):
        """Replay the Krylov step as a CUDA graph (default) or launch its kernels one by one."""
        self._check(self.lib.psfd_set_graphs(self.ctx, int(bool(enable))))

    def autotune(self, force: bool = False) -> dict:
        """Time the candidate tile shapes on this context's grid and keep the fastest
        (process-wide, per grid and precision); returns the report."""
        r = TuneReport()
        self._check(self.lib.psfd_autotune(self.ctx, int(bool(force)), ctypes.byref(r)))
        return {"default_ms": r.default_ms, "tuned_ms": r.tuned_ms, "zx": r.zx, "rb": r.rb, "cx": r.cx,
                "pf": r.pf, "candidates": r.candidates}

    def set_device_loop(self, enable: bool):
        """Run each Krylov sweep as one graph launch that loops on the device (default) or
        return to the host after every check_every iterations."""
        self._check(self.lib.psfd_set_device_loop(self.ctx, int(bool(enable))))

    def set_residual_arith(self, kind: int):
        """RESID_DFLOAT (default): the refined solve's FP64 residual runs its z transforms and
        dyadic products (and the y transforms of split planes) in double-float; RESID_FP64: all
        in FP64."""
        self._check(self.lib.psfd_set_residual_arith(self.ctx, int(kind)))

    def set_illumination(self, theta_deg, phi_deg, pol):
        th = np.ascontiguousarray(theta_deg, dtype=np.float64).reshape(-1)
        ph = np.ascontiguousarray(phi_deg, dtype=np.float64).reshape(-1)
        po = np.ascontiguousarray(pol, dtype=np.int32).reshape(-1)
        self._check(self.lib.psfd_set_illumination(self.ctx, int(th.size), _dptr(th), _dptr(ph),
                                                   po.ctypes.data_as(_IP)))
        self.n_rhs = int(th.size)

    def solve(self, tol=1e-10, max_iter=500, max_outer=12, inner_tol=1e-4, check_every=4, raise_on_error=True,
              krylov=BICGSTAB, restart=0):
        o = SolveOpts(float(tol), int(max_iter), int(max_outer), float(inner_tol), int(check_every), int(krylov),
                      int(restart))
        r = Report()
        st = self.lib.psfd_solve(self.ctx, ctypes.byref(o), ctypes.byref(r))
        rep = {"iterations": r.iterations, "outer": r.outer, "relres": r.relres, "seconds": r.seconds,
               "status": st}
        if raise_on_error and st != OK:
            self._check(st)
        return rep

    def solve_fixed_point(self, tol=1e-10, max_steps=50, step_tol=0.0, max_iter=500, max_outer=12, inner_tol=1e-4,
                          check_every=4, raise_on_error=True, krylov=BICGSTAB, restart=0):
        """The outer fixed-point iteration of Eq. (8): free-space solves with R rebuilt from the
        previous step's mask field, until the folded residual is below tol. "outer" in the
        report counts the outer steps, "iterations" the Krylov iterations over all of them."""
        o = SolveOpts(float(tol), int(max_iter), int(max_outer), float(inner_tol), int(check_every), int(krylov),
                      int(restart))
        r = Report()
        st = self.lib.psfd_solve_fixed_point(self.ctx, ctypes.byref(o), int(max_steps), float(step_tol),
                                             ctypes.byref(r))
        rep = {"iterations": r.iterations, "outer": r.outer, "relres": r.relres, "seconds": r.seconds,
               "status": st}
        if raise_on_error and st != OK:
            self._check(st)
        return rep

    def num_orders(self, rhs: int) -> int:
        n = ctypes.c_int(0)
        self._check(self.lib.psfd_num_orders(self.ctx, int(rhs), ctypes.byref(n)))
        return n.value

    def diffraction_orders(self, rhs: int = 0):
        cap = self.num_orders(rhs)
        n = ctypes.c_int(0)
        mn = np.zeros(2 * max(cap, 1), np.int32)
        amp = np.zeros(6 * max(cap, 1), np.float64)
        sp = np.zeros(4 * max(cap, 1), np.float64)
        eff = np.zeros(max(cap, 1), np.float64)
        self._check(self.lib.psfd_diffraction_orders(self.ctx, int(rhs), cap, ctypes.byref(n), mn.ctypes.data_as(_IP),
                                                     _dptr(amp), _dptr(sp), _dptr(eff)))
        k = n.value
        a = amp[:6 * k].view(np.complex128).reshape(k, 3)
        s = sp[:4 * k].view(np.complex128).reshape(k, 2)
        return {"m": mn[0:2 * k:2].copy(), "n": mn[1:2 * k:2].copy(), "amp": a.copy(), "a_s": s[:, 0].copy(),
                "a_p": s[:, 1].copy(), "eff": eff[:k].copy()}

    def apply(self, u, out, rhs0: int = 0, precision: int | None = None):
        """out = A u on device tensors (complex128 for FP64, complex64 for FP32)."""
        import torch
        if precision is None:
            precision = FP64 if u.dtype == torch.complex128 else FP32_REFINED
        nrhs = u.shape[0]
        self._check(self.lib.psfd_apply(self.ctx, int(precision), int(rhs0), int(nrhs),
                                        ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(out.data_ptr())))
        return out

    def _field_shape(self):
        g = self.grid
        return (3, g.nslab, g.ny, g.nx)

    def get_solution(self, rhs: int = 0) -> np.ndarray:
        out = np.zeros(self._field_shape(), np.complex128)
        self._check(self.lib.psfd_get_solution(self.ctx, int(rhs), out.ctypes.data_as(ctypes.c_void_p), HOST))
        return out

    def set_initial_guess(self, rhs, x):
        """Warm start of illumination rhs: x is a complex128 numpy array or CUDA tensor of the
        field shape; the next solve starts from it."""
        if hasattr(x, "is_cuda") and x.is_cuda:
            self._check(self.lib.psfd_set_initial_guess(self.ctx, int(rhs), ctypes.c_void_p(x.data_ptr()), DEVICE))
        else:
            a = np.ascontiguousarray(x, dtype=np.complex128)
            if a.shape != self._field_shape():
                raise ValueError(f"initial guess of shape {a.shape}, expected {self._field_shape()}")
            self._check(self.lib.psfd_set_initial_guess(self.ctx, int(rhs), a.ctypes.data_as(ctypes.c_void_p), HOST))

    def residual_history(self, rhs: int = 0):
        """Convergence curve of the latest solve: iteration, kind (1 = FP64 residual, 0 = Krylov
        estimate, 2 = folded residual after an outer fixed-point step) and relative residual per
        recorded point."""
        n = ctypes.c_int(0)
        self._check(self.lib.psfd_residual_history(self.ctx, int(rhs), 0, ctypes.byref(n), None, None, None))
        cap = n.value
        it = np.zeros(max(cap, 1), np.int32)
        kind = np.zeros(max(cap, 1), np.int32)
        rel = np.zeros(max(cap, 1), np.float64)
        self._check(self.lib.psfd_residual_history(self.ctx, int(rhs), cap, ctypes.byref(n), it.ctypes.data_as(_IP),
                                                   kind.ctypes.data_as(_IP), _dptr(rel)))
        k = min(cap, n.value)
        return {"iteration": it[:k].copy(), "kind": kind[:k].copy(), "relres": rel[:k].copy()}

    def get_rhs(self, rhs: int = 0) -> np.ndarray:
        out = np.zeros(self._field_shape(), np.complex128)
        self._check(self.lib.psfd_get_rhs(self.ctx, int(rhs), out.ctypes.data_as(ctypes.c_void_p), HOST))
        return out

    def mode_tables(self, rhs: int = 0):
        g = self.grid
        beta = np.zeros((g.ny, g.nx), np.complex128)
        rs = np.zeros_like(beta)
        rp = np.zeros_like(beta)
        self._check(self.lib.psfd_get_mode_tables(self.ctx, int(rhs), _dptr(beta.view(np.float64)),
                                                  _dptr(rs.view(np.float64)), _dptr(rp.view(np.float64))))
        return beta, rs, rp


def fft_inplace(data, inverse: bool = False):
    """In-place FFT of the rows of a (count, n) complex CUDA tensor with the library's kernels."""
    import torch
    fp64 = data.dtype == torch.complex128
    st = load().psfd_test_fft(int(data.shape[-1]), int(data.numel() // data.shape[-1]), int(inverse), int(fp64),
                              ctypes.c_void_p(data.data_ptr()))
    if st != OK:
        raise PsfdError(st, strerror(st))
    return data


class Server:
    """Serving loop: queue mask-clip requests, drive progress(), collect orders per request."""

    def __init__(self, precision: int = FP32_REFINED, hbm_budget: int = 0, slots_per_context: int = 18,
                 tol=1e-8, max_iter=400, max_outer=12, inner_tol=1e-4, check_every=4, krylov=BICGSTAB, restart=0):
        self.lib = load()
        self.h = ctypes.c_void_p()
        o = SolveOpts(float(tol), int(max_iter), int(max_outer), float(inner_tol), int(check_every), int(krylov),
                      int(restart))
        st = self.lib.psfd_server_create(ctypes.byref(self.h), int(precision), ctypes.c_size_t(int(hbm_budget)),
                                         int(slots_per_context), ctypes.byref(o))
        if st != OK:
            raise PsfdError(st, strerror(st))

    def _check(self, st):
        if st != OK:
            raise PsfdError(st, strerror(st))

    def close(self):
        if self.h:
            self.lib.psfd_server_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_rounds(self, ticks_per_round: int):
        """Fused rounds: one graph launch per round advances every bucket inside a Krylov sweep
        by up to ticks_per_round ticks (0: buckets advance independently)."""
        self._check(self.lib.psfd_server_set_rounds(self.h, int(ticks_per_round)))

    def set_max_running(self, n: int):
        """Requests in flight at once (0: as many as fit)."""
        self._check(self.lib.psfd_server_set_max_running(self.h, int(n)))

    def submit(self, prob, theta=None, phi=None, pol=None) -> int:
        """Queue one clip (a layouts.Problem); illuminations default to the problem's."""
        th = np.ascontiguousarray(prob.theta_deg if theta is None else theta, dtype=np.float64).reshape(-1)
        ph = np.ascontiguousarray(prob.phi_deg if phi is None else phi, dtype=np.float64).reshape(-1)
        po = np.ascontiguousarray(prob.pol if pol is None else pol, dtype=np.int32).reshape(-1)
        n = _c128(prob.n_layers).reshape(-1)
        nn = n.view(np.float64) if n.size else np.zeros(2, np.float64)
        d = np.ascontiguousarray(prob.d_layers, dtype=np.float64).reshape(-1)
        d = d if d.size else np.zeros(1)
        ns = np.array([complex(prob.n_sub).real, complex(prob.n_sub).imag], dtype=np.float64)
        eps = _c128(prob.eps)
        g = make_grid(prob.nx, prob.ny, prob.nslab, prob.nf, prob.dx, prob.dy, prob.dz, prob.wavelength,
                      prob.eps_bg)
        q = Request(g, int(n.size), _dptr(nn), _dptr(d), _dptr(ns), _dptr(eps.view(np.float64)), int(th.size),
                    _dptr(th), _dptr(ph), po.ctypes.data_as(_IP))
        t = ctypes.c_longlong(0)
        self._check(self.lib.psfd_server_submit(self.h, ctypes.byref(q), ctypes.byref(t)))
        return int(t.value)

    def progress(self) -> int:
        n = ctypes.c_int(0)
        self._check(self.lib.psfd_server_progress(self.h, ctypes.byref(n)))
        return n.value

    def status(self, ticket: int):
        state, status = ctypes.c_int(0), ctypes.c_int(0)
        self._check(self.lib.psfd_server_status(self.h, ctypes.c_longlong(ticket), ctypes.byref(state),
                                                ctypes.byref(status)))
        return state.value, status.value

    def orders(self, ticket: int, rhs: int = 0, capacity: int = 65536):
        n = ctypes.c_int(0)
        mn = np.zeros(2 * capacity, np.int32)
        amp = np.zeros(6 * capacity, np.float64)
        sp = np.zeros(4 * capacity, np.float64)
        eff = np.zeros(capacity, np.float64)
        self._check(self.lib.psfd_server_orders(self.h, ctypes.c_longlong(ticket), int(rhs), int(capacity),
                                                ctypes.byref(n), mn.ctypes.data_as(_IP), _dptr(amp), _dptr(sp),
                                                _dptr(eff)))
        k = n.value
        a = amp[:6 * k].view(np.complex128).reshape(k, 3)
        s = sp[:4 * k].view(np.complex128).reshape(k, 2)
        return {"m": mn[0:2 * k:2].copy(), "n": mn[1:2 * k:2].copy(), "amp": a.copy(), "a_s": s[:, 0].copy(),
                "a_p": s[:, 1].copy(), "eff": eff[:k].copy()}

    def release(self, ticket: int):
        self._check(self.lib.psfd_server_release(self.h, ctypes.c_longlong(ticket)))

    def memory(self):
        used, n = ctypes.c_size_t(0), ctypes.c_int(0)
        self._check(self.lib.psfd_server_memory(self.h, ctypes.byref(used), ctypes.byref(n)))
        return int(used.value), n.value

    def run_until_done(self, max_steps: int = 100000) -> int:
        for k in range(max_steps):
            if self.progress() == 0:
                return k + 1
        raise RuntimeError("server did not finish")
