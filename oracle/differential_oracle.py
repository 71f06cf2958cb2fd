"""Plain FP64 CPU oracle of the conventional (differential) PSFD formulation of the mask
problem and of the preconditioner comparison it is measured with (Sec. 3, Eqs. (4)-(7), (10)
and the preconditioner table).

Test infrastructure only: imported by ``tests/`` (and nothing on the product path). It shares
no code with the CUDA path; its transforms are the oracle's own (``oracle/fft.py``).

Problem: a periodic clip in free space (no stack), scattered-field form of Eq. (3),
    curl curl E_s - k0^2 eps E_s = k0^2 (eps - eps_bg) E_inc,
for the Bloch envelope of E_s on a z column that holds the absorber between vacuum spacers and
perfectly matched layers (PMLs) at both ends. Derivatives are spectral (Eq. (6)): along x and y
exact per transverse mode (d/dx -> i q_x with q = q_inc + 2 pi m / P), along z by FFT on the
column, divided by the PML stretch s(z) = 1 + i sigma(z) (Eq. (7)).
Readings (the paper gives neither the PML profile nor its strength): sigma(z) =
sigma_max (depth/L_pml)^3 inside the layers, sigma_max = -4 ln(1e-8) / (2 kb L_pml) (a
normal-incidence round-trip reflection of 1e-8); the absorber sits on the lowest slab
planes, as in the LS form; the incident envelope is e exp(-i beta z).
Preconditioners compared (the table of Sec. 3): none; the isotropic spectral damping
D(k) = min(1, kb^2 / |k|^2) applied on the left in the 3-D Fourier domain of the column; and
the Lippmann-Schwinger form itself (the free-space Green's function as left preconditioner,
Eq. (10)), whose operator is psfd_oracle.apply_operator without the stack.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import fft as offt
from .psfd_oracle import triad, upper_sqrt

__all__ = ["DiffProblem", "diff_problem_from_clip", "apply_differential", "differential_rhs",
           "spectral_damping", "gmres_restarted", "reflected_amplitude_film", "preconditioner_study"]


@dataclasses.dataclass
class DiffProblem:
    nx: int
    ny: int
    nz: int            # planes of the whole column (PML + spacer + slab + spacer + PML)
    dx: float
    dy: float
    dz: float
    wavelength: float
    eps_bg: float
    eps: np.ndarray    # (nz, ny, nx)
    n_pml: int         # PML planes at each end
    theta: float = 6.0
    phi: float = 0.0
    pol: int = 0


def diff_problem_from_clip(prob, i: int = 0, spacer: float = 20.0, pml: float = 30.0) -> DiffProblem:
    """The column for a clip of the LS form (layouts.Problem, eps on nslab planes): PML of
    `pml` nm, vacuum spacer of `spacer` nm, the slab, spacer, PML (z grows upward)."""
    ns = int(round(spacer / prob.dz))
    npml = int(round(pml / prob.dz))
    nz = 2 * npml + 2 * ns + prob.nslab
    eps = np.full((nz, prob.ny, prob.nx), prob.eps_bg, np.complex128)
    eps[npml + ns:npml + ns + prob.nslab] = prob.eps
    return DiffProblem(prob.nx, prob.ny, nz, prob.dx, prob.dy, prob.dz, prob.wavelength, prob.eps_bg, eps, npml,
                       float(prob.theta_deg[i]), float(prob.phi_deg[i]), int(prob.pol[i]))


def _geometry(p: DiffProblem):
    k0 = 2 * math.pi / p.wavelength
    kb = k0 * math.sqrt(p.eps_bg)
    th, ph = math.radians(p.theta), math.radians(p.phi)
    qix, qiy = kb * math.sin(th) * math.cos(ph), kb * math.sin(th) * math.sin(ph)
    qx = qix + 2 * math.pi * offt.fftfreq(p.nx, p.dx)
    qy = qiy + 2 * math.pi * offt.fftfreq(p.ny, p.dy)
    kz = 2 * math.pi * offt.fftfreq(p.nz, p.dz)
    # PML stretch, cubic profile over n_pml planes at both ends
    Lp = p.n_pml * p.dz
    smax = -4.0 * math.log(1e-8) / (2.0 * kb * Lp) if p.n_pml > 0 else 0.0
    z = (np.arange(p.nz) + 0.5) * p.dz
    depth = np.maximum(np.maximum(Lp - z, z - (p.nz * p.dz - Lp)), 0.0)
    s = 1.0 + 1j * smax * (depth / max(Lp, 1e-300)) ** 3
    return k0, kb, qix, qiy, qx, qy, kz, s


def _d(f, axis, p, g):
    """Spectral derivative of f (nz, ny, nx) along x (axis 2), y (1) or z (0, stretched)."""
    k0, kb, qix, qiy, qx, qy, kz, s = g
    if axis == 2:
        return offt.ifft(1j * qx[None, None, :] * offt.fft(f, axis=2), axis=2)
    if axis == 1:
        return offt.ifft(1j * qy[None, :, None] * offt.fft(f, axis=1), axis=1)
    return offt.ifft(1j * kz[:, None, None] * offt.fft(f, axis=0), axis=0) / s[:, None, None]


def _curl(E, p, g):
    Ex, Ey, Ez = E
    return np.stack([_d(Ez, 1, p, g) - _d(Ey, 0, p, g),
                     _d(Ex, 0, p, g) - _d(Ez, 2, p, g),
                     _d(Ey, 2, p, g) - _d(Ex, 1, p, g)])


def apply_differential(p: DiffProblem, E: np.ndarray, g=None) -> np.ndarray:
    """curl curl E - k0^2 eps E with the spectral (PML-stretched) derivatives; E (3, nz, ny, nx)."""
    g = g or _geometry(p)
    k0 = g[0]
    return _curl(_curl(E, p, g), p, g) - k0 * k0 * p.eps[None] * E


def differential_rhs(p: DiffProblem, g=None) -> np.ndarray:
    """k0^2 (eps - eps_bg) E_inc with E_inc = e exp(-i beta z) (Bloch envelope)."""
    g = g or _geometry(p)
    k0, kb, qix, qiy = g[:4]
    beta = upper_sqrt(np.array([[kb * kb - qix * qix - qiy * qiy]], np.complex128))
    s_hat, p_up, p_dn = triad(np.array([[qix]]), np.array([[qiy]]), beta, kb, math.radians(p.phi))
    e = (s_hat if p.pol == 0 else p_dn)[:, 0, 0]
    z = np.arange(p.nz) * p.dz
    inc = e[:, None] * np.exp(-1j * beta[0, 0] * z)[None]
    return k0 * k0 * (p.eps - p.eps_bg)[None] * inc[:, :, None, None]


def spectral_damping(p: DiffProblem, r: np.ndarray, g=None) -> np.ndarray:
    """D(k) r with D = min(1, kb^2/|k|^2) on the 3-D Fourier grid of the column."""
    g = g or _geometry(p)
    kb, qx, qy, kz = g[1], g[4], g[5], g[6]
    k2 = qx[None, None, :] ** 2 + qy[None, :, None] ** 2 + kz[:, None, None] ** 2
    D = np.minimum(1.0, kb * kb / np.maximum(k2, 1e-300))
    return offt.ifftn(D[None] * offt.fftn(r, axes=(1, 2, 3)), axes=(1, 2, 3))


def gmres_restarted(apply, b: np.ndarray, rtol: float = 1e-8, restart: int = 60, maxiter: int = 20000):
    """GMRES(restart) with modified Gram-Schmidt and Givens rotations. Returns (x, matvecs,
    relative residual of the (left-preconditioned) system)."""
    shape = b.shape
    bv = b.reshape(-1)
    bn = np.linalg.norm(bv)
    x = np.zeros_like(bv)
    if bn == 0:
        return x.reshape(shape), 0, 0.0
    mv = 0
    res = 1.0
    while mv < maxiter:
        r = bv - apply(x.reshape(shape)).reshape(-1) if mv else bv.copy()
        beta = np.linalg.norm(r)
        res = beta / bn
        if res <= rtol:
            break
        m = min(restart, maxiter - mv)
        Q = np.zeros((m + 1, bv.size), np.complex128)
        H = np.zeros((m + 1, m), np.complex128)
        cs, sn = np.zeros(m, np.complex128), np.zeros(m, np.float64)
        gvec = np.zeros(m + 1, np.complex128)
        gvec[0] = beta
        Q[0] = r / beta
        j = 0
        for j in range(m):
            w = apply(Q[j].reshape(shape)).reshape(-1)
            mv += 1
            for i in range(j + 1):
                H[i, j] = np.vdot(Q[i], w)
                w = w - H[i, j] * Q[i]
            hn = np.linalg.norm(w)
            if hn != 0:
                Q[j + 1] = w / hn
            # earlier rotations G_i = [[conj(c), s], [-s, c]] (s real), then the new one
            for i in range(j):
                t = np.conj(cs[i]) * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = math.hypot(abs(H[j, j]), hn)
            cs[j] = H[j, j] / den if den else 1.0
            sn[j] = hn / den if den else 0.0
            H[j, j] = den
            gvec[j + 1] = -sn[j] * gvec[j]
            gvec[j] = np.conj(cs[j]) * gvec[j]
            res = abs(gvec[j + 1]) / bn
            if res <= rtol:
                break
        y = np.linalg.solve(np.triu(H[:j + 1, :j + 1]), gvec[:j + 1])
        x = x + Q[:j + 1].T @ y
        if res <= rtol:
            break
    return x.reshape(shape), mv, float(res)


def reflected_amplitude_film(p: DiffProblem, E_s: np.ndarray, z_top: float, g=None) -> complex:
    """Reflection coefficient of a laterally uniform column (nx = ny = 1, pol 0) from its
    scattered field: in the upper spacer E_s = r E_inc(z_top) exp(i beta (z - z_top)) s_hat, so
    r = s_hat . E_s(z) exp(-i beta (z - z_top)) / exp(-i beta z_top), averaged over the spacer
    planes outside the PML."""
    g = g or _geometry(p)
    kb, qix, qiy = g[1], g[2], g[3]
    beta = upper_sqrt(np.array([[kb * kb - qix * qix - qiy * qiy]], np.complex128))
    s_hat = triad(np.array([[qix]]), np.array([[qiy]]), beta, kb, math.radians(p.phi))[0][:, 0, 0]
    b = beta[0, 0]
    top = p.nz - p.n_pml
    zs = np.arange(p.nz) * p.dz
    idx = [k for k in range(p.nz) if zs[k] > z_top + p.dz and k < top - 1]
    vals = [(s_hat @ E_s[:, k, 0, 0]) * np.exp(-1j * b * (zs[k] - z_top)) / np.exp(-1j * b * z_top) for k in idx]
    return complex(np.mean(vals))


def preconditioner_study(prob, i: int = 0, rtol: float = 1e-8, restart: int = 60, maxiter: int = 20000,
                         spacer: float = 20.0, pml: float = 30.0):
    """Operator applications GMRES(restart) needs to reach rtol for illumination i of a clip in
    free space: the differential PSFD without and with the spectral damping preconditioner,
    and the Lippmann-Schwinger form (the Green's function as preconditioner, the periodic
    operator of psfd_oracle without the stack). Returns a dict of (matvecs, residual)."""
    from .psfd_oracle import apply_operator, rhs_vector, setup_rhs
    p = diff_problem_from_clip(prob, i, spacer, pml)
    g = _geometry(p)
    b = differential_rhs(p, g)
    out = {}
    _, mv, res = gmres_restarted(lambda v: apply_differential(p, v, g), b, rtol, restart, maxiter)
    out["none"] = (mv, res)
    Db = spectral_damping(p, b, g)
    _, mv, res = gmres_restarted(lambda v: spectral_damping(p, apply_differential(p, v, g), g), Db, rtol, restart,
                                 maxiter)
    out["spectral_damping"] = (mv, res)
    ctx = setup_rhs(prob, i, reflection=False)
    bl = rhs_vector(ctx)
    _, mv, res = gmres_restarted(lambda v: apply_operator(ctx, v), bl, rtol, restart, maxiter)
    out["lippmann_schwinger"] = (mv, res)
    return out
