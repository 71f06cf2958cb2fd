"""Plain FP64 CPU oracle of the isolated (non-periodic) clip: the Lippmann-Schwinger operator
with the paper's spherically windowed dyadic Green's function (Sec. 3, Eqs. (13)-(18)).

Test infrastructure only: imported by ``tests/`` (and nothing on the product path). It
shares no code with the CUDA path; its transforms are the oracle's own (``oracle/fft.py``).

The problem: a scatterer of permittivity eps on a box grid, free space eps_bg around it, a
plane wave E_inc. With V = k0^2 (eps - eps_bg) and the total field u,
    u - G_R * (V u) = E_inc                                  (Eqs. (11), (12), (18))
where G_R is the dyadic Green's function (I + grad grad / kb^2) g, g = exp(i kb r)/(4 pi r),
truncated to |r| < R (Eq. (13)). The grid is the padded computational box: V vanishes outside
the scatterer, and the periodic FFT convolution equals the linear one as long as every
period exceeds the scatterer's extent plus R (Sec. 3, discussion of Eq. (18)).

Reading of Eq. (16), whose constants are garbled in the text: the transform is
    F[G_R](k) = A(k) I + B(k) khat khat^T,
    A = F[g_R](k) + h(k),  B = -F[g_R](k) - 3 h(k) - 1/kb^2  (k > 0),  A(0) = F[g_R](0) + h(0),
    B(0) = 0,  h(k) = 4 pi R^2 g'(R) j1(kR) / (kb^2 kR),
derived here from grad grad (chi g) = chi grad grad g + (grad chi)(grad g) + (grad g)(grad chi)
+ g grad grad chi for the window chi and the angular integrals of the shell terms; the
factor R^2 (not R) in h and the factor 4 pi in A(0) follow from that derivation and are
pinned by a direct real-space quadrature in tests/test_oracle_isolated.py.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import fft as offt
from .psfd_oracle import gmres, triad, upper_sqrt

__all__ = ["windowed_scalar_spectrum", "windowed_dyadic_coefficients", "dyadic_green_realspace",
           "IsolatedProblem", "isolated_kernel", "isolated_rhs", "apply_isolated", "solve_isolated"]


def _phi1(z):
    """(e^z - 1)/z with its limit 1 at z = 0 (expm1 keeps the small-z values accurate)."""
    z = np.asarray(z, dtype=np.complex128)
    small = np.abs(z) < 1e-8
    safe = np.where(small, 1.0, z)
    return np.where(small, 1.0 + z / 2, np.expm1(safe) / safe)


def windowed_scalar_spectrum(k, kb, R):
    """F[g_R](k) = int_{|r|<R} g(r) exp(-i k.r) d^3r for |k| = k >= 0 (Eq. (17)).

    After the angular integral, F = (1/k) int_0^R exp(i kb r) sin(k r) dr; writing the sine as
    two exponentials gives (1/(2ik)) [R phi1(i(kb+k)R) - R phi1(i(kb-k)R)], which stays finite
    through k = kb (the removable singularity of the closed form). k = 0: int_0^R r exp(i kb r) dr.
    """
    k = np.asarray(k, dtype=np.float64)
    kb = complex(kb)
    zero = k < 1e-12 * abs(kb)
    ks = np.where(zero, 1.0, k)
    general = (R * _phi1(1j * (kb + ks) * R) - R * _phi1(1j * (kb - ks) * R)) / (2j * ks)
    at0 = (np.exp(1j * kb * R) * (1.0 - 1j * kb * R) - 1.0) / (kb * kb)
    return np.where(zero, at0, general)


def _j1_over_x(x):
    """j1(x)/x = (sin x - x cos x)/x^3, by its Taylor series for small x."""
    x = np.asarray(x, dtype=np.float64)
    small = x < 1e-2
    xs = np.where(small, 1.0, x)
    series = 1.0 / 3.0 - x ** 2 / 30.0 + x ** 4 / 840.0 - x ** 6 / 45360.0
    return np.where(small, series, (np.sin(xs) - xs * np.cos(xs)) / xs ** 3)


def windowed_dyadic_coefficients(k, kb, R):
    """(A(k), B(k)) of F[G_R](k) = A I + B khat khat^T (Eqs. (15)-(17), reading in the header)."""
    k = np.asarray(k, dtype=np.float64)
    kb = complex(kb)
    f = windowed_scalar_spectrum(k, kb, R)
    g_R = np.exp(1j * kb * R) / (4 * math.pi * R)
    dg_R = g_R * (1j * kb - 1.0 / R)  # g'(R)
    h = 4 * math.pi * R * R * dg_R * _j1_over_x(k * R) / (kb * kb)
    A = f + h
    B = np.where(k < 1e-12 * abs(kb), 0.0, -f - 3.0 * h - 1.0 / (kb * kb))
    return A, B


def dyadic_green_realspace(rvec, kb):
    """G(r) = (I + grad grad / kb^2) exp(i kb r)/(4 pi r) for r != 0 (Eq. (14)), rvec (..., 3):
    g [(1 + i/(kb r) - 1/(kb r)^2) I + (3/(kb r)^2 - 3i/(kb r) - 1) rhat rhat^T]."""
    rvec = np.asarray(rvec, dtype=np.float64)
    r = np.linalg.norm(rvec, axis=-1)
    rh = rvec / r[..., None]
    x = complex(kb) * r
    g = np.exp(1j * x) / (4 * math.pi * r)
    a = g * (1.0 + 1j / x - 1.0 / x ** 2)
    b = g * (3.0 / x ** 2 - 3j / x - 1.0)
    return a[..., None, None] * np.eye(3) + b[..., None, None] * rh[..., :, None] * rh[..., None, :]


@dataclasses.dataclass
class IsolatedProblem:
    """Padded box grid (nz, ny, nx) at spacing (dz, dy, dx) nm; eps (nz, ny, nx) equals eps_bg
    outside the scatterer; window radius R (nm); one plane wave (theta, phi deg, pol 0 = s)."""
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    wavelength: float
    eps_bg: float
    eps: np.ndarray
    R: float
    theta: float = 0.0
    phi: float = 0.0
    pol: int = 0
    # Bloch envelopes: the unknown is the field times exp(-i q_inc . r_perp), so the kernel is
    # taken at k + q_inc and E_inc becomes e exp(-i beta z) (the same linear convolution, on a
    # k-grid shifted by q_inc)
    bloch: bool = False


def _q_inc(p: IsolatedProblem):
    kb = 2 * math.pi / p.wavelength * math.sqrt(p.eps_bg)
    th, ph = math.radians(p.theta), math.radians(p.phi)
    return kb * math.sin(th) * math.cos(ph), kb * math.sin(th) * math.sin(ph)


def isolated_kernel(p: IsolatedProblem) -> np.ndarray:
    """F[G_R] at the grid wavenumbers (shifted by q_inc for Bloch envelopes), (3, 3, nz, ny, nx)."""
    kb = 2 * math.pi / p.wavelength * math.sqrt(p.eps_bg)
    qix, qiy = _q_inc(p) if p.bloch else (0.0, 0.0)
    kx = qix + 2 * math.pi * offt.fftfreq(p.nx, p.dx)
    ky = qiy + 2 * math.pi * offt.fftfreq(p.ny, p.dy)
    kz = 2 * math.pi * offt.fftfreq(p.nz, p.dz)
    KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
    kk = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    A, B = windowed_dyadic_coefficients(kk, kb, p.R)
    safe = np.where(kk > 0, kk, 1.0)
    kh = [KX / safe, KY / safe, KZ / safe]
    G = np.empty((3, 3) + kk.shape, dtype=np.complex128)
    for a in range(3):
        for b in range(3):
            G[a, b] = (A if a == b else 0.0) + B * kh[a] * kh[b]
    return G


def isolated_rhs(p: IsolatedProblem) -> np.ndarray:
    """E_inc = e exp(i k_inc . r) on the grid (3, nz, ny, nx); k_inc = kb (sin t cos f,
    sin t sin f, -cos t), e = s (pol 0) or p- (pol 1) of the same triad as the periodic case."""
    kb = 2 * math.pi / p.wavelength * math.sqrt(p.eps_bg)
    th, ph = math.radians(p.theta), math.radians(p.phi)
    qx, qy = kb * math.sin(th) * math.cos(ph), kb * math.sin(th) * math.sin(ph)
    beta = upper_sqrt(np.array([[kb * kb - qx * qx - qy * qy]], np.complex128))
    s_hat, p_up, p_dn = triad(np.array([[qx]]), np.array([[qy]]), beta, kb, ph)
    e = (s_hat if p.pol == 0 else p_dn)[:, 0, 0]
    z = np.arange(p.nz) * p.dz
    y = np.arange(p.ny) * p.dy
    x = np.arange(p.nx) * p.dx
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    if p.bloch:
        phase = np.exp(-1j * beta[0, 0] * Z)
    else:
        phase = np.exp(1j * (qx * X + qy * Y - beta[0, 0] * Z))
    return e[:, None, None, None] * phase[None]


def apply_isolated(p: IsolatedProblem, u: np.ndarray, G: np.ndarray | None = None) -> np.ndarray:
    """u - IFFT(F[G_R] . FFT(V u)) (Eq. (18)); u (3, nz, ny, nx)."""
    if G is None:
        G = isolated_kernel(p)
    k0 = 2 * math.pi / p.wavelength
    V = k0 * k0 * (np.asarray(p.eps, np.complex128) - p.eps_bg)
    J = offt.fftn(V[None] * u, axes=(1, 2, 3))
    W = np.einsum("ab...,b...->a...", G, J)
    return u - offt.ifftn(W, axes=(1, 2, 3))


def solve_isolated(p: IsolatedProblem, rtol: float = 1e-12, maxiter: int = 400, direct: bool = False):
    """Total field u of the isolated clip; returns (u, info)."""
    G = isolated_kernel(p)
    b = isolated_rhs(p)
    if direct:
        n = b.size
        A = np.empty((n, n), np.complex128)
        for j in range(n):
            e = np.zeros(n, np.complex128)
            e[j] = 1.0
            A[:, j] = apply_isolated(p, e.reshape(b.shape), G).reshape(-1)
        u = np.linalg.solve(A, b.reshape(-1)).reshape(b.shape)
        return u, {"iterations": 0, "relres": float(np.linalg.norm(A @ u.reshape(-1) - b.reshape(-1))
                                                      / np.linalg.norm(b))}
    u, its, res = gmres(lambda v: apply_isolated(p, v, G), b, rtol=rtol, maxiter=maxiter)
    return u, {"iterations": its, "relres": res}
