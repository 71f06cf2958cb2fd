"""Pins of the isolated-clip oracle (spherically windowed dyadic Green's function, Sec. 3,
Eqs. (13)-(18)) against what the mathematics fixes: radial quadrature of the windowed scalar
kernel, a real-space quadrature of the windowed dyadic kernel around a target whose window
cuts through the source (the shell terms of the transform, h(k), matter there), continuity at
k = 0, exactness of the padded periodic convolution, and the dense direct solve."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import isolated_oracle as iso

LAM = 13.5
KB = 2 * math.pi / LAM


@pytest.mark.parametrize("kb", [KB, KB * (1.0 + 0.02j)])
def test_windowed_scalar_spectrum_matches_radial_quadrature(kb):
    """F[g_R](k) = (1/k) int_0^R exp(i kb r) sin(k r) dr (and int_0^R r exp(i kb r) dr at k = 0),
    including k = kb, where the closed form of Eq. (17) is 0/0."""
    R = 40.0
    kr = kb.real if isinstance(kb, complex) else kb
    for k in [0.0, 0.3 * kr, kr * (1 - 1e-9), kr, kr * (1 + 1e-7), 1.7 * kr, 5.0 * kr]:
        got = complex(iso.windowed_scalar_spectrum(np.array([k]), kb, R)[0])
        if k == 0.0:
            f = lambda r: r * np.exp(1j * kb * r)  # noqa: E731
        else:
            f = lambda r: np.exp(1j * kb * r) * math.sin(k * r) / k  # noqa: E731
        re = integrate.quad(lambda r: f(r).real, 0.0, R, limit=400, epsabs=0, epsrel=1e-13)[0]
        im = integrate.quad(lambda r: f(r).imag, 0.0, R, limit=400, epsabs=0, epsrel=1e-13)[0]
        ref = complex(re, im)
        assert abs(got - ref) < 1e-11 * abs(ref), (k, got, ref)


def test_dyadic_coefficients_are_continuous_at_k_zero():
    """A(k) -> A(0) = F[g_R](0) + 4 pi R^2 g'(R) / (3 kb^2) and B(k) -> 0 as k -> 0: the k = 0
    values are the limits of the k > 0 formulas, not separate definitions."""
    R = 25.0
    k = np.array([0.0, 1e-5, 1e-4, 1e-3])
    A, B = iso.windowed_dyadic_coefficients(k, KB, R)
    assert B[0] == 0
    kR2 = (k * R) ** 2  # both are even in k: the gap closes like (kR)^2
    for i in (1, 2, 3):
        assert abs(A[i] - A[0]) < kR2[i] * abs(A[0]), i
        assert abs(B[i]) < kR2[i] * abs(A[0]), i


@pytest.mark.parametrize("comp", [0, 2])
def test_windowed_dyadic_transform_matches_realspace_quadrature(comp):
    """G_R * J at a grid point through the FFT with A I + B khat khat^T, against a direct
    quadrature of int_{|s|<R} G(s) J(x0 - s) d^3s in spherical coordinates about x0 with the
    analytic dyadic G (Eq. (14)). The source (a Gaussian of 3 nm) sits 32 nm from the target
    and the 40 nm window cuts through it, so the shell terms h(k) of the transform enter:
    leaving h out changes the result by about 4 %. The 108 nm period keeps every image of the
    source farther than R from the target, so the periodic FFT convolution is the linear one."""
    n, d, R = 72, 1.5, 40.0
    p = iso.IsolatedProblem(nx=n, ny=n, nz=n, dx=d, dy=d, dz=d, wavelength=LAM, eps_bg=1.0,
                            eps=np.ones((n, n, n)), R=R)
    G = iso.isolated_kernel(p)
    sig = 2 * d
    c = np.array([14, 14, 14])             # source centre, grid index (z, y, x)
    x0 = c + np.array([14, 10, 13])        # target
    Dv = (x0 - c) * d
    D = float(np.linalg.norm(Dv))
    assert D < R < D + 3 * sig
    z = np.arange(n) * d
    Z, Y, X = np.meshgrid(z, z, z, indexing="ij")
    cz, cy, cx = c * d
    gauss = np.exp(-((Z - cz) ** 2 + (Y - cy) ** 2 + (X - cx) ** 2) / (2 * sig ** 2))
    J = np.zeros((3, n, n, n), np.complex128)
    J[comp] = gauss
    W = np.fft.ifftn(np.einsum("ab...,b...->a...", G, np.fft.fftn(J, axes=(1, 2, 3))), axes=(1, 2, 3))
    w_fft = W[:, x0[0], x0[1], x0[2]]
    # quadrature about x0, polar axis toward the source centre (the source is negligible
    # beyond 8 sigma / D from the axis and at the target itself)
    ax = -Dv / D
    e1 = np.cross(ax, np.array([1.0, 0.0, 0.0]))
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(ax, e1)
    rn, rw = np.polynomial.legendre.leggauss(240)
    rr, rwt = 0.5 * R * (rn + 1), 0.5 * R * rw
    tmax = 8 * sig / D
    tn, tw = np.polynomial.legendre.leggauss(80)
    th, thw = 0.5 * tmax * (tn + 1), 0.5 * tmax * tw
    nph = 96
    phs = 2 * math.pi * np.arange(nph) / nph
    RR, TH, PH = np.meshgrid(rr, th, phs, indexing="ij")
    WW = (rwt[:, None, None] * rr[:, None, None] ** 2) * (thw[None, :, None] * np.sin(th)[None, :, None]) \
        * (2 * math.pi / nph)
    dirs = np.cos(TH)[..., None] * ax + np.sin(TH)[..., None] * (np.cos(PH)[..., None] * e1
                                                                 + np.sin(PH)[..., None] * e2)
    S = RR[..., None] * dirs                # from the target toward the source points, (z, y, x)
    Jv = np.exp(-np.sum((x0 * d + S - c * d) ** 2, -1) / (2 * sig ** 2))
    Gs = iso.dyadic_green_realspace(-S[..., ::-1], KB)  # argument x0 - r' in (x, y, z)
    w_dir = np.einsum("ijkb,ijk->b", Gs[..., :, comp], Jv * WW)
    assert np.max(np.abs(w_fft - w_dir)) < 1e-9 * np.max(np.abs(w_dir)), (w_fft, w_dir)


def _cube_problem(n, nz, R, L=6, Lz=4, d=2.0, eps=None):
    e = np.ones((nz, n, n), np.complex128)
    e[:Lz, :L, :L] = (0.94 + 0.04j) ** 2 if eps is None else eps
    return iso.IsolatedProblem(nx=n, ny=n, nz=nz, dx=d, dy=d, dz=d, wavelength=LAM, eps_bg=1.0, eps=e, R=R,
                               theta=6.0, phi=20.0, pol=0)


def _bump_problem(n, R, d=1.0, sig=2.0, c=10.0):
    """A smooth scatterer: eps - 1 a Gaussian of 2 nm (negligible beyond 8 nm from its centre)."""
    z = np.arange(n) * d
    Z, Y, X = np.meshgrid(z, z, z, indexing="ij")
    g = np.exp(-((Z - c) ** 2 + (Y - c) ** 2 + (X - c) ** 2) / (2 * sig ** 2))
    return iso.IsolatedProblem(nx=n, ny=n, nz=n, dx=d, dy=d, dz=d, wavelength=LAM, eps_bg=1.0,
                               eps=1.0 + (-0.12 + 0.08j) * g, R=R, theta=6.0, phi=20.0, pol=1)


def test_isolated_solution_does_not_depend_on_the_padding():
    """Eq. (13) with the padding of Sec. 3: once R exceeds the scatterer's diameter and every
    period exceeds its extent plus R, the periodic FFT convolution is the linear one, so the
    field on the scatterer no longer changes with the box (checked on a smooth scatterer, whose
    spectrum is resolved: the 16 nm support and R = 27.7 nm need a 44 nm box). A box below that
    bound sees the scatterer's images through the window and differs."""
    R = 16.0 * math.sqrt(3)
    sub = (slice(None), slice(0, 21), slice(0, 21), slice(0, 21))
    u40, _ = iso.solve_isolated(_bump_problem(40, R), rtol=1e-13)
    u48, _ = iso.solve_isolated(_bump_problem(48, R), rtol=1e-13)
    u56, _ = iso.solve_isolated(_bump_problem(56, R), rtol=1e-13)
    ref = np.max(np.abs(u56[sub]))
    assert np.max(np.abs(u48[sub] - u56[sub])) < 1e-7 * ref
    assert np.max(np.abs(u40[sub] - u56[sub])) > 1e-4 * ref
    # and the scatterer does scatter
    assert np.max(np.abs(u56[sub] - iso.isolated_rhs(_bump_problem(56, R))[sub])) > 1e-2 * ref


def test_isolated_gmres_matches_dense_direct_solve():
    p = _cube_problem(8, 6, R=9.0, L=3, Lz=2)
    u_it, info = iso.solve_isolated(p, rtol=1e-14)
    u_lu, _ = iso.solve_isolated(p, direct=True)
    assert np.max(np.abs(u_it - u_lu)) < 1e-12 * np.max(np.abs(u_lu))


def test_no_scatterer_leaves_the_incident_field():
    """V = 0: the operator is the identity exactly and the solve returns E_inc."""
    p = _cube_problem(8, 6, R=9.0, eps=1.0)
    b = iso.isolated_rhs(p)
    assert np.array_equal(iso.apply_isolated(p, b), b)
    u, info = iso.solve_isolated(p)
    assert info["iterations"] <= 1 and np.max(np.abs(u - b)) < 1e-15 * np.max(np.abs(b))


# ---------------------------------------------------------------------------
# Bloch envelopes (the form the CUDA path solves): u_B = u exp(-i q_inc . r_perp), the kernel
# taken at k + q_inc and E_inc = e exp(-i beta z). On a grid where q_inc is a grid frequency
# (q_inc = 2 pi m / (n dx)) the envelope problem is the plain problem with its spectrum moved
# by m bins, which fixes the sign of the shift in the kernel and of the envelope phase.
# ---------------------------------------------------------------------------
_NB, _DB = 40, 1.0
_THB = math.degrees(math.asin(LAM / (_NB * _DB)))  # sin(theta) = lambda / (n dx): one bin


def _grid_wave_problem(phi, bloch, R=12.0, pol=1):
    """A weak scatterer whose permittivity is a raised cosine over the box, (1 - cos)/2 along
    each axis: its spectrum occupies bins -1, 0, 1 only, so each order of multiple scattering
    widens the field's transverse spectrum by one bin, and the Nyquist bins (20 bins away from
    the incident one) are reached only at order ~20, suppressed far below rounding."""
    n, d = _NB, _DB
    t = (1.0 - np.cos(2 * math.pi * np.arange(n) / n)) / 2
    h = t[:, None, None] * t[None, :, None] * t[None, None, :]
    eps = 1.0 + (-0.03 + 0.02j) * h
    return iso.IsolatedProblem(nx=n, ny=n, nz=n, dx=d, dy=d, dz=d, wavelength=LAM, eps_bg=1.0, eps=eps, R=R,
                               theta=_THB, phi=phi, pol=pol, bloch=bloch)


def _bin_shift(phi):
    return {0.0: (1, 0), 90.0: (0, 1), 180.0: (-1, 0)}[phi]


@pytest.mark.parametrize("phi", [0.0, 90.0, 180.0])
def test_bloch_kernel_is_the_plain_kernel_one_bin_over(phi):
    """isolated_kernel(bloch=True) at bin j equals the plain kernel at bin j + m (m the incident
    wavevector in bins), wherever j + m does not wrap past the Nyquist bin. A shift of the wrong
    sign would match bin j - m instead."""
    sx, sy = _bin_shift(phi)
    Gb = iso.isolated_kernel(_grid_wave_problem(phi, True))
    Gp = iso.isolated_kernel(_grid_wave_problem(phi, False))
    n = _NB
    f = np.where(np.arange(n) < n // 2, np.arange(n), np.arange(n) - n)
    okx = (f + sx >= -(n // 2)) & (f + sx < n // 2)
    oky = (f + sy >= -(n // 2)) & (f + sy < n // 2)
    shifted = np.roll(np.roll(Gp, -sx, axis=4), -sy, axis=3)
    sel = (slice(None), slice(None), slice(None), oky, slice(None))
    a = Gb[sel][..., okx]
    b = shifted[sel][..., okx]
    assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(b))
    wrong = np.roll(np.roll(Gp, sx, axis=4), sy, axis=3)[sel][..., okx]
    assert np.max(np.abs(a - wrong)) > 1e-3 * np.max(np.abs(b))


@pytest.mark.parametrize("phi", [0.0, 90.0])
def test_bloch_rhs_is_the_plain_rhs_times_the_envelope(phi):
    pb, pp = _grid_wave_problem(phi, True), _grid_wave_problem(phi, False)
    n, d = _NB, _DB
    qx, qy = iso._q_inc(pp)
    x = np.arange(n) * d
    env = np.exp(1j * (qx * x[None, None, :] + qy * x[None, :, None]))
    assert np.max(np.abs(iso.isolated_rhs(pb) * env[None] - iso.isolated_rhs(pp))) < 1e-13


@pytest.mark.parametrize("phi", [0.0, 90.0])
def test_bloch_solution_times_the_envelope_is_the_plain_solution(phi):
    """With no field spectrum left at the Nyquist bins (the band-limited scatterer above), the
    envelope problem and the plain one are the same problem, so u_B exp(i q_inc . r) = u to
    the solver tolerance. A sign error in the kernel's shift or in the envelope phase changes
    the scattered field at order one."""
    pb, pp = _grid_wave_problem(phi, True), _grid_wave_problem(phi, False)
    ub, _ = iso.solve_isolated(pb, rtol=1e-13)
    up, _ = iso.solve_isolated(pp, rtol=1e-13)
    n, d = _NB, _DB
    qx, qy = iso._q_inc(pp)
    x = np.arange(n) * d
    env = np.exp(1j * (qx * x[None, None, :] + qy * x[None, :, None]))
    scat = up - iso.isolated_rhs(pp)
    assert np.max(np.abs(scat)) > 1e-3 * np.max(np.abs(up))  # the scatterer does scatter
    assert np.max(np.abs(ub * env[None] - up)) < 1e-10 * np.max(np.abs(scat))
