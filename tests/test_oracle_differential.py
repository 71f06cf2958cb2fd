"""Pins of the differential (curl-curl) PSFD oracle and the preconditioner comparison of Sec. 3:
the spectral curl-curl of a single Fourier mode, convergence of a film's reflection to the
stack recursion through the PML-terminated column, and the ordering of the preconditioners
(none, spectral damping, Lippmann-Schwinger) on a small synthetic clip."""
import math

import numpy as np

import oracle
from oracle import differential_oracle as dif
from paper_2606_25541_b300 import layouts

LAM = 13.5
K0 = 2 * math.pi / LAM


def test_curl_curl_of_a_fourier_mode():
    """Without PML, curl curl (v exp(i k.r)) = (|k|^2 v - k (k.v)) exp(i k.r) for every grid mode
    (Bloch offset included): the spectral derivatives of Eq. (6) reproduce it to rounding."""
    p = dif.DiffProblem(nx=8, ny=6, nz=10, dx=3.0, dy=2.5, dz=2.0, wavelength=LAM, eps_bg=1.0,
                        eps=np.ones((10, 6, 8), np.complex128), n_pml=0, theta=7.0, phi=30.0)
    g = dif._geometry(p)
    k0, kb, qix, qiy, qx, qy, kz, s = g
    z, y, x = np.arange(p.nz) * p.dz, np.arange(p.ny) * p.dy, np.arange(p.nx) * p.dx
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    v = np.array([0.3 + 0.1j, -0.7 + 0.2j, 0.5 - 0.4j])
    for m, n, l in [(2, -1, 3), (0, 0, 0), (-4, 3, -5), (1, 2, 5)]:
        kvec = np.array([qx[m], qy[n], kz[l]])
        ph = np.exp(1j * ((qx[m] - qix) * X + (qy[n] - qiy) * Y + kz[l] * Z))
        E = v[:, None, None, None] * ph[None]
        expect = ((kvec @ kvec) * v - kvec * (kvec @ v) - k0 * k0 * v)[:, None, None, None] * ph[None]
        got = dif.apply_differential(p, E, g)
        assert np.max(np.abs(got - expect)) < 1e-13 * np.max(np.abs(expect)), (m, n, l)


def test_film_reflection_converges_to_the_stack_recursion():
    """An 8 nm absorber film in vacuum, normal incidence, s: the reflected amplitude read in the
    upper spacer of the PML-terminated column approaches the Parratt value at second order in
    dz (cell-centred film boundaries)."""
    n, t = 0.94 + 0.04j, 8.0
    r_ex = complex(oracle.parratt_reflection(K0, np.array(0.0), 1.0, np.array([n * n]), np.array([t]), 1.0 + 0j, 0))
    errs = []
    for dz in (1.0, 0.5, 0.25):
        npml, ns, nsl = int(round(40 / dz)), int(round(20 / dz)), int(round(t / dz))
        nz = 2 * npml + 2 * ns + nsl
        eps = np.ones((nz, 1, 1), np.complex128)
        a = npml + ns
        eps[a:a + nsl] = n * n
        p = dif.DiffProblem(nx=1, ny=1, nz=nz, dx=10.0, dy=10.0, dz=dz, wavelength=LAM, eps_bg=1.0, eps=eps,
                            n_pml=npml, theta=0.0, phi=0.0, pol=0)
        g = dif._geometry(p)
        E, mv, res = dif.gmres_restarted(lambda v: dif.apply_differential(p, v, g), dif.differential_rhs(p, g),
                                         rtol=1e-11, restart=200)
        assert res <= 1e-11
        r = dif.reflected_amplitude_film(p, E, (a + nsl - 0.5) * dz, g)
        errs.append(abs(r - r_ex) / abs(r_ex))
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs
    assert errs[2] < 3e-3, errs


def test_green_function_preconditioner_needs_far_fewer_iterations():
    """The comparison of Sec. 3 (its preconditioner table) on a seeded 8 x 8 x 8 clip at 4 nm in
    free space, GMRES(60) to 1e-8: the Lippmann-Schwinger form needs over ten times fewer
    operator applications than the spectrally damped differential system, which needs fewer
    than the unpreconditioned one."""
    p = layouts.small_clip(nx=8, ny=8, nslab=8, dx=4.0, dz=4.0, seed=3, stack=layouts.empty_stack(),
                           theta=(6.0,), pol=(0,))
    out = dif.preconditioner_study(p, 0, rtol=1e-8, restart=60, maxiter=30000)
    assert all(res <= 1e-8 for _, res in out.values()), out
    none, damp, ls = out["none"][0], out["spectral_damping"][0], out["lippmann_schwinger"][0]
    assert none > damp > 10 * ls, out
