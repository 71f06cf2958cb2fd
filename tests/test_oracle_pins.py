"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms,
an independent route (characteristic matrices, quadrature, explicit DFT sums, a
dense direct solve), invariants and limits. A dropped term, a wrong sign, index or
transposed operand anywhere in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2606_25541_b300 import layouts

K0 = 2 * math.pi / 13.5


def _problem(eps, stack, theta, phi, pol, dx, dz, nf=None):
    nslab, ny, nx = eps.shape
    return layouts.Problem(nx=nx, ny=ny, nslab=nslab, nf=nf or layouts.padded_nf(nslab),
                           dx=dx, dy=dx, dz=dz, wavelength=13.5, eps_bg=1.0, eps=eps,
                           n_layers=stack[0], d_layers=stack[1], n_sub=stack[2],
                           theta_deg=np.array([theta], float), phi_deg=np.array([phi], float),
                           pol=np.array([pol], np.int32))


# ---------------------------------------------------------------------------
# stack response (Sec. 2: transfer matrices / generalized reflection coefficients)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("pol", [0, 1])
def test_parratt_matches_characteristic_matrices_full_stack(pol):
    n_l, d_l, n_s = layouts.ru_mosi_stack(40)
    th = np.radians(np.linspace(0.0, 12.0, 7))
    q2 = (K0 * np.sin(th)) ** 2
    r1 = oracle.parratt_reflection(K0, q2, 1.0, n_l ** 2, d_l, n_s ** 2, pol)
    r2 = oracle.tmm_reflection(K0, q2, 1.0, n_l ** 2, d_l, n_s ** 2, pol)
    assert np.max(np.abs(r1 - r2) / np.abs(r2)) < 1e-12
    # a Bragg mirror: near-normal reflectance of 40 Mo/Si pairs is large
    assert np.all(np.abs(r1) ** 2 > 0.3)


@pytest.mark.parametrize("n_pairs", [1, 4, 9])
def test_quarter_wave_stack_closed_form(n_pairs):
    """Normal incidence on (H L)^N quarter-wave pairs: r = (n0 - Y)/(n0 + Y), Y = (nH/nL)^2N ns."""
    lam = 13.5
    nH, nL, ns = 1.3, 1.1, 1.2
    n_l, d_l = [], []
    for _ in range(n_pairs):
        n_l += [nH, nL]
        d_l += [lam / (4 * nH), lam / (4 * nL)]
    Y = (nH / nL) ** (2 * n_pairs) * ns
    expect = (1.0 - Y) / (1.0 + Y)
    eps = np.array(n_l, complex) ** 2
    r_s = oracle.parratt_reflection(K0, 0.0, 1.0, eps, np.array(d_l), ns ** 2, 0)
    r_p = oracle.parratt_reflection(K0, 0.0, 1.0, eps, np.array(d_l), ns ** 2, 1)
    assert abs(r_s - expect) < 1e-13
    assert abs(r_p + expect) < 1e-13  # H-field convention: r_p = -r_s at normal incidence


def test_brewster_angle_zeroes_p_reflection():
    n = 1.5
    th = math.atan(n)
    q2 = (K0 * math.sin(th)) ** 2
    r_p = oracle.parratt_reflection(K0, q2, 1.0, [], np.zeros(0), n * n, 1)
    r_s = oracle.parratt_reflection(K0, q2, 1.0, [], np.zeros(0), n * n, 0)
    assert abs(r_p) < 1e-14
    assert abs(r_s) > 0.1


@pytest.mark.parametrize("pol", [0, 1])
def test_total_reflection_from_lossless_stack(pol):
    """Substrate index below the ambient's: past the critical angle a lossless stack reflects fully."""
    n_l = np.array([0.95, 0.99, 0.95], complex)
    d_l = np.array([3.0, 4.0, 3.0])
    th = math.radians(75.0)
    q2 = (K0 * math.sin(th)) ** 2
    r = oracle.parratt_reflection(K0, q2, 1.0, n_l ** 2, d_l, 0.9 ** 2, pol)
    assert abs(abs(r) - 1.0) < 1e-13


def test_thick_absorbing_layer_hides_what_is_below():
    n_l = np.array([0.9 + 0.2j, 1.3], complex)
    d_l = np.array([400.0, 5.0])
    r = oracle.parratt_reflection(K0, 0.0, 1.0, n_l ** 2, d_l, 2.0, 0)
    fresnel_top = (1.0 - n_l[0]) / (1.0 + n_l[0])
    assert abs(r - fresnel_top) < 1e-12


# ---------------------------------------------------------------------------
# polarisation triad and reflection matrix (Eq. (9)'s T_R)
# ---------------------------------------------------------------------------
def test_triad_is_bilinear_orthonormal_also_for_evanescent_modes():
    qx = np.array([0.1, 0.9, -1.3])
    qy = np.array([0.2, -0.4, 0.7])
    beta = oracle.upper_sqrt(K0 ** 2 - qx ** 2 - qy ** 2)
    assert beta[1].imag > 0 and beta[2].imag > 0
    s, pu, pd = oracle.triad(qx, qy, beta, K0, 0.0)
    kd = np.stack([qx, qy, -beta])
    ku = np.stack([qx, qy, beta])
    dot = lambda a, b: np.sum(a * b, axis=0)  # noqa: E731
    np.testing.assert_allclose(dot(s, s), 1, atol=1e-14)
    np.testing.assert_allclose(dot(pd, pd), 1, atol=1e-14)
    np.testing.assert_allclose(dot(pu, pu), 1, atol=1e-14)
    np.testing.assert_allclose(dot(s, pd), 0, atol=1e-14)
    np.testing.assert_allclose(dot(kd, pd), 0, atol=1e-14)
    np.testing.assert_allclose(dot(ku, pu), 0, atol=1e-14)
    np.testing.assert_allclose(dot(kd, s), 0, atol=1e-14)


@pytest.mark.parametrize("phi", [0.0, 30.0, 90.0])
def test_normal_incidence_reflection_is_isotropic(phi):
    """At q = 0 the E-field reflection matrix is r_s (xx + yy) whatever the azimuth."""
    eps = np.ones((2, 2, 2), complex)
    p = _problem(eps, layouts.ru_mosi_stack(5), 0.0, phi, 0, 4.0, 2.0)
    ctx = oracle.setup_rhs(p, 0)
    T = ctx.TR[:, :, 0, 0]
    expect = ctx.r_s[0, 0] * np.diag([1, 1, 0])
    np.testing.assert_allclose(T, expect, atol=1e-15)


# ---------------------------------------------------------------------------
# windowed Green's function (Eqs. (13)-(17), one-dimensional periodic reading)
# ---------------------------------------------------------------------------
def _quad_c(f, a, b, points=None):
    re = integrate.quad(lambda t: f(t).real, a, b, points=points, limit=400, epsabs=1e-14,
                        epsrel=1e-13)[0]
    im = integrate.quad(lambda t: f(t).imag, a, b, points=points, limit=400, epsabs=1e-14,
                        epsrel=1e-13)[0]
    return re + 1j * im


def _g1(beta):
    return lambda z: 1j * np.exp(1j * beta * abs(z)) / (2 * beta)


BETAS = [0.4629, 0.21 + 0.0j, 0.0 + 0.8j, 0.3 + 0.02j]


@pytest.mark.parametrize("beta", BETAS)
@pytest.mark.parametrize("l", [0, 1, 5, -8])
def test_green_scalar_matches_quadrature(beta, l):
    nf, dz = 16, 1.0
    L = nf * dz / 2
    kz = 2 * math.pi * l / (nf * dz)
    g1 = _g1(beta)
    ref = 2 * _quad_c(lambda z: g1(z) * math.cos(kz * z), 0.0, L)
    got = oracle.green_scalar(np.array(beta), np.array(l), nf, dz)
    assert abs(got - ref) <= 1e-11 * abs(ref)


def test_green_scalar_removable_limit_is_continuous():
    nf, dz = 32, 1.0
    l = 3
    kap = 2 * math.pi * l / (nf * dz)
    vals = [oracle.green_scalar(np.array(kap + d + 0j), np.array(l), nf, dz)
            for d in (0.0, 1e-12, 1e-9, 1e-6, 1e-4)]
    L = nf * dz / 2
    assert abs(vals[0] - 1j * L / (2 * kap)) < 1e-14 * L / kap
    for d, v in zip((1e-12, 1e-9, 1e-6, 1e-4), vals[1:]):
        g1 = _g1(kap + d)
        ref = 2 * _quad_c(lambda z: g1(z) * math.cos(kap * z), 0.0, L)
        assert abs(v - ref) < 1e-11 * abs(ref)


@pytest.mark.parametrize("beta_idx", range(3))
def test_green_dyadic_matches_quadrature_of_the_spatial_kernel(beta_idx):
    """Each entry of F[G_L] against quadrature of (I + grad grad / kb^2) g1 windowed in z.

    d/dz g1 = -sgn(z) exp(i beta |z|)/2, and d^2/dz^2 g1 = -beta^2 g1 - delta(z); the delta
    sits inside the window and contributes -1/kb^2 to the zz entry.
    """
    nf, dz = 16, 1.0
    L = nf * dz / 2
    kb = K0
    qx, qy = [(0.1, -0.2), (0.35, 0.3), (0.9, 0.4)][beta_idx]
    beta = complex(oracle.upper_sqrt(kb * kb - qx * qx - qy * qy))
    G = oracle.green_dyadic(np.array([[qx]]), np.array([[qy]]), np.array([[beta]]), nf, dz, kb)
    g1 = _g1(beta)
    for l in (0, 2, -3, 7):
        li = l % nf
        kz = 2 * math.pi * l / (nf * dz)
        S = 2 * _quad_c(lambda z: g1(z) * math.cos(kz * z), 0.0, L)
        dg = -2j * _quad_c(lambda z: (-np.exp(1j * beta * z) / 2) * math.sin(kz * z), 0.0, L)
        ref = np.empty((3, 3), complex)
        ref[0, 0] = (1 - qx * qx / kb ** 2) * S
        ref[1, 1] = (1 - qy * qy / kb ** 2) * S
        ref[0, 1] = ref[1, 0] = -qx * qy / kb ** 2 * S
        ref[0, 2] = ref[2, 0] = 1j * qx / kb ** 2 * dg
        ref[1, 2] = ref[2, 1] = 1j * qy / kb ** 2 * dg
        ref[2, 2] = (1 - beta * beta / kb ** 2) * S - 1 / kb ** 2
        got = G[:, :, li, 0, 0]
        assert np.max(np.abs(got - ref)) < 1e-10 * np.max(np.abs(ref)), (l, got, ref)


# ---------------------------------------------------------------------------
# the operator (Eq. (18) with Eq. (9) folded in)
# ---------------------------------------------------------------------------
def test_operator_fft_equals_explicit_dft_sums():
    p = layouts.small_clip(nx=4, ny=6, nslab=3, seed=5, theta=(8.0,), phi=(30.0,), pol=(1,))
    ctx = oracle.setup_rhs(p, 0)
    u = layouts.random_field((3, 3, 6, 4), seed=1)
    a = oracle.apply_operator(ctx, u)
    b = oracle.apply_operator_dft(ctx, u)
    assert np.max(np.abs(a - b)) < 1e-13 * np.max(np.abs(a))


@pytest.mark.parametrize("pol", [0, 1])
def test_gmres_matches_dense_direct_solve(pol):
    p = layouts.small_clip(nx=4, ny=4, nslab=3, seed=7, theta=(6.0,), phi=(20.0,), pol=(pol,))
    o_it, x_it, info = oracle.solve(p, 0, rtol=1e-14)
    o_lu, x_lu, _ = oracle.solve(p, 0, direct=True)
    assert np.max(np.abs(x_it - x_lu)) < 1e-12 * np.max(np.abs(x_lu))
    assert np.max(np.abs(o_it["amp"] - o_lu["amp"])) < 1e-12 * np.max(np.abs(o_lu["amp"]))


def test_absorber_removed_gives_zero_mask_field_and_stack_reflection():
    """V = 0: G*(V u) vanishes bitwise, only the specular order is left and it is r_s / r_p."""
    st = layouts.ru_mosi_stack(40)
    for pol in (0, 1):
        eps = np.ones((5, 4, 4), complex)
        p = _problem(eps, st, 6.0, 0.0, pol, 2.0, 2.0)
        orders, x, info = oracle.solve(p, 0)
        assert np.all(info["E0"] == 0) and np.all(info["Etop"] == 0)
        spec = (orders["m"] == 0) & (orders["n"] == 0)
        assert np.all(orders["amp"][~spec] == 0)
        q2 = (K0 * math.sin(math.radians(6.0))) ** 2
        r = oracle.parratt_reflection(K0, q2, 1.0, st[0] ** 2, st[1], st[2] ** 2, pol)
        a = orders["a_s"][spec][0] if pol == 0 else orders["a_p"][spec][0]
        assert abs(a - r) < 1e-14


@pytest.mark.parametrize("pol,theta", [(0, 6.0), (1, 6.0), (0, 30.0)])
def test_uniform_film_converges_to_parratt_with_film_on_top(pol, theta):
    """A laterally uniform absorber film is a 1-D problem: the LS solution must approach the
    stack recursion with the film as an extra top layer, at second order in dz."""
    n_abs, h = 0.94 + 0.04j, 12.0
    st = layouts.ru_mosi_stack(3)
    errs = []
    for dz in (1.0, 0.5, 0.25):
        nslab = int(round(h / dz))
        eps = np.full((nslab, 1, 1), n_abs ** 2, complex)
        p = _problem(eps, st, theta, 0.0, pol, 10.0, dz)
        orders, _, info = oracle.solve(p, 0)
        ctx = info["ctx"]
        q2 = ctx.qx[0, 0] ** 2 + ctx.qy[0, 0] ** 2
        r = oracle.parratt_reflection(K0, q2, 1.0, np.concatenate([[n_abs ** 2], st[0] ** 2]),
                                      np.concatenate([[h], st[1]]), st[2] ** 2, pol)
        ref = r * np.exp(-2j * ctx.beta00 * h)
        got = orders["a_s"][0] if pol == 0 else orders["a_p"][0]
        errs.append(abs(got - ref) / abs(ref))
    assert errs[-1] < 2e-3
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5


def test_uniform_film_excites_only_the_specular_order():
    st = layouts.ru_mosi_stack(2)
    eps = np.full((4, 4, 4), (0.94 + 0.04j) ** 2, complex)
    p = _problem(eps, st, 6.0, 35.0, 1, 4.0, 2.0)
    orders, _, _ = oracle.solve(p, 0)
    spec = (orders["m"] == 0) & (orders["n"] == 0)
    assert np.max(np.abs(orders["amp"][~spec])) < 1e-13
    assert np.max(np.abs(orders["amp"][spec])) > 1e-2


def test_lossless_absorber_without_stack_conserves_energy():
    eps = layouts.extrude(layouts.contact_hole_mask(8, 8, 4, 4), 8, n_abs=0.94)
    p = _problem(eps, layouts.empty_stack(), 6.0, 0.0, 1, 4.0, 1.0)
    orders, _, info = oracle.solve(p, 0)
    trans = oracle.transmitted_orders(info["ctx"], info["E0"])
    total = orders["eff"].sum() + trans["eff"].sum()
    assert abs(total - 1.0) < 1e-3
    # a lossy absorber must lose energy
    eps2 = layouts.extrude(layouts.contact_hole_mask(8, 8, 4, 4), 8, n_abs=0.94 + 0.04j)
    o2, _, i2 = oracle.solve(_problem(eps2, layouts.empty_stack(), 6.0, 0.0, 1, 4.0, 1.0), 0)
    t2 = oracle.transmitted_orders(i2["ctx"], i2["E0"])
    assert o2["eff"].sum() + t2["eff"].sum() < 0.9


def test_mirror_symmetric_layout_at_normal_incidence_gives_mirrored_orders():
    """x -> -x symmetric layout, theta = 0, s along y: A(-m, n) = diag(-1, 1, 1) A(m, n).
    An odd grid has no Nyquist bin, so the symmetry is exact to rounding."""
    nx = ny = 9
    rng = np.random.default_rng(1)
    cols = rng.random((ny, 5)) < 0.5
    mask = np.stack([cols[:, min(i, nx - i)] for i in range(nx)], axis=1)
    assert (mask == mask[:, (-np.arange(nx)) % nx]).all()
    p = _problem(layouts.extrude(mask, 3), layouts.ru_mosi_stack(2), 0.0, 0.0, 0, 2.5, 2.0, nf=8)
    orders, _, _ = oracle.solve(p, 0)
    amp = {(m, n): a for m, n, a in zip(orders["m"], orders["n"], orders["amp"])}
    assert len(amp) > 4
    err = max(np.max(np.abs(amp[(-m, n)] - np.array([-1, 1, 1]) * a)) for (m, n), a in amp.items())
    assert err < 1e-15


@pytest.mark.parametrize("pol", [0, 1])
def test_rotated_layout_and_illumination_give_rotated_orders(pol):
    """Rotating the layout by 90 deg about z together with phi -> phi + 90 deg maps order
    (m, n) to (-n, m) and rotates its amplitude vector, (Ax, Ay, Az) -> (-Ay, Ax, Az). Odd
    square grid (no Nyquist bin), dx = dy: exact to the solver tolerance."""
    n = 9
    rng = np.random.default_rng(7)
    mask = rng.random((n, n)) < 0.45
    eps = layouts.extrude(mask, 3)
    # eps_rot[y', x'] = eps[y, x] with (x', y') = (-y, x)
    eps_rot = np.ascontiguousarray(eps[:, (-np.arange(n)) % n, :].transpose(0, 2, 1))
    assert np.allclose(eps_rot[:, 2, (-5) % n], eps[:, 5, 2])
    st = layouts.ru_mosi_stack(3)
    p0 = _problem(eps, st, 6.0, 20.0, pol, 2.5, 2.0, nf=8)
    p1 = _problem(eps_rot, st, 6.0, 110.0, pol, 2.5, 2.0, nf=8)
    o0, _, _ = oracle.solve(p0, 0, rtol=1e-14)
    o1, _, _ = oracle.solve(p1, 0, rtol=1e-14)
    a0 = {(m, k): a for m, k, a in zip(o0["m"], o0["n"], o0["amp"])}
    a1 = {(m, k): a for m, k, a in zip(o1["m"], o1["n"], o1["amp"])}
    assert len(a0) == len(a1) > 4
    rot = np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1]])
    scale = max(np.max(np.abs(a)) for a in a0.values())
    err = max(np.max(np.abs(a1[(-k, m)] - rot @ a)) for (m, k), a in a0.items())
    assert err < 1e-11 * scale


def test_rayleigh_anomaly_is_reported():
    eps = np.ones((2, 9, 9), complex)
    p = _problem(eps, layouts.ru_mosi_stack(1), 0.0, 0.0, 0, 13.5 / 9 * 2, 2.0)
    with pytest.raises(oracle.AnomalyError):
        oracle.setup_rhs(p, 0)


# ---------------------------------------------------------------------------
# P7: the decomposition against a conventional PSFD with the stack in the domain
# ---------------------------------------------------------------------------
def _full_domain_error(dz, pol, theta, n_bilayers=2):
    p = layouts.small_clip(nx=8, ny=8, nslab=int(round(4.0 / dz)), dx=4.0, dz=dz, seed=5,
                           stack=layouts.ru_mosi_stack(n_bilayers), theta=(theta,), pol=(pol,))
    o_dec, _, _ = oracle.solve(p, 0, rtol=1e-12, maxiter=800)
    pf, depth = oracle.full_domain_problem(p)
    o_full, _, info = oracle.solve(pf, 0, rtol=1e-12, maxiter=800)
    o_full = oracle.orders_at_old_reference(o_full, info["ctx"], depth)
    key = {(m, n): k for k, (m, n) in enumerate(zip(o_dec["m"], o_dec["n"]))}
    idx = [key[(m, n)] for m, n in zip(o_full["m"], o_full["n"])]
    assert len(idx) == len(key) > 4
    return float(np.linalg.norm(o_full["amp"] - o_dec["amp"][idx]) / np.linalg.norm(o_dec["amp"]))


@pytest.mark.parametrize("pol,theta", [(0, 6.0), (1, 8.0)])
def test_stack_in_the_domain_converges_to_the_decomposition(pol, theta):
    """Sec. 4 compares the background-field method with a conventional PSFD that meshes
    the Mo/Si stack: here Ru + 2 bilayers are voxelised (thickness-weighted permittivity per
    cell, layers not aligned with the grid) below the absorber, the reflection operator keeps
    only the substrate interface, and the reflected orders (moved to the same reference plane)
    approach those of the analytic-stack decomposition as dz shrinks."""
    errs = [_full_domain_error(dz, pol, theta) for dz in (0.5, 0.25, 0.125)]
    assert errs[1] < errs[0] / 2 and errs[2] < errs[1] / 1.8, errs
    assert errs[2] < 1.5e-3, errs


def test_single_mode_restriction_equals_the_full_operator():
    """The one-mode form used to check large grids mode by mode reproduces the xy spectrum
    of u - A u of the full (pinned) operator, including the Nyquist index and modes whose
    signed indices wrap around."""
    p = layouts.small_clip(nx=16, ny=8, nslab=5, dx=2.0, dz=1.5, seed=3, stack=layouts.ru_mosi_stack(10))
    p = p.with_illumination([7.0], [20.0], [1])
    u = layouts.random_field((3, 5, 8, 16), seed=2)
    W = np.fft.fft2(u - oracle.apply_operator(oracle.setup_rhs(p, 0), u), axes=(2, 3))
    for m, n in [(0, 0), (3, -2), (-8, 3), (7, -4), (-1, -4)]:
        got = oracle.scattered_spectrum_mode(p, 0, u, m, n)
        ref = W[:, :, n % 8, m % 16]
        assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()


# ---------------------------------------------------------------------------
# the outer fixed-point iteration of Eq. (8)
# ---------------------------------------------------------------------------
def _fixed_point_clip(stack, pol=1):
    return layouts.small_clip(nx=4, ny=4, nslab=3, seed=7, theta=(6.0,), phi=(20.0,), pol=(pol,),
                              stack=stack)


@pytest.mark.parametrize("n_bilayers,pol", [(3, 1), (40, 0)])
def test_fixed_point_converges_to_the_folded_dense_solution(n_bilayers, pol):
    """At the fixed point of Eq. (8) E_mask stops changing, so R[E_inc + E_mask] is
    consistent with the solution and the loop lands on the folded system A u = b, here
    solved by dense LU; the orders agree as well."""
    p = _fixed_point_clip(layouts.ru_mosi_stack(n_bilayers), pol)
    o_fp, u_fp, info = oracle.solve_fixed_point(p, 0, rtol=1e-12)
    o_lu, u_lu, _ = oracle.solve(p, 0, direct=True)
    assert info["converged"] and 3 <= info["outer"] <= 30
    assert np.max(np.abs(u_fp - u_lu)) < 1e-10 * np.max(np.abs(u_lu))
    assert np.max(np.abs(o_fp["amp"] - o_lu["amp"])) < 1e-10 * np.max(np.abs(o_lu["amp"]))
    ch = info["changes"]
    assert all(b < a for a, b in zip(ch, ch[1:])), ch  # a contraction on this clip


def test_fixed_point_iterates_follow_the_operator_splitting():
    """Outer step k solves M u_k = b + (M - A) u_(k-1), u_0 = 0, with M the free-space
    operator (dense, from the reflection-free operator) and A the folded one (dense): the
    reflection of the previous mask field built from plane 0, T_R and exp(i beta z) must
    equal (M - A) u_(k-1) on the absorber planes, and the reported change is its step."""
    p = _fixed_point_clip(layouts.ru_mosi_stack(5))
    ctx, free = oracle.setup_rhs(p, 0), oracle.setup_rhs(p, 0, reflection=False)
    A = oracle.dense_operator(ctx)
    M = oracle.dense_operator(free, lambda v: oracle.apply_operator(free, v))
    b = oracle.rhs_vector(ctx).reshape(-1)
    u_prev = np.zeros_like(b)
    for k in (1, 2, 3):
        u_k = np.linalg.solve(M, b + (M - A) @ u_prev)
        _, u, info = oracle.solve_fixed_point(p, 0, rtol=0.0, max_outer=k, inner_rtol=1e-15)
        assert info["outer"] == k and not info["converged"]
        assert np.max(np.abs(u.reshape(-1) - u_k)) < 1e-12 * np.max(np.abs(u_k)), k
        step = np.linalg.norm((M - A) @ (u_k - u_prev)) / np.linalg.norm(b)
        assert abs(info["changes"][-1] - step) < 1e-9 * step, (k, info["changes"], step)
        u_prev = u_k


def test_fixed_point_without_stack_is_a_single_free_space_solve():
    """No stack and a vacuum substrate: T_R = 0, R vanishes, the first outer step already
    has a zero change and its field is the plain free-space solution."""
    p = _fixed_point_clip(layouts.empty_stack())
    o_fp, u_fp, info = oracle.solve_fixed_point(p, 0, rtol=1e-12)
    o_lu, u_lu, _ = oracle.solve(p, 0, direct=True)
    assert info["outer"] == 1 and info["changes"] == [0.0]
    assert np.max(np.abs(u_fp - u_lu)) < 1e-11 * np.max(np.abs(u_lu))
