"""Plain FP64 CPU oracle of the background-field Lippmann-Schwinger PSFD method.

Test infrastructure only: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``; nothing on the product path may call it.

Everything is complex128, written for reading rather than speed. The discrete Fourier
transforms are the oracle's own (``oracle/fft.py``, pinned against the direct sums) and dense
linear algebra serves as a library primitive; there is no blocking, fusion or
reordering beyond the steps below. Paper references are to arXiv 2606.25541
(Lee, Gillijns, Kim: "Pseudo-spectral frequency-domain method with background field
decomposition and Green's function preconditioner ..."), by section and equation.

The discrete problem (the same on the CUDA side, derived independently there):

* Sec. 2, Eq. (3): the mask field solves a free-space scattering problem driven by
  the incident field plus the stack reflection R[E_inc + E_mask].
* Sec. 3, Eqs. (11)-(12), (18): Lippmann-Schwinger form x - G*(V x) = G*(V b) with
  V = k0^2 (eps - eps_bg), evaluated with FFTs and a windowed Green's function.
* Sec. 3, Eq. (9): R acts per transverse Fourier mode with the stack's reflection
  matrix T_R and propagates upward with exp(i k_z (z - z_top)).

Readings where the paper is silent or written for another geometry (each is stated
again at the function that uses it):

* periodic clips: the transverse directions are Bloch-periodic (diffraction orders),
  so the Green's function is taken per transverse mode q exactly and windowed only
  in z, |z| < L = nf*dz/2 -- the one-dimensional analogue of the windowed kernel of
  Eqs. (13)-(17);
* R is folded into the operator: the unknown u is the total field on the absorber
  planes and A u = u - (I + R) G*(V u); this has the fixed point of the outer
  iteration of Eq. (8);
* absorber planes are cell centred, z_p = (p - 1/2) dz above z_top for p = 1..nslab;
  plane 0 (z = -dz/2) samples the downgoing mask field for R, plane nslab+1 the
  upgoing field for the reflected orders;
* p polarisation uses the H-field Fresnel coefficients and the bilinear triad
  s, p+-, so T_R = r_s s s^T + r_p p+ p-^T.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import fft as offt

__all__ = [
    "upper_sqrt", "fft_integers", "parratt_reflection", "tmm_reflection", "triad",
    "green_scalar", "green_dyadic", "RhsContext", "setup_rhs", "apply_operator",
    "apply_operator_dft", "rhs_vector", "gmres", "dense_operator", "diffraction_orders",
    "transmitted_orders", "solve", "solve_all", "AnomalyError", "full_domain_problem",
    "orders_at_old_reference", "scattered_spectrum_mode", "reflected_field", "solve_fixed_point",
]


class AnomalyError(ValueError):
    """A diffraction order grazes the interface (beta = 0, a Rayleigh anomaly)."""


# ---------------------------------------------------------------------------
# elementary pieces
# ---------------------------------------------------------------------------
def upper_sqrt(z):
    """Square root on the branch with Im >= 0 (outgoing or decaying wave)."""
    s = np.sqrt(np.asarray(z, dtype=np.complex128))
    flip = (s.imag < 0) | ((s.imag == 0) & (s.real < 0))
    return np.where(flip, -s, s)


def fft_integers(n: int) -> np.ndarray:
    """Signed integer frequency of each FFT bin (numpy order; the Nyquist bin is negative)."""
    return np.rint(offt.fftfreq(n) * n).astype(np.int64)


# ---------------------------------------------------------------------------
# stack response, Sec. 2 ("transfer matrix method or generalized reflection
# coefficients") and Eq. (9)'s T_R
# ---------------------------------------------------------------------------
def _fresnel(kz_i, kz_j, eps_i, eps_j, pol):
    if pol == 0:  # s: E-field amplitude ratio
        return (kz_i - kz_j) / (kz_i + kz_j)
    # p: H-field amplitude ratio
    return (eps_j * kz_i - eps_i * kz_j) / (eps_j * kz_i + eps_i * kz_j)


def parratt_reflection(k0, q2, eps_amb, eps_layers, d_layers, eps_sub, pol):
    """Reflection coefficient of a planar stack seen from the ambient medium at z_top.

    Generalized reflection coefficients (Parratt/Airy recursion) from the substrate
    upward: Gamma_M = r_{M,M+1}, Gamma_{j-1} = (r + Gamma_j e)/(1 + r Gamma_j e) with
    r = r_{j-1,j} and e = exp(2 i k_zj d_j). `q2` is the squared transverse wavenumber
    (array), media top to bottom are ambient, layers 1..M, substrate.
    """
    eps_all = [complex(eps_amb)] + [complex(e) for e in eps_layers] + [complex(eps_sub)]
    kz = [upper_sqrt(k0 * k0 * e - q2) for e in eps_all]
    m = len(eps_layers)
    gamma = _fresnel(kz[m], kz[m + 1], eps_all[m], eps_all[m + 1], pol)
    for j in range(m, 0, -1):
        e = np.exp(2j * kz[j] * d_layers[j - 1])
        r = _fresnel(kz[j - 1], kz[j], eps_all[j - 1], eps_all[j], pol)
        gamma = (r + gamma * e) / (1.0 + r * gamma * e)
    return gamma


def tmm_reflection(k0, q2, eps_amb, eps_layers, d_layers, eps_sub, pol):
    """Same reflection coefficient by 2x2 characteristic matrices (an independent route).

    The tangential pair (psi, psi'/c) -- psi = E_y, c = 1 for s; psi = H_y, c = eps for p
    -- is carried from a purely transmitted wave in the substrate up through every
    layer; in the ambient it is split into downgoing (a) and upgoing (b) parts, r = b/a.
    Only usable where no layer is strongly evanescent (the matrices grow exponentially).
    """
    q2 = np.asarray(q2, dtype=np.complex128)

    def c_of(e):
        return 1.0 if pol == 0 else e

    ks = upper_sqrt(k0 * k0 * eps_sub - q2)
    psi = np.ones_like(q2)
    dpsi = -1j * ks / c_of(complex(eps_sub))
    for j in range(len(eps_layers) - 1, -1, -1):
        e = complex(eps_layers[j])
        k = upper_sqrt(k0 * k0 * e - q2)
        c = c_of(e)
        cs, sn = np.cos(k * d_layers[j]), np.sin(k * d_layers[j])
        psi, dpsi = cs * psi + (c / k) * sn * dpsi, -(k / c) * sn * psi + cs * dpsi
    k_a = upper_sqrt(k0 * k0 * eps_amb - q2)
    diff = dpsi * c_of(complex(eps_amb)) / (1j * k_a)  # = b - a
    a = 0.5 * (psi - diff)
    b = 0.5 * (psi + diff)
    return b / a


def triad(qx, qy, beta, kb, phi_rad):
    """Bilinear polarisation triad of each transverse mode.

    s = z x q/|q| (at q = 0: the azimuth of the illumination breaks the tie), and
    p+- = k+- x s / kb with k+- = (qx, qy, +-beta). Dot products are bilinear (no
    conjugation) so s.s = p-.p- = 1 also for evanescent beta.
    """
    qn = np.sqrt(qx * qx + qy * qy)
    zero = qn == 0
    safe = np.where(zero, 1.0, qn)
    qhx = np.where(zero, math.cos(phi_rad), qx / safe)
    qhy = np.where(zero, math.sin(phi_rad), qy / safe)
    s_hat = np.stack([-qhy, qhx, np.zeros_like(qhx)]).astype(np.complex128)
    k_up = np.stack([qx + 0j, qy + 0j, beta])
    k_dn = np.stack([qx + 0j, qy + 0j, -beta])
    p_up = np.cross(k_up, s_hat, axis=0) / kb
    p_dn = np.cross(k_dn, s_hat, axis=0) / kb
    return s_hat, p_up, p_dn


# ---------------------------------------------------------------------------
# windowed Green's function, Sec. 3 Eqs. (13)-(17), periodic-transverse reading
# ---------------------------------------------------------------------------
def green_scalar(beta, l_int, nf, dz):
    """S = int_{-L}^{L} g1(z) exp(-i kz z) dz with g1 = i exp(i beta |z|)/(2 beta), L = nf dz/2.

    For kz = 2 pi l/(nf dz) one has kz L = pi l and
        S = (1 - (-1)^l exp(i beta L)) / (kz^2 - beta^2),
    the one-dimensional analogue of the k != k_bg branch of Eq. (17). At kz^2 = beta^2
    the singularity is removable: with w = i(beta - |kz|) L,
        S = i L phi1(w) / (|kz| + beta),  phi1(w) = (e^w - 1)/w,
    which is used (as a Taylor series of phi1) wherever |w| is small.
    """
    L = 0.5 * nf * dz
    kz = 2.0 * math.pi * np.asarray(l_int, dtype=np.float64) / (nf * dz)
    sign = np.where(np.asarray(l_int) % 2 == 0, 1.0, -1.0)
    beta = np.asarray(beta, dtype=np.complex128)
    kap = np.abs(kz)
    w = 1j * (beta - kap) * L
    near = np.abs(w) < 1e-2
    denom = kz * kz - beta * beta
    plain = (1.0 - sign * np.exp(1j * beta * L)) / np.where(near, 1.0, denom)
    phi1 = 1.0 + w / 2 + w ** 2 / 6 + w ** 3 / 24 + w ** 4 / 120 + w ** 5 / 720 + w ** 6 / 5040 \
        + w ** 7 / 40320
    series = 1j * L * phi1 / (kap + beta)
    return np.where(near, series, plain)


def green_dyadic(qx, qy, beta, nf, dz, kb):
    """Windowed dyadic Green's function per (kz_l, mode): array (3, 3, nf, ny, nx).

    G = (I + grad grad / kb^2) g (Eq. (14)) with grad -> (i qx, i qy, d/dz) per
    transverse mode; windowing after differentiation (Eq. (13)) gives, with
    k = (qx, qy, kz_l) and E = (-1)^l exp(i beta L):
        F[G_L] = S (I - k k^T / kb^2) - (E / kb^2) z z^T,
    where the z z^T term is the boundary value of d/dz g1 at |z| = L together with the
    delta function of d^2/dz^2 g1 at z = 0 (inside the window).
    """
    l_int = fft_integers(nf)
    L = 0.5 * nf * dz
    kz = 2.0 * math.pi * l_int / (nf * dz)
    S = green_scalar(beta[None, :, :], l_int[:, None, None], nf, dz)  # (nf, ny, nx)
    sign = np.where(l_int % 2 == 0, 1.0, -1.0)[:, None, None]
    E = sign * np.exp(1j * beta[None] * L)
    kvec = [np.broadcast_to(qx[None], S.shape), np.broadcast_to(qy[None], S.shape),
            np.broadcast_to(kz[:, None, None], S.shape)]
    G = np.empty((3, 3) + S.shape, dtype=np.complex128)
    for a in range(3):
        for b in range(3):
            G[a, b] = S * ((1.0 if a == b else 0.0) - kvec[a] * kvec[b] / (kb * kb))
    G[2, 2] -= E / (kb * kb)
    return G


# ---------------------------------------------------------------------------
# per right-hand-side set-up
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class RhsContext:
    nx: int
    ny: int
    nslab: int
    nf: int
    dz: float
    k0: float
    kb: float
    qx: np.ndarray
    qy: np.ndarray
    beta: np.ndarray  # (ny, nx)
    V: np.ndarray  # (nslab, ny, nx)
    G: np.ndarray  # (3, 3, nf, ny, nx)
    TR: np.ndarray  # (3, 3, ny, nx)
    r_s: np.ndarray
    r_p: np.ndarray
    s_hat: np.ndarray
    p_up: np.ndarray
    p_dn: np.ndarray
    e_inc: np.ndarray  # (3,)
    beta00: complex
    mi: np.ndarray  # signed order index along x, (nx,)
    ni: np.ndarray  # signed order index along y, (ny,)


def _mode_tables(prob, i: int, mi: np.ndarray, ni: np.ndarray, reflection: bool = True):
    """Wavevectors, beta, stack reflection and triad of the transverse modes (ni, mi) (2-D
    arrays of signed order indices) for illumination i."""
    k0 = 2.0 * math.pi / prob.wavelength
    kb = k0 * math.sqrt(prob.eps_bg)
    th = math.radians(float(prob.theta_deg[i]))
    ph = math.radians(float(prob.phi_deg[i]))
    qix = kb * math.sin(th) * math.cos(ph)
    qiy = kb * math.sin(th) * math.sin(ph)
    qx = qix + 2.0 * math.pi * mi / (prob.nx * prob.dx)
    qy = qiy + 2.0 * math.pi * ni / (prob.ny * prob.dy)
    q2 = qx * qx + qy * qy
    beta = upper_sqrt(kb * kb - q2)
    if np.any(np.abs(beta) < 1e-9 * k0):
        raise AnomalyError("a diffraction order has beta = 0 (Rayleigh anomaly)")
    eps_l = np.asarray(prob.n_layers, np.complex128) ** 2
    eps_s = complex(prob.n_sub) ** 2
    if reflection:
        r_s = parratt_reflection(k0, q2, prob.eps_bg, eps_l, prob.d_layers, eps_s, 0)
        r_p = parratt_reflection(k0, q2, prob.eps_bg, eps_l, prob.d_layers, eps_s, 1)
    else:
        r_s = np.zeros_like(beta)
        r_p = np.zeros_like(beta)
    s_hat, p_up, p_dn = triad(qx, qy, beta, kb, ph)
    TR = r_s[None, None] * s_hat[:, None] * s_hat[None, :] \
        + r_p[None, None] * p_up[:, None] * p_dn[None, :]
    return k0, kb, qx, qy, beta, r_s, r_p, s_hat, p_up, p_dn, TR


def setup_rhs(prob, i: int, reflection: bool = True) -> RhsContext:
    """Mode wavevectors, stack tables, Green's function and potential for one illumination."""
    mi = fft_integers(prob.nx)
    ni = fft_integers(prob.ny)
    k0, kb, qx, qy, beta, r_s, r_p, s_hat, p_up, p_dn, TR = _mode_tables(
        prob, i, mi[None, :] + 0 * ni[:, None], ni[:, None] + 0 * mi[None, :], reflection)
    e_inc = s_hat[:, 0, 0] if int(prob.pol[i]) == 0 else p_dn[:, 0, 0]
    V = k0 * k0 * (np.asarray(prob.eps, np.complex128) - prob.eps_bg)
    G = green_dyadic(qx, qy, beta, prob.nf, prob.dz, kb)
    return RhsContext(prob.nx, prob.ny, prob.nslab, prob.nf, prob.dz, k0, kb, qx, qy, beta, V,
                      G, TR, r_s, r_p, s_hat, p_up, p_dn, np.array(e_inc), complex(beta[0, 0]),
                      mi, ni)


# ---------------------------------------------------------------------------
# the operator, Eq. (18) with Eq. (9) folded in
# ---------------------------------------------------------------------------
def _reflect_and_invert(ctx: RhsContext, Wt: np.ndarray):
    """Add R (Eq. (9)) to the z-inverse-transformed field and undo the xy transform.

    Wt holds the xy spectrum (unnormalised DFT convention) on all nf z planes. Plane 0
    (z = -dz/2) carries the downgoing mask field; it is moved to z_top by
    exp(-i beta dz/2), reflected with T_R and propagated up to plane p
    (z = (p - 1/2) dz) by exp(i beta (p - 1/2) dz): in total exp(i beta (p - 1) dz).
    """
    n = ctx.nslab
    R0 = np.einsum("abyx,byx->ayx", ctx.TR, Wt[:, 0])
    steps = np.arange(n, dtype=np.float64)[:, None, None]
    phase = np.exp(1j * ctx.beta[None] * ctx.dz * steps)
    W_slab = Wt[:, 1:n + 1] + R0[:, None] * phase[None]
    return offt.ifft2(W_slab, axes=(2, 3))


def apply_operator(ctx: RhsContext, u: np.ndarray, return_side: bool = False):
    """A u = u - (I + R) G*(V u) on the absorber planes; u has shape (3, nslab, ny, nx).

    Eq. (18): FFT_xyz, the dyadic product per wavevector, inverse FFT; numpy's
    unnormalised forward / 1/N inverse convention realises the convolution integral
    without explicit cell-volume factors. z is zero padded from nslab to nf planes
    (the padding of Sec. 3 that turns the periodic into a linear convolution).
    Optionally returns the normalised xy Fourier coefficients of G*(V u) on plane 0
    and plane nslab+1 (used for the diffraction orders).
    """
    n = ctx.nslab
    J = np.zeros((3, ctx.nf, ctx.ny, ctx.nx), dtype=np.complex128)
    J[:, 1:n + 1] = ctx.V[None] * u
    Jh = offt.fftn(J, axes=(1, 2, 3))
    Wh = np.einsum("ablyx,blyx->alyx", ctx.G, Jh)
    Wt = offt.ifft(Wh, axis=1)
    w = _reflect_and_invert(ctx, Wt)
    Au = u - w
    if return_side:
        norm = 1.0 / (ctx.nx * ctx.ny)
        return Au, Wt[:, 0] * norm, Wt[:, n + 1] * norm
    return Au


def _dft_matrix(n, sign):
    k = np.arange(n)
    return np.exp(sign * 2j * math.pi * np.outer(k, k) / n)


def apply_operator_dft(ctx: RhsContext, u: np.ndarray) -> np.ndarray:
    """The same operator with every transform written as an explicit O(N^2) DFT sum."""
    n = ctx.nslab
    J = np.zeros((3, ctx.nf, ctx.ny, ctx.nx), dtype=np.complex128)
    J[:, 1:n + 1] = ctx.V[None] * u
    Fz, Fy, Fx = _dft_matrix(ctx.nf, -1), _dft_matrix(ctx.ny, -1), _dft_matrix(ctx.nx, -1)
    Jh = np.einsum("lz,ky,mx,czyx->clkm", Fz, Fy, Fx, J)
    Wh = np.einsum("ablyx,blyx->alyx", ctx.G, Jh)
    Wt = np.einsum("zl,clyx->czyx", _dft_matrix(ctx.nf, +1), Wh) / ctx.nf
    R0 = np.einsum("abyx,byx->ayx", ctx.TR, Wt[:, 0])
    steps = np.arange(n, dtype=np.float64)[:, None, None]
    W_slab = Wt[:, 1:n + 1] + R0[:, None] * np.exp(1j * ctx.beta[None] * ctx.dz * steps)[None]
    Gy, Gx = _dft_matrix(ctx.ny, +1), _dft_matrix(ctx.nx, +1)
    w = np.einsum("yk,xm,czkm->czyx", Gy, Gx, W_slab) / (ctx.nx * ctx.ny)
    return u - w


def rhs_vector(ctx: RhsContext) -> np.ndarray:
    """b = E_inc + R[E_inc] on the absorber planes (Eqs. (3), (9)); uniform in x, y.

    E_inc = e exp(-i beta00 z) (downgoing, Bloch envelope); its reflection is
    T_R(q00) e exp(+i beta00 z); z_p = (p - 1/2) dz.
    """
    zc = (np.arange(1, ctx.nslab + 1) - 0.5) * ctx.dz
    down = np.exp(-1j * ctx.beta00 * zc)
    up = np.exp(1j * ctx.beta00 * zc)
    refl = ctx.TR[:, :, 0, 0] @ ctx.e_inc
    col = ctx.e_inc[:, None] * down[None] + refl[:, None] * up[None]  # (3, nslab)
    return np.ascontiguousarray(np.broadcast_to(col[:, :, None, None],
                                                (3, ctx.nslab, ctx.ny, ctx.nx))).astype(np.complex128)


# ---------------------------------------------------------------------------
# Krylov solver and dense cross-check, Sec. 3 (GMRES, Saad & Schultz)
# ---------------------------------------------------------------------------
def gmres(apply, b: np.ndarray, rtol: float = 1e-13, maxiter: int = 500, history=None):
    """Unrestarted GMRES with modified Gram-Schmidt; the small least-squares problem is
    solved directly at every step. Returns (x, iterations, relative residual)."""
    shape = b.shape
    bv = b.reshape(-1)
    bnorm = np.linalg.norm(bv)
    if bnorm == 0.0:
        return np.zeros_like(b), 0, 0.0
    Q = [bv / bnorm]
    H = np.zeros((maxiter + 1, maxiter), dtype=np.complex128)
    y = np.zeros(0, np.complex128)
    res = 1.0
    j = 0
    for j in range(maxiter):
        w = apply(Q[j].reshape(shape)).reshape(-1)
        for i in range(j + 1):
            H[i, j] = np.vdot(Q[i], w)
            w = w - H[i, j] * Q[i]
        H[j + 1, j] = np.linalg.norm(w)
        e1 = np.zeros(j + 2, np.complex128)
        e1[0] = bnorm
        y, *_ = np.linalg.lstsq(H[:j + 2, :j + 1], e1, rcond=None)
        res = np.linalg.norm(e1 - H[:j + 2, :j + 1] @ y) / bnorm
        if history is not None:
            history.append(res)
        if res <= rtol or H[j + 1, j] == 0:
            break
        Q.append(w / H[j + 1, j])
    x = np.zeros_like(bv)
    for i, yi in enumerate(y):
        x = x + yi * Q[i]
    return x.reshape(shape), j + 1, float(res)


def dense_operator(ctx: RhsContext, apply=None) -> np.ndarray:
    """The operator as a dense matrix, built column by column from unit vectors."""
    apply = apply or (lambda v: apply_operator(ctx, v))
    shape = (3, ctx.nslab, ctx.ny, ctx.nx)
    n = int(np.prod(shape))
    A = np.empty((n, n), dtype=np.complex128)
    for k in range(n):
        e = np.zeros(n, np.complex128)
        e[k] = 1.0
        A[:, k] = apply(e.reshape(shape)).reshape(-1)
    return A


# ---------------------------------------------------------------------------
# diffraction orders, Eqs. (3), (9)
# ---------------------------------------------------------------------------
def diffraction_orders(ctx: RhsContext, E0: np.ndarray, Etop: np.ndarray):
    """Reflected plane-wave amplitudes, referenced to z_top, of every propagating order.

    A_mn = T_R (delta_{mn,00} e + E0 exp(-i beta dz/2)) + Etop exp(-i beta (nslab+1/2) dz):
    the stack reflects the incident wave and the downgoing mask field (known on plane 0),
    and the upgoing mask field is read on plane nslab+1 above the absorber.
    Returns a dict of arrays over the propagating orders.
    """
    n = ctx.nslab
    inc = np.zeros((3, ctx.ny, ctx.nx), np.complex128)
    inc[:, 0, 0] = ctx.e_inc
    down = inc + E0 * np.exp(-0.5j * ctx.beta * ctx.dz)[None]
    A = np.einsum("abyx,byx->ayx", ctx.TR, down) \
        + Etop * np.exp(-1j * ctx.beta * (n + 0.5) * ctx.dz)[None]
    prop = (ctx.qx ** 2 + ctx.qy ** 2) < ctx.kb ** 2
    ys, xs = np.nonzero(prop)
    amp = A[:, ys, xs].T  # (n_orders, 3)
    a_s = np.einsum("oa,ao->o", amp, ctx.s_hat[:, ys, xs])
    a_p = np.einsum("oa,ao->o", amp, ctx.p_up[:, ys, xs])
    eff = np.sum(np.abs(amp) ** 2, axis=1) * ctx.beta[ys, xs].real / ctx.beta00.real
    return {"m": ctx.mi[xs], "n": ctx.ni[ys], "amp": amp, "a_s": a_s, "a_p": a_p, "eff": eff}


def transmitted_orders(ctx: RhsContext, E0: np.ndarray):
    """Downgoing amplitudes at z_top (meaningful when there is no stack, T_R = 0)."""
    inc = np.zeros((3, ctx.ny, ctx.nx), np.complex128)
    inc[:, 0, 0] = ctx.e_inc
    T = inc + E0 * np.exp(-0.5j * ctx.beta * ctx.dz)[None]
    prop = (ctx.qx ** 2 + ctx.qy ** 2) < ctx.kb ** 2
    ys, xs = np.nonzero(prop)
    amp = T[:, ys, xs].T
    eff = np.sum(np.abs(amp) ** 2, axis=1) * ctx.beta[ys, xs].real / ctx.beta00.real
    return {"m": ctx.mi[xs], "n": ctx.ni[ys], "amp": amp, "eff": eff}


def solve(prob, i: int = 0, rtol: float = 1e-13, maxiter: int = 500, direct: bool = False,
          reflection: bool = True, history=None):
    """Solve one illumination; returns (orders, solution u, info dict). `history`, if given,
    receives GMRES's relative residual after every iteration."""
    ctx = setup_rhs(prob, i, reflection=reflection)
    b = rhs_vector(ctx)
    if direct:
        A = dense_operator(ctx)
        x = np.linalg.solve(A, b.reshape(-1)).reshape(b.shape)
        its, res = 0, float(np.linalg.norm(A @ x.reshape(-1) - b.reshape(-1)) / np.linalg.norm(b))
    else:
        x, its, res = gmres(lambda v: apply_operator(ctx, v), b, rtol=rtol, maxiter=maxiter, history=history)
    _, E0, Etop = apply_operator(ctx, x, return_side=True)
    orders = diffraction_orders(ctx, E0, Etop)
    return orders, x, {"iterations": its, "relres": res, "ctx": ctx, "E0": E0, "Etop": Etop}


# ---------------------------------------------------------------------------
# the outer fixed-point iteration of Eq. (8)
# ---------------------------------------------------------------------------
def reflected_field(ctx: RhsContext, D: np.ndarray) -> np.ndarray:
    """R[E] on the absorber planes, Eq. (9), for a downgoing field given by its normalised
    xy Fourier coefficients D (shape (3, ny, nx)) at z_top:
    FFT_xy^-1[T_R D] exp(i beta (z_p - z_top)), z_p = (p - 1/2) dz, p = 1..nslab."""
    zc = (np.arange(1, ctx.nslab + 1) - 0.5) * ctx.dz
    up = np.exp(1j * ctx.beta[None] * zc[:, None, None])          # (nslab, ny, nx)
    TD = np.einsum("abyx,byx->ayx", ctx.TR, D)
    return offt.ifft2(TD[:, None] * up[None], axes=(2, 3)) * (ctx.nx * ctx.ny)


def solve_fixed_point(prob, i: int = 0, rtol: float = 1e-10, max_outer: int = 50,
                      inner_rtol: float = 1e-13, maxiter: int = 500):
    """The background-field method as the paper runs it (Sec. 3, Eqs. (8)-(9)): an outer
    fixed-point loop in which the stack reflection is built from the mask field of the
    previous outer step, and each outer step solves a free-space Lippmann-Schwinger problem.

    Outer step k (E_mask^(0) = 0):
      b_k = E_inc + R[E_inc + E_mask^(k-1)]      on the absorber planes, with R of Eq. (9)
      u_k - G*(V u_k) = b_k                      (free space: no R in the operator), GMRES
      E_mask^(k) = G*(V u_k); its downgoing part at z_top comes from plane 0, moved up by
      exp(-i beta dz/2)
    and the loop stops when the reflected field changes by at most rtol between steps:
    ||R[E_mask^(k)] - R[E_mask^(k-1)]|| <= rtol ||b_1|| (b_1 = E_inc + R[E_inc], the driving
    field of the folded system; the paper leaves the norm and the tolerance open).
    u_k is the total field on the absorber planes, the unknown of the folded solve, which
    this loop converges to (Sec. 3: its fixed point is A u = b_1 with A = I - (I + R) G*V).

    Returns (orders, u, info) like solve(); info["changes"] lists the relative change per
    outer step, info["outer"] the steps taken, info["converged"] whether rtol was met.
    """
    ctx = setup_rhs(prob, i)                       # T_R for R and the orders
    free = setup_rhs(prob, i, reflection=False)    # the free-space operator u - G*(V u)
    n = ctx.nslab
    zc = (np.arange(1, n + 1) - 0.5) * ctx.dz
    E_inc = ctx.e_inc[:, None, None, None] * np.exp(-1j * ctx.beta00 * zc)[None, :, None, None] \
        * np.ones((1, 1, ctx.ny, ctx.nx))
    D_inc = np.zeros((3, ctx.ny, ctx.nx), np.complex128)
    D_inc[:, 0, 0] = ctx.e_inc                     # E_inc at z_top, normalised coefficients
    R_inc = reflected_field(ctx, D_inc)
    b1 = E_inc + R_inc
    b1n = np.linalg.norm(b1)
    R_mask = np.zeros_like(b1)                     # R[E_mask^(0)] = 0
    changes, inner = [], 0
    u = np.zeros_like(b1)
    converged = False
    k = 0
    for k in range(1, max_outer + 1):
        b_k = E_inc + R_inc + R_mask
        u, its, _ = gmres(lambda v: apply_operator(free, v), b_k, rtol=inner_rtol, maxiter=maxiter)
        inner += its
        _, E0, _ = apply_operator(free, u, return_side=True)
        D_mask = E0 * np.exp(-0.5j * ctx.beta * ctx.dz)[None]
        R_new = reflected_field(ctx, D_mask)
        change = float(np.linalg.norm(R_new - R_mask) / b1n)
        changes.append(change)
        R_mask = R_new
        if change <= rtol:
            converged = True
            break
    _, E0, Etop = apply_operator(free, u, return_side=True)
    orders = diffraction_orders(ctx, E0, Etop)
    return orders, u, {"outer": k, "inner_iterations": inner, "changes": changes,
                       "converged": converged, "ctx": ctx, "E0": E0, "Etop": Etop}


# ---------------------------------------------------------------------------
# conventional PSFD with the stack inside the domain (cross-check of the decomposition)
# ---------------------------------------------------------------------------
def _smooth_length(n: int) -> int:
    """Smallest 2^a 3^b 5^c >= n."""
    m = n
    while True:
        k = m
        for f in (2, 3, 5):
            while k % f == 0:
                k //= f
        if k == 1:
            return m
        m += 1


def full_domain_problem(prob, nf: int | None = None):
    """The clip with its multilayer stack meshed into the domain (Sec. 4's comparison).

    The voxelisation (thickness-weighted permittivity per cell, substrate-only reflection
    below the new bottom) is input construction and comes from the seeded input module;
    this picks the z length (smallest 2^a 3^b 5^c >= 2 nslab + 2 unless given). Returns
    (problem, D) with D the depth of the new reference plane below the old z_top.
    """
    from paper_2606_25541_b300 import layouts
    m = int(math.ceil(float(np.sum(prob.d_layers)) / prob.dz - 1e-9))
    if nf is None:
        nf = _smooth_length(max(prob.nf, 2 * (prob.nslab + m) + 2))
    return layouts.stack_in_domain(prob, nf)


def orders_at_old_reference(orders_full: dict, ctx_full: RhsContext, D: float) -> dict:
    """Reflected amplitudes of the full-domain solve referred to the decomposition's z_top.

    The full-domain solve references the incident wave and the upgoing orders to z = -D;
    moving both references up by D multiplies each order by exp(i (beta_mn + beta00) D).
    """
    out = dict(orders_full)
    beta = np.array([ctx_full.beta[(ctx_full.ni == n).argmax(), (ctx_full.mi == m).argmax()]
                     for m, n in zip(orders_full["m"], orders_full["n"])])
    ph = np.exp(1j * (beta + ctx_full.beta00) * D)
    out["amp"] = orders_full["amp"] * ph[:, None]
    out["a_s"] = orders_full["a_s"] * ph
    out["a_p"] = orders_full["a_p"] * ph
    return out


def scattered_spectrum_mode(prob, i: int, u: np.ndarray, m: int, n: int) -> np.ndarray:
    """xy Fourier coefficient (unnormalised DFT) at the single transverse mode (m, n) of the
    scattered part (I + R) G*(V u) = u - A u on the absorber planes; shape (3, nslab).

    The steps of apply_operator restricted to one mode, for grids too large for the full
    oracle: the xy transform of V u at (m, n) is written as a direct sum over the plane,
    then zero padding and the z transform, the dyadic Green's function of that mode, the
    inverse z transform and the reflection of the plane-0 field (Eqs. (9), (18)).
    """
    mi = np.array([[m]])
    ni = np.array([[n]])
    k0, kb, qx, qy, beta, r_s, r_p, s_hat, p_up, p_dn, TR = _mode_tables(prob, i, mi, ni)
    V = k0 * k0 * (np.asarray(prob.eps, np.complex128) - prob.eps_bg)
    x = np.arange(prob.nx)
    y = np.arange(prob.ny)
    phase = np.exp(-2j * math.pi * (n * y[:, None] / prob.ny + m * x[None, :] / prob.nx))
    J = np.zeros((3, prob.nf), np.complex128)
    for p in range(prob.nslab):
        J[:, p + 1] = np.einsum("cyx,yx->c", V[p][None] * u[:, p], phase)
    G = green_dyadic(qx, qy, beta, prob.nf, prob.dz, kb)[:, :, :, 0, 0]  # (3, 3, nf)
    Wt = offt.ifft(np.einsum("abl,bl->al", G, offt.fft(J, axis=1)), axis=1)
    R0 = TR[:, :, 0, 0] @ Wt[:, 0]
    steps = np.arange(prob.nslab, dtype=np.float64)
    return Wt[:, 1:prob.nslab + 1] + R0[:, None] * np.exp(1j * beta[0, 0] * prob.dz * steps)[None]


def solve_all(prob, rtol: float = 1e-13):
    """Every illumination of the problem, one after another."""
    return [solve(prob, i, rtol=rtol)[0] for i in range(prob.n_rhs)]
