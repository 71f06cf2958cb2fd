"""Seeded synthetic EUV-mask workloads.

This module only generates inputs: permittivity grids of the absorber layer, the
multilayer stack description and illumination lists. It holds none of the
solver's arithmetic (no Green's function, no FFT, no stack recursion), so that
both the CUDA path and the FP64 CPU oracle can be fed from it.

Conventions shared by every generator:

* lengths in nm, time convention exp(-i w t), a lossy medium has Im n > 0;
* permittivity eps = n**2 (non-magnetic media);
* absorber grids are complex128 arrays shaped ``(nslab, ny, nx)``; plane 0 is the
  plane directly above the stack interface z_top, x is the fastest axis;
* the stack is listed top to bottom as ``(n_layers complex[M], d_layers[M])`` plus a
  substrate index;
* illuminations are ``(theta_deg, phi_deg, pol)`` with pol 0 = s, 1 = p.

The paper evaluates its solver on LithoBench layouts (Sec. 3, 760 x 760 nm^2 clips
on a 4 nm grid, 50 nm Ta absorber on 40 Mo/Si bilayers, 6 deg TE illumination).
That dataset is not available here; the seeded layouts below stand in for it
with the same scale of features, absorber thickness and stack.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

N_ABSORBER = 0.94 + 0.04j
N_RU = 0.886 + 0.017j
N_MO = 0.921 + 0.0064j
N_SI = 0.999 + 0.0018j
WAVELENGTH_NM = 13.5


@dataclasses.dataclass
class Problem:
    """One mask clip: grid, absorber permittivity, stack and illuminations."""

    nx: int
    ny: int
    nslab: int
    nf: int
    dx: float
    dy: float
    dz: float
    wavelength: float
    eps_bg: float
    eps: np.ndarray  # complex128 (nslab, ny, nx)
    n_layers: np.ndarray  # complex128 (M,) top -> bottom
    d_layers: np.ndarray  # float64 (M,)
    n_sub: complex
    theta_deg: np.ndarray  # (n_rhs,)
    phi_deg: np.ndarray  # (n_rhs,)
    pol: np.ndarray  # int32 (n_rhs,)
    name: str = ""

    @property
    def n_rhs(self) -> int:
        return int(len(self.theta_deg))

    @property
    def unknowns_per_rhs(self) -> int:
        return 3 * self.nx * self.ny * self.nslab

    def with_illumination(self, theta, phi, pol) -> "Problem":
        return dataclasses.replace(
            self,
            theta_deg=np.asarray(theta, dtype=np.float64).reshape(-1),
            phi_deg=np.asarray(phi, dtype=np.float64).reshape(-1),
            pol=np.asarray(pol, dtype=np.int32).reshape(-1),
        )


# ---------------------------------------------------------------------------
# z padding
# ---------------------------------------------------------------------------
# FFT lengths the CUDA kernels are instantiated for (psfd_supported_length).
SUPPORTED_LENGTHS = (4, 8, 16, 32, 64, 96, 128, 160, 192, 256, 320, 384, 512, 640, 768, 1024)


def padded_nf(nslab: int, nz_min: int = 0) -> int:
    """Smallest supported FFT length >= max(nz_min, 2*nslab + 2).

    The z window of the periodic Green's function has half-width L = nf*dz/2 and
    must cover every source/observation separation of the slab plus the two
    extraction planes, hence nf >= 2*nslab + 2.
    """
    need = max(int(nz_min), 2 * int(nslab) + 2)
    for n in SUPPORTED_LENGTHS:
        if n >= need:
            return n
    raise ValueError(f"no supported z length >= {need}")


# ---------------------------------------------------------------------------
# stacks
# ---------------------------------------------------------------------------
def ru_mosi_stack(n_bilayers: int = 40, with_cap: bool = True):
    """Ru cap 2.5 nm on n_bilayers x [Mo 2.78 nm, Si 4.17 nm] on a Si substrate."""
    n, d = [], []
    if with_cap:
        n.append(N_RU)
        d.append(2.5)
    for _ in range(n_bilayers):
        n += [N_MO, N_SI]
        d += [2.78, 4.17]
    return np.array(n, dtype=np.complex128), np.array(d, dtype=np.float64), complex(N_SI)


def empty_stack(n_sub: complex = 1.0 + 0.0j):
    """No layers; the substrate index alone (1.0 means no reflection at all)."""
    return np.zeros(0, np.complex128), np.zeros(0, np.float64), complex(n_sub)


# ---------------------------------------------------------------------------
# absorber layouts (2-D masks extruded over the absorber planes)
# ---------------------------------------------------------------------------
def extrude(mask2d: np.ndarray, nslab: int, n_abs=N_ABSORBER, eps_bg: float = 1.0,
            n_map: np.ndarray | None = None) -> np.ndarray:
    """Permittivity grid of a z-invariant absorber: eps = n**2 where mask, eps_bg elsewhere."""
    mask2d = np.asarray(mask2d, dtype=bool)
    if n_map is None:
        eps2d = np.where(mask2d, complex(n_abs) ** 2, eps_bg + 0j)
    else:
        eps2d = np.where(mask2d, np.asarray(n_map, np.complex128) ** 2, eps_bg + 0j)
    return np.ascontiguousarray(np.broadcast_to(eps2d, (nslab,) + mask2d.shape)).astype(np.complex128)


def contact_hole_mask(nx: int, ny: int, hole_x: int, hole_y: int) -> np.ndarray:
    """Absorber everywhere except a centred rectangular hole of hole_x x hole_y cells."""
    m = np.ones((ny, nx), dtype=bool)
    x0 = (nx - hole_x) // 2
    y0 = (ny - hole_y) // 2
    m[y0:y0 + hole_y, x0:x0 + hole_x] = False
    return m


def line_space_mask(nx: int, ny: int, dx: float, pitch_nm: float, width_nm: float) -> np.ndarray:
    """Absorber lines along y, one per pitch, centred in x; width snapped to the grid."""
    w = int(round(width_nm / dx))
    per = int(round(pitch_nm / dx))
    m = np.zeros((ny, nx), dtype=bool)
    for start in range(0, nx, per):
        c = start + per // 2
        lo = max(0, c - w // 2)
        m[:, lo:min(nx, lo + w)] = True
    return m


def manhattan_mask(nx: int, ny: int, rng: np.random.Generator, fill_lo=0.30, fill_hi=0.50,
                   snap: int = 4, min_feat: int = 8, max_feat: int | None = None):
    """Random axis-aligned rectangles on a `snap`-cell lattice until the fill target is met.

    Returns (mask, labels) where labels numbers the rectangle that last covered each
    cell (-1 = open), so per-feature properties can be attached.
    """
    if max_feat is None:
        max_feat = max(min_feat + snap, min(nx, ny) // 3)
    target = rng.uniform(fill_lo, fill_hi)
    m = np.zeros((ny, nx), dtype=bool)
    labels = -np.ones((ny, nx), dtype=np.int32)
    k = 0
    for _ in range(100000):
        if m.mean() >= target:
            break
        w = int(rng.integers(min_feat // snap, max_feat // snap + 1)) * snap
        h = int(rng.integers(min_feat // snap, max_feat // snap + 1)) * snap
        x0 = int(rng.integers(0, max(1, nx // snap))) * snap
        y0 = int(rng.integers(0, max(1, ny // snap))) * snap
        xs = np.arange(x0, x0 + w) % nx
        ys = np.arange(y0, y0 + h) % ny
        m[np.ix_(ys, xs)] = True
        labels[np.ix_(ys, xs)] = k
        k += 1
    return m, labels


def curvilinear_mask(nx: int, ny: int, rng: np.random.Generator, corr_cells: float = 12.0,
                     fill: float = 0.4) -> np.ndarray:
    """Thresholded smooth random field (ILT-like curvilinear contours), periodic."""
    noise = rng.standard_normal((ny, nx))
    kx = np.fft.fftfreq(nx)[None, :]
    ky = np.fft.fftfreq(ny)[:, None]
    filt = np.exp(-0.5 * (kx ** 2 + ky ** 2) * (2 * math.pi * corr_cells) ** 2)
    field = np.real(np.fft.ifft2(np.fft.fft2(noise) * filt))
    thr = np.quantile(field, 1.0 - fill)
    return field > thr


# ---------------------------------------------------------------------------
# the workloads
# ---------------------------------------------------------------------------
def _problem(nx, ny, nslab, nf, dx, dz, eps, stack, theta, phi, pol, name):
    n_l, d_l, n_s = stack
    return Problem(nx=nx, ny=ny, nslab=nslab, nf=nf, dx=dx, dy=dx, dz=dz,
                   wavelength=WAVELENGTH_NM, eps_bg=1.0, eps=eps, n_layers=n_l,
                   d_layers=d_l, n_sub=n_s,
                   theta_deg=np.asarray(theta, np.float64).reshape(-1),
                   phi_deg=np.asarray(phi, np.float64).reshape(-1),
                   pol=np.asarray(pol, np.int32).reshape(-1), name=name)


def contact_hole_clip() -> Problem:
    """64 x 64 nm contact-hole clip at 2 nm: 32 x 32 x 30 absorber planes, nf = 64.

    60 nm absorber (n = 0.94+0.04i) with a centred 32 x 32 nm hole, Ru/40x(Mo/Si)
    stack, one s-polarised plane wave at 6 deg polar / 0 deg azimuth.
    """
    nx = ny = 32
    dx = dz = 2.0
    nslab = 30
    eps = extrude(contact_hole_mask(nx, ny, 16, 16), nslab)
    return _problem(nx, ny, nslab, padded_nf(nslab, 64), dx, dz, eps, ru_mosi_stack(),
                    [6.0], [0.0], [0], "contact_hole_32x32x30")


def line_space_clip(seed: int = 2) -> Problem:
    """128 x 128 nm line/space clip at 1 nm: 60 absorber planes, nf = 128, 18 RHS.

    One absorber line per 128 nm pitch with seeded width U{16..48} nm; 9 angles on a
    3 x 3 grid (polar 0/4/8 deg, azimuth 0/45/90 deg) times s/p polarisation.
    """
    rng = np.random.default_rng(seed)
    nx = ny = 128
    dx = dz = 1.0
    nslab = 60
    width = int(rng.integers(16, 49))
    eps = extrude(line_space_mask(nx, ny, dx, 128.0, width), nslab)
    th, ph, po = [], [], []
    for t in (0.0, 4.0, 8.0):
        for p in (0.0, 45.0, 90.0):
            for s in (0, 1):
                th.append(t)
                ph.append(p)
                po.append(s)
    return _problem(nx, ny, nslab, padded_nf(nslab, 96), dx, dz, eps, ru_mosi_stack(),
                    th, ph, po, f"line_space_128x128x60_w{width}")


def manhattan_clip(n: int = 256, seed: int = 3, nslab: int = 60, nz: int = 128,
                   jitter: float = 0.02) -> Problem:
    """n x n Manhattan clip at 1 nm (30-50 % fill, 4 nm snap, +-2 % index jitter), 6 deg s/p."""
    rng = np.random.default_rng(seed)
    mask, labels = manhattan_mask(n, n, rng)
    nfeat = int(labels.max()) + 1
    scale = 1.0 + rng.uniform(-jitter, jitter, size=max(nfeat, 1))
    n_map = np.where(labels >= 0, N_ABSORBER * scale[np.maximum(labels, 0)], 1.0)
    eps = extrude(mask, nslab, n_map=n_map)
    return _problem(n, n, nslab, padded_nf(nslab, nz), 1.0, 1.0, eps, ru_mosi_stack(),
                    [6.0, 6.0], [0.0, 0.0], [0, 1], f"manhattan_{n}x{n}x{nslab}")


def curvilinear_clip(n: int = 1024, seed: int = 5, nslab: int = 60, nf: int = 160) -> Problem:
    """n x n curvilinear (ILT-like) clip at 1 nm: a thresholded smooth random field extruded
    over 60 absorber planes (n = 0.94 + 0.04i), nf = 160; 4 polar angles (0, 3, 6, 9 deg at
    azimuth 0) times s/p polarisation."""
    rng = np.random.default_rng(seed)
    eps = extrude(curvilinear_mask(n, n, rng, corr_cells=12.0, fill=0.4), nslab)
    th = [t for t in (0.0, 3.0, 6.0, 9.0) for _ in (0, 1)]
    po = [s for _ in range(4) for s in (0, 1)]
    return _problem(n, n, nslab, padded_nf(nslab, nf), 1.0, 1.0, eps, ru_mosi_stack(), th,
                    [0.0] * 8, po, f"curvilinear_{n}x{n}x{nslab}")


def small_clip(nx=8, ny=8, nslab=4, dx=4.0, dz=2.0, seed=0, stack=None, theta=(6.0,), phi=(0.0,),
               pol=(0,), nz_min=0) -> Problem:
    """Tiny seeded Manhattan-like clip for exhaustive element-wise checks."""
    rng = np.random.default_rng(seed)
    mask = rng.random((ny, nx)) < 0.5
    mask[0, 0] = True
    nmap = N_ABSORBER * (1.0 + rng.uniform(-0.02, 0.02, size=(ny, nx)))
    eps = extrude(mask, nslab, n_map=nmap)
    # vary along z as well so that nothing relies on z invariance
    eps = eps * (1.0 + 0.01 * rng.standard_normal((nslab, 1, 1)))
    if stack is None:
        stack = ru_mosi_stack(3)
    return _problem(nx, ny, nslab, padded_nf(nslab, nz_min), dx, dz, eps.astype(np.complex128),
                    stack, theta, phi, pol, f"small_{nx}x{ny}x{nslab}_s{seed}")


def stack_in_domain(prob: Problem, nf: int | None = None):
    """The clip with its multilayer stack meshed into the domain (the conventional PSFD of
    the paper's comparison): the stack of total thickness T below z_top is covered by
    M = ceil(T/dz) cells that extend the domain downward, each with the thickness-weighted
    mean permittivity of the layers (and substrate) it overlaps; below the new bottom only
    the substrate remains (an empty stack). nf defaults to the smallest supported length.
    Returns (problem, D) with D = M dz, the depth of the new reference plane."""
    d = np.asarray(prob.d_layers, np.float64)
    eps_l = np.asarray(prob.n_layers, np.complex128) ** 2
    eps_s = complex(prob.n_sub) ** 2
    M = int(math.ceil(float(d.sum()) / prob.dz - 1e-9))
    D = M * prob.dz
    tops = -np.concatenate([[0.0], np.cumsum(d)])  # layer j spans [tops[j+1], tops[j]]
    cells = np.empty(M, np.complex128)
    for p in range(M):  # cell p (from the bottom) spans [lo, hi]
        lo, hi = -D + p * prob.dz, -D + (p + 1) * prob.dz
        acc, covered = 0.0 + 0.0j, 0.0
        for j in range(len(d)):
            ov = max(0.0, min(hi, tops[j]) - max(lo, tops[j + 1]))
            acc += ov * eps_l[j]
            covered += ov
        acc += (prob.dz - covered) * eps_s  # what is left of the cell lies in the substrate
        cells[p] = acc / prob.dz
    eps = np.concatenate([np.broadcast_to(cells[:, None, None], (M, prob.ny, prob.nx)),
                          np.asarray(prob.eps, np.complex128)], axis=0)
    nslab = prob.nslab + M
    full = dataclasses.replace(prob, nslab=nslab, nf=nf or padded_nf(nslab), eps=eps,
                               n_layers=np.zeros(0, np.complex128), d_layers=np.zeros(0, np.float64),
                               name=prob.name + "_stack_in_domain")
    return full, D


def random_field(shape, seed: int, dtype=np.complex128) -> np.ndarray:
    """Seeded complex Gaussian test vector (for operator-level parity checks)."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(dtype)


def serving_requests(n: int, seed: int = 4, sizes=(64, 128), z_choices=(64, 96, 128), max_rhs: int = 18,
                     slab_quantum: int = 8):
    """Seeded stream of mask-clip requests for the serving loop.

    Transverse sizes from `sizes` (independently in x and y) at 1 nm, a z extent from
    `z_choices`, an absorber of U{50..70} nm with a Manhattan layout (30-50 % fill, 4 nm snap,
    +-2 % index jitter) placed on the lowest planes of a slab rounded up to a multiple of
    `slab_quantum` planes (vacuum above; requests of similar thickness then share a grid),
    and 1..max_rhs illuminations (polar 0..8 deg, azimuth 0..90 deg, s or p).
    """
    rng = np.random.default_rng(seed)
    out = []
    stack = ru_mosi_stack()
    for k in range(n):
        nx = int(sizes[rng.integers(len(sizes))])
        ny = int(sizes[rng.integers(len(sizes))])
        nz = int(z_choices[rng.integers(len(z_choices))])
        thick = int(rng.integers(50, 71))
        nslab = slab_quantum * ((thick + slab_quantum - 1) // slab_quantum)
        mask, labels = manhattan_mask(nx, ny, rng)
        nfeat = int(labels.max()) + 1
        scale = 1.0 + rng.uniform(-0.02, 0.02, size=max(nfeat, 1))
        n_map = np.where(labels >= 0, N_ABSORBER * scale[np.maximum(labels, 0)], 1.0)
        eps = extrude(mask, nslab, n_map=n_map)
        eps[thick:] = 1.0
        n_rhs = int(rng.integers(1, max_rhs + 1))
        th = np.round(rng.uniform(0.0, 8.0, n_rhs), 1)
        ph = np.round(rng.uniform(0.0, 90.0, n_rhs), 0)
        po = rng.integers(0, 2, n_rhs)
        out.append(_problem(nx, ny, nslab, padded_nf(nslab, nz), 1.0, 1.0, eps, stack, th, ph, po,
                            f"request_{k}_{nx}x{ny}x{nslab}_{n_rhs}rhs"))
    return out
