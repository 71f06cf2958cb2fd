// tables.cu -- FP64 set-up and post-processing kernels: scattering potential, per-mode
// stack reflection (Parratt recursion), right-hand side, diffraction orders, the
// defect-correction helpers, and the FFT test hook.
#include <vector>

#include "fft.cuh"
#include "krylov.cuh"
#include "tables.h"
#include "dfloat.cuh"

namespace psfd {

// Counts one kernel launch and reports whether it was accepted.
static int launched() {
  count_launch();
  return cudaGetLastError() == cudaSuccess ? PSFD_OK : PSFD_E_CUDA;
}

// ---------------------------------------------------------------------------
// V = k0^2 (eps - eps_bg) in FP64 and FP32 (Sec. 2, Eq. (1); Sec. 3, Eq. (10))
// ---------------------------------------------------------------------------
__global__ void k_potential(size_t n, const double2* eps, double k02, double eps_bg, double2* V64, float2* V32,
                            float4* Vdf) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double2 e = eps[i];
    const double2 v = make_double2(k02 * (e.x - eps_bg), k02 * e.y);
    V64[i] = v;
    V32[i] = to_c32(v);
    if (Vdf) {  // the pairs the residual's double-float row pass multiplies by (once per potential)
      const dfc d = to_dfc(v);
      Vdf[i] = make_float4(d.x.hi, d.x.lo, d.y.hi, d.y.lo);
    }
  }
}

int launch_potential(size_t n, const double2* eps, double k02, double eps_bg, double2* V64, float2* V32, float4* Vdf,
                     cudaStream_t st) {
  k_potential<<<592, 256, 0, st>>>(n, eps, k02, eps_bg, V64, V32, Vdf);
  return launched();
}

// ---------------------------------------------------------------------------
// Stack response per transverse mode (Sec. 2: generalized reflection coefficients /
// transfer-matrix method; Sec. 3, Eq. (9): T_R). Media: 0 = background, 1..M layers
// top to bottom, M+1 substrate; k_zj = sqrt(k0^2 eps_j - q^2) with Im >= 0.
//   s: r_ij = (k_zi - k_zj) / (k_zi + k_zj)                       (E field)
//   p: r_ij = (eps_j k_zi - eps_i k_zj) / (eps_j k_zi + eps_i k_zj) (H field)
//   Gamma_M = r_{M,M+1},  Gamma_{j-1} = (r + Gamma_j e) / (1 + r Gamma_j e),
//   r = r_{j-1,j}, e = exp(2 i k_zj d_j); the reflection at z_top is Gamma_0.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double2 fresnel_d(double2 kzi, double2 kzj, double2 ei, double2 ej, int pol) {
  if (pol == 0) return cdiv(csub(kzi, kzj), cadd(kzi, kzj));
  const double2 a = cmul(ej, kzi), b = cmul(ei, kzj);
  return cdiv(csub(a, b), cadd(a, b));
}

__device__ __forceinline__ double2 kz_of(double k02, double2 eps, double q2) {
  return csqrt_upper_d(make_double2(k02 * eps.x - q2, k02 * eps.y));
}

__device__ double2 parratt_d(double k02, double q2, double2 eps_amb, const StackDev& st, int pol) {
  const int M = st.n_layers;
  double2 e_j = M > 0 ? st.eps[M - 1] : eps_amb;
  double2 kz_j = kz_of(k02, e_j, q2);
  double2 gam = fresnel_d(kz_j, kz_of(k02, st.eps_sub, q2), e_j, st.eps_sub, pol);
  for (int j = M; j >= 1; --j) {
    const double2 e_a = (j >= 2) ? st.eps[j - 2] : eps_amb;
    const double2 kz_a = kz_of(k02, e_a, q2);
    const double2 ph = cexp_d(make_double2(-2.0 * kz_j.y * st.d[j - 1], 2.0 * kz_j.x * st.d[j - 1]));
    const double2 r = fresnel_d(kz_a, kz_j, e_a, e_j, pol);
    const double2 ge = cmul(gam, ph);
    gam = cdiv(cadd(r, ge), cadd(make_double2(1.0, 0.0), cmul(r, ge)));
    kz_j = kz_a;
    e_j = e_a;
  }
  return gam;
}

// 2 x 2 complex matrices acting on the reflection coefficient as Moebius maps.
struct Mobius2 {
  double2 a, b, c, d;  // G -> (a G + b) / (c G + d)
};
__device__ __forceinline__ Mobius2 mobius_layer(double2 e, double2 r) {
  return {e, r, cmul(r, e), make_double2(1.0, 0.0)};
}
__device__ __forceinline__ Mobius2 mobius_mul(const Mobius2& x, const Mobius2& y) {
  return {cadd(cmul(x.a, y.a), cmul(x.b, y.c)), cadd(cmul(x.a, y.b), cmul(x.b, y.d)),
          cadd(cmul(x.c, y.a), cmul(x.d, y.c)), cadd(cmul(x.c, y.b), cmul(x.d, y.d))};
}
__device__ __forceinline__ Mobius2 mobius_rescale(const Mobius2& x) {
  const double m = fmax(fmax(cabs2(x.a), cabs2(x.b)), fmax(cabs2(x.c), cabs2(x.d)));
  const double s = m > 0.0 ? 1.0 / sqrt(m) : 1.0;
  return {cscale(x.a, s), cscale(x.b, s), cscale(x.c, s), cscale(x.d, s)};
}
__device__ __forceinline__ Mobius2 mobius_pow(Mobius2 x, int k) {
  Mobius2 r = {make_double2(1.0, 0.0), make_double2(0.0, 0.0), make_double2(0.0, 0.0), make_double2(1.0, 0.0)};
  while (k > 0) {
    if (k & 1) r = mobius_rescale(mobius_mul(r, x));
    k >>= 1;
    if (k) x = mobius_rescale(mobius_mul(x, x));
  }
  return r;
}
__device__ __forceinline__ double2 mobius_apply(const Mobius2& m, double2 g) {
  return cdiv(cadd(cmul(m.a, g), m.b), cadd(cmul(m.c, g), m.d));
}

// The same recursion for s and p at once, with the square roots, Fresnel coefficients
// and layer phase factors taken once per distinct medium / interface / layer class.
__device__ void parratt_dedup_d(double k02, double q2, const StackDev& st, double2& rs, double2& rp) {
  double2 kz[kMaxMat], fs[kMaxIface], fp[kMaxIface], ph[kMaxPh];
  for (int m = 0; m < st.n_mat; ++m) kz[m] = kz_of(k02, st.mat_eps[m], q2);
  for (int i = 0; i < st.n_iface; ++i) {
    const int ia = st.iface_a[i], ib = st.iface_b[i];
    fs[i] = fresnel_d(kz[ia], kz[ib], st.mat_eps[ia], st.mat_eps[ib], 0);
    fp[i] = fresnel_d(kz[ia], kz[ib], st.mat_eps[ia], st.mat_eps[ib], 1);
  }
  for (int p = 0; p < st.n_ph; ++p) {
    const double2 k = kz[st.ph_mat[p]];
    ph[p] = cexp_d(make_double2(-2.0 * k.y * st.ph_d[p], 2.0 * k.x * st.ph_d[p]));
  }
  const int M = st.n_layers;
  double2 gs = fs[st.iface_of[M]], gp = fp[st.iface_of[M]];
  const double2 one = make_double2(1.0, 0.0);
  // one recursion step through layer j: G <- (r + G e) / (1 + r G e)
  auto step = [&](int j) {
    const double2 e = ph[st.layer_ph[j - 1]];
    const int f = st.iface_of[j - 1];
    const double2 ges = cmul(gs, e), gep = cmul(gp, e);
    gs = cdiv(cadd(fs[f], ges), cadd(one, cmul(fs[f], ges)));
    gp = cdiv(cadd(fp[f], gep), cadd(one, cmul(fp[f], gep)));
  };
  const int rb = st.run_k ? st.run_top + 2 * st.run_k - 1 : 0;  // bottom layer of the run
  for (int j = M; j > rb; --j) step(j);
  if (st.run_k) {
    // The step through layer j is the Moebius map of [[e, r], [r e, 1]]; a unit (upper
    // layer a, lower layer b) is their product, and run_k units are its run_k-th power
    // (by squaring, rescaled to unit max entry: the map ignores a common factor).
    const int ja = st.run_top, jb = st.run_top + 1;
    const double2 ea = ph[st.layer_ph[ja - 1]], eb = ph[st.layer_ph[jb - 1]];
    const int fa = st.iface_of[ja - 1], fb = st.iface_of[jb - 1];
    Mobius2 qs = mobius_mul(mobius_layer(ea, fs[fa]), mobius_layer(eb, fs[fb]));
    Mobius2 qp = mobius_mul(mobius_layer(ea, fp[fa]), mobius_layer(eb, fp[fb]));
    gs = mobius_apply(mobius_pow(qs, st.run_k), gs);
    gp = mobius_apply(mobius_pow(qp, st.run_k), gp);
  }
  if (st.run_k)
    for (int j = st.run_top - 1; j >= 1; --j) step(j);
  rs = gs;
  rp = gp;
}

void stack_dedup(StackDev& st, const double2* eps_layers, const double* d_layers, int n_layers, double2 eps_amb,
                 double2 eps_sub) {
  st.n_mat = st.n_iface = st.n_ph = 0;
  st.run_top = st.run_k = 0;
  if (n_layers > kStackMaxLayers) return;
  int med[kStackMaxLayers + 2];
  auto mat_id = [&](double2 e) -> int {
    for (int m = 0; m < st.n_mat; ++m)
      if (st.mat_eps[m].x == e.x && st.mat_eps[m].y == e.y) return m;
    if (st.n_mat == kMaxMat) return -1;
    st.mat_eps[st.n_mat] = e;
    return st.n_mat++;
  };
  for (int j = 0; j < n_layers + 2; ++j) {
    const double2 e = j == 0 ? eps_amb : (j == n_layers + 1 ? eps_sub : eps_layers[j - 1]);
    med[j] = mat_id(e);
    if (med[j] < 0) { st.n_mat = 0; return; }
  }
  for (int j = 0; j <= n_layers; ++j) {
    int id = -1;
    for (int i = 0; i < st.n_iface; ++i)
      if (st.iface_a[i] == med[j] && st.iface_b[i] == med[j + 1]) id = i;
    if (id < 0) {
      if (st.n_iface == kMaxIface) { st.n_mat = 0; return; }
      id = st.n_iface++;
      st.iface_a[id] = (unsigned char)med[j];
      st.iface_b[id] = (unsigned char)med[j + 1];
    }
    st.iface_of[j] = (unsigned char)id;
  }
  for (int j = 0; j < n_layers; ++j) {
    int id = -1;
    for (int p = 0; p < st.n_ph; ++p)
      if (st.ph_mat[p] == med[j + 1] && st.ph_d[p] == d_layers[j]) id = p;
    if (id < 0) {
      if (st.n_ph == kMaxPh) { st.n_mat = 0; return; }
      id = st.n_ph++;
      st.ph_mat[id] = (unsigned char)med[j + 1];
      st.ph_d[id] = d_layers[j];
    }
    st.layer_ph[j] = (unsigned char)id;
  }
  // longest periodic two-layer run: 1-based layers top .. top + 2k - 1 with layer j and j + 2
  // alike for every j in the run, and medium top - 1 alike medium top + 1 (so that every
  // unit of the run sits below the same interface)
  auto same = [&](int j1, int j2) {  // 1-based layers j1, j2 <= n_layers: medium and thickness
    return med[j1] == med[j2] && d_layers[j1 - 1] == d_layers[j2 - 1];
  };
  for (int top = 1; top + 3 <= n_layers; ++top) {
    if (med[top - 1] != med[top + 1]) continue;
    int k = 0;
    while (top + 2 * k + 1 <= n_layers && same(top + 2 * k, top) && same(top + 2 * k + 1, top + 1)) ++k;
    if (k > st.run_k) {
      st.run_k = k;
      st.run_top = top;
    }
  }
  if (st.run_k < 3) st.run_k = 0;
}

// grid (ceil(nx / 128), ny, n_slots)
__global__ void k_modes(ModesArgs a) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  const int slot = a.slots ? a.slots[blockIdx.z] : a.slot0 + blockIdx.z;
  if (x >= a.nx) return;
  const double two_pi = 6.283185307179586476925286766559;
  const double* sp = a.slot_par + 4 * slot;
  const double qx = sp[0] + two_pi * fft_freq(x, a.nx) / (a.nx * a.dx);
  const double qy = sp[1] + two_pi * fft_freq(y, a.ny) / (a.ny * a.dy);
  const double q2 = qx * qx + qy * qy;
  const double kb2 = a.k0 * a.k0 * a.eps_bg;
  const double2 beta = csqrt_upper_d(make_double2(kb2 - q2, 0.0));
  if (sqrt(cabs2(beta)) < 1e-9 * a.k0) atomicOr(a.anomaly, 1);
  ModeEntry m;
  m.beta = beta;
  m.ebL = cexp_d(make_double2(-beta.y * a.L, beta.x * a.L));
  const double k02 = a.k0 * a.k0;
  const double2 eb = make_double2(a.eps_bg, 0.0);
  if (!a.stack.reflect) {
    m.rs = make_double2(0.0, 0.0);
    m.rp = make_double2(0.0, 0.0);
  } else if (a.stack.n_mat > 0) {
    parratt_dedup_d(k02, q2, a.stack, m.rs, m.rp);
  } else {
    m.rs = parratt_d(k02, q2, eb, a.stack, 0);
    m.rp = parratt_d(k02, q2, eb, a.stack, 1);
  }
  const size_t idx = ((size_t)slot * a.ny + y) * a.nx + x;
  a.modes[idx] = m;
  if (!a.modes32 && !a.modesdf) return;
  // per-column constants of the z pass, evaluated once in FP64 for both copies
  const double2 e1 = cexp_d(make_double2(-beta.y * a.dz, beta.x * a.dz));
  const double2 e8 = cexp_d(make_double2(-8.0 * beta.y * a.dz, 8.0 * beta.x * a.dz));
  const double qn = sqrt(q2);
  const double hx = qn > 0.0 ? qx / qn : sp[2];
  const double hy = qn > 0.0 ? qy / qn : sp[3];
  const double qnk = qn / a.kb;
  const double2 bq = cscale(beta, 1.0 / a.kb);
  if (a.modes32) {
    ModeF32 f;
    f.qx = (float)qx;
    f.qy = (float)qy;
    split_hi_lo(beta, f.bh, f.bl);
    f.ebL = to_c32(m.ebL);
    f.e1 = to_c32(e1);
    f.e8 = to_c32(e8);
    f.rs = to_c32(m.rs);
    f.rp = to_c32(m.rp);
    f.hx = (float)hx;
    f.hy = (float)hy;
    f.qnk = (float)qnk;
    f.pad = 0.f;
    f.bq = to_c32(bq);
    a.modes32[idx] = f;
  }
  if (a.modesdf) {
    // the same quantities as pairs, each converted once from its FP64 value
    auto c4 = [](double2 v) {
      const dfc d = to_dfc(v);
      return make_float4(d.x.hi, d.x.lo, d.y.hi, d.y.lo);
    };
    auto r2 = [](double v) {
      const dfr d = to_dfr(v);
      return make_float2(d.hi, d.lo);
    };
    ModeDF f;
    f.beta = c4(beta);
    f.ebL = c4(m.ebL);
    f.e1 = c4(e1);
    f.e8 = c4(e8);
    f.rs = c4(m.rs);
    f.rp = c4(m.rp);
    f.bq = c4(bq);
    f.qx = r2(qx);
    f.qy = r2(qy);
    f.hx = r2(hx);
    f.hy = r2(hy);
    f.qnk = r2(qnk);
    f.pad = make_float2(0.f, 0.f);
    a.modesdf[idx] = f;
  }
}

// (e^z - 1)/z for z = i a (a real): sin(a)/a + i 2 sin^2(a/2)/a, by its Taylor series near 0.
__device__ __forceinline__ double2 phi1_imag(double a) {
  if (fabs(a) < 1e-3) {
    const double a2 = a * a;
    return make_double2(1.0 - a2 / 6.0 + a2 * a2 / 120.0, a / 2.0 - a * a2 / 24.0 + a * a2 * a2 / 720.0);
  }
  const double s = sin(0.5 * a);
  return make_double2(sin(a) / a, 2.0 * s * s / a);
}

// One thread per (mode, l): A(|k|) and B(|k|)/|k|^2 of the windowed dyadic kernel.
//   F[g_R](k) = (1/k) int_0^R exp(i kb r) sin(k r) dr: (E - 1)/(kb^2 - k^2) with
//   E = exp(i kb R)(cos kR - i (kb/k) sin kR), or, near k = kb, R (phi1(i(kb+k)R) -
//   phi1(i(kb-k)R)) / (2ik); at k = 0, (exp(i kb R)(1 - i kb R) - 1)/kb^2.
//   h(k) = 4 pi R^2 g'(R) j1(kR)/(kb^2 kR) = exp(i kb R)(i kb R - 1) j1(kR)/(kR kb^2),
//   A = F[g_R] + h, B = -F[g_R] - 3h - 1/kb^2 (k > 0); B khat khat^T vanishes at k = 0.
__global__ void k_sph_table(SphArgs a) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, sl = blockIdx.z;
  const int HF = a.nf / 2;
  if (x >= a.nx) return;
  const int slot = a.slot0 + sl;
  const double two_pi = 6.283185307179586476925286766559;
  const double qx = a.slot_par[4 * slot] + two_pi * fft_freq(x, a.nx) / (a.nx * a.dx);
  const double qy = a.slot_par[4 * slot + 1] + two_pi * fft_freq(y, a.ny) / (a.ny * a.dy);
  const double kb = a.kb, R = a.R, kb2 = kb * kb;
  const double2 ekR = make_double2(cos(kb * R), sin(kb * R));
  const double scale = 1.0 / ((double)a.nf * a.nx * a.ny);
  for (int l = 0; l <= HF; ++l) {
    const double kz = two_pi * l / (a.nf * a.dz);
    const double k2 = qx * qx + qy * qy + kz * kz, k = sqrt(k2);
    double2 f;
    if (k < 1e-12 * kb) {
      f = cscale(csub(cmul(ekR, make_double2(1.0, -kb * R)), make_double2(1.0, 0.0)), 1.0 / kb2);
    } else if (fabs(k - kb) * R < 0.5) {
      const double2 d = csub(phi1_imag((kb + k) * R), phi1_imag((kb - k) * R));
      f = make_double2(R * d.y / (2.0 * k), -R * d.x / (2.0 * k));  // R d / (2 i k)
    } else {
      const double2 E = cmul(ekR, make_double2(cos(k * R), -(kb / k) * sin(k * R)));
      f = cscale(csub(E, make_double2(1.0, 0.0)), 1.0 / (kb2 - k2));
    }
    const double x1 = k * R;
    const double j1x = x1 < 1e-2 ? 1.0 / 3.0 - x1 * x1 / 30.0 + x1 * x1 * x1 * x1 / 840.0
                                 : (sin(x1) - x1 * cos(x1)) / (x1 * x1 * x1);
    const double2 h = cscale(cmul(ekR, make_double2(-1.0, kb * R)), j1x / kb2);
    const double2 A = cadd(f, h);
    double2 Bt = make_double2(0.0, 0.0);
    if (k >= 1e-12 * kb) {
      const double2 B = csub(csub(cneg(f), cscale(h, 3.0)), make_double2(1.0 / kb2, 0.0));
      Bt = cscale(B, 1.0 / k2);
    }
    const size_t o = (((size_t)slot * (HF + 1) + l) * a.ny + y) * a.nx + x;
    a.t64[2 * o] = cscale(A, scale);
    a.t64[2 * o + 1] = cscale(Bt, scale);
    if (a.t32)
      a.t32[o] = make_float4((float)(A.x * scale), (float)(A.y * scale), (float)(Bt.x * scale), (float)(Bt.y * scale));
  }
}

int launch_sph_table(const SphArgs& a, int n_slots, cudaStream_t st) {
  dim3 grid((a.nx + 127) / 128, a.ny, n_slots);
  k_sph_table<<<grid, 128, 0, st>>>(a);
  return launched();
}

int launch_modes(const ModesArgs& a, int n_slots, cudaStream_t st) {
  dim3 grid((a.nx + 127) / 128, a.ny, n_slots);
  k_modes<<<grid, 128, 0, st>>>(a);
  return launched();
}

// Bilinear triad of a mode: s = z x qhat, p+- = (-+beta qhat, |q|)/kb.
struct Triad {
  double sx, sy;
  double2 pp[3], pm[3];
};
__device__ __forceinline__ Triad triad_d(double qx, double qy, double2 beta, double kb, double cphi, double sphi) {
  const double qn = sqrt(qx * qx + qy * qy);
  const double hx = qn > 0.0 ? qx / qn : cphi;
  const double hy = qn > 0.0 ? qy / qn : sphi;
  Triad t;
  t.sx = -hy;
  t.sy = hx;
  const double2 bq = cscale(beta, 1.0 / kb);
  t.pp[0] = cscale(bq, -hx);
  t.pp[1] = cscale(bq, -hy);
  t.pp[2] = make_double2(qn / kb, 0.0);
  t.pm[0] = cscale(bq, hx);
  t.pm[1] = cscale(bq, hy);
  t.pm[2] = t.pp[2];
  return t;
}

// T_R v = r_s s (s.v) + r_p p+ (p-.v)
__device__ __forceinline__ void apply_TR(const Triad& t, double2 rs, double2 rp, const double2 v[3], double2 out[3]) {
  const double2 sv = cadd(cscale(v[0], t.sx), cscale(v[1], t.sy));
  const double2 pv = cadd(cadd(cmul(t.pm[0], v[0]), cmul(t.pm[1], v[1])), cmul(t.pm[2], v[2]));
  const double2 as = cmul(rs, sv), ap = cmul(rp, pv);
  out[0] = cadd(cscale(as, t.sx), cmul(ap, t.pp[0]));
  out[1] = cadd(cscale(as, t.sy), cmul(ap, t.pp[1]));
  out[2] = cmul(ap, t.pp[2]);
}

// One thread per illumination: incident vector e (s or p-) and its reflection T_R e.
__global__ void k_rhs_params(int rhs0, int nrhs, RhsParam* rp, const ModeEntry* modes, int nx, int ny, double kb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrhs) return;
  RhsParam p = rp[rhs0 + i];
  const ModeEntry m = modes[(size_t)p.slot * ny * nx];  // mode (0, 0)
  const Triad t = triad_d(p.qix, p.qiy, m.beta, kb, p.cphi, p.sphi);
  if (p.pol == 0) {
    p.e_inc[0] = make_double2(t.sx, 0.0);
    p.e_inc[1] = make_double2(t.sy, 0.0);
    p.e_inc[2] = make_double2(0.0, 0.0);
  } else {
    for (int c = 0; c < 3; ++c) p.e_inc[c] = t.pm[c];
  }
  apply_TR(t, m.rs, m.rp, p.e_inc, p.r_inc);
  p.beta00 = m.beta;
  rp[rhs0 + i] = p;
}

// b = E_inc + R[E_inc] on the absorber planes (Eqs. (3), (9)): uniform in (x, y),
// e exp(-i beta00 z_p) + T_R e exp(+i beta00 z_p), z_p = (p + 1/2) dz.
// grid (3 nslab, nrhs): one CTA per (component, plane); the value is evaluated once.
__global__ void k_build_rhs(int rhs0, const RhsParam* rp, int nslab, int plane, double dz, double2* b) {
  __shared__ double2 val;
  const int cp = blockIdx.x, lr = blockIdx.y;
  const int c = cp / nslab, p = cp % nslab;
  if (threadIdx.x == 0) {
    const RhsParam& q = rp[rhs0 + lr];
    const double z = (p + 0.5) * dz;
    const double2 bz = cscale(q.beta00, z);
    const double2 down = cexp_d(make_double2(bz.y, -bz.x));  // exp(-i beta00 z)
    const double2 up = cexp_d(make_double2(-bz.y, bz.x));    // exp(+i beta00 z)
    val = cadd(cmul(q.e_inc[c], down), cmul(q.r_inc[c], up));
  }
  __syncthreads();
  const double2 v = val;
  double2* dst = b + ((size_t)lr * 3 * nslab + cp) * plane;
  for (int i = threadIdx.x; i < plane; i += blockDim.x) dst[i] = v;
}

int launch_rhs(int rhs0, int nrhs, RhsParam* rp, const ModeEntry* modes, int nx, int ny, int nslab, double dz,
               double kb, double2* b, cudaStream_t st) {
  k_rhs_params<<<(nrhs + 63) / 64, 64, 0, st>>>(rhs0, nrhs, rp, modes, nx, ny, kb);
  if (launched() != PSFD_OK) return PSFD_E_CUDA;
  k_build_rhs<<<dim3(3 * nslab, nrhs), 256, 0, st>>>(rhs0, rp, nslab, nx * ny, dz, b);
  return launched();
}

// ---------------------------------------------------------------------------
// Diffraction orders (Eqs. (3), (9)): amplitude at z_top of every propagating order,
//   A = T_R (delta_{mn,00} e + E0 exp(-i beta dz/2)) + Etop exp(-i beta (nslab + 1/2) dz),
// E0 / Etop being the normalised spectra of G*(V u) on plane 0 (z = -dz/2) and plane
// nslab+1. Output per order: A (3 complex), a_s, a_p (s . A, p+ . A), efficiency.
// ---------------------------------------------------------------------------
__global__ void k_orders(OrdersArgs a) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x, g = blockIdx.y;
  if (k >= a.n_orders[g] || (a.mask && !a.mask[g])) return;
  const int mi = a.mn[((size_t)g * a.max_orders + k) * 2], ni = a.mn[((size_t)g * a.max_orders + k) * 2 + 1];
  const int x = (mi + a.nx) % a.nx, y = (ni + a.ny) % a.ny;
  const RhsParam p = a.rhsp[g];
  const ModeEntry m = a.modes[((size_t)p.slot * a.ny + y) * a.nx + x];
  const double two_pi = 6.283185307179586476925286766559;
  const double qx = p.qix + two_pi * mi / (a.nx * a.dx);
  const double qy = p.qiy + two_pi * ni / (a.ny * a.dy);
  const Triad t = triad_d(qx, qy, m.beta, a.kb, p.cphi, p.sphi);
  const size_t plane = (size_t)a.ny * a.nx;
  const size_t o0 = ((size_t)g * 2 * 3) * plane + (size_t)y * a.nx + x;
  const double2 bh = cscale(m.beta, 0.5 * a.dz);
  const double2 ph0 = cexp_d(make_double2(bh.y, -bh.x));  // exp(-i beta dz/2)
  const double2 bt = cscale(m.beta, (a.nslab + 0.5) * a.dz);
  const double2 pht = cexp_d(make_double2(bt.y, -bt.x));
  double2 down[3], A[3];
  for (int c = 0; c < 3; ++c) {
    down[c] = cmul(a.side[o0 + c * plane], ph0);
    if (mi == 0 && ni == 0) down[c] = cadd(down[c], p.e_inc[c]);
  }
  apply_TR(t, m.rs, m.rp, down, A);
  for (int c = 0; c < 3; ++c) A[c] = cadd(A[c], cmul(a.side[o0 + (3 + c) * plane], pht));
  double* out = a.out + ((size_t)g * a.max_orders + k) * 12;
  for (int c = 0; c < 3; ++c) {
    out[2 * c] = A[c].x;
    out[2 * c + 1] = A[c].y;
  }
  const double2 as = cadd(cscale(A[0], t.sx), cscale(A[1], t.sy));
  const double2 ap = cadd(cadd(cmul(t.pp[0], A[0]), cmul(t.pp[1], A[1])), cmul(t.pp[2], A[2]));
  out[6] = as.x;
  out[7] = as.y;
  out[8] = ap.x;
  out[9] = ap.y;
  out[10] = (cabs2(A[0]) + cabs2(A[1]) + cabs2(A[2])) * m.beta.x / p.beta00.x;
  out[11] = 0.0;
}

int launch_orders(const OrdersArgs& a, int nrhs, cudaStream_t st) {
  dim3 grid((a.max_orders + 127) / 128, nrhs);
  k_orders<<<grid, 128, 0, st>>>(a);
  return launched();
}

// ---------------------------------------------------------------------------
// defect correction helpers (FP64 outer loop around the FP32 Krylov solve)
// ---------------------------------------------------------------------------
// partial ||v||^2 per block into slot 2
__global__ void __launch_bounds__(VEC_NT) k_norm2_partials(int n, int nblk, int rhs0, const int* mask,
                                                            const double2* v, double2* partials, int maxblk) {
  const int blk = blockIdx.x, lr = blockIdx.y, g = rhs0 + lr;
  if (mask && !mask[g]) return;
  const size_t off = (size_t)lr * n;
  const int chunk = (n + nblk - 1) / nblk;
  const int lo = blk * chunk, hi = min(n, lo + chunk);
  double2 d2 = make_double2(0.0, 0.0);
  for (int i = lo + threadIdx.x; i < hi; i += VEC_NT) d2.x += cabs2(v[off + i]);
  vec_block_dots<double2>(make_double2(0.0, 0.0), d2, DOT_OUT_OUT, partials + ((size_t)g * NDOT) * maxblk + blk,
                          maxblk);
}

// mode 0: bnorm2 = rnorm2 = sum (initial residual = b); mode 1: rnorm2 = sum.
// act = rnorm2 > tol2 * bnorm2. Right-hand sides outside mask (null = all) are untouched.
__global__ void __launch_bounds__(VEC_NT) k_norm_finish(int rhs0, int nblk, const int* mask, const double2* partials,
                                                         int maxblk, int mode, double tol2, KScal* sc, int* act) {
  __shared__ double2 sh[33];
  const int g = rhs0 + blockIdx.x;
  if (mask && !mask[g]) return;
  const double2 s = block_sum_fixed(slot_ptr(partials, g, 2, maxblk), nblk, sh);
  if (threadIdx.x == 0) {
    if (mode == 0) sc[g].bnorm2 = s.x;
    sc[g].rnorm2 = s.x;
    act[g] = (s.x > tol2 * sc[g].bnorm2) && isfinite(s.x);
  }
}

int launch_norm(int n, int nblk, int rhs0, int nrhs, const int* mask, const double2* v, double2* partials,
                int maxblk, int mode, double tol2, KScal* sc, int* act, cudaStream_t st) {
  if (v) {
    k_norm2_partials<<<dim3(nblk, nrhs), VEC_NT, 0, st>>>(n, nblk, rhs0, mask, v, partials, maxblk);
    if (launched() != PSFD_OK) return PSFD_E_CUDA;
  }
  k_norm_finish<<<nrhs, VEC_NT, 0, st>>>(rhs0, nblk, mask, partials, maxblk, mode, tol2, sc, act);
  return launched();
}

// FP32 <-> FP64 of one value by integer operations (df_f32_rn / df_f64_of), falling back to
// the conversion instruction outside their range: this GPU's FP64 pipe, which runs those
// instructions, is far slower than its integer and FP32 pipes.
__device__ __forceinline__ float f32_of(double d) {
  float f;
  return df_f32_rn(d, f) ? f : (float)d;
}
__device__ __forceinline__ double f64_of(float f) {
  double d;
  return df_f64_of(f, d) ? d : (double)f;
}

// rs = r64 / ||r64|| in the Krylov precision (right-hand sides selected by act). 1/||r64|| is
// formed once per CTA. In FP32 each element is rounded to FP32 and scaled there (when the scale
// is moderate, so that no element that matters leaves the FP32 range): no FP64 arithmetic per
// element, against one FP64 scaling before the rounding otherwise.
template <typename C>
__global__ void k_ref_scale(int n, int rhs0, const int* act, const KScal* sc, const double2* r64, C* rs) {
  const int lr = blockIdx.y, g = rhs0 + lr;
  if (!act[g]) return;
  __shared__ double s_inv;
  if (threadIdx.x == 0) s_inv = 1.0 / sqrt(sc[g].rnorm2);
  __syncthreads();
  const double inv = s_inv;
  const size_t off = (size_t)lr * n;
  if constexpr (sizeof(C) == sizeof(float2)) {
    if (inv > 0x1p-60 && inv < 0x1p60) {
      const float fi = f32_of(inv);
      for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double2 r = r64[off + i];
        rs[off + i] = make_float2(f32_of(r.x) * fi, f32_of(r.y) * fi);
      }
      return;
    }
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    rs[off + i] = from_c64<C>(cscale(r64[off + i], inv));
}

// x64 += ||r64|| xc (the FP32 correction widened exactly by integer operations; ||r64|| once
// per CTA)
template <typename C>
__global__ void k_ref_update(int n, int rhs0, const int* act, const KScal* sc, double2* x64, const C* xc) {
  const int lr = blockIdx.y, g = rhs0 + lr;
  if (!act[g]) return;
  __shared__ double s_s;
  if (threadIdx.x == 0) s_s = sqrt(sc[g].rnorm2);
  __syncthreads();
  const double s = s_s;
  const size_t off = (size_t)lr * n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double2 d;
    if constexpr (sizeof(C) == sizeof(float2)) {
      const C v = xc[off + i];
      d = make_double2(f64_of(v.x), f64_of(v.y));
    } else {
      d = xc[off + i];
    }
    x64[off + i] = cadd(x64[off + i], cscale(d, s));
  }
}

__global__ void k_vec_add(int n, int rhs0, const int* mask, double2* a, const double2* b) {
  const int lr = blockIdx.y, g = rhs0 + lr;
  if (mask && !mask[g]) return;
  const size_t off = (size_t)lr * n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    a[off + i] = cadd(a[off + i], b[off + i]);
}

int launch_vec_add(int n, int rhs0, int nrhs, const int* mask, double2* a, const double2* b, cudaStream_t st) {
  const int bx = (n + 256 * 8 - 1) / (256 * 8);
  k_vec_add<<<dim3(bx, nrhs), 256, 0, st>>>(n, rhs0, mask, a, b);
  return launched();
}

template <typename C>
int launch_ref_scale(int n, int rhs0, int nrhs, const int* act, const KScal* sc, const double2* r64, C* rs,
                     cudaStream_t st) {
  const int bx = (n + 256 * 8 - 1) / (256 * 8);
  k_ref_scale<C><<<dim3(bx, nrhs), 256, 0, st>>>(n, rhs0, act, sc, r64, rs);
  return launched();
}

template <typename C>
int launch_ref_update(int n, int rhs0, int nrhs, const int* act, const KScal* sc, double2* x64, const C* xc,
                      cudaStream_t st) {
  const int bx = (n + 256 * 8 - 1) / (256 * 8);
  k_ref_update<C><<<dim3(bx, nrhs), 256, 0, st>>>(n, rhs0, act, sc, x64, xc);
  return launched();
}
template int launch_ref_scale<float2>(int, int, int, const int*, const KScal*, const double2*, float2*, cudaStream_t);
template int launch_ref_scale<double2>(int, int, int, const int*, const KScal*, const double2*, double2*,
                                       cudaStream_t);
template int launch_ref_update<float2>(int, int, int, const int*, const KScal*, double2*, const float2*,
                                       cudaStream_t);
template int launch_ref_update<double2>(int, int, int, const int*, const KScal*, double2*, const double2*,
                                        cudaStream_t);

// ---------------------------------------------------------------------------
// FFT test hook: `count` contiguous length-N transforms, B per CTA.
// ---------------------------------------------------------------------------
template <typename C, int N, bool INV>
__global__ void __launch_bounds__(256) k_test_fft(C* data, int count, const double2* tw64) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int B = N >= 2048 ? 1 : 2048 / N;
  C* tile = reinterpret_cast<C*>(smem);
  constexpr int PN = fft_phys(N);
  C* tw = tile + B * PN;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = from_c64<C>(tw64[i]);
  const int f0 = blockIdx.x * B;
  const int nb = min(B, count - f0);
  for (int i = threadIdx.x; i < nb * N; i += blockDim.x) tile[(i / N) * PN + fpad(i % N)] = data[(size_t)f0 * N + i];
  __syncthreads();
  cta_fft<C, N, INV>(tile, nb, PN, tw);
  __syncthreads();
  for (int i = threadIdx.x; i < nb * N; i += blockDim.x) data[(size_t)f0 * N + i] = tile[(i / N) * PN + fpad(i % N)];
}

template <typename C, int N>
int run_test_fft(C* data, int count, bool inv, const double2* tw) {
  constexpr int B = N >= 2048 ? 1 : 2048 / N;
  const size_t smem = (size_t)(B * fft_phys(N) + N) * sizeof(C);
  const int grid = (count + B - 1) / B;
  if (inv) {
    auto k = k_test_fft<C, N, true>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<grid, 256, smem>>>(data, count, tw);
  } else {
    auto k = k_test_fft<C, N, false>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<grid, 256, smem>>>(data, count, tw);
  }
  return launched();
}

int launch_test_fft(int n, int count, bool inv, bool fp64, void* data, const double2* tw) {
  switch (n) {
#define X(v)                                                                              \
  case v:                                                                                 \
    return fp64 ? run_test_fft<double2, v>((double2*)data, count, inv, tw)                \
                : run_test_fft<float2, v>((float2*)data, count, inv, tw);
    X(4) X(8) X(16) X(32) X(64) X(96) X(128) X(160) X(192) X(256) X(320) X(384) X(512) X(640) X(768) X(1024)
#undef X
  }
  return PSFD_E_ARG;
}

}  // namespace psfd
