// solver.cuh -- host side of the batched BiCGStab loop (one instantiation per precision).
//
// Per iteration: v = A p with p = r + beta (p - omega v) formed inside K1; alpha;
// t = A s with s = r - alpha v formed inside K1; omega; x and r updated with their dot
// products; rho, beta and the convergence test. All scalars and the per-RHS activity
// flags stay on the device: iterations are enqueued without any host synchronisation,
// and right-hand sides that converged (or were never started) are skipped by every
// kernel, so illuminations at different stages of their solve can share the launches.
#pragma once

#include "krylov.cuh"
#include "op_launch.cuh"

namespace psfd {

template <typename C>
int vec_blocks(const KrylovCall<C>& k) {
  int nblk = (k.n + 8191) / 8192;
  if (nblk > k.op.maxblk) nblk = k.op.maxblk;
  return nblk < 1 ? 1 : nblk;
}

template <typename C>
int bicg_start_impl(const KrylovCall<C>& k, const int* mask) {
  const OpCall<C>& base = k.op;
  cudaStream_t st = base.stream;
  const int nblk = vec_blocks(k);
  k_bicg_init<C><<<dim3(nblk, base.nrhs), VEC_NT, 0, st>>>(k.n, nblk, base.rhs0, mask, k.b, k.x, k.r, k.r0, k.p,
                                                            k.v, base.partials, base.maxblk);
  PSFD_CHECK_LAUNCH();
  k_scal_init<<<base.nrhs, VEC_NT, 0, st>>>(base.rhs0, nblk, base.partials, base.maxblk, mask, k.tol, k.tol_slot,
                                            k.sc, k.act);
  PSFD_CHECK_LAUNCH();
  return PSFD_OK;
}

template <typename C>
int bicg_iterate_impl(const KrylovCall<C>& k, int iters) {
  const OpCall<C>& base = k.op;
  cudaStream_t st = base.stream;
  const int nrhs = base.nrhs, rhs0 = base.rhs0;
  const int nblk = vec_blocks(k);

  OpCall<C> pv = base;  // v = A p
  pv.active = k.act;
  pv.in_mode = IN_PUPDATE;
  pv.u = k.p;
  // Half-plane K1 kernels read every element of p from two CTAs: the updated p goes to
  // pn there, and the x/r update copies it back into p.
  pv.ustore = use_half<C>(base.nx, base.ny) ? k.pn : k.p;
  pv.r = k.r;
  pv.v = k.v;
  pv.sc = k.sc;
  pv.work = k.work;
  pv.epi = EPI_AU;
  pv.out = k.v;
  pv.r0 = k.r0;
  pv.dot_mask = DOT_R0_OUT;
  pv.side = nullptr;

  OpCall<C> ts = pv;  // t = A s
  ts.in_mode = IN_SUPDATE;
  ts.u = nullptr;
  ts.ustore = k.s;
  ts.out = k.t;
  ts.dot_mask = DOT_OUT_U | DOT_OUT_OUT;

  for (int it = 0; it < iters; ++it) {
    int nb = op_apply_impl<C>(pv);
    if (nb < 0) return nb;
    k_scal_alpha<<<nrhs, VEC_NT, 0, st>>>(rhs0, nb, base.partials, base.maxblk, k.sc, k.act);
    PSFD_CHECK_LAUNCH();
    nb = op_apply_impl<C>(ts);
    if (nb < 0) return nb;
    k_scal_omega<<<nrhs, VEC_NT, 0, st>>>(rhs0, nb, base.partials, base.maxblk, k.sc, k.act);
    PSFD_CHECK_LAUNCH();
    const int vcls = sizeof(C) == 16 ? PK_VEC64 : PK_VEC32;
    unsigned* ctac = prof_begin(vcls, st);
    k_bicg_xr<C><<<dim3(nblk, nrhs), VEC_NT, 0, st>>>(k.n, nblk, rhs0, k.act, k.sc, k.x, pv.ustore, k.p, k.s, k.t,
                                                       k.r, k.r0, base.partials, base.maxblk, ctac);
    PSFD_CHECK_LAUNCH();
    // reads x, p, s, t, r0; writes x, r (and p when the update went to pn)
    const double nvec = pv.ustore == k.p ? 7.0 : 8.0;
    prof_end(vcls, st, nvec * nrhs * (double)k.n * sizeof(C), 24.0 * nrhs * (double)k.n, (double)nblk * nrhs);
    k_scal_rho<<<nrhs, VEC_NT, 0, st>>>(rhs0, nblk, base.partials, base.maxblk, k.max_iter, k.sc, k.act);
    PSFD_CHECK_LAUNCH();
  }
  return PSFD_OK;
}

}  // namespace psfd
