// solver.cuh -- host driver of the batched BiCGStab loop (one instantiation per precision).
//
// Per iteration: v = A p with p = r + beta (p - omega v) formed inside K1; alpha;
// t = A s with s = r - alpha v formed inside K1; omega; x and r updated with their dot
// products; rho, beta and the convergence test. All scalars stay on the device; the
// host reads the per-RHS activity flags every check_every iterations only.
#pragma once

#include "krylov.cuh"
#include "op_launch.cuh"

namespace psfd {

template <typename C>
int bicgstab_impl(const KrylovCall<C>& k) {
  const OpCall<C>& base = k.op;
  cudaStream_t st = base.stream;
  const int nrhs = base.nrhs, rhs0 = base.rhs0;
  int nblk = (k.n + 8191) / 8192;
  if (nblk > base.maxblk) nblk = base.maxblk;
  if (nblk < 1) nblk = 1;
  k_bicg_init<C><<<dim3(nblk, nrhs), VEC_NT, 0, st>>>(k.n, nblk, rhs0, k.b, k.x, k.r, k.r0, k.p, k.v,
                                                       base.partials, base.maxblk);
  PSFD_CHECK_LAUNCH();
  k_scal_init<<<nrhs, VEC_NT, 0, st>>>(rhs0, nblk, base.partials, base.maxblk, k.act_in, k.sc, k.act);
  PSFD_CHECK_LAUNCH();

  OpCall<C> pv = base;  // v = A p
  pv.active = k.act;
  pv.in_mode = IN_PUPDATE;
  pv.u = k.p;
  pv.ustore = k.p;
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

  const double tol2 = k.tol * k.tol;
  const int every = k.check_every > 0 ? k.check_every : 4;
  for (int it = 0; it < k.max_iter; ++it) {
    int nb = op_apply_impl<C>(pv);
    if (nb < 0) return nb;
    k_scal_alpha<<<nrhs, VEC_NT, 0, st>>>(rhs0, nb, base.partials, base.maxblk, k.sc, k.act);
    PSFD_CHECK_LAUNCH();
    nb = op_apply_impl<C>(ts);
    if (nb < 0) return nb;
    k_scal_omega<<<nrhs, VEC_NT, 0, st>>>(rhs0, nb, base.partials, base.maxblk, k.sc, k.act);
    PSFD_CHECK_LAUNCH();
    const int vcls = sizeof(C) == 16 ? PK_VEC64 : PK_VEC32;
    prof_begin(vcls, st);
    k_bicg_xr<C><<<dim3(nblk, nrhs), VEC_NT, 0, st>>>(k.n, nblk, rhs0, k.act, k.sc, k.x, k.p, k.s, k.t, k.r,
                                                       k.r0, base.partials, base.maxblk);
    PSFD_CHECK_LAUNCH();
    // reads x, p, s, t, r0; writes x, r
    prof_end(vcls, st, 7.0 * nrhs * (double)k.n * sizeof(C), 24.0 * nrhs * (double)k.n);
    k_scal_rho<<<nrhs, VEC_NT, 0, st>>>(rhs0, nblk, base.partials, base.maxblk, tol2, k.max_iter, k.sc, k.act);
    PSFD_CHECK_LAUNCH();
    if ((it + 1) % every == 0 || it + 1 == k.max_iter) {
      if (cudaMemcpyAsync(k.h_act + rhs0, k.act + rhs0, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, st) !=
          cudaSuccess)
        return PSFD_E_CUDA;
      if (cudaStreamSynchronize(st) != cudaSuccess) return PSFD_E_CUDA;
      bool any = false;
      for (int i = 0; i < nrhs; ++i) any = any || k.h_act[rhs0 + i];
      if (!any) break;
    }
  }
  return PSFD_OK;
}

}  // namespace psfd
