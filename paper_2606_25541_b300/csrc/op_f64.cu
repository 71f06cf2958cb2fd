// op_f64.cu -- complex FP64 instantiation of the operator and the Krylov solvers.
#include "dfloat_ops.h"
#include "gmres.cuh"
#include "solver.cuh"

namespace psfd {
template <> int op_apply<double2>(const OpCall<double2>& a) { return op_apply_impl<double2>(a); }
template <> int bicg_start<double2>(const KrylovCall<double2>& k, const int* mask) {
  return bicg_start_impl<double2>(k, mask);
}
template <> int bicg_iterate<double2>(const KrylovCall<double2>& k, int iters) {
  return bicg_iterate_impl<double2>(k, iters);
}
template <> int gmres_start<double2>(const KrylovCall<double2>& k, const int* mask) {
  return gmres_start_impl<double2>(k, mask);
}
template <> int gmres_iterate<double2>(const KrylovCall<double2>& k, int iters) {
  return gmres_iterate_impl<double2>(k, iters);
}
template <> int gmres_finish<double2>(const KrylovCall<double2>& k, const int* mask) {
  return gmres_finish_impl<double2>(k, mask);
}

// Row passes of FP64 split planes, for op_apply_df.
template <int IN>
static int rows_fwd64(const OpCall<double2>& a) {
  switch (a.nx) {
#define X(n) \
  case n:    \
    return launch_rows_fwd<double2, n, IN>(a);
    PSFD_FOR_EACH_LENGTH(X)
#undef X
  }
  return PSFD_E_ARG;
}
template <int EPI>
static int rows_inv64(const OpCall<double2>& a, const double2* uin) {
  switch (a.nx) {
#define X(n) \
  case n:    \
    return launch_rows_inv<double2, n, EPI>(a, uin);
    PSFD_FOR_EACH_LENGTH(X)
#undef X
  }
  return PSFD_E_ARG;
}

// The FP64 operator with the double-float passes where their kernels handle the call: the z
// pass (zcol_df.cu), the column passes of split planes (cols_df.cu) and their row passes
// (rows_df.cu); fused planes as in op_apply<double2>, the profile class of each pass
// unchanged. When all five passes are double-float, the spectral work array carries
// double-float pairs between them (only x, V, b and the output are converted).
int op_apply_df(const OpCall<double2>& a0) {
  const bool zdf = zcol_df_supported(a0);
  const bool ydf = !use_fused<double2>(a0.nx, a0.ny) && cols_df_supported(a0);
  const bool xdf = ydf && rows_df_supported(a0);
  const bool wdf = xdf && zdf;
  if (!zdf && !ydf) return op_apply_impl<double2>(a0);
  const bool prof = prof_on();
  OpCall<double2> a = a0;
  PassCost cost;
  double cx = 0, cz = 0;
  if (prof) {
    cost = pass_cost(a);
    pass_ctas(a, &cx, &cz);
  }
  int rc;
  a.ctac = prof ? prof_begin(PK_FWD64, a.stream) : nullptr;
  switch (a.in_mode) {
    case IN_PLAIN:
      rc = xdf ? launch_rows_fwd_df(a, wdf) : (ydf ? rows_fwd64<IN_PLAIN>(a) : dispatch_fwd<double2, IN_PLAIN>(a));
      break;
    case IN_PUPDATE: rc = ydf ? rows_fwd64<IN_PUPDATE>(a) : dispatch_fwd<double2, IN_PUPDATE>(a); break;
    case IN_SUPDATE: rc = ydf ? rows_fwd64<IN_SUPDATE>(a) : dispatch_fwd<double2, IN_SUPDATE>(a); break;
    default: return PSFD_E_ARG;
  }
  if (rc) return rc;
  if (ydf && (rc = launch_cols_df(a, false, wdf))) return rc;
  if (prof) prof_end(PK_FWD64, a.stream, cost.bytes[0], cost.flops[0], cx);
  a.ctac = prof ? prof_begin(PK_Z64, a.stream) : nullptr;
  if ((rc = zdf ? launch_zcol_df(a, wdf) : dispatch_z<double2>(a))) return rc;
  if (prof) prof_end(PK_Z64, a.stream, cost.bytes[1], cost.flops[1], cz);
  if (a.epi == EPI_NONE) return blocks_per_rhs_t<double2>(a.nx, a.ny, a.nslab);
  const double2* uin = a.in_mode == IN_PLAIN ? a.u : a.ustore;
  a.ctac = prof ? prof_begin(PK_INV64, a.stream) : nullptr;
  if (ydf && (rc = launch_cols_df(a, true, wdf))) return rc;
  if (xdf) {
    rc = launch_rows_inv_df(a, uin, wdf);
  } else {
    switch (a.epi) {
      case EPI_AU: rc = ydf ? rows_inv64<EPI_AU>(a, uin) : dispatch_inv<double2, EPI_AU>(a, uin); break;
      case EPI_RESID: rc = ydf ? rows_inv64<EPI_RESID>(a, uin) : dispatch_inv<double2, EPI_RESID>(a, uin); break;
      default: return PSFD_E_ARG;
    }
  }
  if (rc) return rc;
  if (prof) prof_end(PK_INV64, a.stream, cost.bytes[2], cost.flops[2], cx);
  return blocks_per_rhs_t<double2>(a.nx, a.ny, a.nslab);
}

int op_blocks_per_rhs(int nx, int ny, int nslab, bool fp64) {
  return fp64 ? blocks_per_rhs_t<double2>(nx, ny, nslab) : blocks_per_rhs_t<float2>(nx, ny, nslab);
}

bool fft_length_supported(int n) {
  switch (n) {
#define X(v) case v: return true;
    PSFD_FOR_EACH_LENGTH(X)
#undef X
  }
  return false;
}
}  // namespace psfd
