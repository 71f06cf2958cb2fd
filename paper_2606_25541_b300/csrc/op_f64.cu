// op_f64.cu -- complex FP64 instantiation of the operator and the Krylov solvers.
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
