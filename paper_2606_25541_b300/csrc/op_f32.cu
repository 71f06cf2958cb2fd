// op_f32.cu -- complex FP32 instantiation of the operator and the Krylov solvers (bulk path).
#include "gmres.cuh"
#include "solver.cuh"

namespace psfd {
template <> int op_apply<float2>(const OpCall<float2>& a) { return op_apply_impl<float2>(a); }
template <> int bicg_start<float2>(const KrylovCall<float2>& k, const int* mask) {
  return bicg_start_impl<float2>(k, mask);
}
template <> int bicg_iterate<float2>(const KrylovCall<float2>& k, int iters) {
  return bicg_iterate_impl<float2>(k, iters);
}
template <> int gmres_start<float2>(const KrylovCall<float2>& k, const int* mask) {
  return gmres_start_impl<float2>(k, mask);
}
template <> int gmres_iterate<float2>(const KrylovCall<float2>& k, int iters) {
  return gmres_iterate_impl<float2>(k, iters);
}
template <> int gmres_finish<float2>(const KrylovCall<float2>& k, const int* mask) {
  return gmres_finish_impl<float2>(k, mask);
}
}  // namespace psfd
