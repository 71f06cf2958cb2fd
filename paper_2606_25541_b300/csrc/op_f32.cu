// op_f32.cu -- complex FP32 instantiation of the operator and BiCGStab (bulk path).
#include "solver.cuh"

namespace psfd {
template <> int op_apply<float2>(const OpCall<float2>& a) { return op_apply_impl<float2>(a); }
template <> int bicgstab<float2>(const KrylovCall<float2>& k) { return bicgstab_impl<float2>(k); }
}  // namespace psfd
