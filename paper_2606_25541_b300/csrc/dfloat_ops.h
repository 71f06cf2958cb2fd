// dfloat_ops.h -- the FP64 residual operator with its z pass in double-float arithmetic.
#pragma once

#include "internal.h"

namespace psfd {

// Whether launch_zcol_df handles this call (nf 64 or 128, periodic kernel, x tiles that
// divide nx); otherwise the FP64 z pass runs.
bool zcol_df_supported(const OpCall<double2>& a);
// K2 of an FP64 operator call with the z transforms and dyadic products in double-float.
int launch_zcol_df(const OpCall<double2>& a);
// op_apply<double2> with launch_zcol_df as its z pass where supported (the refined solve's
// residual); returns the partial-sum blocks per RHS or a negative status, like op_apply.
int op_apply_df(const OpCall<double2>& a);

}  // namespace psfd
