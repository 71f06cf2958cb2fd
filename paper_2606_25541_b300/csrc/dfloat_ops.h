// dfloat_ops.h -- the FP64 residual operator with its z pass in double-float arithmetic.
#pragma once

#include "internal.h"

namespace psfd {

// wdf = true: the spectral work array a.work holds double-float pairs (dfc) instead of FP64 on
// the pass's input and output (every pass of the chain is double-float, see op_apply_df).

// Whether launch_zcol_df handles this call (nf 64 or 128, periodic kernel, x tiles that
// divide nx); otherwise the FP64 z pass runs.
bool zcol_df_supported(const OpCall<double2>& a);
// K2 of an FP64 operator call with the z transforms and dyadic products in double-float.
int launch_zcol_df(const OpCall<double2>& a, bool wdf = false);
// Whether launch_cols_df handles the column pass of this call's split planes (ny 128 or 256,
// nx a multiple of 8); the pass transforms in place along y (inverse = 1: unnormalised inverse).
bool cols_df_supported(const OpCall<double2>& a);
int launch_cols_df(const OpCall<double2>& a, bool inverse, bool wdf = false);
// Whether the row passes of this call's split planes run in double-float (nx 64, 128 or 256,
// plain input stage, epilogue u - w or b - (u - w)); the forward pass forms J = V u and
// transforms along x, the inverse transforms back and applies the epilogue with its dots.
bool rows_df_supported(const OpCall<double2>& a);
int launch_rows_fwd_df(const OpCall<double2>& a, bool wdf);
int launch_rows_inv_df(const OpCall<double2>& a, const double2* uin, bool wdf);
// op_apply<double2> with launch_zcol_df as its z pass and launch_cols_df as the column passes
// of split planes where supported (the refined solve's residual); returns the partial-sum
// blocks per RHS or a negative status, like op_apply.
int op_apply_df(const OpCall<double2>& a);

}  // namespace psfd
