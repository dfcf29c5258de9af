/* Prints the size and every field offset of the structs of include/dfm.h, one
 * "struct field offset" line each, and "struct sizeof size"; read by
 * tests/test_abi_layout.py to check that the Python binding's ctypes mirrors
 * match the C layout. */
#include <stddef.h>
#include <stdio.h>

#include "dfm.h"

#define F(S, f) printf(#S " " #f " %zu\n", offsetof(S, f))
#define Z(S) printf(#S " sizeof %zu\n", sizeof(S))

int main(void) {
  F(dfm_mesh_info_t, n_verts); F(dfm_mesh_info_t, n_tets); F(dfm_mesh_info_t, n_rows);
  F(dfm_mesh_info_t, n_boundary_rows); F(dfm_mesh_info_t, min_abs_volume); F(dfm_mesh_info_t, total_volume);
  Z(dfm_mesh_info_t);
  F(dfm_params, Np); F(dfm_params, mu); F(dfm_params, mu_uniform); F(dfm_params, quad_order);
  F(dfm_params, max_patch_deg); F(dfm_params, precision); F(dfm_params, moment); F(dfm_params, c);
  F(dfm_params, rho_f);
  Z(dfm_params);
  F(dfm_op_info_t, Np); F(dfm_op_info_t, nb); F(dfm_op_info_t, precision); F(dfm_op_info_t, n_rows);
  F(dfm_op_info_t, row_stride); F(dfm_op_info_t, vals); F(dfm_op_info_t, bytes);
  Z(dfm_op_info_t);
  F(dfm_solve_opts, method); F(dfm_solve_opts, tol); F(dfm_solve_opts, max_iter); F(dfm_solve_opts, restart);
  F(dfm_solve_opts, use_x0); F(dfm_solve_opts, inner_tol); F(dfm_solve_opts, transpose);
  F(dfm_solve_opts, poly_degree); F(dfm_solve_opts, precond_precision); F(dfm_solve_opts, batch);
  F(dfm_solve_opts, block); F(dfm_solve_opts, coarse);
  Z(dfm_solve_opts);
  F(dfm_solve_info, iters); F(dfm_solve_info, outer); F(dfm_solve_info, resid);
  Z(dfm_solve_info);
  return 0;
}
