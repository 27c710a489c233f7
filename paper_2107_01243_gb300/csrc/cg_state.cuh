// Transitions of the device-side CG state (CGState), each run by the one
// thread that holds a grid reduction's totals; shared by every kernel that
// finishes a CG reduction (vector kernels, element kernels with a fused
// <p, H p>, the batched kernels).
#pragma once
#include "sem_internal.cuh"

namespace sem {

// after <r, z>, <r, r> of the starting residual (tot = {rz, rr})
__device__ __forceinline__ void st_after_init(CGState* st, const double (&tot)[2], double tol,
                                              int maxit, int bb_from_rr) {
  st->rz = tot[0];
  st->rr = tot[1];
  if (bb_from_rr) st->bb = tot[1];
  st->tol2 = tol * tol * st->bb;
  st->iter = 0;
  st->status = SEM_OK;
  st->maxit = maxit;
  st->alpha = st->beta = 0.0;
  st->done = (tot[1] <= st->tol2 || st->bb == 0.0 || maxit <= 0) ? 1 : 0;
  if (st->done && !(tot[1] <= st->tol2 || st->bb == 0.0)) st->status = SEM_ERR_NOCONV;
}

// after <p, w>: alpha, or breakdown
__device__ __forceinline__ void st_after_pw(CGState* st, double pw) {
  st->pw = pw;
  if (!(pw > 0.0)) {
    st->status = SEM_ERR_BREAKDOWN;
    st->done = 1;
  } else {
    st->alpha = st->rz / pw;
  }
}

// after the x, r update (tot = {<r, z>, <r, r>}): stop test, beta
__device__ __forceinline__ void st_after_update(CGState* st, const double (&tot)[2]) {
  st->iter += 1;
  st->rr = tot[1];
  if (!(tot[1] == tot[1]) || !(tot[0] == tot[0])) {
    st->status = SEM_ERR_BREAKDOWN;
    st->done = 1;
  } else if (tot[1] <= st->tol2) {
    st->done = 1;
  } else if (st->iter >= st->maxit) {
    st->status = SEM_ERR_NOCONV;
    st->done = 1;
  } else {
    st->beta = tot[0] / st->rz;
    st->rz = tot[0];
  }
}

}  // namespace sem
