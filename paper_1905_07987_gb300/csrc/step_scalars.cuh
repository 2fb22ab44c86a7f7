// Device-side time-step scalars shared by the per-context kernels (common.cu) and the ensemble's
// persistent launches: the time-step finalisation of Eq. (7) and the time advance.
#pragma once
#include "ader_internal.h"

namespace ader {

// dt = CFL_N / (d (2N+1)) * min_d h_d / lambda_max  (or the fixed dt), clipped to t_end.
__device__ __forceinline__ void dt_finalize_one(const StepArgs& A) {
  DevScalars* s = A.dev;
  double dt;
  if (A.dt_fixed > 0.0) {
    dt = A.dt_fixed;
  } else {
    const double lam = __longlong_as_double((long long)s->lam_bits);
    double hmin = A.g.h[0];
    for (int d = 1; d < A.g.dim; ++d) hmin = fmin(hmin, A.g.h[d]);
    dt = A.cfl / (double)(A.g.dim * (2 * A.g.order + 1)) * hmin / lam;
  }
  if (A.t_end > 0.0) dt = fmin(dt, A.t_end - s->t);
  if (dt < 0.0) dt = 0.0;
  if (!isfinite(dt)) {
    atomicOr(&s->status, ST_NONFINITE);
    dt = 0.0;
  }
  s->dt = dt;
  s->lam_bits = 0ull;
  s->lam_lo_bits = 0u;
  s->n_troubled = 0;
  s->fv_retry = 0;
}

__device__ __forceinline__ void advance_one(DevScalars* s, int receivers_on) {
  s->t += s->dt;
  s->nstep += 1;
  if (receivers_on) s->seismo_row += 1;
}

}  // namespace ader
