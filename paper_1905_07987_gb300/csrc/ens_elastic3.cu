// Batched ensemble step of the 3-D elastic family with the FP64 predictor, orders 1-5 (one
// persistent launch per phase for all runs).
#include "kernels_ensemble.cuh"

namespace ader {

cudaError_t ens_step_elastic3_fp64(const StepArgs* R, const EnsTable& E, const Tables& T,
                                   const TablesF& F, int order, cudaStream_t s) {
  switch (order) {
    case 1: return ens_step_n<Elastic, 3, 1, false>(R, E, T, F, s);
    case 2: return ens_step_n<Elastic, 3, 2, false>(R, E, T, F, s);
    case 3: return ens_step_n<Elastic, 3, 3, false>(R, E, T, F, s);
    case 4: return ens_step_n<Elastic, 3, 4, false>(R, E, T, F, s);
    case 5: return ens_step_n<Elastic, 3, 5, false>(R, E, T, F, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t ens_fused_elastic3_fp64(const StepArgs* R, const EnsTable& E, const Tables& T, const TablesF& F, int order,
               int steps, void* bar, long long limit, int bps, cudaStream_t s) {
  GridBar* b = static_cast<GridBar*>(bar);
  switch (order) {
    case 1: return ens_fused_n<Elastic, 3, 1, false>(R, E, T, F, steps, b, limit, bps, s);
    case 2: return ens_fused_n<Elastic, 3, 2, false>(R, E, T, F, steps, b, limit, bps, s);
    case 3: return ens_fused_n<Elastic, 3, 3, false>(R, E, T, F, steps, b, limit, bps, s);
    case 4: return ens_fused_n<Elastic, 3, 4, false>(R, E, T, F, steps, b, limit, bps, s);
    case 5: return ens_fused_n<Elastic, 3, 5, false>(R, E, T, F, steps, b, limit, bps, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace ader
