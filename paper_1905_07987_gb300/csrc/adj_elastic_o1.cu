// Adjoint kernels of the elastic step (Picard and Cauchy-Kowalevski predictors), order 1
// (own translation unit to keep builds parallel).
#include "kernels_adjoint_ck_mixed.cuh"

namespace ader {
template <>
cudaError_t adj_run_n<1>(const StepArgs& a, const AdjArgs& j, const Tables& t, int blocks, cudaStream_t s) {
  return AdjLaunch<1>::run(a, j, t, blocks, s);
}
template <>
long long adj_scratch_n<1>(int iters) { return AdjLaunch<1>::scratch_per_block(iters); }
template <>
int adj_bps_n<1>() { return AdjLaunch<1>::blocks_per_sm(); }
template <>
cudaError_t adj_run_ck_n<1>(const StepArgs& a, const AdjArgs& j, const Tables& t, cudaStream_t s) {
  return AdjLaunchCK<1>::run(a, j, t, s);
}
template <>
cudaError_t adj_run_ck_mixed_n<1>(const StepArgs& a, const AdjArgs& j, const Tables& t,
                                  const TablesF& f, cudaStream_t s) {
  return AdjLaunchCKM<1>::run(a, j, t, f, s);
}
}  // namespace ader
