// Adjoint kernels of the elastic step (Picard and Cauchy-Kowalevski predictors), order 4
// (own translation unit to keep builds parallel).
#include "kernels_adjoint_ck_mixed.cuh"

namespace ader {
template <>
cudaError_t adj_run_n<4>(const StepArgs& a, const AdjArgs& j, const Tables& t, int blocks, cudaStream_t s) {
  return AdjLaunch<4>::run(a, j, t, blocks, s);
}
template <>
long long adj_scratch_n<4>(int iters) { return AdjLaunch<4>::scratch_per_block(iters); }
template <>
int adj_bps_n<4>() { return AdjLaunch<4>::blocks_per_sm(); }
template <>
cudaError_t adj_run_ck_n<4>(const StepArgs& a, const AdjArgs& j, const Tables& t, cudaStream_t s) {
  return AdjLaunchCK<4>::run(a, j, t, s);
}
template <>
cudaError_t adj_run_ck_mixed_n<4>(const StepArgs& a, const AdjArgs& j, const Tables& t,
                                  const TablesF& f, cudaStream_t s) {
  return AdjLaunchCKM<4>::run(a, j, t, f, s);
}
}  // namespace ader
