// Kernel family: linear elasticity in 3D, orders 1-6, with the adjoint step (orders 1-5).
#include "kernels_adjoint.cuh"

namespace ader {
namespace {
cudaError_t adj_run(const StepArgs& a, const AdjArgs& j, const Tables& t, int blocks, cudaStream_t s) {
  switch (a.g.order) {
    case 1: return AdjLaunch<1>::run(a, j, t, blocks, s);
    case 2: return AdjLaunch<2>::run(a, j, t, blocks, s);
    case 3: return AdjLaunch<3>::run(a, j, t, blocks, s);
    case 4: return AdjLaunch<4>::run(a, j, t, blocks, s);
    case 5: return AdjLaunch<5>::run(a, j, t, blocks, s);
  }
  return cudaErrorInvalidValue;
}
long long adj_scratch(int order, int iters) {
  switch (order) {
    case 1: return AdjLaunch<1>::scratch_per_block(iters);
    case 2: return AdjLaunch<2>::scratch_per_block(iters);
    case 3: return AdjLaunch<3>::scratch_per_block(iters);
    case 4: return AdjLaunch<4>::scratch_per_block(iters);
    case 5: return AdjLaunch<5>::scratch_per_block(iters);
  }
  return 0;
}
int adj_bps(int order) {
  switch (order) {
    case 1: return AdjLaunch<1>::blocks_per_sm();
    case 2: return AdjLaunch<2>::blocks_per_sm();
    case 3: return AdjLaunch<3>::blocks_per_sm();
    case 4: return AdjLaunch<4>::blocks_per_sm();
    case 5: return AdjLaunch<5>::blocks_per_sm();
  }
  return 0;
}
}  // namespace

const Family* family_elastic3() {
  static Family f = [] {
    Family g = *FamilyImpl<Elastic, 3>::get();
    g.adj_run = &adj_run;
    g.adj_scratch_per_block = &adj_scratch;
    g.adj_blocks_per_sm = &adj_bps;
    return g;
  }();
  return &f;
}
}  // namespace ader
