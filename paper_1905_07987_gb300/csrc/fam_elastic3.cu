// Kernel family: linear elasticity in 3D, orders 1-6, with the adjoint step (orders 1-5, Picard
// and Cauchy-Kowalevski forms) and the Cauchy-Kowalevski predictor (orders 1-6).
#include "kernels.cuh"

namespace ader {
struct AdjArgs;
cudaError_t ens_step_elastic3_fp64(const StepArgs* R, const EnsTable& E, const Tables& T,
                                   const TablesF& F, int order, cudaStream_t s);
cudaError_t ens_step_elastic3_mixed(const StepArgs* R, const EnsTable& E, const Tables& T,
                                    const TablesF& F, int order, cudaStream_t s);
cudaError_t predictor_ck_elastic3(const StepArgs& a, const Tables& t, const TablesF& f, int prec,
                                  cudaStream_t s);
cudaError_t ens_fused_elastic3_fp64(const StepArgs* R, const EnsTable& E, const Tables& T,
                                    const TablesF& F, int order, int steps, void* bar,
                                    long long limit, int bps, cudaStream_t s);
cudaError_t ens_fused_elastic3_mixed(const StepArgs* R, const EnsTable& E, const Tables& T,
                                     const TablesF& F, int order, int steps, void* bar,
                                     long long limit, int bps, cudaStream_t s);
template <int N>
cudaError_t adj_run_n(const StepArgs& a, const AdjArgs& j, const Tables& t, int blocks, cudaStream_t s);
template <int N>
long long adj_scratch_n(int iters);
template <int N>
int adj_bps_n();
template <int N>
cudaError_t adj_run_ck_n(const StepArgs& a, const AdjArgs& j, const Tables& t, cudaStream_t s);
template <int N>
cudaError_t adj_run_ck_mixed_n(const StepArgs& a, const AdjArgs& j, const Tables& t,
                               const TablesF& f, cudaStream_t s);
namespace {
cudaError_t adj_run(const StepArgs& a, const AdjArgs& j, const Tables& t, int blocks, cudaStream_t s) {
  switch (a.g.order) {
    case 1: return adj_run_n<1>(a, j, t, blocks, s);
    case 2: return adj_run_n<2>(a, j, t, blocks, s);
    case 3: return adj_run_n<3>(a, j, t, blocks, s);
    case 4: return adj_run_n<4>(a, j, t, blocks, s);
    case 5: return adj_run_n<5>(a, j, t, blocks, s);
  }
  return cudaErrorInvalidValue;
}
// prec: 0 the FP64 adjoint; otherwise the mixed-precision one
cudaError_t adj_run_ck(const StepArgs& a, const AdjArgs& j, const Tables& t, const TablesF& f,
                       int prec, cudaStream_t s) {
  if (prec != 0) {
    switch (a.g.order) {
      case 1: return adj_run_ck_mixed_n<1>(a, j, t, f, s);
      case 2: return adj_run_ck_mixed_n<2>(a, j, t, f, s);
      case 3: return adj_run_ck_mixed_n<3>(a, j, t, f, s);
      case 4: return adj_run_ck_mixed_n<4>(a, j, t, f, s);
      case 5: return adj_run_ck_mixed_n<5>(a, j, t, f, s);
    }
    return cudaErrorInvalidValue;
  }
  switch (a.g.order) {
    case 1: return adj_run_ck_n<1>(a, j, t, s);
    case 2: return adj_run_ck_n<2>(a, j, t, s);
    case 3: return adj_run_ck_n<3>(a, j, t, s);
    case 4: return adj_run_ck_n<4>(a, j, t, s);
    case 5: return adj_run_ck_n<5>(a, j, t, s);
  }
  return cudaErrorInvalidValue;
}
long long adj_scratch(int order, int iters) {
  switch (order) {
    case 1: return adj_scratch_n<1>(iters);
    case 2: return adj_scratch_n<2>(iters);
    case 3: return adj_scratch_n<3>(iters);
    case 4: return adj_scratch_n<4>(iters);
    case 5: return adj_scratch_n<5>(iters);
  }
  return 0;
}
int adj_bps(int order) {
  switch (order) {
    case 1: return adj_bps_n<1>();
    case 2: return adj_bps_n<2>();
    case 3: return adj_bps_n<3>();
    case 4: return adj_bps_n<4>();
    case 5: return adj_bps_n<5>();
  }
  return 0;
}
cudaError_t ens_step(const StepArgs* R, const EnsTable& E, const Tables& T, const TablesF& F,
                     int prec, int order, cudaStream_t s) {
  if (order > 5) return cudaErrorInvalidValue;
  return prec == 1 ? ens_step_elastic3_mixed(R, E, T, F, order, s)
                   : ens_step_elastic3_fp64(R, E, T, F, order, s);
}
cudaError_t ens_fused(const StepArgs* R, const EnsTable& E, const Tables& T, const TablesF& F,
                      int prec, int order, int steps, void* bar, long long limit, int bps,
                      cudaStream_t s) {
  if (order > 5) return cudaErrorInvalidValue;
  return prec == 1 ? ens_fused_elastic3_mixed(R, E, T, F, order, steps, bar, limit, bps, s)
                   : ens_fused_elastic3_fp64(R, E, T, F, order, steps, bar, limit, bps, s);
}
}  // namespace

const Family* family_elastic3() {
  static Family f = [] {
    Family g = *FamilyImpl<Elastic, 3>::get();
    g.adj_run = &adj_run;
    g.adj_run_ck = &adj_run_ck;
    g.adj_scratch_per_block = &adj_scratch;
    g.adj_blocks_per_sm = &adj_bps;
    g.ens_step = &ens_step;
    g.predictor_ck = &predictor_ck_elastic3;
    g.ens_fused = &ens_fused;
    return g;
  }();
  return &f;
}
}  // namespace ader
