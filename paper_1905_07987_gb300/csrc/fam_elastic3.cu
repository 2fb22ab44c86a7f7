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
cudaError_t ens_step_ck_elastic3(const StepArgs* R, const EnsTable& E, const Tables& T,
                                 const TablesF& F, int prec, int order, cudaStream_t s);
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

// The per-face material terms of the elastic Riemann solver (the wave speed max(vp_L, vp_R), ties
// left, and the 3-point path average of each row's coefficient of B_d), one thread per face, by
// the same operations as the per-step evaluation in riemann_face; a boundary face takes its
// interior cell's material on both sides.
__global__ void __launch_bounds__(256) k_face_material(const __grid_constant__ Geometry g,
                                                       const double* __restrict__ mat,
                                                       const __grid_constant__ Tables T,
                                                       double* __restrict__ out) {
  long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int d = 0;
  long long nf = (long long)(g.n[0] + 1) * FaceIdx::ntrans(g, 0);
  long long base = 0;
  while (d < 2 && f - base >= nf) {
    base += nf;
    ++d;
    nf = (long long)(g.n[d] + 1) * FaceIdx::ntrans(g, d);
  }
  if (f - base >= nf) return;
  const long long fl = f - base;
  const int nd = g.n[d];
  const int kf = (int)(fl % (nd + 1));
  const long long tr = fl / (nd + 1);
  const bool periodic = (g.bc[d][0] == BC_PERIODIC);
  long long cL = -1, cR = -1;
  if (kf > 0) cL = FaceIdx::cell_of(g, tr, d, kf - 1);
  else if (periodic) cL = FaceIdx::cell_of(g, tr, d, nd - 1);
  if (kf < nd) cR = FaceIdx::cell_of(g, tr, d, kf);
  else if (periodic) cR = FaceIdx::cell_of(g, tr, d, 0);
  const long long mcL = cL >= 0 ? cL : cR, mcR = cR >= 0 ? cR : cL;
  const double rL = mat[mcL * 3], lL = mat[mcL * 3 + 1], uL = mat[mcL * 3 + 2];
  const double rR = mat[mcR * 3], lR = mat[mcR * 3 + 1], uR = mat[mcR * 3 + 2];
  double ir[3];
  for (int gq = 0; gq < 3; ++gq) ir[gq] = 1.0 / fma(T.pz[gq], rR - rL, rL);
  const double sL = sqrt((lL + 2.0 * uL) / rL), sR = sqrt((lR + 2.0 * uR) / rR);
  out[f * FMAT] = (sL >= sR) ? sL : sR;
  for (int v = 0; v < 9; ++v) {
    const double bmu = v < 3 ? 0.0 : (v < 6 ? (v - 3 == d ? 2.0 : 0.0) : 1.0);
    double acc = 0.0;
    for (int gq = 0; gq < 3; ++gq) {
      const double z = T.pz[gq];
      const double lz = fma(z, lR - lL, lL), uz = fma(z, uR - uL, uL);
      const double cl = -((v >= 3 && v < 6 ? lz : 0.0) + bmu * uz);
      acc = fma(T.pw[gq], v < 3 ? -ir[gq] : cl, acc);
    }
    out[f * FMAT + 1 + v] = acc;
  }
}

cudaError_t launch_face_material_elastic(const Geometry& g, const double* mat, const Tables& t,
                                         double* out, cudaStream_t s) {
  long long nf = 0;
  for (int d = 0; d < 3; ++d) nf += (long long)(g.n[d] + 1) * (g.ncells / g.n[d]);
  if (nf <= 0) return cudaSuccess;
  k_face_material<<<(unsigned)((nf + 255) / 256), 256, 0, s>>>(g, mat, t, out);
  return cudaGetLastError();
}

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
    g.ens_step_ck = &ens_step_ck_elastic3;
    return g;
  }();
  return &f;
}
}  // namespace ader
