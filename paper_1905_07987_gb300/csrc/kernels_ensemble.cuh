// Ensembles of uneven grids advanced together: one persistent launch per phase of the step for all
// runs.  The work of the runs is concatenated (cells for the predictor and the corrector, faces of
// one direction for the Riemann solver); each work item finds its run by binary search in the
// prefix offsets of the run table and is processed by the same device function as in the
// per-context kernels, with that run's step arguments (from device memory).  Blocks and warps
// loop over the concatenated items (grid sized by the SM count), so small runs share the GPU with
// large ones inside one launch.  No block waits for another.
#pragma once
#include "kernels.cuh"

namespace ader {

// Largest r with off[r] <= item (off[0] = 0, off[nr] = total, item < total).
__device__ __forceinline__ int ens_find(const long long* off, int nr, long long item) {
  int lo = 0, hi = nr - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <class P, int D, int N, bool MIXED>
struct EnsCfg {
  static constexpr int TPB = MIXED ? CfgM<P, D, N>::TPB : Cfg<P, D, N>::TPB;
  static constexpr int MINB = MIXED ? CfgM<P, D, N>::MINB : 1;
  static constexpr size_t SMEM = MIXED ? CfgM<P, D, N>::SMEM : Cfg<P, D, N>::SMEM;
};

template <class P, int D, int N, bool MIXED>
__global__ void __launch_bounds__(EnsCfg<P, D, N, MIXED>::TPB, EnsCfg<P, D, N, MIXED>::MINB)
    k_ens_predictor(const StepArgs* __restrict__ R, const __grid_constant__ EnsTable E,
                    const __grid_constant__ Tables T, const __grid_constant__ TablesF F) {
  const long long total = E.cell0[E.nr];
  for (long long it = blockIdx.x; it < total; it += gridDim.x) {
    const int r = ens_find(E.cell0, E.nr, it);
    if constexpr (MIXED) predictor_mixed_cell<P, D, N>(R[r], T, F, it - E.cell0[r]);
    else predictor_cell<P, D, N>(R[r], T, it - E.cell0[r]);
    __syncthreads();  // the next cell reuses the shared memory
  }
}

template <class P, int D, int N>
__global__ void __launch_bounds__(128) k_ens_riemann(const StepArgs* __restrict__ R,
                                                     const __grid_constant__ EnsTable E,
                                                     const __grid_constant__ Tables T, int d) {
  const long long total = E.face0[d][E.nr];
  const int lane = threadIdx.x & 31;
  for (long long w = (long long)blockIdx.x * 4 + (threadIdx.x >> 5); w < total;
       w += (long long)gridDim.x * 4) {
    const int r = ens_find(E.face0[d], E.nr, w);  // the same for the whole warp
    riemann_face<P, D, N>(R[r], T, d, E.phioff[d][r], w - E.face0[d][r], lane);
  }
}

template <class P, int D, int N>
__global__ void __launch_bounds__(256) k_ens_corrector(const StepArgs* __restrict__ R,
                                                       const __grid_constant__ EnsTable E) {
  constexpr int n = N + 1, NL = Cfg<P, D, N>::NL;
  // dt e0 / (w h_d), dt e1 / (w h_d) of every run
  __shared__ double sw[ENS_MAXR][2][3][n];
  for (int i = threadIdx.x; i < E.nr * 2 * D * n; i += blockDim.x) {
    const int r = i / (2 * D * n), k = (i / (D * n)) % 2, d = (i / n) % D, m = i % n;
    sw[r][k][d][m] = R[r].dev->dt * (k ? R[r].cw1[d][m] : R[r].cw0[d][m]);
  }
  __syncthreads();
  const long long total = E.cell0[E.nr] * NL;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = ens_find(E.cell0, E.nr, e / NL);
    corrector_dof<P, D, N>(R[r], sw[r], E.phioff[1][r], E.phioff[2][r], e - E.cell0[r] * NL);
  }
}

// One step of every run: dt, predictor, Riemann per direction, corrector, time advance.
template <class P, int D, int N, bool MIXED>
cudaError_t ens_step_n(const StepArgs* R, const EnsTable& E, const Tables& T, const TablesF& F,
                       cudaStream_t s) {
  using G = EnsCfg<P, D, N, MIXED>;
  static bool attr = false;
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(k_ens_predictor<P, D, N, MIXED>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)G::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  cudaError_t e = launch_ens_dt(R, E.nr, s);
  if (e != cudaSuccess) return e;
  k_ens_predictor<P, D, N, MIXED><<<E.pblocks, G::TPB, G::SMEM, s>>>(R, E, T, F);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int d = 0; d < D; ++d) {
    k_ens_riemann<P, D, N><<<152 * 16, 128, 0, s>>>(R, E, T, d);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  k_ens_corrector<P, D, N><<<152 * 8, 256, 0, s>>>(R, E);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return launch_ens_advance(R, E.nr, s);
}

}  // namespace ader
