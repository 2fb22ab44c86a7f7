// Batched ensemble step of the 3-D elastic family with the Cauchy-Kowalevski predictor (FP64 and
// mixed precision), orders 4 and 5 (one cell per block): one launch per phase for all runs, as for
// the Picard predictor.  The predictor's blocks take the concatenated cells of the runs (one each)
// and call the per-context kernels' block function with the cell's run; the Riemann solver and
// the corrector are the ensemble's shared persistent kernels.  For these runs the per-run
// launches on forked streams are faster (74.9 against 87.3 ms per step of the 16-run ensemble);
// the autotuner chooses between them.
#include "kernels_ck.cuh"
#include "kernels_ensemble.cuh"

namespace ader {

template <int N, bool MIXED>
struct EnsCKCfg {
  static constexpr int TPB = MIXED ? CfgCKM<N>::TPB : CfgCK<N>::TPB;
  static constexpr int MINB = MIXED ? CfgCKM<N>::MINB : 1;
  static constexpr size_t SMEM = MIXED ? CfgCKM<N>::SMEM : CfgCK<N>::SMEM;
  static_assert((MIXED ? CfgCKM<N>::CPB : CfgCK<N>::CPB) == 1, "one cell per block");
};

template <int N, bool MIXED>
__global__ void __launch_bounds__(EnsCKCfg<N, MIXED>::TPB, EnsCKCfg<N, MIXED>::MINB)
    k_ens_predictor_ck(const StepArgs* __restrict__ R, const __grid_constant__ EnsTable E,
                       const __grid_constant__ Tables T, const __grid_constant__ TablesF F) {
  const long long total = E.cell0[E.nr];
  for (long long it = blockIdx.x; it < total; it += gridDim.x) {
    const int r = ens_find(E.cell0, E.nr, it);
    if constexpr (MIXED) predictor_ck_mixed_block<N>(R[r], T, F, it - E.cell0[r]);
    else predictor_ck_block<N>(R[r], T, it - E.cell0[r]);
    __syncthreads();  // the next cell reuses the shared memory
  }
}

template <int N, bool MIXED>
cudaError_t ens_step_ck_n(const StepArgs* R, const EnsTable& E, const Tables& T, const TablesF& F,
                          cudaStream_t s) {
  using G = EnsCKCfg<N, MIXED>;
  static bool attr = false;
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(k_ens_predictor_ck<N, MIXED>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)G::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  cudaError_t e = launch_ens_dt(R, E.nr, s);
  if (e != cudaSuccess) return e;
  // one block per cell of all runs (the block scheduler overlaps the cells' loads and work better
  // than resident blocks looping over cells)
  const long long total = E.cell0[E.nr];
  if (total > 0x7fffffffLL) return cudaErrorInvalidValue;
  const unsigned blocks = (unsigned)total;
  k_ens_predictor_ck<N, MIXED><<<blocks, G::TPB, G::SMEM, s>>>(R, E, T, F);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int d = 0; d < 3; ++d) {
    k_ens_riemann<Elastic, 3, N><<<152 * 16, 128, 0, s>>>(R, E, T, d);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  k_ens_corrector<Elastic, 3, N><<<152 * 8, 256, 0, s>>>(R, E);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return launch_ens_advance(R, E.nr, s);
}

// prec: 0 FP64, 1 mixed; orders 4 and 5
cudaError_t ens_step_ck_elastic3(const StepArgs* R, const EnsTable& E, const Tables& T,
                                 const TablesF& F, int prec, int order, cudaStream_t s) {
  if (prec == 1) {
    if (order == 4) return ens_step_ck_n<4, true>(R, E, T, F, s);
    if (order == 5) return ens_step_ck_n<5, true>(R, E, T, F, s);
  } else if (prec == 0) {
    if (order == 4) return ens_step_ck_n<4, false>(R, E, T, F, s);
    if (order == 5) return ens_step_ck_n<5, false>(R, E, T, F, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace ader
