// Ensembles of uneven grids advanced together: one persistent launch per phase of the step for all
// runs.  The work of the runs is concatenated (cells for the predictor and the corrector, faces of
// one direction for the Riemann solver); each work item finds its run by binary search in the
// prefix offsets of the run table and is processed by the same device function as in the
// per-context kernels, with that run's step arguments (from device memory).  Blocks and warps
// loop over the concatenated items (grid sized by the SM count), so small runs share the GPU with
// large ones inside one launch.  No block waits for another.
#pragma once
#include "kernels.cuh"
#include "step_scalars.cuh"

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

namespace ader {

// ---- one persistent launch for whole steps ----------------------------------------------------
// Grid-wide barrier of a cooperative launch (every block resident): blocks arrive on a counter,
// the last one resets it and advances the generation; the others poll the generation at most
// `limit` times.  A wait that runs out returns false (the caller latches ST_TIMEOUT and leaves);
// the other blocks then run out at the same barrier, so no block waits forever.  The state is
// zeroed by the host before every launch.
struct GridBar {
  unsigned count;
  unsigned gen;
};

__device__ __forceinline__ bool grid_sync(GridBar* b, unsigned nblocks, long long limit) {
  __syncthreads();
  int ok = 1;
  if (threadIdx.x == 0) {
    volatile unsigned* vg = &b->gen;
    const unsigned g = *vg;
    __threadfence();
    if (atomicAdd(&b->count, 1u) == nblocks - 1) {
      b->count = 0;
      __threadfence();
      atomicAdd(&b->gen, 1u);
    } else {
      long long i = 0;
      while (*vg == g) {
        if (i++ >= limit) {
          ok = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
  }
  return __syncthreads_and(ok) != 0;
}

// `steps` steps of every run in one launch: per step the time-step finalisation, the predictor
// over the concatenated cells, the Riemann solver over the concatenated faces of all directions,
// the corrector over the concatenated degrees of freedom and the time advance, separated by
// grid-wide barriers.  Rsteps: the runs' step arguments of each step ([steps][nr]).
template <class P, int D, int N, bool MIXED>
__global__ void __launch_bounds__(EnsCfg<P, D, N, MIXED>::TPB, EnsCfg<P, D, N, MIXED>::MINB)
    k_ens_fused(const StepArgs* __restrict__ Rsteps, const __grid_constant__ EnsTable E,
                const __grid_constant__ Tables T, const __grid_constant__ TablesF F, int steps,
                GridBar* bar, long long limit) {
  using C = Cfg<P, D, N>;
  constexpr int n = N + 1, NL = C::NL, TPB = EnsCfg<P, D, N, MIXED>::TPB;
  extern __shared__ __align__(16) double fsm[];
  const unsigned nb = gridDim.x;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const long long ncell = E.cell0[E.nr];
  bool ok = true;
  for (int s = 0; s < steps && ok; ++s) {
    const StepArgs* R = Rsteps + (long long)s * E.nr;
    if (blockIdx.x == 0 && (int)threadIdx.x < E.nr) dt_finalize_one(R[threadIdx.x]);
    if (!(ok = grid_sync(bar, nb, limit))) break;
    for (long long it = blockIdx.x; it < ncell; it += nb) {
      const int r = ens_find(E.cell0, E.nr, it);
      if constexpr (MIXED) predictor_mixed_cell<P, D, N>(R[r], T, F, it - E.cell0[r]);
      else predictor_cell<P, D, N>(R[r], T, it - E.cell0[r]);
      __syncthreads();  // the next cell reuses the shared memory
    }
    if (!(ok = grid_sync(bar, nb, limit))) break;
    {
      const long long nf0 = E.face0[0][E.nr], nf1 = E.face0[1][E.nr];
      const long long nft = nf0 + nf1 + (D == 3 ? E.face0[2][E.nr] : 0);
      const long long wpb = TPB / 32;
      for (long long w = (long long)blockIdx.x * wpb + wib; w < nft; w += (long long)nb * wpb) {
        const int d = w < nf0 ? 0 : (w < nf0 + nf1 ? 1 : 2);
        const long long wd = w - (d == 0 ? 0 : (d == 1 ? nf0 : nf0 + nf1));
        const int r = ens_find(E.face0[d], E.nr, wd);  // the same for the whole warp
        riemann_face<P, D, N>(R[r], T, d, E.phioff[d][r], wd - E.face0[d][r], lane);
      }
    }
    if (!(ok = grid_sync(bar, nb, limit))) break;
    {
      // dt e0 / (w h_d), dt e1 / (w h_d) of every run, over the predictor's shared memory
      double (*sw)[2][3][n] = reinterpret_cast<double (*)[2][3][n]>(fsm);
      for (int i = threadIdx.x; i < E.nr * 2 * D * n; i += TPB) {
        const int r = i / (2 * D * n), k = (i / (D * n)) % 2, d = (i / n) % D, m = i % n;
        sw[r][k][d][m] = R[r].dev->dt * (k ? R[r].cw1[d][m] : R[r].cw0[d][m]);
      }
      __syncthreads();
      const long long total = ncell * NL;
      for (long long e = (long long)blockIdx.x * TPB + threadIdx.x; e < total; e += (long long)nb * TPB) {
        const int r = ens_find(E.cell0, E.nr, e / NL);
        corrector_dof<P, D, N>(R[r], sw[r], E.phioff[1][r], E.phioff[2][r], e - E.cell0[r] * NL);
      }
    }
    if (!(ok = grid_sync(bar, nb, limit))) break;
    if (blockIdx.x == 0 && (int)threadIdx.x < E.nr) advance_one(R[threadIdx.x].dev, 0);
    // the next step's finalisation (block 0, same threads) follows the advance in program order
  }
  if (!ok && threadIdx.x == 0)
    for (int r = 0; r < E.nr; ++r) atomicOr(&Rsteps[r].dev->status, ST_TIMEOUT);
}

// Launch `steps` steps of every run as one cooperative kernel (after zeroing the barrier).
template <class P, int D, int N, bool MIXED>
cudaError_t ens_fused_n(const StepArgs* R, const EnsTable& E, const Tables& T, const TablesF& F,
                        int steps, GridBar* bar, long long limit, int blocks_per_sm,
                        cudaStream_t s) {
  using G = EnsCfg<P, D, N, MIXED>;
  constexpr size_t SW = (size_t)ENS_MAXR * 2 * 3 * (N + 1) * sizeof(double);
  constexpr size_t SMEM = G::SMEM > SW ? G::SMEM : SW;
  static int max_bps = 0;
  if (!max_bps) {
    cudaError_t e = cudaFuncSetAttribute(k_ens_fused<P, D, N, MIXED>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
    if (e != cudaSuccess) return e;
    int nbk = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nbk, k_ens_fused<P, D, N, MIXED>, G::TPB, SMEM);
    if (e != cudaSuccess) return e;
    max_bps = nbk < 1 ? 1 : nbk;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int bps = blocks_per_sm < 1 ? 1 : (blocks_per_sm > max_bps ? max_bps : blocks_per_sm);
  cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(GridBar), s);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(sms * bps));
  cfg.blockDim = dim3(G::TPB);
  cfg.dynamicSmemBytes = SMEM;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_ens_fused<P, D, N, MIXED>, R, E, T, F, steps, bar, limit);
}

}  // namespace ader
