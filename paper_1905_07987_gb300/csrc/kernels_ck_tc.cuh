// Cauchy-Kowalevski predictor of the linear elastic system (Sec. 2, Sec. 3.3) with every
// contraction on the tensor cores (ADER_PREC_MIXED_TF32X3): the derivatives of the Taylor
// coefficients along each direction and the extrapolation of the time average to the faces are
// small dense products with the 1-D tables, batched over all lines of a cell,
//   Y[line][i] = sum_m X[line][m] B[i][m],   B rows: D[i][.] (i < n), e0, e1, zero padding,
// run as tcgen05.mma kind::tf32 (M = 128 lines per tile, N = 16, K = 8 >= n) with split operands:
// X = Xh + Xl and B = Bh + Bl (TF32 hi / lo parts), Y = Xh Bh + Xl Bh + Xh Bl accumulated in FP32
// in tensor memory (relative error about 2^-21 of sum_m |X_m| |B_im|: the dropped Xl Bl term and
// the FP32 accumulation).  The cell-constant material combination of the derivatives (the rows of
// B_d), the Taylor recursion a_{k+1} = dt/(k+1) (L a_k + g s_k) and the time average run in
// binary32 on the CUDA cores, and u^{n+1} = u^n + dt vol is formed in FP64.
//
// Data flow per cell (persistent blocks loop over the cells):
//   * the cell's FP64 state arrives in shared memory by a TMA tensor load (cp.async.bulk.tensor),
//     prefetched one cell ahead into a second buffer;
//   * per application of the spatial operator, every thread that owns a node writes its values,
//     split into TF32 hi / lo, into the K-major line matrices (lines of direction d: the six
//     variables its derivative reads); the application to the time average also extrapolates
//     those lines to the faces, and one more pass extrapolates the other three variables;
//   * one thread issues 3 MMAs per 128-line tile and commits them to an mbarrier;
//   * the line owners read their line's outputs from tensor memory (tcgen05.ld) and scatter the
//     derivatives to their nodes (and, last, the face values to the face records);
//   * the node owners combine the 18 derivatives with the material coefficients.
#pragma once
#include <cuda.h>
#include "ader_internal.h"
#include "ff.cuh"
#include "pde.cuh"
#include "tc.cuh"

namespace ader {

template <int N>
struct CfgCKT {
  static constexpr int n = N + 1;
  static constexpr int NS = n * n * n, NV = 9, NL = NS * NV, NF = n * n;
  static constexpr int TPB = 256;                       // 8 warps
  static constexpr int ROWS_L = 3 * 6 * NF;             // lines of an application of L
  static constexpr int ROWS_O = 3 * 3 * NF;             // lines of the other variables (faces)
  static constexpr int TILES_L = (ROWS_L + 127) / 128;
  static constexpr int TILES_O = (ROWS_O + 127) / 128;
  static constexpr int TCOLS_RAW = TILES_L * 16;
  static constexpr int TCOLS = TCOLS_RAW <= 32 ? 32 : (TCOLS_RAW <= 64 ? 64 : (TCOLS_RAW <= 128 ? 128 : 256));
  static constexpr int DVS = 18;                        // derivative slots per node
  // shared memory: A hi | A lo (TILES_L x 4 KB each) | B hi | B lo (1 KB each) | state x 2 | Dv
  static constexpr size_t OFF_AH = 0;
  static constexpr size_t OFF_AL = OFF_AH + (size_t)TILES_L * 4096;
  static constexpr size_t OFF_BH = OFF_AL + (size_t)TILES_L * 4096;
  static constexpr size_t OFF_BL = OFF_BH + 1024;
  static constexpr size_t OFF_ST = OFF_BL + 1024;
  static constexpr size_t ST_BYTES = ((size_t)NL * 8 + 127) / 128 * 128;
  static constexpr size_t OFF_DV = OFF_ST + 2 * ST_BYTES;
  static constexpr size_t SMEM = OFF_DV + (size_t)NS * DVS * 4 + 1024;  // + alignment slack
  static_assert(N % 2 == 1, "TMA box of the cell state needs an even number of nodes per direction");
  static_assert(TILES_O <= TILES_L, "the face pass reuses the operand tiles");
};

// Offset (floats) of element (row r, k) in a K-major line matrix with K = 8: core matrices of 8
// rows x 4 floats, 2 along K per group of 8 rows (group stride 256 bytes).  Lines of direction d
// are rows d * per * NF + q * NF + f (variable slot q, transverse node f fastest), so that the
// nodes of a warp, which differ in f, store into different row slots (fewer bank conflicts).
__device__ __forceinline__ int kmaj_off(int r, int k) {
  return (r >> 3) * 64 + (k >> 2) * 32 + (r & 7) * 4 + (k & 3);
}

// The six variables of direction d whose derivatives the rows of B_d read: v_x, v_y, v_z and
// sigma_{0d}, sigma_{1d}, sigma_{2d}.
__device__ __forceinline__ constexpr int ck_need(int d, int q) {
  return q < 3 ? q : Elastic::sig(q - 3, d);
}

// The three variables of direction d whose derivatives no row of B_d reads (their faces are
// extrapolated in a separate pass): the normal stresses other than sigma_dd and the shear stress
// without a d index.
__device__ __forceinline__ constexpr int ck_other(int d, int q) {
  return d == 0 ? (q == 0 ? 4 : (q == 1 ? 5 : 8))
                : (d == 1 ? (q == 0 ? 3 : (q == 1 ? 5 : 7)) : (q == 0 ? 3 : (q == 1 ? 4 : 6)));
}

// Transverse index of node j on the face of direction d (the face records' node order) and the
// node's position along d.
template <int n>
__device__ __forceinline__ int face_node(int j, int d, int& jd) {
  const int st = d == 0 ? 1 : (d == 1 ? n : n * n);
  jd = (j / st) % n;
  return (j % st) + (j / (st * n)) * st;
}

constexpr uint32_t CKT_WAIT = 1u << 20;  // polls of a bounded mbarrier wait

template <int N>
__global__ void __launch_bounds__(256, 2)
    k_predictor_ck_tc(const __grid_constant__ StepArgs A, const __grid_constant__ Tables T,
                      const __grid_constant__ CUtensorMap tmap) {
  using C = CfgCKT<N>;
  constexpr int n = C::n, NS = C::NS, NV = C::NV, NL = C::NL, NF = C::NF, TPB = C::TPB;
  constexpr int FR = NF * NV;  // doubles per face record (elastic: q only)
  extern __shared__ unsigned char smem_raw[];
  // 1024-byte alignment of the operand matrices
  unsigned char* sm = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float* AH = reinterpret_cast<float*>(sm + C::OFF_AH);
  float* AL = reinterpret_cast<float*>(sm + C::OFF_AL);
  float* BH = reinterpret_cast<float*>(sm + C::OFF_BH);
  float* BL = reinterpret_cast<float*>(sm + C::OFF_BL);
  float* Dv = reinterpret_cast<float*>(sm + C::OFF_DV);  // [18][NS] derivatives at the nodes
  __shared__ __align__(8) uint64_t bar_tma[2], bar_mma;
  __shared__ uint32_t s_tmem;
  __shared__ float s_cf[3][4];   // {1/(rho h_d), (lam + 2 mu)/h_d, lam/h_d, mu/h_d}
  __shared__ float s_sk[n + 1];  // Taylor coefficients of the wavelet's interpolant, its average

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long ncells = A.g.ncells;

  // ---- set-up: B tables (D rows, e0, e1; TF32 hi / lo), zero K padding of A, barriers, TMEM ----
  for (int e = tid; e < 16 * 8; e += TPB) {
    const int i = e / 8, m = e % 8;
    double b = 0.0;
    if (m < n) b = i < n ? T.D[i][m] : (i == n ? T.e0[m] : (i == n + 1 ? T.e1[m] : 0.0));
    const float h = tc::to_tf32((float)b);
    BH[kmaj_off(i, m)] = h;
    BL[kmaj_off(i, m)] = tc::to_tf32((float)(b - (double)h));
  }
  for (int e = tid; e < C::TILES_L * 128 * (8 - n); e += TPB) {
    const int r = e / (8 - n), k = n + e % (8 - n);
    AH[kmaj_off(r, k)] = 0.f;
    AL[kmaj_off(r, k)] = 0.f;
  }
  if (tid == 0) {
    tc::mbar_init(&bar_tma[0], 1);
    tc::mbar_init(&bar_tma[1], 1);
    tc::mbar_init(&bar_mma, 1);
    tc::mbar_fence_init();
  }
  if (warp == 0) tc::tmem_alloc(&s_tmem, C::TCOLS);
  tc::fence_async_smem();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t sAH = tc::smem_addr(AH), sAL = tc::smem_addr(AL);
  const uint64_t dBH = tc::sdesc_kmajor(tc::smem_addr(BH), 128, 256);
  const uint64_t dBL = tc::sdesc_kmajor(tc::smem_addr(BL), 128, 256);
  constexpr uint32_t IDESC = tc::idesc_tf32(128, 16);
  constexpr uint32_t CELL_BYTES = (uint32_t)NL * 8;

  // first cell's state
  long long c = blockIdx.x;
  bool pending[2] = {false, false};  // TMA loads issued and not yet waited for (thread 0)
  if (tid == 0 && c < ncells) {
    tc::mbar_arrive_expect_tx(&bar_tma[0], CELL_BYTES);
    tc::tma_load_3d(sm + C::OFF_ST, &tmap, 0, 0, (int)c, &bar_tma[0]);
    pending[0] = true;
  }
  uint32_t tma_phase[2] = {0u, 0u}, mma_phase = 0u;
  bool mma_pending = false, failed = false;
  const double dt = A.dev->dt;
  const double tn = A.dev->t;
  const float dtf = (float)dt;

  const bool node_owner = tid < NS;
  const int j = node_owner ? tid : 0;
  // loop-invariant staging positions of the owned node: first line row of each direction (six-
  // and three-variable line sets) and the K part of the offset (position along the direction)
  int rbl[3], kt[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    int jd;
    const int jp = face_node<n>(j, d, jd);
    rbl[d] = d * 6 * NF + jp;   // + q NF; the three-variable rows: rbl[d] - d 3 NF + q NF
    kt[d] = (jd >> 2) * 32 + (jd & 3);
  }
  // loop-invariant rows of the line owner (tiles t = warp / 4 + 2 i): the first node of the line
  // in Dv, its node stride, and its derivative slot
  constexpr int LR = (C::TILES_L + 1) / 2;
  int lrow_dv[LR], lrow_st[LR];
#pragma unroll
  for (int i = 0; i < LR; ++i) {
    const int r = ((warp >> 2) + 2 * i) * 128 + (warp & 3) * 32 + lane;
    lrow_dv[i] = -1;
    lrow_st[i] = 0;
    if (r < C::ROWS_L) {
      const int d = r / (6 * NF), rr = r - d * 6 * NF;
      const int q = rr / NF, f = rr - q * NF;
      const int st = d == 0 ? 1 : (d == 1 ? n : n * n);
      // Dv is slot-major ([slot][node], node fastest): the lines of a warp store to nearby nodes
      lrow_dv[i] = (d * 6 + q) * NS + (f % st) + (f / st) * st * n;
      lrow_st[i] = st;
    }
  }

  for (int it = 0; c < ncells; ++it, c += gridDim.x) {
    const int buf = it & 1;
    const double* ST = reinterpret_cast<const double*>(sm + C::OFF_ST + buf * C::ST_BYTES);
    // prefetch the next cell into the other buffer (its previous contents were read before the
    // last barrier of the previous cell)
    const long long cn = c + gridDim.x;
    if (tid == 0 && cn < ncells) {
      tc::mbar_arrive_expect_tx(&bar_tma[buf ^ 1], CELL_BYTES);
      tc::tma_load_3d(sm + C::OFF_ST + (buf ^ 1) * C::ST_BYTES, &tmap, 0, 0, (int)cn,
                      &bar_tma[buf ^ 1]);
      pending[buf ^ 1] = true;
    }
    // per-cell coefficients (one FP64 division per cell, by a thread other than the one that
    // issues the copies) and the point source
    if (tid == 32) {
      const double irho = 1.0 / A.mat[c * 3 + 0], lam = A.mat[c * 3 + 1], mu = A.mat[c * 3 + 2];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const double ih = A.g.inv_h[d];
        s_cf[d][0] = (float)(irho * ih);
        s_cf[d][1] = (float)((lam + 2.0 * mu) * ih);
        s_cf[d][2] = (float)(lam * ih);
        s_cf[d][3] = (float)(mu * ih);
      }
    }
    const bool srcc = (A.src.cell == c);  // uniform over the block
    float g[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (srcc) {
      if (tid == 0) {
        double ric[n], sbar = 0.0;
#pragma unroll
        for (int t = 0; t < n; ++t) {
          const double tau = fma(T.x[t], dt, tn) - A.src.t0;
          const double a = (M_PI * A.src.f0 * tau) * (M_PI * A.src.f0 * tau);
          ric[t] = (1.0 - 2.0 * a) * exp(-a);
          sbar = fma(T.w[t], ric[t], sbar);
        }
#pragma unroll
        for (int k = 0; k < n; ++k) {
          double s = 0.0;
#pragma unroll
          for (int t = 0; t < n; ++t) s = fma(T.Vi[k][t], ric[t], s);
          s_sk[k] = (float)s;
        }
        s_sk[n] = (float)sbar;
      }
      if (node_owner)
#pragma unroll
        for (int i = 0; i < 6; ++i) g[i] = (float)(-A.src.M[i] * A.src.phi[j]);
    }
    // wait for this cell's state: one thread polls the barrier, the block waits at bar.sync
    // (no issue slots taken from the other resident block)
    bool tma_ok = true;
    if (tid == 0) {
      tma_ok = tc::mbar_wait(&bar_tma[buf], tma_phase[buf], CKT_WAIT);
      pending[buf] = !tma_ok;
    }
    tma_phase[buf] ^= 1u;
    if (__syncthreads_or(!tma_ok)) {
      failed = true;
      break;
    }
    float a[NV], qb[NV];
    if (node_owner) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        a[v] = ff_split_int(ST[j * NV + v]).h;  // leading 24 bits, on the integer pipe
        qb[v] = a[v];
      }
    }

    // ---- applications: a_1 .. a_N (k < N); L qbar with the faces of its lines (k = N); the
    // faces of the other variables (k = N + 1) ----
#pragma unroll 1
    for (int k = 0; k <= N + 1; ++k) {
      const bool vol = (k == N), oth = (k == N + 1);
      // (1) the node's values into the line matrices, split into TF32 hi / lo
      if (node_owner) {
        const float* x = (vol || oth) ? qb : a;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          if (oth) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
              const int r = rbl[d] - d * 3 * NF + q * NF;
              const int o = (r >> 3) * 64 + (r & 7) * 4 + kt[d];
              const float xv = x[ck_other(d, q)];
              const float h = tc::to_tf32(xv);
              AH[o] = h;
              AL[o] = tc::to_tf32(xv - h);
            }
          } else {
#pragma unroll
            for (int q = 0; q < 6; ++q) {
              const int r = rbl[d] + q * NF;
              const int o = (r >> 3) * 64 + (r & 7) * 4 + kt[d];
              const float xv = x[ck_need(d, q)];
              const float h = tc::to_tf32(xv);
              AH[o] = h;
              AL[o] = tc::to_tf32(xv - h);
            }
          }
        }
      }
      tc::fence_async_smem();
      tc::tc_fence_before();
      __syncthreads();
      // (2) one thread issues the MMAs of every tile: hi x hi, lo x hi, hi x lo
      const int tiles = oth ? C::TILES_O : C::TILES_L;
      if (tid == 0) {
        tc::tc_fence_after();
        for (int t = 0; t < tiles; ++t) {
          const uint32_t d_tmem = tmem + (uint32_t)(t * 16);
          const uint64_t ah = tc::sdesc_kmajor(sAH + t * 4096, 128, 256);
          const uint64_t al = tc::sdesc_kmajor(sAL + t * 4096, 128, 256);
          tc::mma_tf32(d_tmem, ah, dBH, IDESC, 0u);
          tc::mma_tf32(d_tmem, al, dBH, IDESC, 1u);
          tc::mma_tf32(d_tmem, ah, dBL, IDESC, 1u);
        }
        tc::mma_commit(&bar_mma);
      }
      // the issuing thread waits for the MMAs; the block waits at bar.sync
      bool mma_ok = true;
      if (tid == 0) {
        mma_pending = true;
        mma_ok = tc::mbar_wait(&bar_mma, mma_phase, CKT_WAIT);
        if (mma_ok) mma_pending = false;
        tc::tc_fence_before();
      }
      if (__syncthreads_or(!mma_ok)) {
        failed = true;
        break;
      }
      mma_phase ^= 1u;
      tc::tc_fence_after();
      // (3) line owners: derivatives to the nodes, face values to the face records
      {
        const int quarter = warp & 3;
#pragma unroll
        for (int i = 0; i < LR; ++i) {
          const int t = (warp >> 2) + 2 * i;
          if (t >= tiles) break;
          float y[8];
          tc::tmem_ld8(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(t * 16), y);
          tc::tmem_wait_ld();
          const int r = t * 128 + quarter * 32 + lane;
          const int per = oth ? 3 : 6;
          if (!oth && lrow_dv[i] >= 0) {
#pragma unroll
            for (int m = 0; m < n; ++m) Dv[lrow_dv[i] + m * lrow_st[i]] = y[m];
          }
          if (r < (oth ? C::ROWS_O : C::ROWS_L)) {
            const int d = r / (per * NF), rr = r - d * per * NF;
            const int q = rr / NF, f = rr - q * NF;
            if (vol || oth) {
              const int v = oth ? ck_other(d, q) : ck_need(d, q);
              double* fc = A.face + c * (3 * 2 * FR) + (d * 2) * FR + f * NV + v;
              fc[0] = f2d_int(y[n]);
              fc[FR] = f2d_int(y[n + 1]);
            }
          }
        }
      }
      tc::tc_fence_before();
      __syncthreads();
      // (4) node owners: R = L x at the node (+ the source), next Taylor coefficient / volume term
      if (node_owner && !oth) {
        float R[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) R[v] = 0.f;
        float dd[18];
#pragma unroll
        for (int i = 0; i < 18; ++i) dd[i] = Dv[i * NS + j];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const float* dv = dd + d * 6;      // d/dx_d of v_0, v_1, v_2
          const float* ds = dd + d * 6 + 3;  // d/dx_d of sigma_{0d}, sigma_{1d}, sigma_{2d}
          const float c0 = s_cf[d][0], c1 = s_cf[d][1], c2 = s_cf[d][2], c3 = s_cf[d][3];
          R[0] = fmaf(c0, ds[0], R[0]);
          R[1] = fmaf(c0, ds[1], R[1]);
          R[2] = fmaf(c0, ds[2], R[2]);
#pragma unroll
          for (int i = 0; i < 3; ++i) R[3 + i] = fmaf(i == d ? c1 : c2, dv[d], R[3 + i]);
#pragma unroll
          for (int v = 6; v < 9; ++v) {
            const int s = Elastic::src(d, v);
            if (s >= 0) R[v] = fmaf(c3, dv[s], R[v]);
          }
        }
        if (!vol) {
          if (srcc) {
#pragma unroll
            for (int v = 3; v < NV; ++v) R[v] = fmaf(g[v - 3], s_sk[k], R[v]);
          }
          const float f = dtf * (1.0f / (k + 1));
          const float wk = 1.0f / (k + 2);
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            a[v] = f * R[v];
            qb[v] = fmaf(wk, a[v], qb[v]);
          }
        } else {
          if (srcc) {
#pragma unroll
            for (int v = 3; v < NV; ++v) R[v] = fmaf(g[v - 3], s_sk[n], R[v]);
          }
          // u^n again from this cell's buffer (the prefetch writes the other one)
          double* un = A.u_next + c * NL + j * NV;
#pragma unroll
          for (int v = 0; v < NV; ++v) un[v] = fma(dt, f2d_int(R[v]), ST[j * NV + v]);
        }
      }
      // no barrier here: the next staging writes only the line matrices (their MMAs are done),
      // and its barrier orders this step's reads of Dv before the next scatter into it
    }
    if (failed) break;
  }
  // ---- tear-down (bounded): after a wait that gave up, the MMAs and the prefetch still in
  // flight are waited for before the tensor memory is released and the block exits ----
  if (failed) {
    if (tid == 0) {
      atomicOr(&A.dev->status, ST_TIMEOUT);
      if (mma_pending) tc::mbar_wait(&bar_mma, mma_phase, CKT_WAIT);
      for (int b = 0; b < 2; ++b)
        if (pending[b]) tc::mbar_wait(&bar_tma[b], tma_phase[b], CKT_WAIT);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, C::TCOLS);
}

// Tensor map of the state as [cells][NL / 8][8] doubles, box = one cell.
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn tensor_map_encoder();

template <int N>
cudaError_t launch_predictor_ck_tc_n(const StepArgs& a, const Tables& t, cudaStream_t s) {
  using C = CfgCKT<N>;
  static int blocks_per_sm = 0;
  if (!blocks_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(k_predictor_ck_tc<N>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return e;
    // the whole unified L1 / shared memory as shared memory, so that two blocks fit per SM
    e = cudaFuncSetAttribute(k_predictor_ck_tc<N>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_predictor_ck_tc<N>, C::TPB, C::SMEM);
    if (e != cudaSuccess) return e;
    // tensor memory: every resident block holds TCOLS of the SM's 512 columns.  Two blocks per
    // SM are launched even where the occupancy query reports one: the blocks never wait for each
    // other, so extra blocks that are not resident simply start later
    const int cap = 512 / C::TCOLS;
    blocks_per_sm = nb < 2 ? 2 : nb;
    if (blocks_per_sm > cap) blocks_per_sm = cap;
  }
  EncodeTiledFn enc = tensor_map_encoder();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap map;
  const cuuint64_t dims[3] = {8, (cuuint64_t)(C::NL / 8), (cuuint64_t)a.g.ncells};
  const cuuint64_t strides[2] = {8 * sizeof(double), (cuuint64_t)C::NL * sizeof(double)};
  const cuuint32_t box[3] = {8, (cuuint32_t)(C::NL / 8), 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, (void*)a.u, dims, strides, box,
                         estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long grid = (long long)sms * blocks_per_sm;
  if (grid > a.g.ncells) grid = a.g.ncells;
  if (grid < 1) return cudaSuccess;
  k_predictor_ck_tc<N><<<(unsigned)grid, C::TPB, C::SMEM, s>>>(a, t, map);
  return cudaGetLastError();
}

}  // namespace ader
