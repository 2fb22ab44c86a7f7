// Adjoint of the linear-elastic ADER-DG step (Sec. 3.3), for gradients of a receiver misfit.
//
// With a fixed dt the step is affine, u^{n+1} = A(m) u^n + b^n(M, m).  One adjoint step maps
// lambda^{n+1} -> lambda^n = A^T lambda^{n+1} (+ dJ/du^n) and accumulates the material gradient
// (per cell rho, lambda, mu) and the moment-tensor gradient.  The transposes are written by hand,
// in the reverse order of the forward kernels:
//   k_adj_riemann  one warp per face: adjoint of the corrector's face terms and of the
//                  path-conservative Rusanov fluctuation; material gradient of the wave speed
//                  s = max(vp_L, vp_R) (ties: left) and of the path-averaged matrix Bbar.
//   k_adj_cell     persistent blocks over the cells: recompute the Picard iterates of the forward
//                  predictor (kept in a per-block global scratch slab), then the adjoint of the
//                  volume term, of the face extrapolation, and of the Picard iteration in reverse.
// The forward face data q_bar of the step are recomputed by the forward predictor kernel first.
// With the Cauchy-Kowalevski predictor (kernels_adjoint_ck.cuh) k_adj_riemann runs in two halves
// around the cell kernel, which forms the forward face data itself.
#pragma once
#include "kernels.cuh"

namespace ader {

// Rows r of B_d whose single non-zero sits in column k (B_d^T has these entries in row k).
struct RowsT {
  signed char r[3][9][3];
};
__host__ __device__ constexpr RowsT make_rows() {
  RowsT t{};
  for (int d = 0; d < 3; ++d)
    for (int k = 0; k < 9; ++k) {
      int m = 0;
      for (int q = 0; q < 3; ++q) t.r[d][k][q] = -1;
      for (int r = 0; r < 9; ++r)
        if (Elastic::src(d, r) == k) t.r[d][k][m++] = (signed char)r;
    }
  return t;
}
static __constant__ RowsT c_rows = make_rows();

// d coef(d, v) / d (rho, lambda, mu)
__device__ __forceinline__ void dcoef(int d, int v, double rho, double* g) {
  g[0] = g[1] = g[2] = 0.0;
  if (v < 3) {
    g[0] = 1.0 / (rho * rho);
  } else if (v < 6) {
    g[1] = -1.0;
    g[2] = (v - 3 == d) ? -2.0 : 0.0;
  } else {
    g[2] = -1.0;
  }
}

// MODE 0: the whole face adjoint (the Picard form): lambda's face projections read from the
// cells' lambda, the forward face data from A.face.  The Cauchy-Kowalevski form splits it around
// its cell kernel, which produces the forward face data, and reads lambda's face projections from
// J.lproj (k_adj_proj): MODE 1 writes the face adjoints (they need lambda and the material only),
// MODE 2 forms the face material gradient from the projections and the forward face data.  In
// modes 1 and 2 every face record a warp needs is staged in shared memory by coalesced loads.
// DIR: the face normal (a template parameter, so that every row index of B_d is a constant).
template <int D, int N, int MODE, int DIR>
__global__ void __launch_bounds__(128) k_adj_riemann(const __grid_constant__ StepArgs A,
                                                     const __grid_constant__ AdjArgs J,
                                                     const __grid_constant__ Tables T,
                                                     long long gface_off) {
  constexpr int d = DIR;
  using C = Cfg<Elastic, 3, N>;
  constexpr int n = C::n, NV = 9, NF = C::NF, FR = C::FR, NL = C::NL;
  constexpr int PER = (NF + 31) / 32;
  // per warp: the projections of both sides (modes 1, 2) and the face data of both sides (mode 2)
  constexpr int NSTAGE = MODE == 0 ? 1 : (MODE == 1 ? 2 : 4);
  __shared__ double stage[4][NSTAGE][MODE == 0 ? 1 : FR];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const long long f = (long long)blockIdx.x * 4 + warp;
  const Geometry& g = A.g;
  const int nd = g.n[d];
  const long long nfaces = (long long)(nd + 1) * FaceIdx::ntrans(g, d);
  if (f >= nfaces) return;
  const int kf = (int)(f % (nd + 1));
  const long long tr = f / (nd + 1);
  const bool periodic = (g.bc[d][0] == BC_PERIODIC);
  double* gf = J.gface + (gface_off + f) * 6;
  if (periodic && kf == nd) {
    if (MODE != 1 && lane < 6) gf[lane] = 0.0;
    return;
  }
  long long cL = -1, cR = -1;
  if (kf > 0) cL = FaceIdx::cell_of(g, tr, d, kf - 1);
  else if (periodic) cL = FaceIdx::cell_of(g, tr, d, nd - 1);
  if (kf < nd) cR = FaceIdx::cell_of(g, tr, d, kf);
  else if (periodic) cR = FaceIdx::cell_of(g, tr, d, 0);
  if (MODE != 0) {
    // stage[0] / [1]: lambda's projection onto the face from the left cell (its right side) and
    // from the right cell (its left side); stage[2] / [3]: the forward face data of both sides
    double* sw = &stage[warp][0][0];
    for (int e = lane; e < FR; e += 32) {
      sw[e] = cL >= 0 ? J.lproj[((cL * 3 + d) * 2 + 1) * (long long)FR + e] : 0.0;
      sw[FR + e] = cR >= 0 ? J.lproj[((cR * 3 + d) * 2 + 0) * (long long)FR + e] : 0.0;
      if (MODE == 2) {
        sw[2 * FR + e] = cL >= 0 ? A.face[cL * (long long)(3 * 2 * FR) + (d * 2 + 1) * FR + e] : 0.0;
        sw[3 * FR + e] = cR >= 0 ? A.face[cR * (long long)(3 * 2 * FR) + (d * 2 + 0) * FR + e] : 0.0;
      }
    }
    __syncwarp();
  }
  const long long mcL = cL >= 0 ? cL : cR, mcR = cR >= 0 ? cR : cL;
  const double rL = A.mat[mcL * 3], lL = A.mat[mcL * 3 + 1], uL = A.mat[mcL * 3 + 2];
  const double rR = A.mat[mcR * 3], lR = A.mat[mcR * 3 + 1], uR = A.mat[mcR * 3 + 2];
  // the face's speed and path-averaged coefficients: from the per-face table when the material
  // has been set (the same values), else formed here; the speeds of both sides only where the
  // material gradient needs them (modes 0 and 2)
  const double* fm = A.fmat ? A.fmat + (gface_off + f) * FMAT : nullptr;
  double sL = 0.0, sR = 0.0, s = 0.0;
  bool left_max = true;
  if (MODE != 1 || !fm) {
    sL = Elastic::vp(rL, lL, uL);
    sR = Elastic::vp(rR, lR, uR);
    left_max = sL >= sR;
    s = left_max ? sL : sR;
  } else {
    s = fm[0];
  }
  double cb[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double acc = 0.0;
    if (fm) {
      acc = fm[1 + v];
    } else {
#pragma unroll
      for (int gq = 0; gq < 3; ++gq) {
        const double z = T.pz[gq];
        acc = fma(T.pw[gq], Elastic::coef(d, v, fma(z, rR - rL, rL), fma(z, lR - lL, lL), fma(z, uR - uL, uL)), acc);
      }
    }
    cb[v] = acc;
  }
  const double dt = A.dev->dt;
  const double dih = dt * A.g.inv_h[d];
  const int st = d == 0 ? 1 : (d == 1 ? n : n * n);
  double S1 = 0.0;   // sum over nodes and variables of dq (gL + gR)
  double S2[NV];     // per row v: sum over nodes of dq[src] (gL - gR)[v]
#pragma unroll
  for (int v = 0; v < NV; ++v) S2[v] = 0.0;
  double dqh[PER][NV];
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    const int jp = lane + 32 * r;
    if (jp >= NF) continue;
    const int jbase = (jp % st) + (jp / st) * st * n;
    double gL[NV], gR[NV], qL[NV], qR[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      if (MODE == 0) {
        double aL = 0.0, aR = 0.0;
        if (cL >= 0) {
          const double* lam = J.lam + cL * NL;
#pragma unroll
          for (int m = 0; m < n; ++m) aL = fma(T.c1[m], lam[(jbase + m * st) * NV + v], aL);
        }
        if (cR >= 0) {
          const double* lam = J.lam + cR * NL;
#pragma unroll
          for (int m = 0; m < n; ++m) aR = fma(T.c0[m], lam[(jbase + m * st) * NV + v], aR);
        }
        gL[v] = -dih * aL;
        gR[v] = dih * aR;
        qL[v] = cL >= 0 ? A.face[cL * (long long)(3 * 2 * FR) + (d * 2 + 1) * FR + jp * NV + v] : 0.0;
        qR[v] = cR >= 0 ? A.face[cR * (long long)(3 * 2 * FR) + (d * 2 + 0) * FR + jp * NV + v] : 0.0;
      } else {
        gL[v] = -dih * stage[warp][0][jp * NV + v];
        gR[v] = dih * stage[warp][1][jp * NV + v];
        if (MODE == 2) {
          qL[v] = stage[warp][NSTAGE == 4 ? 2 : 0][jp * NV + v];
          qR[v] = stage[warp][NSTAGE == 4 ? 3 : 0][jp * NV + v];
        }
      }
    }
    if (MODE != 2) {
      // adjoint of dq = qR - qL:  dqh = -s/2 (gL + gR) + 1/2 Bbar^T (gL - gR)
#pragma unroll
      for (int k = 0; k < NV; ++k) dqh[r][k] = -0.5 * s * (gL[k] + gR[k]);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const int sv = Elastic::src(d, v);
        if (sv >= 0) dqh[r][sv] += 0.5 * cb[v] * (gL[v] - gR[v]);
      }
      if (MODE == 0) {
        if (cL >= 0)
#pragma unroll
          for (int v = 0; v < NV; ++v) J.adjf[((cL * 3 + d) * 2 + 1) * (long long)FR + jp * NV + v] = -dqh[r][v];
        if (cR >= 0)
#pragma unroll
          for (int v = 0; v < NV; ++v) J.adjf[((cR * 3 + d) * 2 + 0) * (long long)FR + jp * NV + v] = dqh[r][v];
      }
    }
    if (MODE != 1) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const double dq = qR[v] - qL[v];
        S1 = fma(dq, gL[v] + gR[v], S1);
        const int sv = Elastic::src(d, v);
        if (sv >= 0) S2[v] = fma(qR[sv] - qL[sv], gL[v] - gR[v], S2[v]);
      }
    }
  }
  if (MODE == 1) {
    // the face adjoints through the staging area (coalesced stores to both cells' records)
    __syncwarp();
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      const int jp = lane + 32 * r;
      if (jp < NF)
#pragma unroll
        for (int v = 0; v < NV; ++v) stage[warp][0][jp * NV + v] = dqh[r][v];
    }
    __syncwarp();
    for (int e = lane; e < FR; e += 32) {
      const double x = stage[warp][0][e];
      if (cL >= 0) J.adjf[((cL * 3 + d) * 2 + 1) * (long long)FR + e] = -x;
      if (cR >= 0) J.adjf[((cR * 3 + d) * 2 + 0) * (long long)FR + e] = x;
    }
    return;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    S1 += __shfl_xor_sync(0xffffffffu, S1, o);
#pragma unroll
    for (int v = 0; v < NV; ++v) S2[v] += __shfl_xor_sync(0xffffffffu, S2[v], o);
  }
  // d/dm of  -1/2 s S1 + 1/2 sum_v cb[v] S2[v] (every lane holds S1 and S2 after the reduction):
  // lane q < 27 takes the term (v, gq) = (q / 3, q % 3) of the path average, lane 0 also the wave
  // speed; the six partial sums are then reduced over the warp
  double gLm[3] = {0.0, 0.0, 0.0}, gRm[3] = {0.0, 0.0, 0.0};
  if (lane == 0) {
    // wave speed: vp = sqrt((lam + 2 mu) / rho)
    const double sr = left_max ? rL : rR, sv = s;
    const double dv[3] = {-sv / (2.0 * sr), 1.0 / (2.0 * sr * sv), 1.0 / (sr * sv)};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (left_max) gLm[k] = -0.5 * S1 * dv[k];
      else gRm[k] = -0.5 * S1 * dv[k];
    }
  }
  if (lane < 27) {
    const int v = lane / 3, gq = lane % 3;
    if (Elastic::src(d, v) >= 0) {
      double s2 = 0.0;  // S2[v] selected without a dynamically indexed array
#pragma unroll
      for (int u = 0; u < NV; ++u)
        if (u == v) s2 = S2[u];
      const double z = T.pz[gq];
      const double rho = fma(z, rR - rL, rL);
      double dc[3];
      dcoef(d, v, rho, dc);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double w = 0.5 * s2 * T.pw[gq] * dc[k];
        gLm[k] = fma(w, 1.0 - z, gLm[k]);
        gRm[k] = fma(w, z, gRm[k]);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      gLm[k] += __shfl_xor_sync(0xffffffffu, gLm[k], o);
      gRm[k] += __shfl_xor_sync(0xffffffffu, gRm[k], o);
    }
  }
  if (lane == 0) {
    // ghost side: the exterior material is the interior one
    if (cL < 0) for (int k = 0; k < 3; ++k) { gRm[k] += gLm[k]; gLm[k] = 0.0; }
    if (cR < 0) for (int k = 0; k < 3; ++k) { gLm[k] += gRm[k]; gRm[k] = 0.0; }
    for (int k = 0; k < 3; ++k) {
      gf[k] = gLm[k];
      gf[3 + k] = gRm[k];
    }
  }
}

// lambda's projections onto the six faces of every cell (the transposes of the corrector's face
// terms before the face weights): J.lproj[c][d][0] = sum_m c0[m] lambda along the lines of
// direction d, [1] with c1; one block per cell (several at low order), lambda staged in shared
// memory by a coalesced load, stores coalesced.
template <int N>
struct CfgProj {
  static constexpr int NS = (N + 1) * (N + 1) * (N + 1);
  static constexpr int CPB = NS >= 96 ? 1 : 128 / NS;  // cells per block
  static constexpr int TPB = (CPB * NS + 31) / 32 * 32;
};

template <int N>
__global__ void __launch_bounds__(CfgProj<N>::TPB)
    k_adj_proj(const __grid_constant__ StepArgs A, const __grid_constant__ AdjArgs J,
               const __grid_constant__ Tables T) {
  constexpr int n = N + 1, NS = n * n * n, NV = 9, NL = NS * NV, NF = n * n, FR = NF * NV;
  constexpr int CPB = CfgProj<N>::CPB, TPB = CfgProj<N>::TPB;
  __shared__ double sl[CPB][NL];
  const long long c0 = (long long)blockIdx.x * CPB;
  const int ncb = (int)(A.g.ncells - c0 < CPB ? A.g.ncells - c0 : CPB);
  for (int e = threadIdx.x; e < ncb * NL; e += TPB) (&sl[0][0])[e] = J.lam[c0 * NL + e];
  __syncthreads();
  for (int e = threadIdx.x; e < ncb * 3 * FR; e += TPB) {
    const int s = e / (3 * FR), r = e - s * (3 * FR);
    const int d = r / FR, q = r - d * FR;
    const int jp = q / NV, v = q - jp * NV;
    const int st = d == 0 ? 1 : (d == 1 ? n : n * n);
    const int jbase = (jp % st) + (jp / st) * st * n;
    double a0 = 0.0, a1 = 0.0;
#pragma unroll
    for (int m = 0; m < n; ++m) {
      const double x = sl[s][(jbase + m * st) * NV + v];
      a0 = fma(T.c0[m], x, a0);
      a1 = fma(T.c1[m], x, a1);
    }
    double* o = J.lproj + ((c0 + s) * 3 + d) * 2 * (long long)FR + q;
    o[0] = a0;
    o[FR] = a1;
  }
}

template <int N>
cudaError_t launch_adj_proj(const StepArgs& a, const AdjArgs& j, const Tables& t, cudaStream_t s) {
  const long long blocks = (a.g.ncells + CfgProj<N>::CPB - 1) / CfgProj<N>::CPB;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  k_adj_proj<N><<<(unsigned)blocks, CfgProj<N>::TPB, 0, s>>>(a, j, t);
  return cudaGetLastError();
}

// The faces of direction d (one warp per face, 4 per block).
template <int N, int MODE>
cudaError_t launch_adj_riemann(const StepArgs& a, const AdjArgs& j, const Tables& t, int d,
                               long long gface_off, cudaStream_t s) {
  const long long nf = (long long)(a.g.n[d] + 1) * (a.g.ncells / a.g.n[d]);
  const unsigned grid = (unsigned)((nf + 3) / 4);
  if (d == 0) k_adj_riemann<3, N, MODE, 0><<<grid, 128, 0, s>>>(a, j, t, gface_off);
  else if (d == 1) k_adj_riemann<3, N, MODE, 1><<<grid, 128, 0, s>>>(a, j, t, gface_off);
  else k_adj_riemann<3, N, MODE, 2><<<grid, 128, 0, s>>>(a, j, t, gface_off);
  return cudaGetLastError();
}

template <int N>
struct CfgA {
  using C = Cfg<Elastic, 3, N>;
  static constexpr int n = C::n, NS = C::NS, NL = C::NL, NV = 9, NF = C::NF;
  static constexpr int TPB = C::TPB, LPT = C::LPT;
  static constexpr size_t SMEM = (size_t)2 * n * NL * sizeof(double);
};

// Per-cell adjoint; blocks loop over cells; scratch slab per block for the forward iterates.
template <int N>
__global__ void __launch_bounds__(Cfg<Elastic, 3, N>::TPB)
    k_adj_cell(const __grid_constant__ StepArgs A, const __grid_constant__ AdjArgs J,
               const __grid_constant__ Tables T, long long off1, long long off2) {
  using M = CfgA<N>;
  constexpr int n = M::n, NV = 9, NL = M::NL, TPB = M::TPB, LPT = M::LPT, NF = M::NF;
  extern __shared__ double sm[];
  double* Q = sm;            // [n][NL] forward iterate
  double* P = sm + n * NL;   // [n][NL] adjoint work (rho), also lambda / q_bar lines
  __shared__ double red[3 * 32 + 6 * 32];
  // D is indexed by per-lane rows and columns: staged in shared memory once per block
  __shared__ double sD[n * n];
  for (int i = threadIdx.x; i < n * n; i += TPB) sD[i] = T.D[i / n][i % n];
  __syncthreads();
  const double dt = A.dev->dt;
  const double tn = A.dev->t;
  double* slab = J.scratch + (long long)blockIdx.x * J.scratch_per_block;
  const int iters = A.iters;
  for (long long c = blockIdx.x; c < A.g.ncells; c += gridDim.x) {
    const double rho = A.mat[c * 3], irho = 1.0 / rho, lamc = A.mat[c * 3 + 1], mu = A.mat[c * 3 + 2];
    const bool has_src = (A.src.cell == c);
    double ric[n], ricbar = 0.0;
#pragma unroll
    for (int t = 0; t < n; ++t) {
      ric[t] = 0.0;
      if (has_src) {
        const double tau = fma(T.x[t], dt, tn) - A.src.t0;
        const double a = (M_PI * A.src.f0 * tau) * (M_PI * A.src.f0 * tau);
        ric[t] = (1.0 - 2.0 * a) * exp(-a);
      }
      ricbar = fma(T.w[t], ric[t], ricbar);
    }
    // ---- forward Picard iterates -----------------------------------------------------
    const double* u = J.u_n + c * NL;
    double ul[LPT];
#pragma unroll
    for (int k = 0; k < LPT; ++k) {
      const int l = threadIdx.x + k * TPB;
      ul[k] = l < NL ? u[l] : 0.0;
      if (l < NL)
#pragma unroll
        for (int t = 0; t < n; ++t) Q[t * NL + l] = ul[k];
    }
    __syncthreads();
    for (int it = 0; it < iters; ++it) {
      double R[LPT][n];
#pragma unroll
      for (int k = 0; k < LPT; ++k)
#pragma unroll
        for (int t = 0; t < n; ++t) R[k][t] = 0.0;
      contract_ncp_elastic<Cfg<Elastic, 3, N>, 0, n>(Q, sD, A.g.inv_h[0], irho, lamc, mu, R, threadIdx.x);
      contract_ncp_elastic<Cfg<Elastic, 3, N>, 1, n>(Q, sD, A.g.inv_h[1], irho, lamc, mu, R, threadIdx.x);
      contract_ncp_elastic<Cfg<Elastic, 3, N>, 2, n>(Q, sD, A.g.inv_h[2], irho, lamc, mu, R, threadIdx.x);
      if (has_src) {
#pragma unroll
        for (int k = 0; k < LPT; ++k) {
          const int l = threadIdx.x + k * TPB;
          if (l < NL && l % NV >= 3) {
            const double amp = -A.src.M[l % NV - 3] * A.src.phi[l / NV];
#pragma unroll
            for (int t = 0; t < n; ++t) R[k][t] = fma(amp, ric[t], R[k][t]);
          }
        }
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < LPT; ++k) {
        const int l = threadIdx.x + k * TPB;
        if (l < NL) {
#pragma unroll
          for (int t = 0; t < n; ++t) {
            double acc = 0.0;
#pragma unroll
            for (int m2 = 0; m2 < n; ++m2) acc = fma(T.Kw[t][m2], R[k][m2], acc);
            const double q = fma(dt, acc, ul[k]);
            Q[t * NL + l] = q;
            if (it + 1 < iters) slab[(long long)it * n * NL + t * NL + l] = q;  // q^{it+1}
          }
        }
      }
      __syncthreads();
    }
    // q_bar of the final iterate -> P[0..NL), lambda -> P[NL..2NL)
    double lam_l[LPT];
#pragma unroll
    for (int k = 0; k < LPT; ++k) {
      const int l = threadIdx.x + k * TPB;
      lam_l[k] = 0.0;
      if (l < NL) {
        double qb = 0.0;
#pragma unroll
        for (int t = 0; t < n; ++t) qb = fma(T.w[t], Q[t * NL + l], qb);
        P[l] = qb;
        lam_l[k] = J.lam[c * NL + l];
        P[NL + l] = lam_l[k];
      }
    }
    __syncthreads();
    double gm[3] = {0.0, 0.0, 0.0}, gM[6] = {0, 0, 0, 0, 0, 0};
    // ---- adjoint of the volume term dt (L q_bar + S_bar) ----------------------------------
    double qh[LPT][n];
#pragma unroll
    for (int k = 0; k < LPT; ++k) {
      const int l = threadIdx.x + k * TPB;
#pragma unroll
      for (int t = 0; t < n; ++t) qh[k][t] = 0.0;
      if (l >= NL) continue;
      const int j = l / NV, v = l % NV;
      double qbh = 0.0;  // adjoint of q_bar[j][v]
#pragma unroll 1
      for (int d = 0; d < 3; ++d) {
        const int st = d == 0 ? 1 : (d == 1 ? n : n * n);
        const int jd = (j / st) % n, j0 = j - jd * st;
        // material: lam[j][v] dt (-1/h) dcoef(d,v) (D_d q_bar)[j][src]
        const int s = Elastic::src(d, v);
        if (s >= 0) {
          double dq = 0.0;
#pragma unroll
          for (int m = 0; m < n; ++m) dq = fma(sD[jd * n + m], P[(j0 + m * st) * NV + s], dq);
          double dc[3];
          dcoef(d, v, rho, dc);
          const double w = lam_l[k] * dt * (-A.g.inv_h[d]) * dq;
          for (int q = 0; q < 3; ++q) gm[q] = fma(w, dc[q], gm[q]);
        }
        // (L^T lam)[j][v] = -(1/h) sum_{rows r with src(d,r) = v} coef(d,r) sum_i D[i][jd] lam[j(i)][r]
#pragma unroll 1
        for (int q = 0; q < 3; ++q) {
          const int r = c_rows.r[d][v][q];
          if (r < 0) break;
          double acc = 0.0;
#pragma unroll
          for (int i = 0; i < n; ++i) acc = fma(sD[i * n + jd], P[NL + (j0 + i * st) * NV + r], acc);
          qbh = fma(-dt * A.g.inv_h[d] * Elastic::coef_ir(d, r, irho, lamc, mu), acc, qbh);
        }
        // face extrapolations of q_bar along d
        const int jp = (j % st) + (j / (st * n)) * st;
        const double* af = J.adjf + (c * 3 + d) * 2 * (long long)(NF * NV);
        qbh = fma(T.e0[jd], af[jp * NV + v], qbh);
        qbh = fma(T.e1[jd], af[NF * NV + jp * NV + v], qbh);
      }
      if (has_src && v >= 3) gM[v - 3] += lam_l[k] * dt * ricbar * (-A.src.phi[j]);
#pragma unroll
      for (int t = 0; t < n; ++t) qh[k][t] = T.w[t] * qbh;  // q_bar = sum_t w_t q^I_t
    }
    __syncthreads();
    // ---- reverse Picard sweep ------------------------------------------------------------
    double uh[LPT];
#pragma unroll
    for (int k = 0; k < LPT; ++k) uh[k] = 0.0;
    for (int r = iters - 1; r >= 0; --r) {
      // q^r into Q (r = 0: 1 (x) u)
#pragma unroll
      for (int k = 0; k < LPT; ++k) {
        const int l = threadIdx.x + k * TPB;
        if (l < NL)
#pragma unroll
          for (int t = 0; t < n; ++t) Q[t * NL + l] = r == 0 ? ul[k] : slab[(long long)(r - 1) * n * NL + t * NL + l];
      }
      // rho = dt Kw^T qh ; uh += sum_t qh
      double rh[LPT][n];
#pragma unroll
      for (int k = 0; k < LPT; ++k) {
        const int l = threadIdx.x + k * TPB;
#pragma unroll
        for (int t = 0; t < n; ++t) {
          double acc = 0.0;
#pragma unroll
          for (int s2 = 0; s2 < n; ++s2) acc = fma(T.Kw[s2][t], qh[k][s2], acc);
          rh[k][t] = dt * acc;
          uh[k] += qh[k][t];
        }
        if (l < NL)
#pragma unroll
          for (int t = 0; t < n; ++t) P[t * NL + l] = rh[k][t];
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < LPT; ++k) {
        const int l = threadIdx.x + k * TPB;
#pragma unroll
        for (int t = 0; t < n; ++t) qh[k][t] = 0.0;
        if (l >= NL) continue;
        const int j = l / NV, v = l % NV;
#pragma unroll 1
        for (int d = 0; d < 3; ++d) {
          const int st = d == 0 ? 1 : (d == 1 ? n : n * n);
          const int jd = (j / st) % n, j0 = j - jd * st;
          const int s = Elastic::src(d, v);
          if (s >= 0) {  // material: rho[t][j][v] (-1/h) dcoef (D_d q^r)[t][j][s]
            double dc[3];
            dcoef(d, v, rho, dc);
            double acc = 0.0;
#pragma unroll
            for (int t = 0; t < n; ++t) {
              double dq = 0.0;
#pragma unroll
              for (int m = 0; m < n; ++m) dq = fma(sD[jd * n + m], Q[t * NL + (j0 + m * st) * NV + s], dq);
              acc = fma(rh[k][t], dq, acc);
            }
            const double w = -A.g.inv_h[d] * acc;
            for (int q = 0; q < 3; ++q) gm[q] = fma(w, dc[q], gm[q]);
          }
#pragma unroll 1
          for (int q = 0; q < 3; ++q) {
            const int rr = c_rows.r[d][v][q];
            if (rr < 0) break;
            const double cf = -A.g.inv_h[d] * Elastic::coef_ir(d, rr, irho, lamc, mu);
#pragma unroll
            for (int t = 0; t < n; ++t) {
              double acc = 0.0;
#pragma unroll
              for (int i = 0; i < n; ++i) acc = fma(sD[i * n + jd], P[t * NL + (j0 + i * st) * NV + rr], acc);
              qh[k][t] = fma(cf, acc, qh[k][t]);
            }
          }
        }
        if (has_src && v >= 3) {
          double acc = 0.0;
#pragma unroll
          for (int t = 0; t < n; ++t) acc = fma(rh[k][t], ric[t], acc);
          gM[v - 3] += acc * (-A.src.phi[j]);
        }
      }
      __syncthreads();
    }
    // q^0 = 1 (x) u
    bool bad = false;
#pragma unroll
    for (int k = 0; k < LPT; ++k) {
      const int l = threadIdx.x + k * TPB;
      if (l >= NL) continue;
#pragma unroll
      for (int t = 0; t < n; ++t) uh[k] += qh[k][t];
      double out = lam_l[k] + uh[k];
      if (J.dJdu) out += J.dJdu[c * NL + l];
      J.lam[c * NL + l] = out;
      bad |= !isfinite(out);
    }
    // a non-finite adjoint or gradient (e.g. from a non-finite forward state) is latched
    if (bad) atomicOr(&A.dev->status, ST_NONFINITE);
    // ---- reductions: material gradient (+ faces), moment tensor ----------------------------
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = TPB >> 5;
#pragma unroll
    for (int q = 0; q < 3; ++q)
      for (int o = 16; o > 0; o >>= 1) gm[q] += __shfl_xor_sync(0xffffffffu, gm[q], o);
    if (has_src)
#pragma unroll
      for (int q = 0; q < 6; ++q)
        for (int o = 16; o > 0; o >>= 1) gM[q] += __shfl_xor_sync(0xffffffffu, gM[q], o);
    if (lane == 0) {
      for (int q = 0; q < 3; ++q) red[q * 32 + warp] = gm[q];
      if (has_src) for (int q = 0; q < 6; ++q) red[96 + q * 32 + warp] = gM[q];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot[3];
      for (int q = 0; q < 3; ++q) {
        tot[q] = 0.0;
        for (int w = 0; w < nw; ++w) tot[q] += red[q * 32 + w];
      }
      // faces of this cell: left face (this cell is R) and right face (this cell is L)
      for (int d = 0; d < 3; ++d) {
        int id;
        const long long trc = FaceIdx::trans_of_cell(A.g, c, d, id);
        const int nd = A.g.n[d];
        int kr = id + 1;
        if (kr == nd && A.g.bc[d][1] == BC_PERIODIC) kr = 0;
        const long long off = d == 0 ? 0 : (d == 1 ? off1 : off2);
        const double* gl = J.gface + (off + id + (long long)(nd + 1) * trc) * 6;   // left face
        const double* gr = J.gface + (off + kr + (long long)(nd + 1) * trc) * 6;   // right face
        for (int q = 0; q < 3; ++q) tot[q] += gl[3 + q] + gr[q];
      }
      for (int q = 0; q < 3; ++q) J.grad_mat[c * 3 + q] += tot[q];
      if (!isfinite(tot[0]) || !isfinite(tot[1]) || !isfinite(tot[2]))
        atomicOr(&A.dev->status, ST_NONFINITE);
      if (has_src)
        for (int q = 0; q < 6; ++q) {
          double s = 0.0;
          for (int w = 0; w < nw; ++w) s += red[96 + q * 32 + w];
          J.grad_M[q] += s;
        }
    }
    __syncthreads();
  }
}

template <int N>
cudaError_t adj_run_n(const StepArgs& a, const AdjArgs& j, const Tables& t, int blocks, cudaStream_t s);
template <int N>
long long adj_scratch_n(int iters);
template <int N>
int adj_bps_n();

template <int N>
struct AdjLaunch {
  static cudaError_t run(const StepArgs& a, const AdjArgs& j, const Tables& t, int blocks,
                         cudaStream_t s) {
    using C = Cfg<Elastic, 3, N>;
    static bool attr = false;
    if (!attr) {
      cudaError_t e = cudaFuncSetAttribute(k_adj_cell<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)CfgA<N>::SMEM);
      if (e != cudaSuccess) return e;
      attr = true;
    }
    long long offs[3] = {0, 0, 0}, off = 0;
    for (int d = 0; d < 3; ++d) {
      offs[d] = off;
      off += (long long)(a.g.n[d] + 1) * (a.g.ncells / a.g.n[d]);
    }
    for (int d = 0; d < 3; ++d) {
      cudaError_t e = launch_adj_riemann<N, 0>(a, j, t, d, offs[d], s);
      if (e != cudaSuccess) return e;
    }
    k_adj_cell<N><<<blocks, C::TPB, CfgA<N>::SMEM, s>>>(a, j, t, offs[1], offs[2]);
    return cudaGetLastError();
  }
  static long long scratch_per_block(int iters) {
    using C = Cfg<Elastic, 3, N>;
    return (long long)(iters > 1 ? iters - 1 : 1) * C::n * C::NL;
  }
  static int blocks_per_sm() {
    cudaFuncSetAttribute(k_adj_cell<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CfgA<N>::SMEM);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_adj_cell<N>, Cfg<Elastic, 3, N>::TPB,
                                                  CfgA<N>::SMEM);
    return nb > 0 ? nb : 1;
  }
};

}  // namespace ader
