// Mixed-precision space-time predictor (Eq. (5)): binary32 increments around float-float base terms.
//
// The predictor is solved for the increment dq = q - u^n, which is O(dt) small:
//   dq^{r+1} = dt Kw [ B0 + dR(dq^r) ],   B0 = R(u^n),   dR(dq) = R(u^n + dq) - R(u^n)
// B0 and every term that carries the O(1) size of the solution (the flux F(u^n), its derivative,
// the face extrapolations of u^n and F(u^n)) are formed in FP64 or in float-float (hi + lo pairs
// of binary32 with error-free transformations, about 44 significant bits) on the FP32 pipe.
// The Picard iterations, their flux increments F(u+dq) - F(u) (written so that no O(1) terms
// cancel), contractions and time solves run in plain binary32 -- each iteration damps the error
// of the previous one by the CFL-sized factor |dt Kw dR/dq|; the last contraction adds the lo
// parts of the tables.  The time average of the last iterate, qbar = sum_t w_t dq_t, is formed in
// float-float directly from the time-averaged solve weights, and every contraction of the
// epilogue runs in float-float, so that no binary32 rounding of the final predictor reaches the
// update.  The time-averaged flux increment is split exactly as
//   sum_t w_t [F(u + dq_t) - F(u)] = A(u) qbar + sum_t w_t N(dq_t),
// with A the flux Jacobian at u^n and N the quadratic remainder: the linear part in float-float
// once per spatial node, the O(dt^2) remainders in binary32 per space-time node.  The FP64 wave
// speeds of the face states (Euler) are evaluated here for the Riemann solver; the corrector,
// Riemann flux, CFL maximum and limiter stay FP64 (other kernels).
#pragma once
#include "kernels.cuh"
#include "ff.cuh"

namespace ader {

// Per-node base data of the Euler increments (float-float; the binary32 iterations use the hi parts).
template <int D>
struct EulerBase {
  ff rho, E, p, j[D], v[D];
};

template <class P, int D, int N>
struct CfgM {
  using C = Cfg<P, D, N>;
  static constexpr int n = C::n, NS = C::NS, NST = C::NST, NV = C::NV, NL = C::NL;
  static constexpr bool EULER = P::CONS && !P::LINEAR;
  // NL / LPD threads per block (about LPD lines per thread), rounded up to 64 threads for Euler
  // and to whole warps otherwise, from sweeps on GB300 (LPD in {2, 3, 4, 6, 8}; 128 to 320
  // threads at orders 3 and 4): Euler 128 threads at order 3 (NL / 3), 320 at order 4 (NL / 2,
  // 96 registers, 20 warps per SM); elastic NL / 6 at order 4, NL / 8 at order 5.
  static constexpr int LPD = EULER ? (N == 4 ? 2 : 3) : (N >= 5 ? 8 : 6);
  static constexpr int RND = EULER ? 64 : 32;
  static constexpr int TPB_E = ((NL + LPD - 1) / LPD + RND - 1) / RND * RND;
  static constexpr int TPB = TPB_E < 64 ? 64 : (TPB_E > 512 ? 512 : TPB_E);
  static constexpr int MINB = TPB <= 128 ? 3 : (TPB <= 320 ? 2 : 1);
  static constexpr int NF = C::NF, FR = C::FR;
  static constexpr int LPT = (NL + TPB - 1) / TPB, NPT = (NST + TPB - 1) / TPB;
  static constexpr int NPS = (NS + TPB - 1) / TPB;
  // v0[D], p0 (float-float) per spatial node; rows padded to an odd number of float-float values
  // so that the 8-byte loads of consecutive nodes fall on distinct banks
  static constexpr int BW = EULER ? ((D + 1) % 2 ? D + 1 : D + 2) : 1;
  static constexpr size_t B_FB0 = P::CONS ? (size_t)D * NL * sizeof(ff) : 0;
  static constexpr size_t B_UFF = (size_t)NL * sizeof(ff);
  static constexpr size_t B_BF = EULER ? (size_t)NS * BW * sizeof(ff) : 0;
  // rounded up to 16 bytes: the region behind it is also read as doubles
  static constexpr size_t B_DQ = ((size_t)n * NL * sizeof(float) + 15) / 16 * 16;
  static constexpr size_t B_F3 = P::CONS ? (size_t)D * n * NL * sizeof(float) : 0;
  static constexpr size_t SMEM = B_FB0 + B_UFF + B_BF + B_DQ + B_F3;
};

template <int D>
__device__ __forceinline__ EulerBase<D> load_base(const ff* uff, const ff* bff, int j) {
  constexpr int NV = D + 2, BW = (D + 1) % 2 ? D + 1 : D + 2;  // row length of bff
  EulerBase<D> b;
  b.rho = uff[j * NV];
  b.E = uff[j * NV + NV - 1];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    b.j[i] = uff[j * NV + 1 + i];
    b.v[i] = bff[j * BW + i];
  }
  b.p = bff[j * BW + D];
  return b;
}

// Flux increments F_d(u + dq) - F_d(u), d = 0..D-1, of the Euler equations in binary32 (hi parts
// of the base), the velocity and pressure increments computed once per node:
//   dv = (dj - v0 drho) / (rho0 + drho),  dp = (gamma-1)(dE - (dj.(v0+dv) + j0.dv)/2),
//   dF = (dj_d, dj (v0_d+dv_d) + j0 dv_d + dp e_d, (dE+dp)(v0_d+dv_d) + (E0+p0) dv_d).
template <int D>
__device__ __forceinline__ void dflux_f_all(const EulerBase<D>& b, const float* dq, float g1h,
                                            float g1l, float (*F)[D + 2]) {
  constexpr int NV = D + 2;
  const float irq = __fdividef(1.0f, b.rho.h + dq[0]);
  float dv[D], djv = 0.f;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    dv[i] = (dq[1 + i] - b.v[i].h * dq[0]) * irq;
    djv = fmaf(dq[1 + i], b.v[i].h + dv[i], fmaf(b.j[i].h, dv[i], djv));
  }
  const float x = dq[NV - 1] - 0.5f * djv;
  const float dp = fmaf(g1h, x, g1l * x);
  const float ep = b.E.h + b.p.h;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const float vd = b.v[d].h + dv[d];
    F[d][0] = dq[1 + d];
#pragma unroll
    for (int i = 0; i < D; ++i) F[d][1 + i] = fmaf(dq[1 + i], vd, b.j[i].h * dv[d]);
    F[d][1 + d] += dp;
    F[d][NV - 1] = fmaf(dq[NV - 1] + dp, vd, ep * dv[d]);
  }
}

// binary32 increments of every direction at the owned space-time nodes: dF3[d][t][NL].
template <class M, class P, int D>
__device__ __forceinline__ void dflux_nodes_all(const float* dqs, const ff* uff, const ff* bff,
                                                const PdeParams& pp, float g1h, float g1l,
                                                float* dF3, int tid) {
  constexpr int NV = M::NV, NS = M::NS, NSL = M::NST * NV;
#pragma unroll
  for (int k = 0; k < M::NPT; ++k) {
    const int node = tid + k * M::TPB;
    if (node < M::NST) {
      float q[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) q[v] = dqs[node * NV + v];
      float F[D][NV];
      if constexpr (M::EULER) {
        dflux_f_all<D>(load_base<D>(uff, bff, node % NS), q, g1h, g1l, F);
      } else {
#pragma unroll
        for (int d = 0; d < D; ++d) F[d][0] = (float)pp.a[d] * q[0];
      }
#pragma unroll
      for (int d = 0; d < D; ++d)
#pragma unroll
        for (int v = 0; v < NV; ++v) dF3[d * NSL + node * NV + v] = F[d][v];
    }
  }
}

// Quadratic remainders of the Euler flux increments, N_d(dq) = F_d(u + dq) - F_d(u) - A_d(u) dq,
// at the owned space-time nodes in binary32 (they are O(dt^2)).  With rho_t = rho0 + drho,
// dv = (dj - v0 drho) / rho_t and dp the exact pressure increment:
//   momentum i: rho_t dv_i dv_d + [i = d] N_p,   N_p = -(gamma-1)/2 rho_t |dv|^2,
//   energy:     N_p v0_d - (E0 + p0) dv_d drho / rho0 + (dE + dp) dv_d,   density: 0.
// NB[d][t][NL].
template <class M, int D>
__device__ __forceinline__ void remainder_nodes(const float* dqs, const ff* uff, const ff* bff,
                                                float g1h, float g1l, float* NB, int tid) {
  constexpr int NV = M::NV, NS = M::NS, NSL = M::NST * NV;
#pragma unroll
  for (int k = 0; k < M::NPT; ++k) {
    const int node = tid + k * M::TPB;
    if (node < M::NST) {
      float q[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) q[v] = dqs[node * NV + v];
      const EulerBase<D> b = load_base<D>(uff, bff, node % NS);
      const float rt = b.rho.h + q[0];
      const float irt = __fdividef(1.0f, rt);
      float dv[D], dv2 = 0.f, djv = 0.f;
#pragma unroll
      for (int i = 0; i < D; ++i) {
        dv[i] = (q[1 + i] - b.v[i].h * q[0]) * irt;
        dv2 = fmaf(dv[i], dv[i], dv2);
        djv = fmaf(q[1 + i], b.v[i].h + dv[i], fmaf(b.j[i].h, dv[i], djv));
      }
      const float x = q[NV - 1] - 0.5f * djv;
      const float dp = fmaf(g1h, x, g1l * x);
      const float np = -0.5f * g1h * rt * dv2;
      const float er = (b.E.h + b.p.h) * q[0] * __fdividef(1.0f, b.rho.h);
      const float ed = q[NV - 1] + dp;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        float* o = NB + d * NSL + node * NV;
        o[0] = 0.f;
        const float rdv = rt * dv[d];
#pragma unroll
        for (int i = 0; i < D; ++i) o[1 + i] = rdv * dv[i] + (i == d ? np : 0.f);
        o[NV - 1] = fmaf(np, b.v[d].h, (ed - er) * dv[d]);
      }
    }
  }
}

// Linear part of the time-averaged flux increments, A_d(u^n) qbar, at the owned spatial nodes in
// float-float (qbar: time average of dq), added to G_d = FB0 over h_d:
//   dv = (jbar - v0 rhobar) / rho0,  dp = (gamma-1)(Ebar - (v0.jbar + j0.dv)/2),
//   A_d qbar = (jbar_d, jbar v0_d + j0 dv_d + dp e_d, (Ebar + dp) v0_d + (E0 + p0) dv_d);
// linear fluxes (advection): a_d qbar.
template <class M, class P, int D>
__device__ __forceinline__ void linear_nodes(const float* qbh, const float* qbl, const ff* uff,
                                             const ff* bff, ff g1, const TablesF& F,
                                             const PdeParams& pp, ff* G, int tid) {
  constexpr int NV = M::NV, NS = M::NS, NL = M::NL;
#pragma unroll
  for (int k = 0; k < M::NPS; ++k) {
    const int j = tid + k * M::TPB;
    if (j < NS) {
      ff qb[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) qb[v] = {qbh[j * NV + v], qbl[j * NV + v]};
      if constexpr (M::EULER) {
        const EulerBase<D> b = load_base<D>(uff, bff, j);
        const ff ir = ff_div({1.f, 0.f}, b.rho);
        ff dv[D], jv = {0.f, 0.f};
#pragma unroll
        for (int i = 0; i < D; ++i) {
          dv[i] = ff_mul(ff_sub(qb[1 + i], ff_mul(b.v[i], qb[0])), ir);
          jv = ff_add(jv, ff_add(ff_mul(qb[1 + i], b.v[i]), ff_mul(b.j[i], dv[i])));
        }
        const ff dp = ff_mul(g1, ff_sub(qb[NV - 1], ff_mulf(jv, 0.5f)));
        const ff ep = ff_add(b.E, b.p);
        const ff ed = ff_add(qb[NV - 1], dp);
#pragma unroll
        for (int d = 0; d < D; ++d) {
          ff Fl[NV];
          Fl[0] = qb[1 + d];
#pragma unroll
          for (int i = 0; i < D; ++i) Fl[1 + i] = ff_add(ff_mul(qb[1 + i], b.v[d]), ff_mul(b.j[i], dv[d]));
          Fl[1 + d] = ff_add(Fl[1 + d], dp);
          Fl[NV - 1] = ff_add(ff_mul(ed, b.v[d]), ff_mul(ep, dv[d]));
          const ff ih = {F.ihh[d], F.ihl[d]};
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            ff* g = G + d * NL + j * NV + v;
            *g = ff_add(*g, ff_mul(Fl[v], ih));
          }
        }
      } else {
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const double a = pp.a[d];
          const float ah = (float)a;
          ff* g = G + d * NL + j * NV;
          *g = ff_add(*g, ff_mul(ff_mul(qb[0], {ah, (float)(a - (double)ah)}), {F.ihh[d], F.ihl[d]}));
        }
      }
    }
  }
}

// R[k][t] += cf[d][v] * sum_m D[j_d][m] X[t][(j, j_d -> m)][src]  in binary32 (D as n x n rows
// in shared memory, hi parts alone and as (hi, lo) pairs: the row index differs between the lanes
// of a warp), with the per-cell
// coefficients cf = {hi[3][NV], lo[3][NV]} in shared memory; with LO the lo parts of the
// coefficient and of the float-float derivative matrix are added (no rounding of fixed tables).
template <class M, int d, bool NCP, bool LO = false>
__device__ __forceinline__ void contract_f(const float* X, const float* Dh, const float2* D2,
                                           const float* cf, float (&R)[M::LPT][M::n], int tid) {
  constexpr int n = M::n, NV = M::NV, NL = M::NL, TPB = M::TPB, st = ipow(n, d);
#pragma unroll
  for (int k = 0; k < M::LPT; ++k) {
    const int l = tid + k * TPB;
    if (l < NL) {
      const int j = l / NV, v = l - (l / NV) * NV;
      int s = v;
      if constexpr (NCP) {
        s = Elastic::src(d, v);
        if (s < 0) continue;
      }
      const float c = cf[d * NV + v], clo = cf[3 * NV + d * NV + v];
      const int jd = digit<n, d>(j);
      const int j0 = j - jd * st;
#pragma unroll
      for (int t = 0; t < n; ++t) {
        float acc = 0.f, lo = 0.f;
#pragma unroll
        for (int m = 0; m < n; ++m) {
          const float x = X[t * NL + (j0 + m * st) * NV + s];
          if constexpr (LO) {
            const float2 dm = D2[jd * n + m];
            acc = fmaf(dm.x, x, acc);
            lo = fmaf(dm.y, x, lo);
          } else {
            acc = fmaf(Dh[jd * n + m], x, acc);
          }
        }
        const float x = acc + lo;
        R[k][t] = fmaf(c, x, LO ? fmaf(clo, x, R[k][t]) : R[k][t]);
      }
    }
  }
}

// Flux increments F_d(u + s) - F_d(u) of every direction at the spatial nodes, for one state
// increment s [NL] (a Runge-Kutta stage of the initial guess), into dF1 [D][NL] (binary32).
template <class M, class P, int D>
__device__ __forceinline__ void dflux_level(const float* sq, const ff* uff, const ff* bff,
                                            const PdeParams& pp, float g1h, float g1l, float* dF1,
                                            int tid) {
  constexpr int NV = M::NV, NS = M::NS, NL = M::NL;
#pragma unroll
  for (int k = 0; k < M::NPS; ++k) {
    const int node = tid + k * M::TPB;
    if (node < NS) {
      float q[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) q[v] = sq[node * NV + v];
      float F[D][NV];
      if constexpr (M::EULER) {
        dflux_f_all<D>(load_base<D>(uff, bff, node), q, g1h, g1l, F);
      } else {
#pragma unroll
        for (int d = 0; d < D; ++d) F[d][0] = (float)pp.a[d] * q[0];
      }
#pragma unroll
      for (int d = 0; d < D; ++d)
#pragma unroll
        for (int v = 0; v < NV; ++v) dF1[d * NL + node * NV + v] = F[d][v];
    }
  }
}

// One time level of contract_f: r[k] += cf[d][v] * sum_m D[j_d][m] X[(j, j_d -> m)][src] (binary32).
template <class M, int d, bool NCP>
__device__ __forceinline__ void contract_level(const float* X, const float* Dh, const float* cf,
                                               float (&r)[M::LPT], int tid) {
  constexpr int n = M::n, NV = M::NV, NL = M::NL, TPB = M::TPB, st = ipow(n, d);
#pragma unroll
  for (int k = 0; k < M::LPT; ++k) {
    const int l = tid + k * TPB;
    if (l < NL) {
      const int j = l / NV, v = l - (l / NV) * NV;
      int s = v;
      if constexpr (NCP) {
        s = Elastic::src(d, v);
        if (s < 0) continue;
      }
      const int jd = digit<n, d>(j);
      const int j0 = j - jd * st;
      float acc = 0.f;
#pragma unroll
      for (int m = 0; m < n; ++m) acc = fmaf(Dh[jd * n + m], X[(j0 + m * st) * NV + s], acc);
      r[k] = fmaf(cf[d * NV + v], acc, r[k]);
    }
  }
}

// One cell c (all threads of the block; called by the per-context kernel and by the persistent
// ensemble kernel).
template <class P, int D, int N>
__device__ __forceinline__ void predictor_mixed_cell(const StepArgs& A, const Tables& T,
                                                     const TablesF& F, long long c) {
  using M = CfgM<P, D, N>;
  constexpr int n = M::n, NS = M::NS, NV = M::NV, NL = M::NL, TPB = M::TPB, LPT = M::LPT;
  constexpr int NF = M::NF, FR = M::FR;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* p = smem_raw;
  ff* FB0 = reinterpret_cast<ff*>(p);  p += M::B_FB0;    // [D][NL] F_d(u)/h_d
  ff* uff = reinterpret_cast<ff*>(p);  p += M::B_UFF;    // [NL] u
  ff* bff = reinterpret_cast<ff*>(p);  p += M::B_BF;     // [NS][BW] v0, p0 (Euler)
  float* dqs = reinterpret_cast<float*>(p);  p += M::B_DQ;  // [n][NL] dq (binary32)
  // [D][n][NL] binary32: flux increments in the iterations, quadratic flux remainders in the
  // epilogue
  float* dF3 = reinterpret_cast<float*>(p);
  constexpr int NSL = n * NL;
  const int tid = threadIdx.x;
  const double dt = A.dev->dt;
  const float dtf = (float)dt;
  const ff dtff = {dtf, (float)(dt - (double)dtf)};
  const double tn = A.dev->t;
  const double* u = A.u + c * NL;
  const ff g1 = {F.g1h, F.g1l};

  double irho = 0.0, lam = 0.0, mu = 0.0;
  if constexpr (P::NCP) {
    irho = 1.0 / A.mat[c * 3 + 0];
    lam = A.mat[c * 3 + 1];
    mu = A.mat[c * 3 + 2];
  }
  // per-cell contraction coefficients: -1/h_d, or -coef(d,v)/h_d for the rows of B_d, as
  // (hi, lo) binary32 pairs
  __shared__ float cf[2 * 3 * NV];
  // tables indexed by a per-lane row (j_d, face side) staged in shared memory
  // (hi, lo) pairs interleaved: one 8-byte load per entry in the float-float contractions
  __shared__ float sDh[n * n], sE[4][n];
  __shared__ float2 sD2[n * n], sW2[n * n];
  for (int i = tid; i < n * n; i += TPB) {
    const int a = i / n, b = i - (i / n) * n;
    sDh[i] = F.Dh[a][b];
    sD2[i] = make_float2(F.Dh[a][b], F.Dl[a][b]);
    sW2[i] = make_float2(F.Wh[a][b], F.Wl[a][b]);
  }
  if (tid < n) {
    sE[0][tid] = F.e0h[tid];
    sE[1][tid] = F.e0l[tid];
    sE[2][tid] = F.e1h[tid];
    sE[3][tid] = F.e1l[tid];
  }
  if (tid < 3 * NV) {
    const int d = tid / NV, v = tid % NV;
    double cd = d < D ? -A.g.inv_h[d] : 0.0;
    if constexpr (P::NCP) cd = -Elastic::coef_ir(d, v, irho, lam, mu) * A.g.inv_h[d];
    const float h = (float)cd;
    cf[tid] = h;
    cf[3 * NV + tid] = (float)(cd - (double)h);
  }
  // point sources exist for the elastic system only (rejected at ader_set_point_source for the
  // others): compiled out of the conservative systems' kernels
  const bool has_src = P::NCP && (A.src.cell == c);
  double ric[n];
#pragma unroll
  for (int t = 0; t < n; ++t) ric[t] = 0.0;
  if (has_src) {
#pragma unroll
    for (int t = 0; t < n; ++t) {
      const double tau = fma(T.x[t], dt, tn) - A.src.t0;
      const double a = (M_PI * A.src.f0 * tau) * (M_PI * A.src.f0 * tau);
      ric[t] = (1.0 - 2.0 * a) * exp(-a);
    }
  }

  // ---- phase 0: base terms at the spatial nodes (FP64 -> float-float) --------------------
  double ul[LPT];
#pragma unroll
  for (int k = 0; k < LPT; ++k) {
    const int l = tid + k * TPB;
    ul[k] = 0.0;
    if (l < NL) {
      ul[k] = u[l];
      uff[l] = ff_split(ul[k]);
    }
  }
  __syncthreads();  // uff complete
  if constexpr (P::CONS) {
    // flux of u^n at the spatial nodes in float-float (scaled by 1/h_d): 1/rho, v, p, F_d
#pragma unroll
    for (int k = 0; k < M::NPS; ++k) {
      const int j = tid + k * TPB;
      if (j < NS) {
        ff q[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) q[v] = uff[j * NV + v];
        if constexpr (M::EULER) {
          const ff ir = ff_div({1.f, 0.f}, q[0]);
          ff vel[D], jv = {0.f, 0.f};
#pragma unroll
          for (int i = 0; i < D; ++i) {
            vel[i] = ff_mul(q[1 + i], ir);
            jv = ff_add(jv, ff_mul(q[1 + i], vel[i]));
          }
          const ff pr = ff_mul(g1, ff_sub(q[NV - 1], ff_mulf(jv, 0.5f)));
#pragma unroll
          for (int i = 0; i < D; ++i) bff[j * M::BW + i] = vel[i];
          bff[j * M::BW + D] = pr;
          const ff ep = ff_add(q[NV - 1], pr);
#pragma unroll
          for (int d = 0; d < D; ++d) {
            const ff ih = {F.ihh[d], F.ihl[d]};
            ff* dst = FB0 + d * NL + j * NV;
            dst[0] = ff_mul(q[1 + d], ih);
#pragma unroll
            for (int i = 0; i < D; ++i) {
              ff f = ff_mul(q[1 + i], vel[d]);
              if (i == d) f = ff_add(f, pr);
              dst[1 + i] = ff_mul(f, ih);
            }
            dst[NV - 1] = ff_mul(ff_mul(ep, vel[d]), ih);
          }
        } else {
#pragma unroll
          for (int d = 0; d < D; ++d) {
            const double ad = A.p.a[d] * A.g.inv_h[d];
            const float ah = (float)ad;
            FB0[d * NL + j * NV] = ff_mul(q[0], {ah, (float)(ad - (double)ah)});
          }
        }
      }
    }
  }
  __syncthreads();

  // B0 = R(u^n) in float-float (hi, lo): flux divergence (conservative form) or the
  // non-conservative product (elastic); the elastic volume term reuses it.
  float b0f[LPT], b0l[LPT];
#pragma unroll
  for (int k = 0; k < LPT; ++k) {
    const int l = tid + k * TPB;
    b0f[k] = 0.f;
    b0l[k] = 0.f;
    if (l < NL) {
      const int j = l / NV, v = l - (l / NV) * NV;
      ff aS = {0.f, 0.f};
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const int st = (d == 0 ? 1 : (d == 1 ? n : n * n));
        const int jd = (j / st) % n;
        const int j0 = j - jd * st;
        if constexpr (P::CONS) {
#pragma unroll
          for (int m = 0; m < n; ++m) {
            const ff f = FB0[d * NL + (j0 + m * st) * NV + v];
            const float2 dm = sD2[jd * n + m];
            ff_mac(aS, dm.x, dm.y, f.h, f.l);
          }
        } else {
          const int s = Elastic::src(d, v);
          if (s >= 0) {
            ff g = {0.f, 0.f};
#pragma unroll
            for (int m = 0; m < n; ++m) {
              const ff f = uff[(j0 + m * st) * NV + s];
              const float2 dm = sD2[jd * n + m];
              ff_mac(g, dm.x, dm.y, f.h, f.l);
            }
            aS = ff_add(aS, ff_mul(ff_norm(g.h, g.l), {cf[d * NV + v], cf[3 * NV + d * NV + v]}));
          }
        }
      }
      // B0 renormalised, without a round trip through FP64 (conservative form: -aS)
      const ff b = ff_norm(aS.h, aS.l);
      b0f[k] = P::CONS ? -b.h : b.h;
      b0l[k] = P::CONS ? -b.l : b.l;
    }
  }

  // ---- continuous extension Runge-Kutta guess (Sec. 5), A.cerk: dq^0 at the time nodes -------
  // Classical four-stage Runge-Kutta on the cell-local ODE dq/dt = R(u + dq) with the stages
  // k_i = B0 + dR(s_i) (+ the point source at the stage time), s = 0, h/2 k_1, h/2 k_2, h k_3,
  // and its natural continuous extension dq(x_t) = h sum_i b_i(x_t) k_i (sum_i b_i = x_t): the
  // stage increments and dR in binary32 (they are O(dt)), B0 from its float-float hi part.
  if (A.cerk) {
    float kd[3][LPT];   // dR of the stages 2, 3, 4
    double rs[4] = {0.0, 0.0, 0.0, 0.0};  // wavelet at the stage times (source cell)
    if (has_src) {
      const double ts[4] = {0.0, 0.5, 0.5, 1.0};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const double tau = fma(ts[i], dt, tn) - A.src.t0;
        const double a = (M_PI * A.src.f0 * tau) * (M_PI * A.src.f0 * tau);
        rs[i] = (1.0 - 2.0 * a) * exp(-a);
      }
    }
#pragma unroll
    for (int st = 0; st < 3; ++st) {
#pragma unroll
      for (int k = 0; k < LPT; ++k) {
        const int l = tid + k * TPB;
        if (l < NL) {
          float kp = b0f[k] + (st > 0 ? kd[st - 1][k] : 0.f);
          if (has_src) {
            const int j = l / NV, v = l - (l / NV) * NV;
            if (v >= 3) kp = fmaf((float)(-A.src.M[v - 3] * A.src.phi[j]), (float)rs[st], kp);
          }
          dqs[l] = (st == 2 ? dtf : 0.5f * dtf) * kp;
        }
      }
      __syncthreads();
      float r[LPT];
#pragma unroll
      for (int k = 0; k < LPT; ++k) r[k] = 0.f;
      if constexpr (P::CONS) {
        dflux_level<M, P, D>(dqs, uff, bff, A.p, F.g1h, F.g1l, dF3, tid);
        __syncthreads();
        contract_level<M, 0, false>(dF3, sDh, cf, r, tid);
        contract_level<M, 1, false>(dF3 + NL, sDh, cf, r, tid);
        if constexpr (D == 3) contract_level<M, 2, false>(dF3 + 2 * NL, sDh, cf, r, tid);
      } else {
        contract_level<M, 0, true>(dqs, sDh, cf, r, tid);
        contract_level<M, 1, true>(dqs, sDh, cf, r, tid);
        contract_level<M, 2, true>(dqs, sDh, cf, r, tid);
      }
#pragma unroll
      for (int k = 0; k < LPT; ++k) kd[st][k] = r[k];
      __syncthreads();  // the stage's reads of dqs / dF3 are done
    }
#pragma unroll
    for (int k = 0; k < LPT; ++k) {
      const int l = tid + k * TPB;
      if (l < NL) {
        float s1 = 0.f, s23 = 0.f, s4 = 0.f;
        if (has_src) {
          const int j = l / NV, v = l - (l / NV) * NV;
          if (v >= 3) {
            const float amp = (float)(-A.src.M[v - 3] * A.src.phi[j]);
            s1 = amp * (float)rs[0];
            s23 = amp * (float)(rs[1] + rs[2]);
            s4 = amp * (float)rs[3];
          }
        }
        const float k23 = kd[0][k] + kd[1][k] + s23, k4 = kd[2][k] + s4;
#pragma unroll
        for (int t = 0; t < n; ++t)
          dqs[t * NL + l] = dtf * fmaf(F.th[t], b0f[k],
                                       fmaf(F.cerk[0][t], s1, fmaf(F.cerk[1][t], k23, F.cerk[2][t] * k4)));
      }
    }
    __syncthreads();
  }

  // ---- Picard iterations on dq ----------------------------------------------------------
  float R[LPT][n];
  ff dqb[P::CONS ? LPT : 1];  // time average of the last iterate (float-float)
#pragma unroll
  for (int k = 0; k < (P::CONS ? LPT : 1); ++k) dqb[k] = {0.f, 0.f};
  for (int it = 0; it < A.iters; ++it) {
#pragma unroll
    for (int k = 0; k < LPT; ++k)
#pragma unroll
      for (int t = 0; t < n; ++t) R[k][t] = 0.f;
    const bool last = (it == A.iters - 1);
    if (it > 0 || A.cerk) {  // dq^0 = 0 gives dR = 0 without a guess
      if constexpr (P::CONS) {
        // all directions at once into dF3
        dflux_nodes_all<M, P, D>(dqs, uff, bff, A.p, F.g1h, F.g1l, dF3, tid);
        __syncthreads();
        if (last) {
          contract_f<M, 0, false, true>(dF3, sDh, sD2, cf, R, tid);
          contract_f<M, 1, false, true>(dF3 + NSL, sDh, sD2, cf, R, tid);
          if constexpr (D == 3) contract_f<M, 2, false, true>(dF3 + 2 * NSL, sDh, sD2, cf, R, tid);
        } else {
          contract_f<M, 0, false>(dF3, sDh, sD2, cf, R, tid);
          contract_f<M, 1, false>(dF3 + NSL, sDh, sD2, cf, R, tid);
          if constexpr (D == 3) contract_f<M, 2, false>(dF3 + 2 * NSL, sDh, sD2, cf, R, tid);
        }
      } else {
        if (last) {
          contract_f<M, 0, true, true>(dqs, sDh, sD2, cf, R, tid);
          contract_f<M, 1, true, true>(dqs, sDh, sD2, cf, R, tid);
          contract_f<M, 2, true, true>(dqs, sDh, sD2, cf, R, tid);
        } else {
          contract_f<M, 0, true>(dqs, sDh, sD2, cf, R, tid);
          contract_f<M, 1, true>(dqs, sDh, sD2, cf, R, tid);
          contract_f<M, 2, true>(dqs, sDh, sD2, cf, R, tid);
        }
      }
    }
    if (has_src) {
#pragma unroll
      for (int k = 0; k < LPT; ++k) {
        const int l = tid + k * TPB;
        if (l < NL) {
          const int j = l / NV, v = l - (l / NV) * NV;
          if (v >= 3) {
            const float amp = (float)(-A.src.M[v - 3] * A.src.phi[j]);
#pragma unroll
            for (int t = 0; t < n; ++t) R[k][t] = fmaf(amp, (float)ric[t], R[k][t]);
          }
        }
      }
    }
    __syncthreads();  // every read of dq of this iteration is done
#pragma unroll
    for (int k = 0; k < LPT; ++k) {
      const int l = tid + k * TPB;
      if (l < NL) {
        // dq_t = dt (kw1_t B0 + sum_m Kw[t][m] R_m); after the last iteration only the flux
        // remainders (conservative form) read the nodal dq_t
        if (!last || P::CONS) {
#pragma unroll
          for (int t = 0; t < n; ++t) {
            float acc = F.kw1[t] * b0f[k];
#pragma unroll
            for (int m = 0; m < n; ++m) acc = fmaf(F.Kw[t][m], R[k][m], acc);
            dqs[t * NL + l] = dtf * acc;
          }
        }
        if (last) {  // the time average qbar in float-float, from the weights averaged over t
          ff acc = {0.f, 0.f};
          ff_mac(acc, F.wk1h, F.wk1l, b0f[k], b0l[k]);
#pragma unroll
          for (int m = 0; m < n; ++m) ff_mac(acc, F.wKh[m], F.wKl[m], R[k][m], 0.f);
          const ff q = ff_mul(dtff, ff_norm(acc.h, acc.l));
          if constexpr (P::CONS) {
            dqb[k] = q;
          } else {  // straight to its place in shared memory (hi, lo over dq)
            dqs[l] = q.h;
            dqs[NL + l] = q.l;
          }
        }
      }
    }
    __syncthreads();
  }

  // ---- epilogue in float-float -------------------------------------------------------------
  float *qbh, *qbl;   // time-averaged dq [NL] (hi, lo)
  if constexpr (P::CONS) {
    // Time-averaged flux increment = A(u^n) qbar + sum_t w_t N(dq_t): the quadratic remainders N
    // per space-time node in binary32, the linear part once per spatial node in float-float.
    float* NB = dF3;  // [D][n][NL] remainders
    if constexpr (M::EULER) {
      remainder_nodes<M, D>(dqs, uff, bff, F.g1h, F.g1l, NB, tid);
      __syncthreads();  // every read of dqs is done: qbar overwrites it
    }
    qbh = dqs;
    qbl = dqs + NL;
#pragma unroll
    for (int k = 0; k < LPT; ++k) {
      const int l = tid + k * TPB;
      if (l < NL) {
        qbh[l] = dqb[k].h;
        qbl[l] = dqb[k].l;
        if constexpr (M::EULER) {
          // FB0 becomes G_d = F_d(u^n)/h_d + (time-averaged increment)_d/h_d; here the remainders
#pragma unroll
          for (int d = 0; d < D; ++d) {
            float nb = 0.f;
#pragma unroll
            for (int t = 0; t < n; ++t) nb = fmaf(F.w[t], NB[d * NSL + t * NL + l], nb);
            ff* g = FB0 + d * NL + l;
            *g = ff_add(*g, {nb * F.ihh[d], 0.f});
          }
        }
      }
    }
    __syncthreads();
    linear_nodes<M, P, D>(qbh, qbl, uff, bff, g1, F, A.p, FB0, tid);
  } else {
    qbh = dqs;  // written by the last time solve
    qbl = dqs + NL;
  }
  __syncthreads();

  double* un = A.u_next + c * NL;
#pragma unroll
  for (int k = 0; k < LPT; ++k) {
    const int l = tid + k * TPB;
    if (l < NL) {
      const int j = l / NV, v = l - (l / NV) * NV;
      ff dvol = {0.f, 0.f};
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const int st = (d == 0 ? 1 : (d == 1 ? n : n * n));
        const int jd = (j / st) % n;
        const int j0 = j - jd * st;
        if constexpr (P::CONS) {
          // weak-form volume term of the time-averaged flux: sum_m W[j_d][m] G_d[m]
#pragma unroll
          for (int m = 0; m < n; ++m) {
            const ff g = FB0[d * NL + (j0 + m * st) * NV + v];
            const float2 wm = sW2[jd * n + m];
            ff_mac(dvol, wm.x, wm.y, g.h, g.l);
          }
        } else {
          const int s = Elastic::src(d, v);
          if (s >= 0) {
            ff a = {0.f, 0.f};
#pragma unroll
            for (int m = 0; m < n; ++m) {
              const int i = (j0 + m * st) * NV + s;
              const float2 dm = sD2[jd * n + m];
              ff_mac(a, dm.x, dm.y, qbh[i], qbl[i]);
            }
            dvol = ff_add(dvol, ff_mul(ff_norm(a.h, a.l), {cf[d * NV + v], cf[3 * NV + d * NV + v]}));
          }
        }
      }
      double vol = ff_to_d(P::CONS ? dvol : ff_add({b0f[k], b0l[k]}, dvol));
      if (has_src && v >= 3) {
        double sbar = 0.0;
#pragma unroll
        for (int t = 0; t < n; ++t) sbar = fma(T.w[t], ric[t], sbar);
        vol = fma(-A.src.M[v - 3] * A.src.phi[j], sbar, vol);
      }
      un[l] = fma(dt, vol, ul[k]);
      uff[l] = ff_add(uff[l], {qbh[l], qbl[l]});  // time-averaged state u^n + qbar for the faces
    }
  }
  __syncthreads();

  // ---- face records: float-float extrapolations of the time-averaged state and flux, both
  // faces of a direction from the same loads --------------------------------------------------
  double* fc = A.face + c * (long long)(D * 2 * FR);
  for (int e = tid; e < NF * NV; e += TPB) {
    const int v = e % NV;
    const int jp = e / NV;
#pragma unroll
    for (int d = 0; d < D; ++d) {  // unrolled: constant index divisors
      const int st = (d == 0 ? 1 : (d == 1 ? n : n * n));
      const int jbase = (jp % st) + (jp / st) * st * n;
      ff qa0 = {0.f, 0.f}, qa1 = {0.f, 0.f}, fa0 = {0.f, 0.f}, fa1 = {0.f, 0.f};
#pragma unroll
      for (int m = 0; m < n; ++m) {
        const int jj = jbase + m * st;
        const ff q = uff[jj * NV + v];
        ff_mac(qa0, sE[0][m], sE[1][m], q.h, q.l);
        ff_mac(qa1, sE[2][m], sE[3][m], q.h, q.l);
        if constexpr (P::CONS) {
          const ff g = FB0[d * NL + jj * NV + v];
          ff_mac(fa0, sE[0][m], sE[1][m], g.h, g.l);
          ff_mac(fa1, sE[2][m], sE[3][m], g.h, g.l);
        }
      }
      double* rec0 = fc + (d * 2) * FR;
      double* rec1 = rec0 + FR;
      const double q0 = ff_to_d(qa0), q1 = ff_to_d(qa1);
      rec0[jp * NV + v] = q0;
      rec1[jp * NV + v] = q1;
      if constexpr (P::CONS) {
        rec0[NF * NV + jp * NV + v] = ff_to_d(fa0) * A.g.h[d];
        rec1[NF * NV + jp * NV + v] = ff_to_d(fa1) * A.g.h[d];
      }
      if constexpr (M::EULER) {  // the face states as written, for the wave speeds below
        double* qs = reinterpret_cast<double*>(dF3);
        qs[((d * 2) * NF + jp) * NV + v] = q0;
        qs[((d * 2 + 1) * NF + jp) * NV + v] = q1;
      }
    }
  }
  if constexpr (M::EULER) {
    // FP64 Rusanov wave speeds |v_d| + c of every face state (the same evaluation as the Riemann
    // solver's on the same face records), for the Riemann solver
    if (A.fspeed) {
      __syncthreads();
      const double* qs = reinterpret_cast<const double*>(dF3);
      double* fs = A.fspeed + c * (long long)(D * 2 * NF);
      for (int e = tid; e < D * 2 * NF; e += TPB) fs[e] = P::speed(qs + e * NV, A.p, e / (2 * NF));
    }
  }
}

template <class P, int D, int N>
__global__ void __launch_bounds__(CfgM<P, D, N>::TPB, CfgM<P, D, N>::MINB)
    k_predictor_mixed(const __grid_constant__ StepArgs A, const __grid_constant__ Tables T,
                      const __grid_constant__ TablesF F) {
  if (A.skip && A.skip[blockIdx.x]) return;  // computes with FV in this step
  predictor_mixed_cell<P, D, N>(A, T, F, blockIdx.x);
}

template <class P, int D, int N>
cudaError_t launch_predictor_mixed_n(const StepArgs& a, const Tables& t, const TablesF& f,
                                     cudaStream_t s) {
  using M = CfgM<P, D, N>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_predictor_mixed<P, D, N>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)M::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (a.g.ncells > 0x7fffffffLL) return cudaErrorInvalidValue;
  k_predictor_mixed<P, D, N><<<(unsigned)a.g.ncells, M::TPB, M::SMEM, s>>>(a, t, f);
  return cudaGetLastError();
}

}  // namespace ader
