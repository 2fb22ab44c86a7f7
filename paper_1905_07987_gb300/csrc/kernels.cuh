// FP64 kernels of one ADER-DG step (Sec. 3.3-3.4), templated on the PDE system, the dimension
// and the order.  One thread block per cell for the predictor (the work is FP64-pipe bound on
// GB300: every cell is an independent dense small contraction problem), one warp per face for
// the Riemann solver, one thread per degree of freedom for the corrector, grid-stride tiles for
// the CFL maximum (Euler: FP64 evaluation only on the nodes that binary32 enclosures cannot rule
// out).  The Riemann solver also serves the mixed-precision form (wave speeds evaluated by its
// predictor).
#pragma once
#include <cstdio>
#include "ader_internal.h"
#include "pde.cuh"

namespace ader {

// Compile-time sizes of the order-N scheme for system P in D dimensions.
template <class P, int D, int N>
struct Cfg {
  static constexpr int DIM = D;
  static constexpr int n = N + 1;               // nodes per direction (and time nodes)
  static constexpr int NS = ipow(n, D);         // spatial nodes per cell
  static constexpr int NST = NS * n;            // space-time nodes per cell
  static constexpr int NV = P::NV;
  static constexpr int NL = NS * NV;            // lines (spatial node, variable)
  static constexpr int NF = ipow(n, D - 1);     // nodes per face
  static constexpr int FR = NF * NV * (P::CONS ? 2 : 1);  // doubles per face record
  static constexpr int NPHI = (P::NCP || P::NCPS) ? 2 : 1;  // numerical fluxes per face node and variable
  static constexpr int TPB_RAW = ((NL + 5) / 6 + 31) / 32 * 32;
  static constexpr int TPB = TPB_RAW < 64 ? 64 : (TPB_RAW > 512 ? 512 : TPB_RAW);
  static constexpr int LPT = (NL + TPB - 1) / TPB;   // lines per thread
  static constexpr int NPT = (NST + TPB - 1) / TPB;  // space-time nodes per thread
  static constexpr int FSLOTS = P::CONS ? cmax(n, D + 1) : 0;
  // shallow water: the surface derivatives d(h + b)/dx_d at every space-time node [NST][D]
  static constexpr int GSLOTS = P::NCPS ? NST * D : 0;
  static constexpr size_t SMEM = ((size_t)(n + FSLOTS) * NL + GSLOTS) * sizeof(double);
};

template <int n, int d>
__device__ __forceinline__ int digit(int j) {
  return (j / ipow(n, d)) % n;
}

// Lines (j, v) owned by this thread: l = tid + k*TPB.
// Accumulate R[k][t] += coef * sum_m D[j_d][m] X[t][(j with j_d -> m)][vsrc]   (X: [n][NL] in smem)
// Dm: D with row stride RS (shared memory, or the kernel-parameter table with RS = MAXN).
template <class C, int d, int RS>
__device__ __forceinline__ void contract_lines(const double* X, const double* Dm, double coef,
                                               double (&R)[C::LPT][C::n], int tid) {
  constexpr int n = C::n, NV = C::NV, NL = C::NL, TPB = C::TPB, st = ipow(n, d);
#pragma unroll
  for (int k = 0; k < C::LPT; ++k) {
    const int l = tid + k * TPB;
    if (l < NL) {
      const int j = l / NV, v = l - (l / NV) * NV;
      const int jd = digit<n, d>(j);
      const int j0 = j - jd * st;
      const double* Dr = Dm + jd * RS;
#pragma unroll
      for (int t = 0; t < n; ++t) {
        double acc = 0.0;
#pragma unroll
        for (int m = 0; m < n; ++m) acc = fma(Dr[m], X[t * NL + (j0 + m * st) * NV + v], acc);
        R[k][t] = fma(coef, acc, R[k][t]);
      }
    }
  }
}

// Elastic: each row v of B_d has one non-zero coef(d,v) at column src(d,v); the NCP term
// B_d dq/dx_d is contracted directly from q (no flux buffer).
template <class C, int d, int RS>
__device__ __forceinline__ void contract_ncp_elastic(const double* X, const double* Dm,
                                                     double inv_h, double irho, double lam,
                                                     double mu, double (&R)[C::LPT][C::n],
                                                     int tid) {
  constexpr int n = C::n, NV = C::NV, NL = C::NL, TPB = C::TPB, st = ipow(n, d);
#pragma unroll
  for (int k = 0; k < C::LPT; ++k) {
    const int l = tid + k * TPB;
    if (l < NL) {
      const int j = l / NV, v = l - (l / NV) * NV;
      const int s = Elastic::src(d, v);
      if (s >= 0) {
        const double coef = -Elastic::coef_ir(d, v, irho, lam, mu) * inv_h;
        const int jd = digit<n, d>(j);
        const int j0 = j - jd * st;
        const double* Dr = Dm + jd * RS;
#pragma unroll
        for (int t = 0; t < n; ++t) {
          double acc = 0.0;
#pragma unroll
          for (int m = 0; m < n; ++m) acc = fma(Dr[m], X[t * NL + (j0 + m * st) * NV + s], acc);
          R[k][t] = fma(coef, acc, R[k][t]);
        }
      }
    }
  }
}

// Shallow water: the derivative of the surface h + b along every direction at the owned
// space-time nodes, G[node][d] = sum_m D[j_d][m] (h + b)(t, j with j_d -> m) (node = t NS + j,
// m ascending), one thread per node so that every lane works; the momentum lines of direction d
// then take g h G (ncp_swe_lines) instead of each forming the sum itself.
template <class C, int RS>
__device__ __forceinline__ void surface_derivs(const double* X, const double* Dm, double* G, int tid) {
  constexpr int n = C::n, NV = C::NV, NL = C::NL, NS = C::NS, D = C::DIM;
#pragma unroll
  for (int k = 0; k < C::NPT; ++k) {
    const int node = tid + k * C::TPB;
    if (node < C::NST) {
      const int t = node / NS, j = node - t * NS;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const int st = d == 0 ? 1 : (d == 1 ? n : n * n);
        const int jd = (j / st) % n;
        const int j0 = j - jd * st;
        const double* Dr = Dm + jd * RS;
        double acc = 0.0;
#pragma unroll
        for (int m = 0; m < n; ++m) {
          const double* q = X + t * NL + (j0 + m * st) * NV;
          acc = fma(Dr[m], q[0] + q[3], acc);
        }
        G[node * D + d] = acc;
      }
    }
  }
}

// Shallow water: row 1 + d of B_d(q) dq/dx_d is g h (dh/dx_d + db/dx_d) with the node's own h
// (state-dependent non-conservative product), accumulated on the momentum line v = 1 + d as
// R -= g h (1/h_d) G[t, j][d].
template <class C, int d>
__device__ __forceinline__ void ncp_swe_lines(const double* X, const double* G, double inv_h,
                                              double grav, double (&R)[C::LPT][C::n], int tid) {
  constexpr int n = C::n, NV = C::NV, NL = C::NL, NS = C::NS, TPB = C::TPB, D = C::DIM;
#pragma unroll
  for (int k = 0; k < C::LPT; ++k) {
    const int l = tid + k * TPB;
    if (l < NL) {
      const int j = l / NV, v = l - (l / NV) * NV;
      if (v == 1 + d) {
#pragma unroll
        for (int t = 0; t < n; ++t)
          R[k][t] = fma(-grav * inv_h * X[t * NL + j * NV], G[(t * NS + j) * D + d], R[k][t]);
      }
    }
  }
}

template <class C, int d, class P>
__device__ __forceinline__ void flux_nodes(const double (&qn)[C::NPT][C::NV],
                                           const typename P::Aux (&ax)[C::NPT],
                                           const PdeParams& pp, double* Fs, int tid) {
#pragma unroll
  for (int k = 0; k < C::NPT; ++k) {
    const int node = tid + k * C::TPB;
    if (node < C::NST) {
      double F[C::NV];
      P::flux(qn[k], ax[k], pp, d, F);
#pragma unroll
      for (int v = 0; v < C::NV; ++v) Fs[node * C::NV + v] = F[v];
    }
  }
}

template <class C, class P>
__device__ __forceinline__ void load_nodes(const double* qs, const PdeParams& pp,
                                           double (&qn)[C::NPT][C::NV],
                                           typename P::Aux (&ax)[C::NPT], int tid) {
#pragma unroll
  for (int k = 0; k < C::NPT; ++k) {
    const int node = tid + k * C::TPB;
    if (node < C::NST) {
#pragma unroll
      for (int v = 0; v < C::NV; ++v) qn[k][v] = qs[node * C::NV + v];
      P::aux(qn[k], pp, ax[k]);
    }
  }
}

// Continuous extension Runge-Kutta guess of the predictor (Sec. 5): the classical four-stage
// Runge-Kutta method on the cell-local ODE dq/dt = R(q) (flux divergence or non-conservative
// product of one time level, point source at the stage time), and its natural continuous
// extension of uniform order 3 evaluated at the time nodes:
//   q_t = u + dt (b1(x_t) k1 + b2(x_t) (k2 + k3) + b4(x_t) k4)   (weights: T.cerk)
// written to the n time slices of qs.  Called once per cell before the Picard iterations (not
// inlined: its registers do not add to the iteration loop's).
template <class P, int D, int N>
__device__ __noinline__ void cerk_guess_cell(const StepArgs& A, const Tables& T, double* qs,
                                             double* Fs, const double* sD, const double* ul,
                                             double irho, double lam, double mu, bool has_src,
                                             int tid) {
  using C = Cfg<P, D, N>;
  constexpr int n = C::n, NV = C::NV, NL = C::NL, NS = C::NS, TPB = C::TPB, LPT = C::LPT;
  const double dt = A.dev->dt;
  const double tn = A.dev->t;
  double kst[4][LPT];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const double ca = i == 0 ? 0.0 : (i == 3 ? 1.0 : 0.5);
    // stage state u + dt a_i k_{i-1} in time slice 0 of qs
#pragma unroll
    for (int k = 0; k < LPT; ++k) {
      const int l = tid + k * TPB;
      if (l < NL) qs[l] = i == 0 ? ul[k] : fma(ca * dt, kst[i > 0 ? i - 1 : 0][k], ul[k]);
    }
    __syncthreads();
    double R1[LPT];
#pragma unroll
    for (int k = 0; k < LPT; ++k) R1[k] = 0.0;
    if constexpr (P::CONS) {
#pragma unroll
      for (int d = 0; d < D; ++d) {
        for (int j = tid; j < NS; j += TPB) {
          double q[NV], f[NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) q[v] = qs[j * NV + v];
          typename P::Aux ax;
          P::aux(q, A.p, ax);
          P::flux(q, ax, A.p, d, f);
#pragma unroll
          for (int v = 0; v < NV; ++v) Fs[j * NV + v] = f[v];
        }
        __syncthreads();
        const int st = d == 0 ? 1 : (d == 1 ? n : n * n);
#pragma unroll
        for (int k = 0; k < LPT; ++k) {
          const int l = tid + k * TPB;
          if (l < NL) {
            const int j = l / NV, v = l - (l / NV) * NV;
            const int jd = (j / st) % n, j0 = j - jd * st;
            double acc = 0.0;
#pragma unroll
            for (int m = 0; m < n; ++m) acc = fma(sD[jd * n + m], Fs[(j0 + m * st) * NV + v], acc);
            R1[k] = fma(-A.g.inv_h[d], acc, R1[k]);
          }
        }
        __syncthreads();
      }
    }
    if constexpr (P::NCP) {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const int st = d == 0 ? 1 : (d == 1 ? n : n * n);
#pragma unroll
        for (int k = 0; k < LPT; ++k) {
          const int l = tid + k * TPB;
          if (l < NL) {
            const int j = l / NV, v = l - (l / NV) * NV;
            const int sv = Elastic::src(d, v);
            if (sv >= 0) {
              const double coef = -Elastic::coef_ir(d, v, irho, lam, mu) * A.g.inv_h[d];
              const int jd = (j / st) % n, j0 = j - jd * st;
              double acc = 0.0;
#pragma unroll
              for (int m = 0; m < n; ++m) acc = fma(sD[jd * n + m], qs[(j0 + m * st) * NV + sv], acc);
              R1[k] = fma(coef, acc, R1[k]);
            }
          }
        }
      }
    }
    if (has_src) {
      const double tau = fma(ca, dt, tn) - A.src.t0;
      const double a = (M_PI * A.src.f0 * tau) * (M_PI * A.src.f0 * tau);
      const double ric = (1.0 - 2.0 * a) * exp(-a);
#pragma unroll
      for (int k = 0; k < LPT; ++k) {
        const int l = tid + k * TPB;
        if (l < NL) {
          const int j = l / NV, v = l - (l / NV) * NV;
          if (v >= 3) R1[k] = fma(-A.src.M[v - 3] * A.src.phi[j], ric, R1[k]);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < LPT; ++k) kst[i][k] = R1[k];
    __syncthreads();  // the next stage overwrites slice 0
  }
#pragma unroll
  for (int k = 0; k < LPT; ++k) {
    const int l = tid + k * TPB;
    if (l < NL) {
#pragma unroll
      for (int t = 0; t < n; ++t)
        qs[t * NL + l] = ul[k] + dt * (T.cerk[0][t] * kst[0][k] + T.cerk[1][t] * (kst[1][k] + kst[2][k]) +
                                       T.cerk[2][t] * kst[3][k]);
    }
  }
}

// Space-time predictor (Eq. (5)) with the fused epilogue: time averages, volume term, the
// cell-local part of the face terms of Eq. (6), and the face extrapolations.
//   q^0 = u (or the continuous extension Runge-Kutta guess, A.cerk);
//   q^{r+1} = u + dt Kw R(q^r)  (Kw = K1^{-1} diag(w), K1^{-1} e0 = 1)
//   R(q) = -sum_d (1/h_d) D_d F_d(q) - sum_d (1/h_d) B_d D_d q + point source
// One cell c (all threads of the block; called by the per-context kernel and by the persistent
// ensemble kernel).
template <class P, int D, int N>
__device__ __forceinline__ void predictor_cell(const StepArgs& A, const Tables& T, long long c) {
  using C = Cfg<P, D, N>;
  constexpr int n = C::n, NV = C::NV, NL = C::NL, TPB = C::TPB, LPT = C::LPT;
  constexpr int NF = C::NF, FR = C::FR;
  extern __shared__ double smem[];
  double* qs = smem;           // [n][NL] space-time predictor (time-major)
  double* Fs = smem + n * NL;  // [FSLOTS][NL] fluxes (conservative systems)
  double* G = Fs + C::FSLOTS * NL;  // [NST][D] surface derivatives (shallow water)
  const int tid = threadIdx.x;
  const double dt = A.dev->dt;
  const double tn = A.dev->t;
  const double* u = A.u + c * NL;
  // D and c0/c1 are indexed by a per-lane row: staged in shared memory
  __shared__ double sD[n * n], sC[2][n];
  for (int i = tid; i < n * n; i += TPB) sD[i] = T.D[i / n][i % n];
  if (tid < n) {
    sC[0][tid] = T.c0[tid];
    sC[1][tid] = T.c1[tid];
  }

  double ul[LPT];
#pragma unroll
  for (int k = 0; k < LPT; ++k) {
    const int l = tid + k * TPB;
    ul[k] = 0.0;
    if (l < NL) {
      ul[k] = u[l];
#pragma unroll
      for (int t = 0; t < n; ++t) qs[t * NL + l] = ul[k];
    }
  }
  double irho = 0.0, lam = 0.0, mu = 0.0;
  if constexpr (P::NCP) {
    irho = 1.0 / A.mat[c * 3 + 0];
    lam = A.mat[c * 3 + 1];
    mu = A.mat[c * 3 + 2];
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
  __syncthreads();
  if (A.cerk) {
    cerk_guess_cell<P, D, N>(A, T, qs, Fs, sD, ul, irho, lam, mu, has_src, tid);
    __syncthreads();
  }

  for (int it = 0; it < A.iters; ++it) {
    double R[LPT][n];
#pragma unroll
    for (int k = 0; k < LPT; ++k)
#pragma unroll
      for (int t = 0; t < n; ++t) R[k][t] = 0.0;
    if constexpr (P::CONS) {
      double qn[C::NPT][NV];
      typename P::Aux ax[C::NPT];
      load_nodes<C, P>(qs, A.p, qn, ax, tid);
      if constexpr (P::NCPS) surface_derivs<C, n>(qs, sD, G, tid);
      flux_nodes<C, 0, P>(qn, ax, A.p, Fs, tid);
      __syncthreads();
      contract_lines<C, 0, n>(Fs, sD, -A.g.inv_h[0], R, tid);
      __syncthreads();
      flux_nodes<C, 1, P>(qn, ax, A.p, Fs, tid);
      __syncthreads();
      contract_lines<C, 1, n>(Fs, sD, -A.g.inv_h[1], R, tid);
      __syncthreads();
      if constexpr (D == 3) {
        flux_nodes<C, 2, P>(qn, ax, A.p, Fs, tid);
        __syncthreads();
        contract_lines<C, 2, n>(Fs, sD, -A.g.inv_h[2], R, tid);
      }
    }
    if constexpr (P::NCP) {
      contract_ncp_elastic<C, 0, n>(qs, sD, A.g.inv_h[0], irho, lam, mu, R, tid);
      contract_ncp_elastic<C, 1, n>(qs, sD, A.g.inv_h[1], irho, lam, mu, R, tid);
      contract_ncp_elastic<C, 2, n>(qs, sD, A.g.inv_h[2], irho, lam, mu, R, tid);
    }
    if constexpr (P::NCPS) {
      ncp_swe_lines<C, 0>(qs, G, A.g.inv_h[0], A.p.grav, R, tid);
      ncp_swe_lines<C, 1>(qs, G, A.g.inv_h[1], A.p.grav, R, tid);
    }
    if (has_src) {
#pragma unroll
      for (int k = 0; k < LPT; ++k) {
        const int l = tid + k * TPB;
        if (l < NL) {
          const int j = l / NV, v = l - (l / NV) * NV;
          if (v >= 3) {
            const double amp = -A.src.M[v - 3] * A.src.phi[j];
#pragma unroll
            for (int t = 0; t < n; ++t) R[k][t] = fma(amp, ric[t], R[k][t]);
          }
        }
      }
    }
    __syncthreads();  // every read of qs of this iteration is done
#pragma unroll
    for (int k = 0; k < LPT; ++k) {
      const int l = tid + k * TPB;
      if (l < NL) {
#pragma unroll
        for (int t = 0; t < n; ++t) {
          double acc = 0.0;
#pragma unroll
          for (int m = 0; m < n; ++m) acc = fma(T.Kw[t][m], R[k][m], acc);
          qs[t * NL + l] = fma(dt, acc, ul[k]);
        }
      }
    }
    __syncthreads();
  }

  // ---- epilogue: time averages -------------------------------------------------------
  double qb[LPT];
#pragma unroll
  for (int k = 0; k < LPT; ++k) {
    const int l = tid + k * TPB;
    qb[k] = 0.0;
    if (l < NL) {
#pragma unroll
      for (int t = 0; t < n; ++t) qb[k] = fma(T.w[t], qs[t * NL + l], qb[k]);
    }
  }
  double* qbs;   // time-averaged q [NL] in smem
  double* FBs;   // time-averaged fluxes [D][NL] in smem (conservative)
  if constexpr (P::CONS) {
    double FB[D][LPT];
    double qn[C::NPT][NV];
    typename P::Aux ax[C::NPT];
    load_nodes<C, P>(qs, A.p, qn, ax, tid);
    if constexpr (P::NCPS) surface_derivs<C, n>(qs, sD, G, tid);  // of the final predictor
#pragma unroll
    for (int d = 0; d < D; ++d) {
      if (d == 0) flux_nodes<C, 0, P>(qn, ax, A.p, Fs, tid);
      if (d == 1) flux_nodes<C, 1, P>(qn, ax, A.p, Fs, tid);
      if constexpr (D == 3)
        if (d == 2) flux_nodes<C, 2, P>(qn, ax, A.p, Fs, tid);
      __syncthreads();
#pragma unroll
      for (int k = 0; k < LPT; ++k) {
        const int l = tid + k * TPB;
        FB[d][k] = 0.0;
        if (l < NL) {
#pragma unroll
          for (int t = 0; t < n; ++t) FB[d][k] = fma(T.w[t], Fs[t * NL + l], FB[d][k]);
        }
      }
      __syncthreads();
    }
    qbs = Fs;
    FBs = Fs + NL;
#pragma unroll
    for (int k = 0; k < LPT; ++k) {
      const int l = tid + k * TPB;
      if (l < NL) {
        qbs[l] = qb[k];
#pragma unroll
        for (int d = 0; d < D; ++d) FBs[d * NL + l] = FB[d][k];
      }
    }
  } else {
    qbs = qs;
    FBs = nullptr;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < LPT; ++k) {
      const int l = tid + k * TPB;
      if (l < NL) qbs[l] = qb[k];
    }
  }
  __syncthreads();

  // ---- volume term and cell-local face terms -> u_next ---------------------------------
  double* un = A.u_next + c * NL;
#pragma unroll
  for (int k = 0; k < LPT; ++k) {
    const int l = tid + k * TPB;
    if (l < NL) {
      const int j = l / NV, v = l - (l / NV) * NV;
      double vol = 0.0;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const int st = (d == 0 ? 1 : (d == 1 ? n : n * n));
        const int jd = (j / st) % n;
        const int j0 = j - jd * st;
        if constexpr (P::CONS) {
          double dF = 0.0, Fp = 0.0, Fm = 0.0;
#pragma unroll
          for (int m = 0; m < n; ++m) {
            const double f = FBs[d * NL + (j0 + m * st) * NV + v];
            dF = fma(sD[jd * n + m], f, dF);
            Fp = fma(T.e1[m], f, Fp);
            Fm = fma(T.e0[m], f, Fm);
          }
          // -(1/h) D F + (1/h)(e1/w F+ - e0/w F-)
          vol += A.g.inv_h[d] * (-dF + sC[1][jd] * Fp - sC[0][jd] * Fm);
        }
        if constexpr (P::NCP) {
          const int s = Elastic::src(d, v);
          if (s >= 0) {
            double dq = 0.0;
#pragma unroll
            for (int m = 0; m < n; ++m) dq = fma(sD[jd * n + m], qbs[(j0 + m * st) * NV + s], dq);
            vol -= A.g.inv_h[d] * Elastic::coef_ir(d, v, irho, lam, mu) * dq;
          }
        }
        if constexpr (P::NCPS) {
          // time average of the state-dependent product taken node by node (sum_t w_t g h_t
          // (D_d (h + b))_t), not of the product of the time averages
          if (v == 1 + d) {
            double nb = 0.0;
#pragma unroll
            for (int t = 0; t < n; ++t)
              nb = fma(T.w[t] * qs[t * NL + j * NV], G[(t * C::NS + j) * D + d], nb);
            vol -= A.g.inv_h[d] * A.p.grav * nb;
          }
        }
      }
      if (has_src && v >= 3) {
        double sbar = 0.0;
#pragma unroll
        for (int t = 0; t < n; ++t) sbar = fma(T.w[t], ric[t], sbar);
        vol = fma(-A.src.M[v - 3] * A.src.phi[j], sbar, vol);
      }
      un[l] = fma(dt, vol, ul[k]);
    }
  }

  // ---- face records: time-averaged q (and F_d) extrapolated to both ends of each direction
  double* fc = A.face + c * (long long)(D * 2 * FR);
  constexpr int NFE = D * 2 * NF * NV;
  for (int e = tid; e < NFE; e += TPB) {
    const int v = e % NV;
    const int jp = (e / NV) % NF;
    const int side = (e / (NV * NF)) % 2;
    const int d = e / (NV * NF * 2);
    const int st = (d == 0 ? 1 : (d == 1 ? n : n * n));
    const int jbase = (jp % st) + (jp / st) * st * n;
    const double* ev = side ? T.e1 : T.e0;
    double qf = 0.0, ff = 0.0;
#pragma unroll
    for (int m = 0; m < n; ++m) {
      const int jj = jbase + m * st;
      qf = fma(ev[m], qbs[jj * NV + v], qf);
      if constexpr (P::CONS) ff = fma(ev[m], FBs[d * NL + jj * NV + v], ff);
    }
    double* rec = fc + (d * 2 + side) * FR;
    rec[jp * NV + v] = qf;
    if constexpr (P::CONS) rec[NF * NV + jp * NV + v] = ff;
  }
}

template <class P, int D, int N>
__global__ void __launch_bounds__(Cfg<P, D, N>::TPB)
    k_predictor(const __grid_constant__ StepArgs A, const __grid_constant__ Tables T) {
  if (A.skip && A.skip[blockIdx.x]) return;  // computes with FV in this step
  predictor_cell<P, D, N>(A, T, blockIdx.x);
}

// Index helpers for faces.  In direction d the faces of one grid line are numbered k = 0..n_d
// (face k is the lower face of cell k); the grid line is the cell index with digit d removed.
struct FaceIdx {
  __device__ static long long trans_of_cell(const Geometry& g, long long c, int d, int& id) {
    const int i0 = (int)(c % g.n[0]);
    const long long r = c / g.n[0];
    const int i1 = (int)(r % g.n[1]);
    const int i2 = (int)(r / g.n[1]);
    if (d == 0) { id = i0; return i1 + (long long)g.n[1] * i2; }
    if (d == 1) { id = i1; return i0 + (long long)g.n[0] * i2; }
    id = i2;
    return i0 + (long long)g.n[0] * i1;
  }
  __device__ static long long cell_of(const Geometry& g, long long tr, int d, int id) {
    if (d == 0) return id + (long long)g.n[0] * tr;
    if (d == 1) {
      const long long i0 = tr % g.n[0], i2 = tr / g.n[0];
      return i0 + (long long)g.n[0] * (id + (long long)g.n[1] * i2);
    }
    const long long i0 = tr % g.n[0], i1 = tr / g.n[0];
    return i0 + (long long)g.n[0] * (i1 + (long long)g.n[1] * id);
  }
  __device__ static long long ntrans(const Geometry& g, int d) {
    return g.ncells / g.n[d];
  }
};

// Ghost state at a non-periodic boundary from the interior face record values.
template <class P>
__device__ __forceinline__ void ghost(int kind, int d, double* q, double* F) {
  if (kind == 1) {  // wall
    P::mirror(q, d);
    if constexpr (P::CONS) P::mirror_flux(F, d);
  } else {          // absorbing
    if constexpr (P::LINEAR) {
#pragma unroll
      for (int v = 0; v < P::NV; ++v) {
        q[v] = 0.0;
        if constexpr (P::CONS) F[v] = 0.0;
      }
    }
  }
}

// Rusanov flux with one wave speed per face (max over face nodes and both sides) and the halved
// path-conservative fluctuation:  Phi_L = G + Bbar dq / 2,  Phi_R = G - Bbar dq / 2.
// One warp per face (warp-shuffle maximum of the speeds); faces of direction d, offset `phi_off`
// in the flux buffer.  With A.fspeed the FP64 speeds of the face states come from the predictor.
// Interior faces whose flux is elementwise (Euler with those speeds, elastic with the face's
// material terms formed once per warp) are walked value by value, coalesced; boundary faces go
// node by node with their ghost states.
template <class P, int D, int N>
__device__ __forceinline__ void riemann_face(const StepArgs& A, const Tables& T, int d,
                                             long long phi_off, long long f, int lane) {
  using C = Cfg<P, D, N>;
  constexpr int NV = C::NV, NF = C::NF, FR = C::FR, NPHI = C::NPHI;
  constexpr int PER = (NF + 31) / 32;
  const Geometry& g = A.g;
  const int nd = g.n[d];
  const long long nfaces = (long long)(nd + 1) * FaceIdx::ntrans(g, d);
  if (f >= nfaces) return;
  const int kf = (int)(f % (nd + 1));
  const long long tr = f / (nd + 1);
  const bool periodic = (g.bc[d][0] == BC_PERIODIC);
  if (periodic && kf == nd) return;  // duplicate of face 0
  long long cL = -1, cR = -1;
  if (kf > 0) cL = FaceIdx::cell_of(g, tr, d, kf - 1);
  else if (periodic) cL = FaceIdx::cell_of(g, tr, d, nd - 1);
  if (kf < nd) cR = FaceIdx::cell_of(g, tr, d, kf);
  else if (periodic) cR = FaceIdx::cell_of(g, tr, d, 0);
  const double* recL = cL >= 0 ? A.face + cL * (long long)(D * 2 * FR) + (d * 2 + 1) * FR : nullptr;
  const double* recR = cR >= 0 ? A.face + cR * (long long)(D * 2 * FR) + (d * 2 + 0) * FR : nullptr;

  if constexpr (P::CONS && !P::LINEAR) {
    // interior face with the speeds already evaluated (mixed form): the flux is elementwise, so the
    // lanes walk the face's NF x NV values contiguously (coalesced loads and stores)
    if (A.fspeed && recL && recR) {
      constexpr int PE = (NF * NV + 31) / 32;  // values per lane; every load issued up front
      double ql[PE], qr[PE], fl[PE], fr[PE];
#pragma unroll
      for (int r = 0; r < PE; ++r) {
        const int e = lane + 32 * r;
        if (e < NF * NV) {
          ql[r] = recL[e];
          qr[r] = recR[e];
          fl[r] = recL[NF * NV + e];
          fr[r] = recR[NF * NV + e];
        }
      }
      const double* sl = A.fspeed + (cL * D + d) * (2 * NF) + NF;
      const double* sr = A.fspeed + (cR * D + d) * (2 * NF);
      double sm = 0.0;
      for (int jp = lane; jp < NF; jp += 32) sm = fmax(sm, fmax(sl[jp], sr[jp]));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sm = fmax(sm, __shfl_xor_sync(0xffffffffu, sm, o));
      double* out = A.phi + phi_off + f * (long long)(NF * NV);
#pragma unroll
      for (int r = 0; r < PE; ++r) {
        const int e = lane + 32 * r;
        if (e < NF * NV) out[e] = 0.5 * (fl[r] + fr[r]) - 0.5 * sm * (qr[r] - ql[r]);
      }
      return;
    }
  }

  // elastic: the face's speed and path-averaged coefficients depend only on the two cells'
  // materials.  The warp forms them without divergent paths (every FP64 instruction costs the
  // whole warp's pipe time): one division per lane (lanes 0-2: 1 / rho at the three path
  // points; lanes 3, 4: (lambda + 2 mu) / rho of the left and right cell), one square root
  // (the P-wave speeds), then lane v < NV accumulates row v's coefficient
  // -(a + b mu(z)) with (a, b) = (lambda(z), 2) on the normal stress of direction d,
  // (lambda(z), 0) on the other normal stresses, (0, 1) on the shear stresses, and -1 / rho(z)
  // on the velocities.  mine_ncp = cb[lane] (lane < NV), s_ncp = the face's speed.
  double s_ncp = 0.0, mine_ncp = 0.0;
  if constexpr (P::NCP) {
   if (A.fmat) {
    // formed when the material was set (the same operations as below)
    long long fo = f;
    for (int dd = 0; dd < d; ++dd) fo += (long long)(g.n[dd] + 1) * FaceIdx::ntrans(g, dd);
    const double* fm = A.fmat + fo * FMAT;
    s_ncp = fm[0];
    mine_ncp = lane < NV ? fm[1 + lane] : 0.0;
   } else {
    const long long mcL = cL >= 0 ? cL : cR, mcR = cR >= 0 ? cR : cL;
    const double rL = A.mat[mcL * 3], lL = A.mat[mcL * 3 + 1], uL = A.mat[mcL * 3 + 2];
    const double rR = A.mat[mcR * 3], lR = A.mat[mcR * 3 + 1], uR = A.mat[mcR * 3 + 2];
    const int gl = lane < 3 ? lane : 0;
    const double num = lane < 3 ? 1.0 : (lane == 3 ? lL + 2.0 * uL : (lane == 4 ? lR + 2.0 * uR : 1.0));
    const double den = lane < 3 ? fma(T.pz[gl], rR - rL, rL) : (lane == 3 ? rL : (lane == 4 ? rR : 1.0));
    const double quo = num / den;
    const double rt = sqrt(quo);
    const double sL = __shfl_sync(0xffffffffu, rt, 3), sR = __shfl_sync(0xffffffffu, rt, 4);
    s_ncp = (sL >= sR) ? sL : sR;
    const int v = lane < NV ? lane : 0;
    const double bmu = v < 3 ? 0.0 : (v < 6 ? (v - 3 == d ? 2.0 : 0.0) : 1.0);
#pragma unroll
    for (int gq = 0; gq < 3; ++gq) {
      const double z = T.pz[gq];
      const double ir = __shfl_sync(0xffffffffu, quo, gq);
      const double lz = fma(z, lR - lL, lL), uz = fma(z, uR - uL, uL);
      const double cl = -((v >= 3 && v < 6 ? lz : 0.0) + bmu * uz);
      mine_ncp = fma(T.pw[gq], v < 3 ? -ir : cl, mine_ncp);
    }
   }
    // interior face: the flux is elementwise over the face's NF x NV values, so the lanes walk
    // them contiguously (coalesced); each lane takes the jump of its row's source variable from
    // the same records and half its coefficient from lane v
    if (recL && recR) {
      constexpr int PE = (NF * NV + 31) / 32;
      const double hcb = 0.5 * mine_ncp;
      const double hs = 0.5 * s_ncp;
      double* out = A.phi + phi_off + f * (long long)(NPHI * NF * NV);
#pragma unroll
      for (int r = 0; r < PE; ++r) {
        const int e = lane + 32 * r;
        const int ve = e % NV;
        const double hc = __shfl_sync(0xffffffffu, hcb, ve);
        if (e < NF * NV) {
          const int sv = Elastic::src(d, ve);
          const int es = e - ve + (sv < 0 ? 0 : sv);
          const double G = -(hs * (recR[e] - recL[e]));
          const double jump = sv >= 0 ? recR[es] - recL[es] : 0.0;
          out[e] = fma(hc, jump, G);
          out[NF * NV + e] = fma(-hc, jump, G);
        }
      }
      return;
    }
  }

  double qL[PER][NV], qR[PER][NV], FL[PER][NV], FR_[PER][NV];
  double smax = 0.0;
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    const int jp = lane + 32 * r;
    if (jp < NF) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const double* a = recL ? recL : recR;
        const double* b = recR ? recR : recL;
        qL[r][v] = a[jp * NV + v];
        qR[r][v] = b[jp * NV + v];
        FL[r][v] = P::CONS ? a[NF * NV + jp * NV + v] : 0.0;
        FR_[r][v] = P::CONS ? b[NF * NV + jp * NV + v] : 0.0;
      }
      if (!recL) ghost<P>(g.bc[d][0], d, qL[r], FL[r]);
      if (!recR) ghost<P>(g.bc[d][1], d, qR[r], FR_[r]);
    }
  }
  if constexpr (P::CONS && !P::LINEAR) {
    if (A.fspeed) {  // mixed form: FP64 speeds of the face states, evaluated by the predictor
      const double* sl = cL >= 0 ? A.fspeed + (cL * D + d) * (2 * NF) + NF : nullptr;
      const double* sr = cR >= 0 ? A.fspeed + (cR * D + d) * (2 * NF) : nullptr;
#pragma unroll
      for (int r = 0; r < PER; ++r) {
        const int jp = lane + 32 * r;
        if (jp < NF) {  // a boundary side has the speed of its interior mirror / copy
          const double a = sl ? sl[jp] : sr[jp], b = sr ? sr[jp] : sl[jp];
          smax = fmax(smax, fmax(a, b));
        }
      }
    } else {
#pragma unroll
      for (int r = 0; r < PER; ++r) {
        const int jp = lane + 32 * r;
        if (jp < NF) smax = fmax(smax, fmax(P::speed(qL[r], A.p, d), P::speed(qR[r], A.p, d)));
      }
    }
  }
  double s;
  double cb[NV];
  if constexpr (P::NCP) {
    s = s_ncp;
#pragma unroll
    for (int v = 0; v < NV; ++v) cb[v] = __shfl_sync(0xffffffffu, mine_ncp, v);
  } else if constexpr (P::LINEAR) {
    s = fabs(A.p.a[d]);
  } else {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
    s = smax;
  }
  double* out = A.phi + phi_off + f * (long long)(NPHI * NF * NV);
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    const int jp = lane + 32 * r;
    if (jp < NF) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const double G = 0.5 * (FL[r][v] + FR_[r][v]) - 0.5 * s * (qR[r][v] - qL[r][v]);
        if constexpr (P::NCPS) {
          // shallow water: the path-conservative fluctuation along the straight segment from qL
          // to qR, int_0^1 g h(z) dz (dh + db) on the momentum of direction d (3-point rule)
          double half = 0.0;
          if (v == 1 + d) {
            const double dh = qR[r][0] - qL[r][0], dhb = dh + (qR[r][3] - qL[r][3]);
            double fl = 0.0;
#pragma unroll
            for (int gq = 0; gq < 3; ++gq) fl = fma(T.pw[gq], A.p.grav * fma(T.pz[gq], dh, qL[r][0]) * dhb, fl);
            half = 0.5 * fl;
          }
          out[jp * NV + v] = G + half;
          out[NF * NV + jp * NV + v] = G - half;
        } else if constexpr (P::NCP) {
          // source variable of row v of B_d, chosen among the three compile-time candidates (the
          // direction d is a run-time value: no dynamic register indexing)
          const int s0 = Elastic::src(0, v), s1 = Elastic::src(1, v), s2 = Elastic::src(2, v);
          const double j0 = s0 >= 0 ? qR[r][s0 < 0 ? 0 : s0] - qL[r][s0 < 0 ? 0 : s0] : 0.0;
          const double j1 = s1 >= 0 ? qR[r][s1 < 0 ? 0 : s1] - qL[r][s1 < 0 ? 0 : s1] : 0.0;
          const double j2 = s2 >= 0 ? qR[r][s2 < 0 ? 0 : s2] - qL[r][s2 < 0 ? 0 : s2] : 0.0;
          const double jump = d == 0 ? j0 : (d == 1 ? j1 : j2);
          const double half = 0.5 * cb[v] * jump;
          out[jp * NV + v] = G + half;
          out[NF * NV + jp * NV + v] = G - half;
        } else {
          out[jp * NV + v] = G;
        }
      }
    }
  }
}

// One warp per face (all lanes of the warp take part).
template <class P, int D, int N>
__global__ void __launch_bounds__(128) k_riemann(const __grid_constant__ StepArgs A,
                                                 const __grid_constant__ Tables T, int d,
                                                 long long phi_off) {
  riemann_face<P, D, N>(A, T, d, phi_off, (long long)blockIdx.x * 4 + (threadIdx.x >> 5),
                        threadIdx.x & 31);
}

// Faces with few nodes (NF <= 16): FPW faces per warp, one lane per (face, node), so that the
// FP64 speed evaluations and flux combinations fill the warp (an FP64 instruction costs the
// whole warp's pipe time, whatever its active lanes).  The node-by-node path of riemann_face
// with the same arithmetic; the face's speed is the maximum over its NF lanes.  For the FP64
// form of the nonlinear conservative systems (Euler, shallow water: no face speeds from the
// predictor).
template <class P, int D, int N>
struct RiemannPack {
  static constexpr int NF = Cfg<P, D, N>::NF;
  static constexpr int FPW = NF <= 16 ? 32 / NF : 1;
  static constexpr bool USE = P::CONS && !P::LINEAR && !P::NCP && FPW >= 2;
};

template <class P, int D, int N>
__global__ void __launch_bounds__(128) k_riemann_packed(const __grid_constant__ StepArgs A,
                                                        const __grid_constant__ Tables T, int d,
                                                        long long phi_off) {
  using C = Cfg<P, D, N>;
  constexpr int NV = C::NV, NF = C::NF, FR = C::FR, NPHI = C::NPHI;
  constexpr int FPW = RiemannPack<P, D, N>::FPW;
  const int lane = threadIdx.x & 31;
  const int slot = lane / NF, jp = lane - slot * NF;
  const Geometry& g = A.g;
  const int nd = g.n[d];
  const long long nfaces = (long long)(nd + 1) * FaceIdx::ntrans(g, d);
  const long long f = ((long long)blockIdx.x * 4 + (threadIdx.x >> 5)) * FPW + slot;
  const bool periodic = (g.bc[d][0] == BC_PERIODIC);
  bool on = slot < FPW && f < nfaces;
  int kf = 0;
  long long tr = 0;
  if (on) {
    kf = (int)(f % (nd + 1));
    tr = f / (nd + 1);
    if (periodic && kf == nd) on = false;  // duplicate of face 0
  }
  double qL[NV], qR[NV], FL[NV], FRv[NV];
  double sp = 0.0;
  if (on) {
    long long cL = -1, cR = -1;
    if (kf > 0) cL = FaceIdx::cell_of(g, tr, d, kf - 1);
    else if (periodic) cL = FaceIdx::cell_of(g, tr, d, nd - 1);
    if (kf < nd) cR = FaceIdx::cell_of(g, tr, d, kf);
    else if (periodic) cR = FaceIdx::cell_of(g, tr, d, 0);
    const double* recL = cL >= 0 ? A.face + cL * (long long)(D * 2 * FR) + (d * 2 + 1) * FR : nullptr;
    const double* recR = cR >= 0 ? A.face + cR * (long long)(D * 2 * FR) + (d * 2 + 0) * FR : nullptr;
    const double* a = recL ? recL : recR;
    const double* b = recR ? recR : recL;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      qL[v] = a[jp * NV + v];
      qR[v] = b[jp * NV + v];
      FL[v] = a[NF * NV + jp * NV + v];
      FRv[v] = b[NF * NV + jp * NV + v];
    }
    // ghost states and speeds with a compile-time direction (the states stay in registers)
#pragma unroll
    for (int dd = 0; dd < D; ++dd) {
      if (dd != d) continue;
      if (!recL) ghost<P>(g.bc[dd][0], dd, qL, FL);
      if (!recR) ghost<P>(g.bc[dd][1], dd, qR, FRv);
      sp = fmax(P::speed(qL, A.p, dd), P::speed(qR, A.p, dd));
    }
  }
  // the face's speed: the maximum over its NF lanes (every lane takes part in the shuffles)
  double s = 0.0;
  const int base = (slot < FPW ? slot : 0) * NF;
#pragma unroll
  for (int k = 0; k < NF; ++k) s = fmax(s, __shfl_sync(0xffffffffu, sp, base + k));
  if (!on) return;
  double* out = A.phi + phi_off + f * (long long)(NPHI * NF * NV);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const double G = 0.5 * (FL[v] + FRv[v]) - 0.5 * s * (qR[v] - qL[v]);
    if constexpr (P::NCPS) {
      // the path-conservative fluctuation of the shallow water equations, as in riemann_face
      double half = 0.0;
      if (v == 1 + d) {
        const double dh = qR[0] - qL[0], dhb = dh + (qR[3] - qL[3]);
        double fl = 0.0;
#pragma unroll
        for (int gq = 0; gq < 3; ++gq) fl = fma(T.pw[gq], A.p.grav * fma(T.pz[gq], dh, qL[0]) * dhb, fl);
        half = 0.5 * fl;
      }
      out[jp * NV + v] = G + half;
      out[NF * NV + jp * NV + v] = G - half;
    } else {
      out[jp * NV + v] = G;
    }
  }
}

// Corrector, face part of Eq. (6) in strong form:
//   u_j -= dt sum_d [ (e1_{j_d}/(w_{j_d} h_d)) Phi_L(right face) - (e0_{j_d}/(w_{j_d} h_d)) Phi_R(left face) ]
// One degree of freedom e of the context; sw = {dt e0/(w h), dt e1/(w h)} of the context.
template <class P, int D, int N>
__device__ __forceinline__ void corrector_dof(const StepArgs& A, const double (*sw)[3][N + 1],
                                              long long off1, long long off2, long long e) {
  using C = Cfg<P, D, N>;
  constexpr int n = C::n, NV = C::NV, NL = C::NL, NF = C::NF, NPHI = C::NPHI;
  const unsigned c = (unsigned)(e / NL);
  const int l = (int)(e - (long long)c * NL);
  const int j = l / NV, v = l - (l / NV) * NV;
  const unsigned n0 = A.g.n[0], n1 = A.g.n[1];
  const unsigned i0 = c % n0, r0 = c / n0, i1 = r0 % n1, i2 = r0 / n1;
  double un = A.u_next[e];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const int st = (d == 0 ? 1 : (d == 1 ? n : n * n));
    const int jd = (j / st) % n;
    const int jp = (j % st) + (j / (st * n)) * st;
    const unsigned id = d == 0 ? i0 : (d == 1 ? i1 : i2);
    const unsigned tr = d == 0 ? i1 + n1 * i2 : (d == 1 ? i0 + n0 * i2 : i0 + n0 * i1);
    const unsigned nd = A.g.n[d];
    unsigned kr = id + 1;
    if (kr == nd && A.g.bc[d][1] == BC_PERIODIC) kr = 0;
    const long long off = d == 0 ? 0 : (d == 1 ? off1 : off2);
    const long long fr = kr + (long long)(nd + 1) * tr;
    const long long fl = id + (long long)(nd + 1) * tr;
    const double PhiL = A.phi[off + fr * (NPHI * NF * NV) + jp * NV + v];
    const double PhiR = A.phi[off + fl * (NPHI * NF * NV) + (NPHI - 1) * NF * NV + jp * NV + v];
    un = fma(-sw[1][d][jd], PhiL, un);
    un = fma(sw[0][d][jd], PhiR, un);
  }
  if constexpr (P::NCP) {
    // The elastic wave speeds come from the material alone, so the CFL kernel does not read the
    // state: the new state is checked here, where it is written (exponent bits, integer pipe;
    // the status word is read before its atomic, so a flood of non-finite values stays cheap).
    if (((__double2hiint(un) >> 20) & 0x7ff) == 0x7ff &&
        !(*(volatile const int*)&A.dev->status & ST_NONFINITE))
      atomicOr(&A.dev->status, ST_NONFINITE);
  }
  A.u_next[e] = un;
}

template <class P, int D, int N>
__global__ void __launch_bounds__(256) k_corrector(const __grid_constant__ StepArgs A,
                                                   const __grid_constant__ Tables T,
                                                   long long off1, long long off2) {
  using C = Cfg<P, D, N>;
  constexpr int n = C::n;
  // dt e0 / (w h_d) and dt e1 / (w h_d) once per block (the row j_d differs between lanes)
  __shared__ double sw[2][3][n];
  if (threadIdx.x < 2 * D * n) {
    const int k = threadIdx.x / (D * n), d = (threadIdx.x / n) % D, m = threadIdx.x % n;
    sw[k][d][m] = A.dev->dt * (k ? A.cw1[d][m] : A.cw0[d][m]);
  }
  __syncthreads();
  const long long e = (long long)blockIdx.x * 256 + threadIdx.x;
  if (e >= A.g.ncells * C::NL) return;
  corrector_dof<P, D, N>(A, sw, off1, off2, e);
}

// Max signal speed of the state (Eq. (7)); NaN / Inf latches ST_NONFINITE.  Euler: one FP64
// division and one square root per node for all directions, on the nodes that the binary32
// enclosures cannot rule out.
template <class P, int D, int N>
__global__ void __launch_bounds__(256) k_cfl(const __grid_constant__ StepArgs A) {
  using C = Cfg<P, D, N>;
  constexpr int NS = C::NS, NV = C::NV;
  double lmax = 0.0;
  bool bad = false;
  if constexpr (P::NCP) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < A.g.ncells;
         i += (long long)gridDim.x * blockDim.x) {
      const double s = Elastic::vp(A.mat[i * 3], A.mat[i * 3 + 1], A.mat[i * 3 + 2]);
      if (!(s >= 0.0) || isinf(s)) bad = true;
      else lmax = fmax(lmax, s);
    }
    // the state's finiteness: checked by the corrector as it writes each new state (a
    // non-finite value of u^n reaches u^{n+1} through the update u^n + dt (...))
  } else if constexpr (P::LINEAR) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < A.g.ncells * NS;
         i += (long long)gridDim.x * blockDim.x) {
      const double* q = A.u + i * NV;
      double s = 0.0;
#pragma unroll
      for (int d = 0; d < D; ++d) s = fmax(s, P::speed(q, A.p, d));
      if (!isfinite(q[0])) bad = true;
      lmax = fmax(lmax, s);
    }
  } else if (A.cfl_filter) {
    // The FP64 maximum, evaluated in FP64 only where it can occur.  Each node
    // gets a binary32 enclosure [lo, hi] of its speed (rounding of the state to binary32 and of
    // every operation bounded, with a factor-4 margin); a device-wide running lower bound of the
    // maximum (the largest lo seen) rules out nodes with hi below it.  The remaining candidates
    // of a tile are queued in shared memory and evaluated by speed_all in FP64 by the first lanes.
    // Non-finite or non-admissible states are always candidates.
    constexpr int TPN = 4;  // nodes per thread and tile
    __shared__ int qn;
    __shared__ long long qidx[256 * TPN];
    __shared__ float tlo[8];
    const float gam = (float)A.p.gamma, g1 = (float)(A.p.gamma - 1.0);
    const float ep = 4.0f * 0x1p-24f;  // four units of binary32 rounding
    const long long total = A.g.ncells * NS;
    const long long tile = (long long)blockDim.x * TPN;
    for (long long base = (long long)blockIdx.x * tile; base < total; base += (long long)gridDim.x * tile) {
      if (threadIdx.x == 0) qn = 0;
      float lo[TPN], hi[TPN];
      bool cand[TPN];
      float wlo = 0.f;
#pragma unroll
      for (int r = 0; r < TPN; ++r) {
        const long long i = base + r * (long long)blockDim.x + threadIdx.x;
        cand[r] = false;
        lo[r] = hi[r] = 0.f;
        if (i < total) {
          const double* q = A.u + i * NV;
          float f[NV];
          bool ok = true;
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            ok = ok && ((__double2hiint(q[v]) & 0x7ff00000) != 0x7ff00000);
            f[v] = __double2float_rn(q[v]);
          }
          ok = ok && (f[0] > 0.f);
          const float ir = __frcp_rn(f[0]);
          float j2 = 0.f, vm = 0.f;
#pragma unroll
          for (int d = 0; d < D; ++d) {
            j2 = fmaf(f[1 + d], f[1 + d], j2);
            vm = fmaxf(vm, fabsf(f[1 + d]));
          }
          const float ke = 0.5f * j2 * ir;
          const float ei = fmaf(-0.5f * j2, ir, f[NV - 1]);
          const float dei = 3.0f * ep * (fabsf(f[NV - 1]) + ke) + ep * fabsf(ei);
          const float p = g1 * ei;
          const float dp = g1 * dei + 2.0f * ep * fabsf(p);
          const float c2 = gam * p * ir;
          const float dc2 = gam * ir * dp + 2.0f * ep * fabsf(c2);
          const float vs = vm * ir;
          const float clo = sqrtf(fmaxf(c2 - dc2, 0.f)) * (1.0f - ep);
          const float chi = sqrtf(fmaxf(c2 + dc2, 0.f)) * (1.0f + ep);
          float l = (vs * (1.0f - 2.0f * ep) + clo) * (1.0f - ep);
          hi[r] = (vs * (1.0f + 2.0f * ep) + chi) * (1.0f + ep);
          ok = ok && (l >= 0.f) && (hi[r] < INFINITY);  // false also for NaN
          if (!ok) l = 0.f;
          lo[r] = l;
          cand[r] = !ok;
          wlo = fmaxf(wlo, l);
        }
      }
      // raise the device-wide lower bound when this tile's largest lo exceeds it
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) wlo = fmaxf(wlo, __shfl_xor_sync(0xffffffffu, wlo, o));
      if ((threadIdx.x & 31) == 0) tlo[threadIdx.x >> 5] = wlo;
      __syncthreads();
      if (threadIdx.x == 0) {
        float m = tlo[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, tlo[w]);
        if (m > __uint_as_float(*(volatile unsigned*)&A.dev->lam_lo_bits))
          atomicMax(&A.dev->lam_lo_bits, __float_as_uint(m));  // non-negative: bits are monotone
      }
      const float thr = __uint_as_float(*(volatile unsigned*)&A.dev->lam_lo_bits);
#pragma unroll
      for (int r = 0; r < TPN; ++r) {
        const long long i = base + r * (long long)blockDim.x + threadIdx.x;
        if (i < total && (cand[r] || !(hi[r] < thr))) qidx[atomicAdd(&qn, 1)] = i;
      }
      __syncthreads();
      for (int k = threadIdx.x; k < qn; k += blockDim.x) {
        const double* q = A.u + qidx[k] * NV;
        double sum = 0.0;
#pragma unroll
        for (int v = 0; v < NV; ++v) sum += q[v];
        const double sp = P::speed_all(q, A.p);
        if (!isfinite(sum) || !(sp >= 0.0) || isinf(sp)) bad = true;
        else lmax = fmax(lmax, sp);
      }
      __syncthreads();
    }
  } else {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < A.g.ncells * NS;
         i += (long long)gridDim.x * blockDim.x) {
      const double* q = A.u + i * NV;
      double sum = 0.0;
#pragma unroll
      for (int v = 0; v < NV; ++v) sum += q[v];
      const double s = P::speed_all(q, A.p);
      if (!isfinite(sum) || !(s >= 0.0) || isinf(s)) bad = true;
      else lmax = fmax(lmax, s);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
  bad = __any_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&A.dev->lam_bits, (unsigned long long)__double_as_longlong(lmax));
    if (bad) atomicOr(&A.dev->status, ST_NONFINITE);
  }
}

// ---- launchers ----------------------------------------------------------------------------
template <class P, int D, int N>
cudaError_t launch_predictor_n(const StepArgs& a, const Tables& t, cudaStream_t s) {
  using C = Cfg<P, D, N>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_predictor<P, D, N>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (a.g.ncells > 0x7fffffffLL) return cudaErrorInvalidValue;
  k_predictor<P, D, N><<<(unsigned)a.g.ncells, C::TPB, C::SMEM, s>>>(a, t);
  return cudaGetLastError();
}

template <class P, int D, int N>
cudaError_t launch_riemann_n(const StepArgs& a, const Tables& t, cudaStream_t s) {
  using C = Cfg<P, D, N>;
  long long off = 0;
  for (int d = 0; d < D; ++d) {
    const long long nf = (long long)(a.g.n[d] + 1) * (a.g.ncells / a.g.n[d]);
    if constexpr (RiemannPack<P, D, N>::USE) {
      if (!a.fspeed) {
        constexpr int FPB = 4 * RiemannPack<P, D, N>::FPW;  // faces per block
        k_riemann_packed<P, D, N><<<(unsigned)((nf + FPB - 1) / FPB), 128, 0, s>>>(a, t, d, off);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        off += nf * (long long)(C::NPHI * C::NF * C::NV);
        continue;
      }
    }
    const long long blocks = (nf + 3) / 4;
    k_riemann<P, D, N><<<(unsigned)blocks, 128, 0, s>>>(a, t, d, off);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    off += nf * (long long)(C::NPHI * C::NF * C::NV);
  }
  return cudaSuccess;
}

template <class P, int D, int N>
cudaError_t launch_corrector_n(const StepArgs& a, const Tables& t, cudaStream_t s) {
  using C = Cfg<P, D, N>;
  long long offs[3] = {0, 0, 0};
  long long off = 0;
  for (int d = 0; d < D; ++d) {
    offs[d] = off;
    off += (long long)(a.g.n[d] + 1) * (a.g.ncells / a.g.n[d]) * (C::NPHI * C::NF * C::NV);
  }
  const long long tot = a.g.ncells * C::NL;
  k_corrector<P, D, N><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(a, t, offs[1], offs[2]);
  return cudaGetLastError();
}

template <class P, int D, int N>
cudaError_t launch_cfl_n(const StepArgs& a, cudaStream_t s) {
  k_cfl<P, D, N><<<152 * 8, 256, 0, s>>>(a);
  return cudaGetLastError();
}

#define ADER_DISPATCH_N(FN, ...)                      \
  switch (a.g.order) {                                \
    case 1: return FN<P, D, 1>(__VA_ARGS__);          \
    case 2: return FN<P, D, 2>(__VA_ARGS__);          \
    case 3: return FN<P, D, 3>(__VA_ARGS__);          \
    case 4: return FN<P, D, 4>(__VA_ARGS__);          \
    case 5: return FN<P, D, 5>(__VA_ARGS__);          \
    case 6: return FN<P, D, 6>(__VA_ARGS__);          \
    default: return cudaErrorInvalidValue;            \
  }

template <class P, int D>
struct FamilyImpl {
  static cudaError_t cfl(const StepArgs& a, cudaStream_t s) { ADER_DISPATCH_N(launch_cfl_n, a, s) }
  static cudaError_t predictor(const StepArgs& a, const Tables& t, const TablesF& f, int prec,
                               cudaStream_t s);
  static cudaError_t riemann(const StepArgs& a, const Tables& t, cudaStream_t s) {
    ADER_DISPATCH_N(launch_riemann_n, a, t, s)
  }
  static cudaError_t corrector(const StepArgs& a, const Tables& t, cudaStream_t s) {
    ADER_DISPATCH_N(launch_corrector_n, a, t, s)
  }
  static size_t smem(int order, int prec);
  static const Family* get() {
    static const Family f = [] {
      Family g{};  // hooks a family does not have stay null
      g.nvar = P::NV;
      g.conservative = P::CONS;
      g.cfl = &cfl;
      g.predictor = &predictor;
      g.riemann = &riemann;
      g.corrector = &corrector;
      g.predictor_smem = &smem;
      g.nphi = Cfg<P, D, 1>::NPHI;
      return g;
    }();
    return &f;
  }
};

}  // namespace ader
#include "kernels_mixed.cuh"
namespace ader {

template <class P, int D>
size_t FamilyImpl<P, D>::smem(int order, int prec) {
#define ADER_SMEM_CASE(NN) \
  case NN: return prec == 1 ? CfgM<P, D, NN>::SMEM : Cfg<P, D, NN>::SMEM;
  if constexpr (P::NCPS) prec = 0;  // FP64 only
  switch (order) {
    ADER_SMEM_CASE(1)
    ADER_SMEM_CASE(2)
    ADER_SMEM_CASE(3)
    ADER_SMEM_CASE(4)
    ADER_SMEM_CASE(5)
    ADER_SMEM_CASE(6)
  }
#undef ADER_SMEM_CASE
  return 0;
}

template <class P, int D>
cudaError_t FamilyImpl<P, D>::predictor(const StepArgs& a, const Tables& t, const TablesF& f,
                                        int prec, cudaStream_t s) {
  if constexpr (!P::NCPS) {
    if (prec == 1) {
      ADER_DISPATCH_N(launch_predictor_mixed_n, a, t, f, s)
    }
  }
  ADER_DISPATCH_N(launch_predictor_n, a, t, s)
}

}  // namespace ader
