// Mixed-precision space-time predictor (the "precision" pattern grown onto Eq. (5)).
//
// The predictor is solved for the increment dq = q - u^n, which is O(dt) small:
//   dq^{r+1} = dt Kw [ B0 + dR(dq^r) ],   B0 = R(u^n),   dR(dq) = R(u^n + dq) - R(u^n)
// B0 and every term that carries the O(1) size of the solution (the flux F(u^n), its derivative,
// the face extrapolations of u^n and F(u^n)) are formed in FP64 or in float-float (hi + lo pairs
// of binary32 with error-free transformations, about 44 significant bits) on the FP32 pipe; the
// Picard iterations, the flux increments F(u+dq) - F(u) (written so that no O(1) terms cancel)
// and their contractions run in binary32.  The corrector, Riemann solver, CFL condition and
// pressure / sound speed of the face states stay FP64 (other kernels).  Rounding in binary32
// therefore perturbs only O(dt) increments: relative error ~1e-7 of the per-step change.
#pragma once
#include "kernels.cuh"

namespace ader {

struct ff {
  float h, l;
};

__device__ __forceinline__ ff ff_split(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double ff_to_d(ff a) { return (double)a.h + (double)a.l; }

// acc += (ah + al) * (bh + bl): exact product of the high parts by FMA, cross terms, two-sum.
__device__ __forceinline__ void ff_mac(ff& acc, float ah, float al, float bh, float bl) {
  const float p = ah * bh;
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  const float s = acc.h + p;
  const float bv = s - acc.h;
  const float err = (acc.h - (s - bv)) + (p - bv);
  acc.h = s;
  acc.l = acc.l + (err + e);
}

// Per-node FP32 base data of the Euler increments.
template <int D>
struct EulerBase {
  float rho, E, p, j[D], v[D];
};

template <class P, int D, int N>
struct CfgM {
  using C = Cfg<P, D, N>;
  static constexpr int n = C::n, NS = C::NS, NST = C::NST, NV = C::NV, NL = C::NL;
  static constexpr int NF = C::NF, FR = C::FR, TPB = C::TPB, LPT = C::LPT, NPT = C::NPT;
  static constexpr int NPS = (NS + TPB - 1) / TPB;
  static constexpr bool EULER = P::CONS && !P::LINEAR;
  static constexpr int BW = EULER ? 2 * D + 3 : 1;
  static constexpr int FS = P::CONS ? cmax(n, D + 1) : 0;
  static constexpr size_t B_FB0 = P::CONS ? (size_t)D * NL * sizeof(ff) : 0;
  static constexpr size_t B_UFF = (size_t)NL * sizeof(ff);
  static constexpr size_t B_BF = EULER ? (size_t)NS * BW * sizeof(float) : 0;
  static constexpr size_t B_DQ = (size_t)n * NL * sizeof(float);
  static constexpr size_t B_DF = (size_t)FS * NL * sizeof(float);
  static constexpr size_t SMEM = B_FB0 + B_UFF + B_BF + B_DQ + B_DF;
};

// Flux increment F_d(u + dq) - F_d(u) in binary32 from the node's base data.
template <class P, int D>
struct Incr;

template <int D>
struct Incr<Euler<D>, D> {
  static constexpr int NV = D + 2;
  struct Aux {
    float dv[D], dp;
  };
  __device__ static void aux(const EulerBase<D>& b, const float* dq, float gm1, Aux& a) {
    const float irq = 1.0f / (b.rho + dq[0]);
    float djv = 0.f;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      a.dv[i] = (dq[1 + i] - b.v[i] * dq[0]) * irq;
      djv = fmaf(dq[1 + i], b.v[i] + a.dv[i], fmaf(b.j[i], a.dv[i], djv));
    }
    a.dp = gm1 * (dq[NV - 1] - 0.5f * djv);
  }
  __device__ static void flux(const EulerBase<D>& b, const float* dq, const Aux& a, int d, float* F) {
    const float vd = b.v[d] + a.dv[d];
    F[0] = dq[1 + d];
#pragma unroll
    for (int i = 0; i < D; ++i) F[1 + i] = fmaf(dq[1 + i], vd, b.j[i] * a.dv[d]);
    F[1 + d] += a.dp;
    F[NV - 1] = fmaf(dq[NV - 1] + a.dp, vd, (b.E + b.p) * a.dv[d]);
  }
};

template <class M, int d, class P, int D>
__device__ __forceinline__ void dflux_nodes(const float* dqs, const float* bf, const PdeParams& pp,
                                            float* dFs, int tid) {
  constexpr int NV = M::NV, NS = M::NS;
#pragma unroll
  for (int k = 0; k < M::NPT; ++k) {
    const int node = tid + k * M::TPB;
    if (node < M::NST) {
      float q[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) q[v] = dqs[node * NV + v];
      float F[NV];
      if constexpr (M::EULER) {
        const int j = node % NS;
        EulerBase<D> b;
        const float* s = bf + j * M::BW;
        b.rho = s[0];
        b.E = s[1];
        b.p = s[2];
#pragma unroll
        for (int i = 0; i < D; ++i) {
          b.j[i] = s[3 + i];
          b.v[i] = s[3 + D + i];
        }
        typename Incr<P, D>::Aux a;
        Incr<P, D>::aux(b, q, (float)(pp.gamma - 1.0), a);
        Incr<P, D>::flux(b, q, a, d, F);
      } else {
        F[0] = (float)pp.a[d] * q[0];
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) dFs[node * NV + v] = F[v];
    }
  }
}

// R[k][t] += coef * sum_m D[j_d][m] X[t][(j, j_d -> m)][src]  in binary32
template <class M, int d, bool NCP>
__device__ __forceinline__ void contract_f(const float* X, const TablesF& T, float coef, double irho,
                                           double lam, double mu, float (&R)[M::LPT][M::n], int tid) {
  constexpr int n = M::n, NV = M::NV, NL = M::NL, TPB = M::TPB, st = ipow(n, d);
#pragma unroll
  for (int k = 0; k < M::LPT; ++k) {
    const int l = tid + k * TPB;
    if (l < NL) {
      const int j = l / NV, v = l - (l / NV) * NV;
      int s = v;
      float c = coef;
      if constexpr (NCP) {
        s = Elastic::src(d, v);
        if (s < 0) continue;
        c = (float)(-Elastic::coef_ir(d, v, irho, lam, mu)) * coef;
      }
      const int jd = digit<n, d>(j);
      const int j0 = j - jd * st;
#pragma unroll
      for (int t = 0; t < n; ++t) {
        float acc = 0.f;
#pragma unroll
        for (int m = 0; m < n; ++m) acc = fmaf(T.Dh[jd][m], X[t * NL + (j0 + m * st) * NV + s], acc);
        R[k][t] = fmaf(c, acc, R[k][t]);
      }
    }
  }
}

template <class P, int D, int N>
__global__ void __launch_bounds__(Cfg<P, D, N>::TPB)
    k_predictor_mixed(const __grid_constant__ StepArgs A, const __grid_constant__ Tables T,
                      const __grid_constant__ TablesF F) {
  using M = CfgM<P, D, N>;
  constexpr int n = M::n, NS = M::NS, NV = M::NV, NL = M::NL, TPB = M::TPB, LPT = M::LPT;
  constexpr int NF = M::NF, FR = M::FR;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ff* FB0 = reinterpret_cast<ff*>(smem_raw);                        // [D][NL] F_d(u)/h_d
  ff* uff = reinterpret_cast<ff*>(smem_raw + M::B_FB0);             // [NL]
  float* bf = reinterpret_cast<float*>(smem_raw + M::B_FB0 + M::B_UFF);  // [NS][BW]
  float* dqs = reinterpret_cast<float*>(smem_raw + M::B_FB0 + M::B_UFF + M::B_BF);  // [n][NL]
  float* dFs = dqs + n * NL;                                         // [FS][NL]
  const long long c = blockIdx.x;
  const int tid = threadIdx.x;
  const double dt = A.dev->dt;
  const float dtf = (float)dt;
  const double tn = A.dev->t;
  const double* u = A.u + c * NL;

  double irho = 0.0, lam = 0.0, mu = 0.0;
  if constexpr (P::NCP) {
    irho = 1.0 / A.mat[c * 3 + 0];
    lam = A.mat[c * 3 + 1];
    mu = A.mat[c * 3 + 2];
  }
  const bool has_src = (A.src.cell == c);
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
  if constexpr (P::CONS) {
#pragma unroll
    for (int k = 0; k < M::NPS; ++k) {
      const int j = tid + k * TPB;
      if (j < NS) {
        double q[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) q[v] = u[j * NV + v];
        typename P::Aux ax;
        P::aux(q, A.p, ax);
#pragma unroll
        for (int d = 0; d < D; ++d) {
          double Fd[NV];
          P::flux(q, ax, A.p, d, Fd);
#pragma unroll
          for (int v = 0; v < NV; ++v) FB0[d * NL + j * NV + v] = ff_split(Fd[v] * A.g.inv_h[d]);
        }
        if constexpr (M::EULER) {
          float* s = bf + j * M::BW;
          s[0] = (float)q[0];
          s[1] = (float)q[NV - 1];
          s[2] = (float)ax.p;
#pragma unroll
          for (int i = 0; i < D; ++i) {
            s[3 + i] = (float)q[1 + i];
            s[3 + D + i] = (float)(q[1 + i] * ax.ir);
          }
        }
      }
    }
  }
  __syncthreads();

  // B0 (strong form, binary32 for the iterations) and the weak-form volume base (FP64).
  float b0f[LPT];
  double b0vol[LPT];
#pragma unroll
  for (int k = 0; k < LPT; ++k) {
    const int l = tid + k * TPB;
    b0f[k] = 0.f;
    b0vol[k] = 0.0;
    if (l < NL) {
      const int j = l / NV, v = l - (l / NV) * NV;
      ff aS = {0.f, 0.f}, aW = {0.f, 0.f};
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const int st = (d == 0 ? 1 : (d == 1 ? n : n * n));
        const int jd = (j / st) % n;
        const int j0 = j - jd * st;
        if constexpr (P::CONS) {
#pragma unroll
          for (int m = 0; m < n; ++m) {
            const ff f = FB0[d * NL + (j0 + m * st) * NV + v];
            ff_mac(aS, F.Dh[jd][m], F.Dl[jd][m], f.h, f.l);
            ff_mac(aW, F.Wh[jd][m], F.Wl[jd][m], f.h, f.l);
          }
        } else {
          const int s = Elastic::src(d, v);
          if (s >= 0) {
            ff g = {0.f, 0.f};
#pragma unroll
            for (int m = 0; m < n; ++m) {
              const ff f = uff[(j0 + m * st) * NV + s];
              ff_mac(g, F.Dh[jd][m], F.Dl[jd][m], f.h, f.l);
            }
            // -(1/h) coef * (D q): scale in FP64 (one multiply per direction)
            b0vol[k] = fma(-A.g.inv_h[d] * Elastic::coef_ir(d, v, irho, lam, mu), ff_to_d(g), b0vol[k]);
          }
        }
      }
      if constexpr (P::CONS) {
        b0f[k] = -(float)ff_to_d(aS);
        b0vol[k] = ff_to_d(aW);
      } else {
        b0f[k] = (float)b0vol[k];
      }
    }
  }

  // ---- Picard iterations on dq (binary32) ----------------------------------------------
  float R[LPT][n];
  for (int it = 0; it < A.iters; ++it) {
#pragma unroll
    for (int k = 0; k < LPT; ++k)
#pragma unroll
      for (int t = 0; t < n; ++t) R[k][t] = 0.f;
    if (it > 0) {
      if constexpr (P::CONS) {
        dflux_nodes<M, 0, P, D>(dqs, bf, A.p, dFs, tid);
        __syncthreads();
        contract_f<M, 0, false>(dFs, F, -(float)A.g.inv_h[0], 0, 0, 0, R, tid);
        __syncthreads();
        dflux_nodes<M, 1, P, D>(dqs, bf, A.p, dFs, tid);
        __syncthreads();
        contract_f<M, 1, false>(dFs, F, -(float)A.g.inv_h[1], 0, 0, 0, R, tid);
        __syncthreads();
        if constexpr (D == 3) {
          dflux_nodes<M, 2, P, D>(dqs, bf, A.p, dFs, tid);
          __syncthreads();
          contract_f<M, 2, false>(dFs, F, -(float)A.g.inv_h[2], 0, 0, 0, R, tid);
        }
      } else {
        contract_f<M, 0, true>(dqs, F, (float)A.g.inv_h[0], irho, lam, mu, R, tid);
        contract_f<M, 1, true>(dqs, F, (float)A.g.inv_h[1], irho, lam, mu, R, tid);
        contract_f<M, 2, true>(dqs, F, (float)A.g.inv_h[2], irho, lam, mu, R, tid);
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
#pragma unroll
        for (int t = 0; t < n; ++t) {
          float acc = F.kw1[t] * b0f[k];
#pragma unroll
          for (int m = 0; m < n; ++m) acc = fmaf(F.Kw[t][m], R[k][m], acc);
          dqs[t * NL + l] = dtf * acc;
        }
      }
    }
    __syncthreads();
  }

  // ---- epilogue --------------------------------------------------------------------------
  float dqb[LPT];
#pragma unroll
  for (int k = 0; k < LPT; ++k) {
    const int l = tid + k * TPB;
    dqb[k] = 0.f;
    if (l < NL) {
#pragma unroll
      for (int t = 0; t < n; ++t) dqb[k] = fmaf(F.w[t], dqs[t * NL + l], dqb[k]);
    }
  }
  float* dqbs;  // time-averaged dq [NL]
  float* dFbs;  // time-averaged flux increments [D][NL]
  if constexpr (P::CONS) {
    float FBv[D][LPT];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      if (d == 0) dflux_nodes<M, 0, P, D>(dqs, bf, A.p, dFs, tid);
      if (d == 1) dflux_nodes<M, 1, P, D>(dqs, bf, A.p, dFs, tid);
      if constexpr (D == 3)
        if (d == 2) dflux_nodes<M, 2, P, D>(dqs, bf, A.p, dFs, tid);
      __syncthreads();
#pragma unroll
      for (int k = 0; k < LPT; ++k) {
        const int l = tid + k * TPB;
        FBv[d][k] = 0.f;
        if (l < NL) {
#pragma unroll
          for (int t = 0; t < n; ++t) FBv[d][k] = fmaf(F.w[t], dFs[t * NL + l], FBv[d][k]);
        }
      }
      __syncthreads();
    }
    dqbs = dFs;
    dFbs = dFs + NL;
#pragma unroll
    for (int k = 0; k < LPT; ++k) {
      const int l = tid + k * TPB;
      if (l < NL) {
        dqbs[l] = dqb[k];
#pragma unroll
        for (int d = 0; d < D; ++d) dFbs[d * NL + l] = FBv[d][k];
      }
    }
  } else {
    dqbs = dqs;
    dFbs = nullptr;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < LPT; ++k) {
      const int l = tid + k * TPB;
      if (l < NL) dqbs[l] = dqb[k];
    }
  }
  __syncthreads();

  double* un = A.u_next + c * NL;
#pragma unroll
  for (int k = 0; k < LPT; ++k) {
    const int l = tid + k * TPB;
    if (l < NL) {
      const int j = l / NV, v = l - (l / NV) * NV;
      float dvol = 0.f;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const int st = (d == 0 ? 1 : (d == 1 ? n : n * n));
        const int jd = (j / st) % n;
        const int j0 = j - jd * st;
        if constexpr (P::CONS) {
          float a = 0.f;
#pragma unroll
          for (int m = 0; m < n; ++m) a = fmaf(F.Wh[jd][m], dFbs[d * NL + (j0 + m * st) * NV + v], a);
          dvol = fmaf((float)A.g.inv_h[d], a, dvol);
        } else {
          const int s = Elastic::src(d, v);
          if (s >= 0) {
            float a = 0.f;
#pragma unroll
            for (int m = 0; m < n; ++m) a = fmaf(F.Dh[jd][m], dqbs[(j0 + m * st) * NV + s], a);
            dvol = fmaf((float)(-A.g.inv_h[d] * Elastic::coef_ir(d, v, irho, lam, mu)), a, dvol);
          }
        }
      }
      double vol = b0vol[k] + (double)dvol;
      if (has_src && v >= 3) {
        double sbar = 0.0;
#pragma unroll
        for (int t = 0; t < n; ++t) sbar = fma(T.w[t], ric[t], sbar);
        vol = fma(-A.src.M[v - 3] * A.src.phi[j], sbar, vol);
      }
      un[l] = fma(dt, vol, ul[k]);
    }
  }

  // ---- face records: FP64-accurate base extrapolation + binary32 increment ----------------
  double* fc = A.face + c * (long long)(D * 2 * FR);
  constexpr int NFE = D * 2 * NF * NV;
  for (int e = tid; e < NFE; e += TPB) {
    const int v = e % NV;
    const int jp = (e / NV) % NF;
    const int side = (e / (NV * NF)) % 2;
    const int d = e / (NV * NF * 2);
    const int st = (d == 0 ? 1 : (d == 1 ? n : n * n));
    const int jbase = (jp % st) + (jp / st) * st * n;
    const float* eh = side ? F.e1h : F.e0h;
    const float* el = side ? F.e1l : F.e0l;
    ff qa = {0.f, 0.f}, fa = {0.f, 0.f};
    float qd = 0.f, fd = 0.f;
#pragma unroll
    for (int m = 0; m < n; ++m) {
      const int jj = jbase + m * st;
      const ff uu = uff[jj * NV + v];
      ff_mac(qa, eh[m], el[m], uu.h, uu.l);
      qd = fmaf(eh[m], dqbs[jj * NV + v], qd);
      if constexpr (P::CONS) {
        const ff f = FB0[d * NL + jj * NV + v];
        ff_mac(fa, eh[m], el[m], f.h, f.l);
        fd = fmaf(eh[m], dFbs[d * NL + jj * NV + v], fd);
      }
    }
    double* rec = fc + (d * 2 + side) * FR;
    rec[jp * NV + v] = ff_to_d(qa) + (double)qd;
    if constexpr (P::CONS) rec[NF * NV + jp * NV + v] = ff_to_d(fa) * A.g.h[d] + (double)fd;
  }
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
