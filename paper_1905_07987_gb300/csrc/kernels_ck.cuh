// Cauchy-Kowalevski space-time predictor of the linear elastic system (Sec. 2 and Sec. 3.3: the
// predictor of linear PDEs is evaluated directly by the Cauchy-Kowalevski procedure).
//
// The local solution's Taylor series in time about t^n is cut after degree N, and every time
// derivative is the spatial operator applied to the previous one.  With
// q(t^n + tau dt) = sum_{k<=N} a_k tau^k:
//   a_0 = u,   a_{k+1} = dt/(k+1) (L a_k + g s_k),   L a = -sum_d (1/h_d) B_d D_d a,
// where g is the point source's spatial factor and s_k are the monomial coefficients (in tau) of
// the degree-N interpolant of the wavelet through the step's time nodes.  The time average is
// qbar = sum_k a_k / (k+1) (Gauss-Legendre weights integrate tau^k exactly).  The epilogue is
// that of the Picard predictor: the volume term dt (L qbar + g sbar) goes into u_next and qbar
// is extrapolated to the faces.
//
// Cost: N+1 applications of L per cell, against (N+1) iterations over n time nodes for Picard.
// One thread per spatial node (several cells per block at low order).  Along direction d the
// thread forms the six derivatives that the eight non-zero rows of B_d read (the three
// velocities and the stresses sigma_{0d}, sigma_{1d}, sigma_{2d}) and combines them:
// 18n + 24 FMA per node and application.  The Taylor coefficients ping-pong between two
// shared-memory buffers of padded node records, 10 doubles per node, read in 16-byte pairs.
#pragma once
#include "ader_internal.h"
#include "pde.cuh"

namespace ader {

template <int N>
struct CfgCK {
  static constexpr int n = N + 1;
  static constexpr int NS = n * n * n;
  static constexpr int NV = 9;
  static constexpr int NL = NS * NV;
  static constexpr int NVP = 10;                        // padded node record (16-byte pairs)
  static constexpr int CPB = NS >= 96 ? 1 : 128 / NS;   // cells per block
  static constexpr int TPB = (CPB * NS + 31) / 32 * 32;
  static constexpr int NF = n * n;
  static constexpr int REC = NS * NVP;                  // doubles per cell and buffer
  static constexpr size_t SMEM = (size_t)CPB * 2 * REC * sizeof(double);
};

// R[v] += row v of -sum_d (1/h_d) B_d D_d X at node j of the cell record X ([NS][NVP]).
// Dr[d][m] = D[j_d][m];  cf[d] = {1/(rho h_d), (lam + 2 mu)/h_d, lam/h_d, mu/h_d}.
template <int N>
__device__ __forceinline__ void ck_apply(const double* X, int j, const double (&Dr)[3][N + 1],
                                         const double (&cf)[3][4], double (&R)[9]) {
  constexpr int n = N + 1, NVP = CfgCK<N>::NVP;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int st = d == 0 ? 1 : (d == 1 ? n : n * n);
    const int jd = (j / st) % n;
    const double* b = X + (j - jd * st) * NVP;
    // stress components sigma_{id}, i = 0..2
    const int s0 = Elastic::sig(0, d), s1 = Elastic::sig(1, d), s2 = Elastic::sig(2, d);
    double dv0 = 0.0, dv1 = 0.0, dv2 = 0.0, ds0 = 0.0, ds1 = 0.0, ds2 = 0.0;
#pragma unroll
    for (int m = 0; m < n; ++m) {
      const double2* p = reinterpret_cast<const double2*>(b + m * st * NVP);
      double r[NVP];
#pragma unroll
      for (int i = 0; i < NVP / 2; ++i) {
        const double2 v = p[i];
        r[2 * i] = v.x;
        r[2 * i + 1] = v.y;
      }
      const double c = Dr[d][m];
      dv0 = fma(c, r[0], dv0);
      dv1 = fma(c, r[1], dv1);
      dv2 = fma(c, r[2], dv2);
      ds0 = fma(c, r[s0], ds0);
      ds1 = fma(c, r[s1], ds1);
      ds2 = fma(c, r[s2], ds2);
    }
    const double dv[3] = {dv0, dv1, dv2};
    // velocities: (1/rho) d sigma_{id} / dx_d
    R[0] = fma(cf[d][0], ds0, R[0]);
    R[1] = fma(cf[d][0], ds1, R[1]);
    R[2] = fma(cf[d][0], ds2, R[2]);
    // normal stresses: (lam + 2 mu [i == d]) dv_d / dx_d
#pragma unroll
    for (int i = 0; i < 3; ++i) R[3 + i] = fma(i == d ? cf[d][1] : cf[d][2], dv[d], R[3 + i]);
    // shear stresses: mu dv_s / dx_d with s = Elastic::src(d, v)
#pragma unroll
    for (int v = 6; v < 9; ++v) {
      const int s = Elastic::src(d, v);
      if (s >= 0) R[v] = fma(cf[d][3], dv[s], R[v]);
    }
  }
}

template <int N>
__global__ void __launch_bounds__(CfgCK<N>::TPB) k_predictor_ck(const __grid_constant__ StepArgs A,
                                                               const __grid_constant__ Tables T) {
  using C = CfgCK<N>;
  constexpr int n = C::n, NS = C::NS, NV = C::NV, NL = C::NL, NVP = C::NVP, CPB = C::CPB;
  constexpr int TPB = C::TPB, REC = C::REC, NF = C::NF, FR = NF * NV;
  extern __shared__ __align__(16) double smem[];  // [CPB][2][NS][NVP]
  const int tid = threadIdx.x;
  const int slot = tid / NS;
  const int j = tid - slot * NS;
  const long long c0 = (long long)blockIdx.x * CPB;
  const int ncb = (int)(A.g.ncells - c0 < CPB ? A.g.ncells - c0 : CPB);  // cells of this block
  const bool act = slot < ncb;
  const long long c = c0 + slot;
  double* Xa = smem + (size_t)(act ? slot : 0) * 2 * REC;
  double* Xb = Xa + REC;
  const double dt = A.dev->dt;
  const double tn = A.dev->t;

  // the block's cells, coalesced, into the padded records of buffer a
  for (int e = tid; e < ncb * NL; e += TPB) {
    const int s = e / NL, r = e - s * NL;
    smem[(size_t)s * 2 * REC + (r / NV) * NVP + r % NV] = A.u[c0 * NL + e];
  }

  // point source of the block (at most one cell): Taylor coefficients s_k of the wavelet's
  // interpolant, its time average, and the spatial factor g of each node
  __shared__ double s_sk[n], s_sbar;
  __shared__ int s_slot;
  const long long sc = A.src.cell - c0;
  const bool srcb = sc >= 0 && sc < ncb;  // uniform over the block
  if (srcb && tid == 0) {
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
      s_sk[k] = s;
    }
    s_sbar = sbar;
    s_slot = (int)sc;
  }

  double Dr[3][n], cf[3][4];
  double qb[NV];
  if (act) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int jd = d == 0 ? j % n : (d == 1 ? (j / n) % n : j / (n * n));
#pragma unroll
      for (int m = 0; m < n; ++m) Dr[d][m] = T.D[jd][m];
    }
    const double irho = 1.0 / A.mat[c * 3 + 0];
    const double lam = A.mat[c * 3 + 1];
    const double mu = A.mat[c * 3 + 2];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double ih = A.g.inv_h[d];
      cf[d][0] = irho * ih;
      cf[d][1] = (lam + 2.0 * mu) * ih;
      cf[d][2] = lam * ih;
      cf[d][3] = mu * ih;
    }
  }
  __syncthreads();
  const bool srcc = srcb && act && s_slot == slot;  // this thread's cell holds the source
  if (act) {
#pragma unroll
    for (int v = 0; v < NV; ++v) qb[v] = Xa[j * NVP + v];
  }

  // Taylor coefficients a_1 .. a_N; qbar accumulates a_k / (k+1)
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const double* Xc = (k & 1) ? Xb : Xa;
    double* Xn = (k & 1) ? Xa : Xb;
    if (act) {
      double R[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) R[v] = 0.0;
      ck_apply<N>(Xc, j, Dr, cf, R);
      if (srcc) {
#pragma unroll
        for (int v = 3; v < NV; ++v) R[v] = fma(-A.src.M[v - 3] * A.src.phi[j], s_sk[k], R[v]);
      }
      const double f = dt * (1.0 / (k + 1));
      const double wk = 1.0 / (k + 2);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const double a = f * R[v];
        qb[v] = fma(wk, a, qb[v]);
        Xn[j * NVP + v] = a;
      }
    }
    __syncthreads();
  }
  // qbar into the buffer that held a_{N-1} (last read before the final barrier)
  double* Xq = ((N - 1) & 1) ? Xb : Xa;
  double* Xo = ((N - 1) & 1) ? Xa : Xb;
  if (act) {
#pragma unroll
    for (int v = 0; v < NV; ++v) Xq[j * NVP + v] = qb[v];
  }
  __syncthreads();

  // volume term: u_next = u + dt (L qbar + g sbar), staged for a coalesced store (u from L2)
  if (act) {
    double R[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) R[v] = 0.0;
    ck_apply<N>(Xq, j, Dr, cf, R);
    if (srcc) {
#pragma unroll
      for (int v = 3; v < NV; ++v) R[v] = fma(-A.src.M[v - 3] * A.src.phi[j], s_sbar, R[v]);
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) Xo[j * NVP + v] = R[v];
  }
  __syncthreads();
  for (int e = tid; e < ncb * NL; e += TPB) {
    const int s = e / NL, r = e - s * NL;
    const double* Xs = smem + (size_t)s * 2 * REC + (((N - 1) & 1) ? 0 : REC);
    A.u_next[c0 * NL + e] = fma(dt, Xs[(r / NV) * NVP + r % NV], A.u[c0 * NL + e]);
  }

  // face records: qbar extrapolated to both ends of every direction
  constexpr int NFE = 3 * 2 * NF * NV;
  for (int e = tid; e < ncb * NFE; e += TPB) {
    const int s = e / NFE, r = e - s * NFE;
    const int v = r % NV;
    const int jp = (r / NV) % NF;
    const int side = (r / (NV * NF)) % 2;
    const int d = r / (NV * NF * 2);
    const int st = (d == 0 ? 1 : (d == 1 ? n : n * n));
    const int jbase = (jp % st) + (jp / st) * st * n;
    const double* ev = side ? T.e1 : T.e0;
    const double* Xs = smem + (size_t)s * 2 * REC + (((N - 1) & 1) ? REC : 0);
    double qf = 0.0;
#pragma unroll
    for (int m = 0; m < n; ++m) qf = fma(ev[m], Xs[(jbase + m * st) * NVP + v], qf);
    A.face[(c0 + s) * (3 * 2 * FR) + (d * 2 + side) * FR + jp * NV + v] = qf;
  }
}

template <int N>
cudaError_t launch_predictor_ck_n(const StepArgs& a, const Tables& t, cudaStream_t s) {
  using C = CfgCK<N>;
  static bool attr = false;
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(
        k_predictor_ck<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const long long blocks = (a.g.ncells + C::CPB - 1) / C::CPB;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  k_predictor_ck<N><<<(unsigned)blocks, C::TPB, C::SMEM, s>>>(a, t);
  return cudaGetLastError();
}

}  // namespace ader
