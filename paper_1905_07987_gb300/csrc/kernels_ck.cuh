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
//
// Mixed-precision form (k_predictor_ck_mixed): only the O(1) base term L u carries the size of the
// solution; it is formed once in float-float (hi + lo binary32 pairs, about 44 bits) and serves
// both a_1 = dt (L u + g s_0) and the volume term.  a_1 is float-float; a_2 .. a_N (O(dt^2) and
// smaller) and L applied to the increment of the time average run in binary32.  The time average
// qbar = u + dbar (dbar = a_1/2 in float-float plus the binary32 sum of the higher terms), its
// face extrapolations and the volume term L u + L dbar + g sbar are float-float, and
// u_next = u + dt vol is formed in FP64.  The FP64 pipe, 1/64 of the FP32 rate, would otherwise
// be the bound: the splits of u into float-float and the exact float -> double conversions of
// the results run on the integer pipe, leaving one FP64 add per face value and an add and an FMA
// per updated value.
#pragma once
#include "ader_internal.h"
#include "ff.cuh"
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
  // + the point source's spatial factor g [NS][6] of the source cell
  static constexpr size_t SMEM = ((size_t)CPB * 2 * REC + (size_t)NS * 6) * sizeof(double);
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

// The CPB cells from c0 of one context (one block); the kernel below and the ensemble's
// persistent kernel call it.
template <int N>
__device__ __forceinline__ void predictor_ck_block(const StepArgs& A, const Tables& T,
                                                   long long c0) {
  using C = CfgCK<N>;
  constexpr int n = C::n, NS = C::NS, NV = C::NV, NL = C::NL, NVP = C::NVP, CPB = C::CPB;
  constexpr int TPB = C::TPB, REC = C::REC, NF = C::NF, FR = NF * NV;
  extern __shared__ __align__(16) double smem[];  // [CPB][2][NS][NVP]
  const int tid = threadIdx.x;
  const int slot = tid / NS;
  const int j = tid - slot * NS;
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
  // g of the source cell's nodes (a loop with no iterations outside the source block: the
  // FP64 products are not issued, predicated off, by every block)
  double* gsrc = smem + (size_t)CPB * 2 * REC;
  for (int i = tid; i < (srcb ? NS * 6 : 0); i += TPB) gsrc[i] = -A.src.M[i % 6] * A.src.phi[i / 6];

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
        for (int v = 3; v < NV; ++v) R[v] = fma(gsrc[j * 6 + v - 3], s_sk[k], R[v]);
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
      for (int v = 3; v < NV; ++v) R[v] = fma(gsrc[j * 6 + v - 3], s_sbar, R[v]);
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

  // face records: qbar extrapolated to both ends of every direction (both ends from one read
  // of the line; the direction loop is unrolled so that every index divisor is a constant)
  for (int e = tid; e < ncb * NF * NV; e += TPB) {
    const int s = e / (NF * NV), r = e - s * (NF * NV);
    const int v = r % NV, jp = r / NV;
    const double* Xs = smem + (size_t)s * 2 * REC + (((N - 1) & 1) ? REC : 0);
    double* fc = A.face + (c0 + s) * (3 * 2 * FR) + jp * NV + v;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int st = (d == 0 ? 1 : (d == 1 ? n : n * n));
      const int jbase = (jp % st) + (jp / st) * st * n;
      double q0 = 0.0, q1 = 0.0;
#pragma unroll
      for (int m = 0; m < n; ++m) {
        const double x = Xs[(jbase + m * st) * NVP + v];
        q0 = fma(T.e0[m], x, q0);
        q1 = fma(T.e1[m], x, q1);
      }
      fc[(d * 2 + 0) * FR] = q0;
      fc[(d * 2 + 1) * FR] = q1;
    }
  }
}

template <int N>
__global__ void __launch_bounds__(CfgCK<N>::TPB) k_predictor_ck(const __grid_constant__ StepArgs A,
                                                               const __grid_constant__ Tables T) {
  predictor_ck_block<N>(A, T, (long long)blockIdx.x * CfgCK<N>::CPB);
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

// ---- mixed precision --------------------------------------------------------------------------

template <int N>
struct CfgCKM {
  static constexpr int n = N + 1;
  static constexpr int NS = n * n * n;
  static constexpr int NV = 9;
  static constexpr int NL = NS * NV;
  static constexpr int NVQ = 10;  // float-float node record: 10 (hi, lo) pairs, 80 bytes
  static constexpr int NVF = 12;  // binary32 node record: 12 floats, 48 bytes (float4 loads)
  static constexpr int CPB = NS >= 96 ? 1 : 128 / NS;
  static constexpr int TPB = (CPB * NS + 31) / 32 * 32;
  static constexpr int MINB = TPB <= 128 ? 4 : (TPB <= 224 ? 3 : 1);  // resident blocks per SM
  static constexpr int NF = n * n;
  // per cell: U (float-float state, then qbar) | A | B (binary32 Taylor coefficients); the
  // float-float volume term is staged over A and B
  static constexpr size_t OFF_A = (size_t)NS * NVQ * 8;
  static constexpr size_t OFF_B = OFF_A + (size_t)NS * NVF * 4;
  static constexpr size_t CELL = OFF_B + (size_t)NS * NVF * 4;
  // + the point source's spatial factor g [NS][6] of the source cell, float-float
  static constexpr size_t SRC_OFF = CPB * CELL;
  static constexpr size_t SMEM = SRC_OFF + (size_t)NS * 6 * 8;
};

// Float-float R[v] += row v of -sum_d (1/h_d) B_d D_d U at node j (U: [NS][NVQ] (hi, lo) pairs).
template <int N>
__device__ __forceinline__ void ck_apply_ff(const float2* U, int j, const float2* D2,
                                            const ff (&cf)[3][4], ff (&R)[9]) {
  constexpr int n = N + 1, NVQ = CfgCKM<N>::NVQ;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int st = d == 0 ? 1 : (d == 1 ? n : n * n);
    const int jd = (j / st) % n;
    const float2* b = U + (j - jd * st) * NVQ;
    const float2* Dr = D2 + jd * n;
    const int s0 = Elastic::sig(0, d), s1 = Elastic::sig(1, d), s2 = Elastic::sig(2, d);
    ff dv[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}}, ds[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
    for (int m = 0; m < n; ++m) {
      const float4* p = reinterpret_cast<const float4*>(b + m * st * NVQ);
      float2 r[NVQ];
#pragma unroll
      for (int i = 0; i < NVQ / 2; ++i) {
        const float4 v = p[i];
        r[2 * i] = make_float2(v.x, v.y);
        r[2 * i + 1] = make_float2(v.z, v.w);
      }
      const float2 c = Dr[m];
      const float ch = c.x, cl = c.y;
#pragma unroll
      for (int i = 0; i < 3; ++i) ff_mac(dv[i], ch, cl, r[i].x, r[i].y);
      ff_mac(ds[0], ch, cl, r[s0].x, r[s0].y);
      ff_mac(ds[1], ch, cl, r[s1].x, r[s1].y);
      ff_mac(ds[2], ch, cl, r[s2].x, r[s2].y);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) ff_mac(R[i], cf[d][0].h, cf[d][0].l, ds[i].h, ds[i].l);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const ff& k = i == d ? cf[d][1] : cf[d][2];
      ff_mac(R[3 + i], k.h, k.l, dv[d].h, dv[d].l);
    }
#pragma unroll
    for (int v = 6; v < 9; ++v) {
      const int s = Elastic::src(d, v);
      if (s >= 0) ff_mac(R[v], cf[d][3].h, cf[d][3].l, dv[s].h, dv[s].l);
    }
  }
}

// Binary32 R[v] += row v of -sum_d (1/h_d) B_d D_d X at node j (X: [NS][NVF] floats).
template <int N>
__device__ __forceinline__ void ck_apply_f(const float* X, int j, const float2* D2,
                                           const ff (&cf)[3][4], float (&R)[9]) {
  constexpr int n = N + 1, NVF = CfgCKM<N>::NVF;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int st = d == 0 ? 1 : (d == 1 ? n : n * n);
    const int jd = (j / st) % n;
    const float* b = X + (j - jd * st) * NVF;
    const float2* Dr = D2 + jd * n;
    const int s0 = Elastic::sig(0, d), s1 = Elastic::sig(1, d), s2 = Elastic::sig(2, d);
    float dv0 = 0.f, dv1 = 0.f, dv2 = 0.f, ds0 = 0.f, ds1 = 0.f, ds2 = 0.f;
#pragma unroll
    for (int m = 0; m < n; ++m) {
      const float4* p = reinterpret_cast<const float4*>(b + m * st * NVF);
      float r[NVF];
#pragma unroll
      for (int i = 0; i < NVF / 4; ++i) {
        const float4 v = p[i];
        r[4 * i] = v.x;
        r[4 * i + 1] = v.y;
        r[4 * i + 2] = v.z;
        r[4 * i + 3] = v.w;
      }
      const float c = Dr[m].x;
      dv0 = fmaf(c, r[0], dv0);
      dv1 = fmaf(c, r[1], dv1);
      dv2 = fmaf(c, r[2], dv2);
      ds0 = fmaf(c, r[s0], ds0);
      ds1 = fmaf(c, r[s1], ds1);
      ds2 = fmaf(c, r[s2], ds2);
    }
    const float dv[3] = {dv0, dv1, dv2};
    R[0] = fmaf(cf[d][0].h, ds0, R[0]);
    R[1] = fmaf(cf[d][0].h, ds1, R[1]);
    R[2] = fmaf(cf[d][0].h, ds2, R[2]);
#pragma unroll
    for (int i = 0; i < 3; ++i) R[3 + i] = fmaf(i == d ? cf[d][1].h : cf[d][2].h, dv[d], R[3 + i]);
#pragma unroll
    for (int v = 6; v < 9; ++v) {
      const int s = Elastic::src(d, v);
      if (s >= 0) R[v] = fmaf(cf[d][3].h, dv[s], R[v]);
    }
  }
}

// The CPB cells from c0 of one context (one block), mixed precision; the kernel below and the
// ensemble's persistent kernel call it.
template <int N>
__device__ __forceinline__ void predictor_ck_mixed_block(const StepArgs& A, const Tables& T,
                                                         const TablesF& F, long long c0) {
  using C = CfgCKM<N>;
  constexpr int n = C::n, NS = C::NS, NV = C::NV, NL = C::NL, CPB = C::CPB, TPB = C::TPB;
  constexpr int NVQ = C::NVQ, NVF = C::NVF, NF = C::NF, FR = NF * NV;
  extern __shared__ __align__(16) unsigned char smem_ck[];  // [CPB][CELL]
  const int tid = threadIdx.x;
  const int slot = tid / NS;
  const int j = tid - slot * NS;
  const int ncb = (int)(A.g.ncells - c0 < CPB ? A.g.ncells - c0 : CPB);
  const bool act = slot < ncb;
  unsigned char* cell = smem_ck + (size_t)(act ? slot : 0) * C::CELL;
  float2* U = reinterpret_cast<float2*>(cell);
  float* XA = reinterpret_cast<float*>(cell + C::OFF_A);
  float* XB = reinterpret_cast<float*>(cell + C::OFF_B);
  float2* V = reinterpret_cast<float2*>(cell + C::OFF_A);  // volume term, over A and B
  const double dt = A.dev->dt;
  const double tn = A.dev->t;

  // the block's cells, coalesced, split into float-float records
  for (int e = tid; e < ncb * NL; e += TPB) {
    const int s = e / NL, r = e - s * NL;
    const ff x = ff_split_int(A.u[c0 * NL + e]);
    reinterpret_cast<float2*>(smem_ck + (size_t)s * C::CELL)[(r / NV) * NVQ + r % NV] =
        make_float2(x.h, x.l);
  }

  // per-cell coefficients {1/(rho h_d), (lam + 2 mu)/h_d, lam/h_d, mu/h_d} in float-float
  __shared__ ff s_cf[CPB][3][4];
  if (tid < ncb) {
    const long long cc = c0 + tid;
    const double irho = 1.0 / A.mat[cc * 3 + 0];
    const double lam = A.mat[cc * 3 + 1];
    const double mu = A.mat[cc * 3 + 2];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double ih = A.g.inv_h[d];
      s_cf[tid][d][0] = ff_split(irho * ih);
      s_cf[tid][d][1] = ff_split((lam + 2.0 * mu) * ih);
      s_cf[tid][d][2] = ff_split(lam * ih);
      s_cf[tid][d][3] = ff_split(mu * ih);
    }
  }
  // point source of the block, as in the FP64 kernel, kept in float-float for the per-node terms
  __shared__ ff s_skf[n], s_sbarf;
  __shared__ int s_slot;
  const long long sc = A.src.cell - c0;
  const bool srcb = sc >= 0 && sc < ncb;
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
      s_skf[k] = ff_split(s);
    }
    s_sbarf = ff_split(sbar);
    s_slot = (int)sc;
  }
  // g of the source cell's nodes in float-float (a loop with no iterations outside the source
  // block: its FP64 products are not issued, predicated off, by every block; the per-node
  // source terms below are FP32 arithmetic)
  float2* gsrc = reinterpret_cast<float2*>(smem_ck + C::SRC_OFF);
  for (int i = tid; i < (srcb ? NS * 6 : 0); i += TPB) {
    const ff g = ff_split(-A.src.M[i % 6] * A.src.phi[i / 6]);
    gsrc[i] = make_float2(g.h, g.l);
  }
  // D as (hi, lo) rows: each lane reads the row of its own node digit
  __shared__ float2 s_D[n * n];
  if (tid < n * n) s_D[tid] = make_float2(F.Dh[tid / n][tid % n], F.Dl[tid / n][tid % n]);
  __syncthreads();
  const bool srcc = srcb && act && s_slot == slot;

  ff cf[3][4];
  ff LU[NV], dbar[NV];
  const ff dtf = ff_split_int(dt);
  if (act) {
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int i = 0; i < 4; ++i) cf[d][i] = s_cf[slot][d][i];
    // base term and a_1 = dt (L u + g s_0) in float-float; dbar starts at a_1 / 2
#pragma unroll
    for (int v = 0; v < NV; ++v) LU[v] = {0.f, 0.f};
    ck_apply_ff<N>(U, j, s_D, cf, LU);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      ff t0 = LU[v];
      if (srcc && v >= 3) {
        const float2 g = gsrc[j * 6 + v - 3];
        t0 = ff_add(t0, ff_mul({g.x, g.y}, s_skf[0]));
      }
      const ff a1 = ff_mul(dtf, t0);
      dbar[v] = {0.5f * a1.h, 0.5f * a1.l};
      XA[j * NVF + v] = a1.h;
    }
  }
  __syncthreads();

  // a_2 .. a_N in binary32; their share of dbar, sum_k a_k / (k+1), in binary32
  float d32[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) d32[v] = 0.f;
#pragma unroll
  for (int k = 1; k < N; ++k) {
    const float* Xc = (k & 1) ? XA : XB;
    float* Xn = (k & 1) ? XB : XA;
    if (act) {
      float R[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) R[v] = 0.f;
      ck_apply_f<N>(Xc, j, s_D, cf, R);
      if (srcc) {
#pragma unroll
        for (int v = 3; v < NV; ++v) R[v] = fmaf(gsrc[j * 6 + v - 3].x, s_skf[k].h, R[v]);
      }
      const float f = dtf.h * (1.0f / (k + 1));
      const float wk = 1.0f / (k + 2);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const float a = f * R[v];
        d32[v] = fmaf(wk, a, d32[v]);
        Xn[j * NVF + v] = a;
      }
    }
    __syncthreads();
  }

  // qbar = u + dbar (float-float, in place: after the base term only the owner reads its node);
  // dbar's hi part into A for the binary32 L dbar
  if (act) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      dbar[v] = ff_add(dbar[v], {d32[v], 0.f});
      const float2 uu = U[j * NVQ + v];
      const ff q = ff_add({uu.x, uu.y}, dbar[v]);
      U[j * NVQ + v] = make_float2(q.h, q.l);
      XA[j * NVF + v] = dbar[v].h;
    }
  }
  __syncthreads();
  ff vol[NV];
  if (act) {
    float R[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) R[v] = 0.f;
    ck_apply_f<N>(XA, j, s_D, cf, R);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      vol[v] = ff_add(LU[v], {R[v], 0.f});
      if (srcc && v >= 3) {
        const float2 g = gsrc[j * 6 + v - 3];
        vol[v] = ff_add(vol[v], ff_mul({g.x, g.y}, s_sbarf));
      }
    }
  }
  __syncthreads();  // every read of A is done before the volume term overwrites it
  if (act) {
#pragma unroll
    for (int v = 0; v < NV; ++v) V[j * NVQ + v] = make_float2(vol[v].h, vol[v].l);
  }
  __syncthreads();

  // u_next = u + dt vol in FP64 (u again from L2), coalesced
  for (int e = tid; e < ncb * NL; e += TPB) {
    const int s = e / NL, r = e - s * NL;
    const float2 w = reinterpret_cast<const float2*>(smem_ck + (size_t)s * C::CELL + C::OFF_A)
        [(r / NV) * NVQ + r % NV];
    A.u_next[c0 * NL + e] = fma(dt, f2d_int(w.x) + f2d_int(w.y), A.u[c0 * NL + e]);
  }

  // face records: qbar extrapolated in float-float to both ends of every direction (both ends
  // from one read of the line; constant index divisors)
  for (int e = tid; e < ncb * NF * NV; e += TPB) {
    const int s = e / (NF * NV), r = e - s * (NF * NV);
    const int v = r % NV, jp = r / NV;
    const float2* Us = reinterpret_cast<const float2*>(smem_ck + (size_t)s * C::CELL);
    double* fc = A.face + (c0 + s) * (3 * 2 * FR) + jp * NV + v;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int st = (d == 0 ? 1 : (d == 1 ? n : n * n));
      const int jbase = (jp % st) + (jp / st) * st * n;
      ff q0 = {0.f, 0.f}, q1 = {0.f, 0.f};
#pragma unroll
      for (int m = 0; m < n; ++m) {
        const float2 q = Us[(jbase + m * st) * NVQ + v];
        ff_mac(q0, F.e0h[m], F.e0l[m], q.x, q.y);
        ff_mac(q1, F.e1h[m], F.e1l[m], q.x, q.y);
      }
      fc[(d * 2 + 0) * FR] = f2d_int(q0.h) + f2d_int(q0.l);
      fc[(d * 2 + 1) * FR] = f2d_int(q1.h) + f2d_int(q1.l);
    }
  }
}

template <int N>
__global__ void __launch_bounds__(CfgCKM<N>::TPB, CfgCKM<N>::MINB)
    k_predictor_ck_mixed(const __grid_constant__ StepArgs A, const __grid_constant__ Tables T,
                         const __grid_constant__ TablesF F) {
  predictor_ck_mixed_block<N>(A, T, F, (long long)blockIdx.x * CfgCKM<N>::CPB);
}

template <int N>
cudaError_t launch_predictor_ck_mixed_n(const StepArgs& a, const Tables& t, const TablesF& f,
                                        cudaStream_t s) {
  using C = CfgCKM<N>;
  static bool attr = false;
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(
        k_predictor_ck_mixed<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const long long blocks = (a.g.ncells + C::CPB - 1) / C::CPB;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  k_predictor_ck_mixed<N><<<(unsigned)blocks, C::TPB, C::SMEM, s>>>(a, t, f);
  return cudaGetLastError();
}

}  // namespace ader
