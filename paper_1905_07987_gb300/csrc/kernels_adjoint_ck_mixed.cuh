// Mixed-precision adjoint of the linear-elastic step with the Cauchy-Kowalevski predictor: the
// recursion of k_adj_cell_ck (kernels_adjoint_ck.cuh) with the split of the mixed forward
// predictor (kernels_ck.cuh), for contexts whose forward step is mixed.
//
// With B = F + dt L^T lambda the adjoint of a_k is
//   mu_k = (B + dt L^T mu_{k+1}) / (k+1),   k = N..0,   mu_{N+1} = 0,   lambda^n = lambda + mu_0.
// Only B carries the size of lambda; it is formed once, in float-float (L^T applied to lambda's
// float-float records, F from the FP64 face adjoints).  dt L^T mu_{k+1} is O(CFL^2) of lambda and
// runs in binary32 on binary32 records of mu; mu_k itself is float-float (B plus that term), and
// lambda^n = lambda + mu_0 is formed in FP64.  The forward recursion is the mixed predictor's:
// L u and a_1 in float-float, a_2 .. a_N and L a_N in binary32, qbar = u + dbar and its face
// extrapolations in float-float (the forward face data, written in FP64).
// Material gradient sum_k f_k (lambda + mu_{k+1})^T (dL/dm) a_k, from P_k = f_k L a_k at the node:
// level 0 (O(CFL) of the state) in float-float from a_1 and lambda + mu_1; levels k >= 1
// (O(CFL^(k+1))) in binary32; the material factors and the sums in FP64.  Moment gradient (the source cell only) in
// FP64.  Relative to the FP64 adjoint the binary32 terms leave about 1e-7 CFL^2 of lambda per step.
//
// Layout per cell (shared memory): the float-float record U ([NS][10] (hi, lo) pairs: u, then
// qbar, then lambda with its stress sum in the tenth pair, then mu_0), the binary32 records of
// a_1 .. a_N and two binary32 records of mu ([NS][12] floats, the stress sum in the tenth);
// after the recursions the a records hold the per-node gradient terms for the fixed-order sums.
#pragma once
#include "kernels_adjoint_ck.cuh"

namespace ader {

template <int N>
struct CfgCKAM {
  static constexpr int n = N + 1;
  static constexpr int NS = n * n * n;
  static constexpr int NV = 9;
  static constexpr int NL = NS * NV;
  static constexpr int NVQ = 10;  // float-float record: 10 (hi, lo) pairs
  static constexpr int NVF = 12;  // binary32 record: 12 floats (float4 loads)
  static constexpr int CPB = NS >= 96 ? 1 : 128 / NS;
  static constexpr int TPB = (CPB * NS + 31) / 32 * 32;
  // resident blocks per SM: 4 at 128 threads (128 registers, a few spilled, measured faster than
  // 3 blocks without spills), 2 at order 5
  static constexpr int MINB = TPB <= 128 ? 4 : 2;
  static constexpr int NF = n * n;
  static constexpr size_t RECF = (size_t)NS * NVF * 4;  // bytes of one binary32 record
  static constexpr size_t OFF_A = (size_t)NS * NVQ * 8; // a_1 .. a_N
  static constexpr size_t OFF_M = OFF_A + (size_t)N * RECF;  // mu records
  static constexpr size_t CELL = OFF_M + 2 * RECF;
  static constexpr size_t SRC_OFF = CPB * CELL;          // g of the source cell, float-float
  static constexpr size_t SMEM = SRC_OFF + (size_t)NS * 6 * 8;
  static_assert(CELL - OFF_A >= (size_t)9 * NS * 8, "gradient staging fits the binary32 records");
};

// Float-float Out[col] += (L^T Y)[j][col] (Y: float-float records, Y[.][9] = Y_3 + Y_4 + Y_5);
// D2[m][i] = (hi, lo) of D[m][i].  The transpose of ck_apply_ff, as ck_apply_T is of ck_apply.
template <int N>
__device__ __forceinline__ void ck_apply_T_ff(const float2* Y, int j, const float2* D2,
                                              const ff (&cf)[3][4], ff (&Out)[9]) {
  constexpr int n = N + 1, NVQ = CfgCKAM<N>::NVQ;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int st = d == 0 ? 1 : (d == 1 ? n : n * n);
    const int jd = (j / st) % n;
    const float2* b = Y + (j - jd * st) * NVQ;
    constexpr int va_[3] = {6, 6, 7}, vb_[3] = {7, 8, 8};
    const int va = va_[d], vb = vb_[d];
    ff t0 = {0.f, 0.f}, t1 = {0.f, 0.f}, t2 = {0.f, 0.f}, tsum = {0.f, 0.f}, tdd = {0.f, 0.f},
       tsa = {0.f, 0.f}, tsb = {0.f, 0.f};
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
      const float2 c = D2[m * n + jd];
      ff_mac(t0, c.x, c.y, r[0].x, r[0].y);
      ff_mac(t1, c.x, c.y, r[1].x, r[1].y);
      ff_mac(t2, c.x, c.y, r[2].x, r[2].y);
      ff_mac(tsum, c.x, c.y, r[9].x, r[9].y);
      ff_mac(tdd, c.x, c.y, r[3 + d].x, r[3 + d].y);
      ff_mac(tsa, c.x, c.y, r[va].x, r[va].y);
      ff_mac(tsb, c.x, c.y, r[vb].x, r[vb].y);
    }
    ff_mac(Out[Elastic::sig(0, d)], cf[d][0].h, cf[d][0].l, t0.h, t0.l);
    ff_mac(Out[Elastic::sig(1, d)], cf[d][0].h, cf[d][0].l, t1.h, t1.l);
    ff_mac(Out[Elastic::sig(2, d)], cf[d][0].h, cf[d][0].l, t2.h, t2.l);
    // (lam + 2 mu) tdd + lam (tsum - tdd) = lam tsum + 2 mu tdd
    ff_mac(Out[d], cf[d][2].h, cf[d][2].l, tsum.h, tsum.l);
    ff_mac(Out[d], 2.f * cf[d][3].h, 2.f * cf[d][3].l, tdd.h, tdd.l);
    ff_mac(Out[Elastic::src(d, va)], cf[d][3].h, cf[d][3].l, tsa.h, tsa.l);
    ff_mac(Out[Elastic::src(d, vb)], cf[d][3].h, cf[d][3].l, tsb.h, tsb.l);
  }
}

// Binary32 Out[col] += (L^T Y)[j][col] (Y: binary32 records, Y[.][9] = Y_3 + Y_4 + Y_5).
template <int N>
__device__ __forceinline__ void ck_apply_T_f(const float* Y, int j, const float2* D2,
                                             const ff (&cf)[3][4], float (&Out)[9]) {
  constexpr int n = N + 1, NVF = CfgCKAM<N>::NVF;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int st = d == 0 ? 1 : (d == 1 ? n : n * n);
    const int jd = (j / st) % n;
    const float* b = Y + (j - jd * st) * NVF;
    constexpr int va_[3] = {6, 6, 7}, vb_[3] = {7, 8, 8};
    const int va = va_[d], vb = vb_[d];
    float t0 = 0.f, t1 = 0.f, t2 = 0.f, tsum = 0.f, tdd = 0.f, tsa = 0.f, tsb = 0.f;
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
      const float c = D2[m * n + jd].x;
      t0 = fmaf(c, r[0], t0);
      t1 = fmaf(c, r[1], t1);
      t2 = fmaf(c, r[2], t2);
      tsum = fmaf(c, r[9], tsum);
      tdd = fmaf(c, r[3 + d], tdd);
      tsa = fmaf(c, r[va], tsa);
      tsb = fmaf(c, r[vb], tsb);
    }
    Out[Elastic::sig(0, d)] = fmaf(cf[d][0].h, t0, Out[Elastic::sig(0, d)]);
    Out[Elastic::sig(1, d)] = fmaf(cf[d][0].h, t1, Out[Elastic::sig(1, d)]);
    Out[Elastic::sig(2, d)] = fmaf(cf[d][0].h, t2, Out[Elastic::sig(2, d)]);
    Out[d] = fmaf(cf[d][2].h, tsum, fmaf(2.f * cf[d][3].h, tdd, Out[d]));
    Out[Elastic::src(d, va)] = fmaf(cf[d][3].h, tsa, Out[Elastic::src(d, va)]);
    Out[Elastic::src(d, vb)] = fmaf(cf[d][3].h, tsb, Out[Elastic::src(d, vb)]);
  }
}

// Binary32 form of ck_dmat_R: the three sums of nu^T (dL/d(rho, lam, mu)) a before the material
// factors, g[0] = sum_i nu_i P_i, g[1] = theta (nu_3 + nu_4 + nu_5) with theta = (P_3 + P_4 +
// P_5) ik, g[2] = sum nu_v P_v - lam theta (nu_3 + nu_4 + nu_5) over the stress rows.
__device__ __forceinline__ void ck_dmat_R_f(const float (&P)[9], const float (&nu)[9], float lam,
                                            float ik, float (&g)[3]) {
  g[0] = fmaf(nu[0], P[0], fmaf(nu[1], P[1], nu[2] * P[2]));
  const float theta = (P[3] + P[4] + P[5]) * ik;
  const float nsum = nu[3] + nu[4] + nu[5];
  g[1] = theta * nsum;
  float s = fmaf(nu[3], P[3], fmaf(nu[4], P[4], nu[5] * P[5]));
  s = fmaf(-lam * theta, nsum, s);
  g[2] = fmaf(nu[6], P[6], fmaf(nu[7], P[7], fmaf(nu[8], P[8], s)));
}

// Float-float form of ck_dmat_R_f (the level-0 pairing, O(CFL) of the state).
__device__ __forceinline__ void ck_dmat_R_ff(const ff (&P)[9], const ff (&nu)[9], ff lam, ff ik,
                                             ff (&g)[3]) {
  g[0] = {0.f, 0.f};
#pragma unroll
  for (int i = 0; i < 3; ++i) ff_mac(g[0], nu[i].h, nu[i].l, P[i].h, P[i].l);
  const ff theta = ff_mul(ff_add(ff_add(P[3], P[4]), P[5]), ik);
  const ff nsum = ff_add(ff_add(nu[3], nu[4]), nu[5]);
  g[1] = ff_mul(theta, nsum);
  ff s = {0.f, 0.f};
#pragma unroll
  for (int v = 3; v < 9; ++v) ff_mac(s, nu[v].h, nu[v].l, P[v].h, P[v].l);
  const ff lt = ff_mul(lam, g[1]);
  g[2] = ff_sub(s, lt);
}

template <int N>
__global__ void __launch_bounds__(CfgCKAM<N>::TPB, CfgCKAM<N>::MINB)
    k_adj_cell_ck_mixed(const __grid_constant__ StepArgs A, const __grid_constant__ AdjArgs J,
                        const __grid_constant__ Tables T, const __grid_constant__ TablesF F) {
  using C = CfgCKAM<N>;
  constexpr int n = C::n, NS = C::NS, NV = C::NV, NL = C::NL, CPB = C::CPB, TPB = C::TPB;
  constexpr int NVQ = C::NVQ, NVF = C::NVF, NF = C::NF, FR = NF * NV;
  extern __shared__ __align__(16) unsigned char smem_am[];  // [CPB][CELL] + g
  __shared__ ff s_cf[CPB][3][4];
  __shared__ double s_mat[CPB][4];  // 1/rho, lam, 1/(3 lam + 2 mu), 1/mu
  __shared__ ff s_skf[n], s_sbarf;
  __shared__ double s_sk[n], s_sbar;
  __shared__ int s_slot;
  __shared__ float2 s_D[n * n];
  __shared__ double s_sum[CPB][9];
  const int tid = threadIdx.x;
  const int slot = tid / NS;
  const int j = tid - slot * NS;
  const long long c0 = (long long)blockIdx.x * CPB;
  const int ncb = (int)(A.g.ncells - c0 < CPB ? A.g.ncells - c0 : CPB);
  const bool act = slot < ncb;
  const long long c = c0 + slot;
  unsigned char* cell = smem_am + (size_t)(act ? slot : 0) * C::CELL;
  float2* U = reinterpret_cast<float2*>(cell);
  float* Arec = reinterpret_cast<float*>(cell + C::OFF_A);  // a_k at Arec + (k - 1) NS NVF
  float* M0 = reinterpret_cast<float*>(cell + C::OFF_M);
  float* M1 = M0 + NS * NVF;
  const double dt = A.dev->dt;
  const double tn = A.dev->t;

  // the block's cells, coalesced, split into float-float records
  for (int e = tid; e < ncb * NL; e += TPB) {
    const int s = e / NL, r = e - s * NL;
    const ff x = ff_split_int(J.u_n[c0 * NL + e]);
    reinterpret_cast<float2*>(smem_am + (size_t)s * C::CELL)[(r / NV) * NVQ + r % NV] =
        make_float2(x.h, x.l);
  }
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
    s_mat[tid][0] = irho;
    s_mat[tid][1] = lam;
    s_mat[tid][2] = 1.0 / (3.0 * lam + 2.0 * mu);
    s_mat[tid][3] = 1.0 / mu;
  }
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
      s_sk[k] = s;
    }
    s_sbarf = ff_split(sbar);
    s_sbar = sbar;
    s_slot = (int)sc;
  }
  float2* gsrc = reinterpret_cast<float2*>(smem_am + C::SRC_OFF);
  for (int i = tid; i < (srcb ? NS * 6 : 0); i += TPB) {
    const ff g = ff_split(-A.src.M[i % 6] * A.src.phi[i / 6]);
    gsrc[i] = make_float2(g.h, g.l);
  }
  if (tid < n * n) s_D[tid] = make_float2(F.Dh[tid / n][tid % n], F.Dl[tid / n][tid % n]);
  __syncthreads();
  const bool srcc = srcb && act && s_slot == slot;

  ff cf[3][4];
  const ff dtf = ff_split_int(dt);
  ff a1[NV], uj[NV];
  if (act) {
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int i = 0; i < 4; ++i) cf[d][i] = s_cf[slot][d][i];
    // a_1 = dt (L u + g s_0) in float-float; its hi part is the binary32 record of level 1
    ff LU[NV];
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
      a1[v] = ff_mul(dtf, t0);
      Arec[j * NVF + v] = a1[v].h;
      const float2 uu = U[j * NVQ + v];
      uj[v] = {uu.x, uu.y};
    }
  }
  __syncthreads();

  // a_2 .. a_N in binary32 (each kept in its record); their share of dbar in binary32
  float d32[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) d32[v] = 0.f;
#pragma unroll 1
  for (int k = 1; k < N; ++k) {
    if (act) {
      float R[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) R[v] = 0.f;
      ck_apply_f<N>(Arec + (k - 1) * NS * NVF, j, s_D, cf, R);
      if (srcc) {
#pragma unroll
        for (int v = 3; v < NV; ++v) R[v] = fmaf(gsrc[j * 6 + v - 3].x, s_skf[k].h, R[v]);
      }
      const float f = dtf.h * (1.0f / (k + 1));
      const float wk = 1.0f / (k + 2);
      float* o = Arec + k * NS * NVF + j * NVF;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const float a = f * R[v];
        d32[v] = fmaf(wk, a, d32[v]);
        o[v] = a;
      }
    }
    __syncthreads();
  }
  // P_N = f_N L a_N at this node (binary32); qbar = u + dbar (float-float) into U (each thread
  // writes its own node; U was last read by the neighbours before the barriers above)
  float PN[NV];
  if (act) {
#pragma unroll
    for (int v = 0; v < NV; ++v) PN[v] = 0.f;
    ck_apply_f<N>(Arec + (N - 1) * NS * NVF, j, s_D, cf, PN);
    const float fN = dtf.h * (1.0f / (N + 1));
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      PN[v] *= fN;
      const ff db = ff_add({0.5f * a1[v].h, 0.5f * a1[v].l}, {d32[v], 0.f});
      const ff q = ff_add(uj[v], db);
      U[j * NVQ + v] = make_float2(q.h, q.l);
    }
  }
  __syncthreads();
  // forward face data: qbar extrapolated in float-float to both ends of every direction
  for (int e = tid; e < ncb * NF * NV; e += TPB) {
    const int s = e / (NF * NV), r = e - s * (NF * NV);
    const int v = r % NV, jp = r / NV;
    const float2* Us = reinterpret_cast<const float2*>(smem_am + (size_t)s * C::CELL);
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
  __syncthreads();
  // lambda^{n+1} into U (float-float, coalesced), then each node's stress sum into its tenth pair
  for (int e = tid; e < ncb * NL; e += TPB) {
    const int s = e / NL, r = e - s * NL;
    const ff x = ff_split_int(J.lam[c0 * NL + e]);
    reinterpret_cast<float2*>(smem_am + (size_t)s * C::CELL)[(r / NV) * NVQ + r % NV] =
        make_float2(x.h, x.l);
  }
  __syncthreads();
  ff lj[NV], Fj[NV];
  if (act) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const float2 x = U[j * NVQ + v];
      lj[v] = {x.x, x.y};
    }
    const ff ls = ff_add(ff_add(lj[3], lj[4]), lj[5]);
    U[j * NVQ + 9] = make_float2(ls.h, ls.l);
    // F: the face adjoints carried back to the nodes, in float-float
#pragma unroll
    for (int v = 0; v < NV; ++v) Fj[v] = {0.f, 0.f};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int st = d == 0 ? 1 : (d == 1 ? n : n * n);
      const int jd = (j / st) % n;
      const int jp = (j % st) + (j / (st * n)) * st;
      const double* af = J.adjf + (c * 3 + d) * 2 * (long long)(NF * NV) + jp * NV;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const ff x0 = ff_split_int(af[v]), x1 = ff_split_int(af[NF * NV + v]);
        ff_mac(Fj[v], F.e0h[jd], F.e0l[jd], x0.h, x0.l);
        ff_mac(Fj[v], F.e1h[jd], F.e1l[jd], x1.h, x1.l);
      }
    }
  }
  __syncthreads();

  // ---- B = F + dt L^T lambda; level N; mu_N ----------------------------------------------
  double gm[3] = {0.0, 0.0, 0.0}, gM[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  const double irho = act ? s_mat[slot][0] : 0.0, lamd = act ? s_mat[slot][1] : 0.0;
  const double ikd = act ? s_mat[slot][2] : 0.0, imud = act ? s_mat[slot][3] : 0.0;
  const float lamf = (float)lamd, ikf = (float)ikd;
  const ff lamff = ff_split(lamd), ikff = ff_split(ikd);
  const double phi = srcc ? A.src.phi[j] : 0.0;
  ff B[NV], mu_c[NV];  // mu_c: mu_{k+1} at this node
  if (act) {
    ff LT[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) LT[v] = {0.f, 0.f};
    ck_apply_T_ff<N>(U, j, s_D, cf, LT);
#pragma unroll
    for (int v = 0; v < NV; ++v) B[v] = ff_add(Fj[v], ff_mul(dtf, LT[v]));
    // level N: f_N lambda^T (dL/dm) a_N
    float nu[NV], g[3];
#pragma unroll
    for (int v = 0; v < NV; ++v) nu[v] = lj[v].h;
    ck_dmat_R_f(PN, nu, lamf, ikf, g);
    gm[0] = -irho * (double)g[0];
    gm[1] = (double)g[1];
    gm[2] = imud * (double)g[2];
    if (srcc) {
#pragma unroll
      for (int a = 0; a < 6; ++a) gM[a] = -phi * dt * s_sbar * ff_to_d(lj[3 + a]);
    }
    const float iN = 1.0f / (N + 1);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      mu_c[v] = ff_mulf(B[v], iN);
      M0[j * NVF + v] = mu_c[v].h;
    }
    M0[j * NVF + 9] = mu_c[3].h + mu_c[4].h + mu_c[5].h;
  }
  __syncthreads();

  // ---- reverse recursion ---------------------------------------------------------------------
#pragma unroll 1
  for (int k = N - 1; k >= 0; --k) {
    const float* Min = ((N - 1 - k) & 1) ? M1 : M0;  // mu_{k+1}
    float* Mout = ((N - 1 - k) & 1) ? M0 : M1;       // mu_k
    if (act) {
      const double f = dt * (1.0 / (k + 1));
      // material: f_k (lambda + mu_{k+1})^T (dL/dm) a_k
      if (k == 0) {
        // float-float from a_1 and lambda + mu_1, the material factors in FP64
        ff P[NV], nu[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          P[v] = a1[v];
          nu[v] = ff_add(lj[v], mu_c[v]);
        }
        if (srcc) {
          const ff fs0 = ff_mul(dtf, s_skf[0]);  // f_0 s_0
#pragma unroll
          for (int a = 0; a < 6; ++a) {
            const float2 g = gsrc[j * 6 + a];
            P[3 + a] = ff_sub(P[3 + a], ff_mul(fs0, {g.x, g.y}));
          }
        }
        ff g[3];
        ck_dmat_R_ff(P, nu, lamff, ikff, g);
        gm[0] = fma(-irho, ff_to_d(g[0]), gm[0]);
        gm[1] += ff_to_d(g[1]);
        gm[2] = fma(imud, ff_to_d(g[2]), gm[2]);
      } else {
        float P[NV], nu[NV], g[3];
        const float* ak = Arec + k * NS * NVF + j * NVF;  // a_{k+1}
        const float fs = (float)(f * s_sk[k]);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          P[v] = ak[v];
          nu[v] = lj[v].h + mu_c[v].h;
        }
        if (srcc) {
#pragma unroll
          for (int a = 0; a < 6; ++a) P[3 + a] = fmaf(-fs, gsrc[j * 6 + a].x, P[3 + a]);
        }
        ck_dmat_R_f(P, nu, lamf, ikf, g);
        gm[0] = fma(-irho, (double)g[0], gm[0]);
        gm[1] += (double)g[1];
        gm[2] = fma(imud, (double)g[2], gm[2]);
      }
      // moment: f_k s_k mu_{k+1}^T (dg/dM)
      if (srcc) {
#pragma unroll
        for (int a = 0; a < 6; ++a) gM[a] = fma(-phi * f * s_sk[k], ff_to_d(mu_c[3 + a]), gM[a]);
      }
      // mu_k = (B + dt L^T mu_{k+1}) / (k+1)
      float Tt[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) Tt[v] = 0.f;
      ck_apply_T_f<N>(Min, j, s_D, cf, Tt);
      const float ik1 = 1.0f / (k + 1);
#pragma unroll
      for (int v = 0; v < NV; ++v) mu_c[v] = ff_mulf(ff_add(B[v], {dtf.h * Tt[v], 0.f}), ik1);
      if (k > 0) {
        float* o = Mout + j * NVF;
#pragma unroll
        for (int v = 0; v < NV; ++v) o[v] = mu_c[v].h;
        o[9] = mu_c[3].h + mu_c[4].h + mu_c[5].h;
      }
    }
    if (k > 0) __syncthreads();
  }
  // lambda^n = lambda^{n+1} + mu_0 (+ dJ/du^n) in FP64; mu_0 staged in U for a coalesced store
  __syncthreads();
  if (act) {
#pragma unroll
    for (int v = 0; v < NV; ++v) U[j * NVQ + v] = make_float2(mu_c[v].h, mu_c[v].l);
  }
  __syncthreads();
  bool bad = false;
  for (int e = tid; e < ncb * NL; e += TPB) {
    const int s = e / NL, r = e - s * NL;
    const float2 m =
        reinterpret_cast<const float2*>(smem_am + (size_t)s * C::CELL)[(r / NV) * NVQ + r % NV];
    double out = J.lam[c0 * NL + e] + (f2d_int(m.x) + f2d_int(m.y));
    if (J.dJdu) out += J.dJdu[c0 * NL + e];
    J.lam[c0 * NL + e] = out;
    bad |= !isfinite(out);
  }
  if (bad) atomicOr(&A.dev->status, ST_NONFINITE);

  // ---- gradients: per-node partial sums -> fixed-order sums per cell -------------------------
  // staged as doubles over the binary32 records (a_k last read at level 1, mu at level 0)
  double* red = reinterpret_cast<double*>(cell + C::OFF_A);
  if (act) {
#pragma unroll
    for (int q = 0; q < 3; ++q) red[q * NS + j] = gm[q];
    if (srcc)
#pragma unroll
      for (int q = 0; q < 6; ++q) red[(3 + q) * NS + j] = gM[q];
  }
  __syncthreads();
  for (int q = j; act && q < (srcc ? 9 : 3); q += NS) {
    double s = 0.0;
    for (int i = 0; i < NS; ++i) s += red[q * NS + i];
    s_sum[slot][q] = s;
  }
  __syncthreads();
  if (act && j == 0) {
    for (int q = 0; q < 3; ++q) J.grad_mat[c * 3 + q] += s_sum[slot][q];
    if (!isfinite(s_sum[slot][0]) || !isfinite(s_sum[slot][1]) || !isfinite(s_sum[slot][2]))
      atomicOr(&A.dev->status, ST_NONFINITE);
    if (srcc)
      for (int q = 0; q < 6; ++q) J.grad_M[q] += s_sum[slot][3 + q];
  }
}

template <int N>
cudaError_t adj_run_ck_mixed_n(const StepArgs& a, const AdjArgs& j, const Tables& t,
                               const TablesF& f, cudaStream_t s);

template <int N>
struct AdjLaunchCKM {
  static cudaError_t run(const StepArgs& a, const AdjArgs& j, const Tables& t, const TablesF& f,
                         cudaStream_t s) {
    using C = CfgCKAM<N>;
    static bool attr = false;
    if (!attr) {
      cudaError_t e = cudaFuncSetAttribute(k_adj_cell_ck_mixed<N>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)C::SMEM);
      if (e != cudaSuccess) return e;
      attr = true;
    }
    long long offs[3] = {0, 0, 0}, off = 0;
    for (int d = 0; d < 3; ++d) {
      offs[d] = off;
      off += (long long)(a.g.n[d] + 1) * (a.g.ncells / a.g.n[d]);
    }
    cudaError_t e0 = launch_adj_proj<N>(a, j, t, s);
    if (e0 != cudaSuccess) return e0;
    for (int d = 0; d < 3; ++d) {
      cudaError_t e = launch_adj_riemann<N, 1>(a, j, t, d, offs[d], s);
      if (e != cudaSuccess) return e;
    }
    const long long blocks = (a.g.ncells + C::CPB - 1) / C::CPB;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_adj_cell_ck_mixed<N><<<(unsigned)blocks, C::TPB, C::SMEM, s>>>(a, j, t, f);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    for (int d = 0; d < 3; ++d) {
      e = launch_adj_riemann<N, 2>(a, j, t, d, offs[d], s);
      if (e != cudaSuccess) return e;
    }
    k_adj_face_sum<N><<<(unsigned)((a.g.ncells + 255) / 256), 256, 0, s>>>(a, j, offs[1], offs[2]);
    return cudaGetLastError();
  }
};

}  // namespace ader
