// Adjoint of the linear-elastic step with the Cauchy-Kowalevski predictor (Sec. 2, Sec. 3.3).
//
// Per cell the forward predictor is linear in the state, the material and the moment tensor:
//   a_0 = u,   a_{k+1} = f_k (L a_k + g s_k),   f_k = dt / (k+1),   k = 0..N-1,
//   qbar = sum_{k<=N} a_k / (k+1),
// followed by the volume term u + dt (L qbar + g sbar) and the face extrapolations E qbar (the
// same epilogue as the Picard form).  Given lambda (the adjoint of the next state) and F, the
// adjoint of the face extrapolations carried back to the nodes (from k_adj_riemann, shared with
// the Picard adjoint), the adjoint of a_k is
//   mu_k = (F + dt L^T lambda) / (k+1) + f_k L^T mu_{k+1}    (mu_{N+1} = 0),
// and since f_k = dt / (k+1) the volume term and the Taylor recursion merge into one recursion on
// nu_k = lambda + mu_k:
//   mu_k = (F + dt L^T nu_{k+1}) / (k+1),   k = N..0,   nu_{N+1} = lambda,
//   lambda^n = nu_0 (+ dJ/du^n).
// The gradients pair each adjoint with the forward quantity that multiplies the parameter; the
// volume term's dt lambda^T (dL/dm) qbar splits over the levels the same way:
//   material   sum_{k=0..N} f_k nu_{k+1}^T (dL/dm) a_k
//   moment     dt sbar lambda^T (dg/dM) + sum_{k<N} f_k s_k mu_{k+1}^T (dg/dM).
// (dL/dm) a needs no contraction of its own: at a node, L a is the material coefficients times
// ten derivative quantities (velocity rows (1/rho) S_i, normal-stress rows lam theta + 2 mu e_i,
// shear rows mu gamma_v), so the derivatives with respect to (rho, lam, mu) follow from R = L a
// itself: -R_i / rho; theta = sum_i R_{3+i} / (3 lam + 2 mu); 2 e_i = (R_{3+i} - lam theta) / mu;
// gamma_v = R_v / mu.  For k < N, f_k L a_k = a_{k+1} - f_k s_k g is already at hand; L a_N costs
// one application.
//
// The forward face data the face terms' material gradient needs come from this kernel too (qbar
// and its extrapolations, as the predictor forms them): the face adjoints, which need lambda and
// the material only, run before it (k_adj_proj, then k_adj_riemann MODE 1), the face material
// gradients after it (MODE 2), so no forward predictor launch precedes the adjoint.
//
// One thread per node, the cells of a block (several at low order) each keep a_0 .. a_N in
// shared memory ((N+2) padded records of 10 doubles per node; the record of a_0 and a spare one
// hold the adjoint nu during the reverse sweep, the tenth double of a nu record its sum
// nu_3 + nu_4 + nu_5), no global scratch.  Work per node: N+1 applications of L (the forward
// recursion and L a_N) and N+1 of L^T; the Picard adjoint recomputes and reverses N+1 iterations
// over n time nodes.  The gradient sums are reduced in a fixed order (no atomics), so repeated
// runs give identical bits.
#pragma once
#include "kernels_adjoint.cuh"
#include "kernels_ck.cuh"

namespace ader {

template <int N>
struct CfgCKA {
  static constexpr int n = N + 1;
  static constexpr int NS = n * n * n;
  static constexpr int NV = 9;
  static constexpr int NL = NS * NV;
  static constexpr int NVP = 10;
  static constexpr int CPB = NS >= 96 ? 1 : 128 / NS;
  static constexpr int TPB = (CPB * NS + 31) / 32 * 32;
  static constexpr int NF = n * n;
  static constexpr int REC = NS * NVP;
  static constexpr int NBUF = N + 2;  // a_0 (then nu) .. a_N, one more nu buffer
  static constexpr size_t SMEM = (size_t)CPB * NBUF * REC * sizeof(double);
};

// Out[col] += (L^T Y)[j][col] for the adjoint record Y ([NS][NVP], Y[.][9] = Y_3 + Y_4 + Y_5)
// at node j.  DT[d][i] = D[i][j_d] (column j_d of the derivative matrix); cf[d] = {1/(rho h_d),
// (lam + 2 mu)/h_d, lam/h_d, mu/h_d}.  Row by row of L (see ck_apply): velocity row i reads
// sigma_{id}, normal-stress rows read v_d, shear row v reads v_{src(d,v)}; the transpose sends
// each row's adjoint back to that column.
template <int N>
__device__ __forceinline__ void ck_apply_T(const double* Y, int j, const double (&DT)[3][N + 1],
                                           const double (&cf)[3][4], double (&Out)[9]) {
  constexpr int n = N + 1, NVP = CfgCKA<N>::NVP;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int st = d == 0 ? 1 : (d == 1 ? n : n * n);
    const int jd = (j / st) % n;
    const double* b = Y + (j - jd * st) * NVP;
    double t0 = 0.0, t1 = 0.0, t2 = 0.0, tsum = 0.0, tdd = 0.0, tsa = 0.0, tsb = 0.0;
    // the two shear rows with a non-zero entry in direction d
    constexpr int va_[3] = {6, 6, 7}, vb_[3] = {7, 8, 8};
    const int va = va_[d], vb = vb_[d];
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
      const double c = DT[d][m];
      t0 = fma(c, r[0], t0);
      t1 = fma(c, r[1], t1);
      t2 = fma(c, r[2], t2);
      tsum = fma(c, r[9], tsum);
      tdd = fma(c, r[3 + d], tdd);
      tsa = fma(c, r[va], tsa);
      tsb = fma(c, r[vb], tsb);
    }
    Out[Elastic::sig(0, d)] = fma(cf[d][0], t0, Out[Elastic::sig(0, d)]);
    Out[Elastic::sig(1, d)] = fma(cf[d][0], t1, Out[Elastic::sig(1, d)]);
    Out[Elastic::sig(2, d)] = fma(cf[d][0], t2, Out[Elastic::sig(2, d)]);
    Out[d] = fma(cf[d][2], tsum, fma(cf[d][1] - cf[d][2], tdd, Out[d]));
    Out[Elastic::src(d, va)] = fma(cf[d][3], tsa, Out[Elastic::src(d, va)]);
    Out[Elastic::src(d, vb)] = fma(cf[d][3], tsb, Out[Elastic::src(d, vb)]);
  }
}

// gm += nu^T (dL/d(rho, lam, mu)) a at one node, given P = w L a there (any weight w: the result
// carries the same factor).  irho = 1/rho, ik = 1/(3 lam + 2 mu), imu = 1/mu.
__device__ __forceinline__ void ck_dmat_R(const double (&P)[9], const double (&nu)[9], double irho,
                                          double lam, double ik, double imu, double (&gm)[3]) {
  gm[0] = fma(-irho, fma(nu[0], P[0], fma(nu[1], P[1], nu[2] * P[2])), gm[0]);
  const double theta = (P[3] + P[4] + P[5]) * ik;
  const double nsum = nu[3] + nu[4] + nu[5];
  gm[1] = fma(theta, nsum, gm[1]);
  double s = fma(nu[3], P[3], fma(nu[4], P[4], nu[5] * P[5]));
  s = fma(-lam * theta, nsum, s);
  s = fma(nu[6], P[6], fma(nu[7], P[7], fma(nu[8], P[8], s)));
  gm[2] = fma(imu, s, gm[2]);
}

template <int N>
__global__ void __launch_bounds__(CfgCKA<N>::TPB)
    k_adj_cell_ck(const __grid_constant__ StepArgs A, const __grid_constant__ AdjArgs J,
                  const __grid_constant__ Tables T) {
  using C = CfgCKA<N>;
  constexpr int n = C::n, NS = C::NS, NV = C::NV, NL = C::NL, NVP = C::NVP, CPB = C::CPB;
  constexpr int TPB = C::TPB, REC = C::REC, NF = C::NF, NBUF = C::NBUF;
  extern __shared__ __align__(16) double smem[];  // [CPB][NBUF][NS][NVP]
  __shared__ double s_sk[n], s_sbar;
  __shared__ double s_sum[CPB][9];  // per-cell gradient sums (3 material, 6 moment)
  const int tid = threadIdx.x;
  const int slot = tid / NS;
  const int j = tid - slot * NS;
  const long long c0 = (long long)blockIdx.x * CPB;
  const int ncb = (int)(A.g.ncells - c0 < CPB ? A.g.ncells - c0 : CPB);
  const bool act = slot < ncb;
  const long long c = c0 + slot;
  double* base = smem + (size_t)(act ? slot : 0) * NBUF * REC;  // a_k at base + k * REC
  double* const spare = base + (N + 1) * REC;
  const double dt = A.dev->dt;
  const double tn = A.dev->t;

  // the block's cells into a_0, lambda^{n+1} into the spare record (coalesced)
  for (int e = tid; e < ncb * NL; e += TPB) {
    const int s = e / NL, r = e - s * NL;
    const size_t o = (size_t)s * NBUF * REC + (r / NV) * NVP + r % NV;
    smem[o] = J.u_n[c0 * NL + e];
    smem[o + (size_t)(N + 1) * REC] = J.lam[c0 * NL + e];
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
      s_sk[k] = s;
    }
    s_sbar = sbar;
  }
  const bool srcc = srcb && act && sc == slot;  // this thread's cell holds the source
  double Dr[3][n], DT[3][n], cf[3][4];
  double irho = 0.0, lam = 0.0, ik = 0.0, imu = 0.0;
  if (act) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int jd = d == 0 ? j % n : (d == 1 ? (j / n) % n : j / (n * n));
#pragma unroll
      for (int m = 0; m < n; ++m) {
        Dr[d][m] = T.D[jd][m];
        DT[d][m] = T.D[m][jd];
      }
    }
    irho = 1.0 / A.mat[c * 3 + 0];
    lam = A.mat[c * 3 + 1];
    const double mu = A.mat[c * 3 + 2];
    ik = 1.0 / (3.0 * lam + 2.0 * mu);
    imu = 1.0 / mu;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double ih = A.g.inv_h[d];
      cf[d][0] = irho * ih;
      cf[d][1] = (lam + 2.0 * mu) * ih;
      cf[d][2] = lam * ih;
      cf[d][3] = mu * ih;
    }
  }
  // the point source's spatial factor g at this node (stress rows): -M_a phi_j
  const double phi = srcc ? A.src.phi[j] : 0.0;
  double mphi[6];
#pragma unroll
  for (int a = 0; a < 6; ++a) mphi[a] = srcc ? -A.src.M[a] * phi : 0.0;
  __syncthreads();

  // ---- forward recursion: a_1 .. a_N; then P = f_N L a_N at this node ------------------------
#pragma unroll
  for (int k = 0; k < N; ++k) {
    if (act) {
      double R[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) R[v] = 0.0;
      ck_apply<N>(base + k * REC, j, Dr, cf, R);
      if (srcc) {
#pragma unroll
        for (int v = 3; v < NV; ++v) R[v] = fma(mphi[v - 3], s_sk[k], R[v]);
      }
      const double f = dt * (1.0 / (k + 1));
#pragma unroll
      for (int v = 0; v < NV; ++v) base[(k + 1) * REC + j * NVP + v] = f * R[v];
    }
    __syncthreads();
  }
  // forward face data of the step (the predictor's epilogue): qbar = sum_k a_k / (k+1) at this
  // node, summed in the predictor's order, into the record of a_0 (each thread reads and writes
  // its own node only), then extrapolated to both ends of every direction
  if (act) {
    double qb[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) qb[v] = base[j * NVP + v];
#pragma unroll
    for (int k = 1; k <= N; ++k) {
      const double wk = 1.0 / (k + 1);
#pragma unroll
      for (int v = 0; v < NV; ++v) qb[v] = fma(wk, base[k * REC + j * NVP + v], qb[v]);
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) base[j * NVP + v] = qb[v];
  }
  __syncthreads();
  for (int e = tid; e < ncb * NF * NV; e += TPB) {
    const int s = e / (NF * NV), r = e - s * (NF * NV);
    const int v = r % NV, jp = r / NV;
    const double* Xs = smem + (size_t)s * NBUF * REC;
    double* fc = A.face + (c0 + s) * (3 * 2 * NF * NV) + jp * NV + v;
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
      fc[(d * 2 + 0) * NF * NV] = q0;
      fc[(d * 2 + 1) * NF * NV] = q1;
    }
  }
  double P[NV];  // f_k L a_k at this node, for the level being reversed
  double lam_j[NV], Fj[NV];
  if (act) {
#pragma unroll
    for (int v = 0; v < NV; ++v) P[v] = 0.0;
    ck_apply<N>(base + N * REC, j, Dr, cf, P);
    const double fN = dt * (1.0 / (N + 1));
#pragma unroll
    for (int v = 0; v < NV; ++v) P[v] *= fN;
    // lambda at this node; its stress sum into the tenth slot of the record
    double* lr = spare + j * NVP;
#pragma unroll
    for (int v = 0; v < NV; ++v) lam_j[v] = lr[v];
    lr[9] = lam_j[3] + lam_j[4] + lam_j[5];
    // F: the face adjoints carried back to the nodes (transposed extrapolation)
#pragma unroll
    for (int v = 0; v < NV; ++v) Fj[v] = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int st = d == 0 ? 1 : (d == 1 ? n : n * n);
      const int jd = (j / st) % n;
      const int jp = (j % st) + (j / (st * n)) * st;
      const double* af = J.adjf + (c * 3 + d) * 2 * (long long)(NF * NV) + jp * NV;
      const double e0 = T.e0[jd], e1 = T.e1[jd];
#pragma unroll
      for (int v = 0; v < NV; ++v) Fj[v] = fma(e0, af[v], fma(e1, af[NF * NV + v], Fj[v]));
    }
  }
  double gm[3] = {0.0, 0.0, 0.0}, gM[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  if (srcc) {
#pragma unroll
    for (int a = 0; a < 6; ++a) gM[a] = -phi * dt * s_sbar * lam_j[3 + a];
  }
  __syncthreads();  // lambda's stress sums are read by the neighbours below

  // ---- reverse recursion on nu_k = lambda + mu_k ---------------------------------------------
  // nu_{k+1} is read from Yin: the spare record at k = N, then alternately the record of a_0 and
  // the spare one (a_0 is not read after the forward recursion).
  double nu_c[NV];  // nu_{k+1} at this node
#pragma unroll
  for (int v = 0; v < NV; ++v) nu_c[v] = lam_j[v];
#pragma unroll
  for (int k = N; k >= 0; --k) {
    const double* Yin = ((N - k) & 1) ? base : spare;
    double* Yout = ((N - k) & 1) ? spare : base;
    if (act) {
      // material: f_k nu_{k+1}^T (dL/dm) a_k, from P = f_k L a_k at this node
      if (k < N) {
        const double f = dt * (1.0 / (k + 1));
#pragma unroll
        for (int v = 0; v < NV; ++v) P[v] = base[(k + 1) * REC + j * NVP + v];
        if (srcc) {
#pragma unroll
          for (int a = 0; a < 6; ++a) {
            P[3 + a] = fma(-f * s_sk[k], mphi[a], P[3 + a]);
            // moment: f_k s_k mu_{k+1}^T (dg/dM), mu_{k+1} = nu_{k+1} - lambda
            gM[a] = fma(-phi * f * s_sk[k], nu_c[3 + a] - lam_j[3 + a], gM[a]);
          }
        }
      }
      ck_dmat_R(P, nu_c, irho, lam, ik, imu, gm);
      double Tt[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) Tt[v] = 0.0;
      ck_apply_T<N>(Yin, j, DT, cf, Tt);
      const double ik1 = 1.0 / (k + 1);
#pragma unroll
      for (int v = 0; v < NV; ++v) nu_c[v] = fma(fma(dt, Tt[v], Fj[v]), ik1, lam_j[v]);
      if (k > 0) {
        double* o = Yout + j * NVP;
#pragma unroll
        for (int v = 0; v < NV; ++v) o[v] = nu_c[v];
        o[9] = nu_c[3] + nu_c[4] + nu_c[5];
      }
    }
    if (k > 0) __syncthreads();
  }
  // lambda^n = nu_0 (+ dJ/du^n), staged in the record of a_1 for a coalesced store (a_1 is last
  // read at level 0, before the barrier below)
  __syncthreads();
  if (act) {
#pragma unroll
    for (int v = 0; v < NV; ++v) base[REC + j * NVP + v] = nu_c[v];
  }
  __syncthreads();
  bool bad = false;
  for (int e = tid; e < ncb * NL; e += TPB) {
    const int s = e / NL, r = e - s * NL;
    double out = smem[(size_t)s * NBUF * REC + REC + (r / NV) * NVP + r % NV];
    if (J.dJdu) out += J.dJdu[c0 * NL + e];
    J.lam[c0 * NL + e] = out;
    bad |= !isfinite(out);
  }
  if (bad) atomicOr(&A.dev->status, ST_NONFINITE);

  // ---- gradients: per-node partial sums -> fixed-order sums per cell -------------------------
  // per-node values staged in the spare record of each cell (last read in the reverse recursion,
  // before the barrier that follows it): [9][NS]
  double* red = spare;
  if (act) {
#pragma unroll
    for (int q = 0; q < 3; ++q) red[q * NS + j] = gm[q];
    if (srcc)
#pragma unroll
      for (int q = 0; q < 6; ++q) red[(3 + q) * NS + j] = gM[q];
  }
  __syncthreads();
  // component q is summed by the cell's thread q mod NS (order 1 has fewer nodes than sums)
  for (int q = j; act && q < (srcc ? 9 : 3); q += NS) {
    double s = 0.0;
    for (int i = 0; i < NS; ++i) s += red[q * NS + i];
    s_sum[slot][q] = s;
  }
  __syncthreads();
  // the cell's own material gradient (its faces' share follows in k_adj_face_sum)
  if (act && j == 0) {
    for (int q = 0; q < 3; ++q) J.grad_mat[c * 3 + q] += s_sum[slot][q];
    if (!isfinite(s_sum[slot][0]) || !isfinite(s_sum[slot][1]) || !isfinite(s_sum[slot][2]))
      atomicOr(&A.dev->status, ST_NONFINITE);
    if (srcc)
      for (int q = 0; q < 6; ++q) J.grad_M[q] += s_sum[slot][3 + q];
  }
}

// grad_mat[c] += the material gradient of the cell's six faces (its left face, where the cell is
// R, and its right face, where it is L, per direction): one thread per cell, fixed order.
template <int N>
__global__ void __launch_bounds__(256) k_adj_face_sum(const __grid_constant__ StepArgs A,
                                                      const __grid_constant__ AdjArgs J,
                                                      long long off1, long long off2) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= A.g.ncells) return;
  double tot[3] = {0.0, 0.0, 0.0};
  for (int d = 0; d < 3; ++d) {
    int id;
    const long long trc = FaceIdx::trans_of_cell(A.g, c, d, id);
    const int nd = A.g.n[d];
    int kr = id + 1;
    if (kr == nd && A.g.bc[d][1] == BC_PERIODIC) kr = 0;
    const long long off = d == 0 ? 0 : (d == 1 ? off1 : off2);
    const double* gl = J.gface + (off + id + (long long)(nd + 1) * trc) * 6;
    const double* gr = J.gface + (off + kr + (long long)(nd + 1) * trc) * 6;
    for (int q = 0; q < 3; ++q) tot[q] += gl[3 + q] + gr[q];
  }
  for (int q = 0; q < 3; ++q) J.grad_mat[c * 3 + q] += tot[q];
  if (!isfinite(tot[0]) || !isfinite(tot[1]) || !isfinite(tot[2]))
    atomicOr(&A.dev->status, ST_NONFINITE);
}

template <int N>
cudaError_t adj_run_ck_n(const StepArgs& a, const AdjArgs& j, const Tables& t, cudaStream_t s);

template <int N>
struct AdjLaunchCK {
  static cudaError_t run(const StepArgs& a, const AdjArgs& j, const Tables& t, cudaStream_t s) {
    using C = CfgCKA<N>;
    static bool attr = false;
    if (!attr) {
      cudaError_t e = cudaFuncSetAttribute(k_adj_cell_ck<N>,
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
    // lambda's projections onto every cell's faces -> face adjoints -> cell kernel (forward face
    // data out) -> face material gradients -> their sums per cell
    cudaError_t e0 = launch_adj_proj<N>(a, j, t, s);
    if (e0 != cudaSuccess) return e0;
    for (int d = 0; d < 3; ++d) {
      cudaError_t e = launch_adj_riemann<N, 1>(a, j, t, d, offs[d], s);
      if (e != cudaSuccess) return e;
    }
    const long long blocks = (a.g.ncells + C::CPB - 1) / C::CPB;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_adj_cell_ck<N><<<(unsigned)blocks, C::TPB, C::SMEM, s>>>(a, j, t);
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
