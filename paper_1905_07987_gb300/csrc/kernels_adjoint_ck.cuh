// Adjoint of the linear-elastic step with the Cauchy-Kowalevski predictor (Sec. 2, Sec. 3.3).
//
// Per cell the forward predictor is linear in the state, the material and the moment tensor:
//   a_0 = u,   a_{k+1} = f_k (L a_k + g s_k),   f_k = dt / (k+1),   k = 0..N-1,
//   qbar = sum_{k<=N} a_k / (k+1),
// followed by the volume term u + dt (L qbar + g sbar) and the face extrapolations E qbar (the
// same epilogue as the Picard form).  Given lambda (the adjoint of the next state) and the
// adjoint of the face extrapolations (k_adj_riemann, shared with the Picard adjoint), the
// transposes are taken in reverse order:
//   lq   = dt L^T lambda + sum_d E_d^T adjf_d                  (adjoint of qbar)
//   mu_N = lq / (N+1),   mu_k = lq / (k+1) + f_k L^T mu_{k+1}   (adjoint of a_k)
//   lambda^n = lambda + mu_0 (+ dJ/du^n)
// and the gradients pair each adjoint with the forward quantity that multiplies the parameter:
//   material   dt lambda^T (dL/dm) qbar + sum_k f_k mu_{k+1}^T (dL/dm) a_k
//   moment     dt sbar lambda^T (dg/dM) + sum_k f_k s_k mu_{k+1}^T (dg/dM).
// (dL/dm) a at a node needs only the derivatives of a at that node (the forward contraction), so
// the material gradient costs one forward-style application per level; L^T needs the adjoint of
// the neighbours along each line: the contraction with the transposed derivative matrix.
//
// One thread per node, the cells of a block (several at low order) each keep a_0 .. a_{N-1}
// and two adjoint buffers in shared memory: (N+2) padded records of 10 doubles per node, no
// global scratch.  Work per node: N forward applications to recompute a_k, then N+1 pairs of
// (L^T, material derivative) applications; the Picard adjoint recomputes and reverses N+1
// iterations over n time nodes.  The gradient sums are reduced in a fixed order (no atomics), so
// repeated runs give identical bits.
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
  static constexpr int NBUF = N + 2;  // a_0 .. a_{N-1}, two adjoint buffers
  static constexpr size_t SMEM = (size_t)CPB * NBUF * REC * sizeof(double);
};

// Out[col] += (L^T Y)[j][col] for the record Y ([NS][NVP]) at node j.  DT[d][i] = D[i][j_d]
// (column j_d of the derivative matrix); cf[d] = {1/(rho h_d), (lam + 2 mu)/h_d, lam/h_d, mu/h_d}.
// Row by row of L (see ck_apply): velocity row i reads sigma_{id}, normal-stress rows read v_d,
// shear row v reads v_{src(d,v)}; the transpose sends each row's adjoint back to that column.
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
      tsum = fma(c, r[3] + r[4] + r[5], tsum);
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

// gm += w * mu^T (dL/d(rho, lam, mu)) X at node j (mu: the adjoint at this node).  The
// derivatives of the record X along each direction are those of ck_apply; ih[d] = 1/h_d.
template <int N>
__device__ __forceinline__ void ck_dmat(const double* X, int j, const double (&Dr)[3][N + 1],
                                        const double (&ih)[3], double irho, const double (&mu)[9],
                                        double w, double (&gm)[3]) {
  constexpr int n = N + 1, NVP = CfgCKA<N>::NVP;
  double grho = 0.0, glam = 0.0, gmu = 0.0;
  const double msum = mu[3] + mu[4] + mu[5];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int st = d == 0 ? 1 : (d == 1 ? n : n * n);
    const int jd = (j / st) % n;
    const double* b = X + (j - jd * st) * NVP;
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
    // velocity rows: (1/rho) d sigma_{id} / dx_d  ->  d/drho = -1/rho^2
    grho = fma(ih[d], fma(mu[0], ds0, fma(mu[1], ds1, mu[2] * ds2)), grho);
    // normal-stress rows: (lam + 2 mu [i == d]) dv_d / dx_d
    glam = fma(ih[d] * dv[d], msum, glam);
    gmu = fma(2.0 * ih[d] * dv[d], mu[3 + d], gmu);
    // shear rows: mu dv_{src(d,v)} / dx_d
#pragma unroll
    for (int v = 6; v < 9; ++v) {
      const int s = Elastic::src(d, v);
      if (s >= 0) gmu = fma(ih[d] * dv[s], mu[v], gmu);
    }
  }
  gm[0] = fma(w, -irho * irho * grho, gm[0]);
  gm[1] = fma(w, glam, gm[1]);
  gm[2] = fma(w, gmu, gm[2]);
}

template <int N>
__global__ void __launch_bounds__(CfgCKA<N>::TPB)
    k_adj_cell_ck(const __grid_constant__ StepArgs A, const __grid_constant__ AdjArgs J,
                  const __grid_constant__ Tables T, long long off1, long long off2) {
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
  double* base = smem + (size_t)(act ? slot : 0) * NBUF * REC;
  double* P = base + N * REC;  // adjoint buffers P, Q
  double* Q = P + REC;
  const double dt = A.dev->dt;
  const double tn = A.dev->t;

  // the block's cells into a_0 (coalesced)
  for (int e = tid; e < ncb * NL; e += TPB) {
    const int s = e / NL, r = e - s * NL;
    smem[(size_t)s * NBUF * REC + (r / NV) * NVP + r % NV] = J.u_n[c0 * NL + e];
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
  double Dr[3][n], DT[3][n], cf[3][4], ih[3], irho = 0.0;
  double phi = 0.0, Mt[6];
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
    const double lam = A.mat[c * 3 + 1];
    const double mu = A.mat[c * 3 + 2];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      ih[d] = A.g.inv_h[d];
      cf[d][0] = irho * ih[d];
      cf[d][1] = (lam + 2.0 * mu) * ih[d];
      cf[d][2] = lam * ih[d];
      cf[d][3] = mu * ih[d];
    }
  }
#pragma unroll
  for (int a = 0; a < 6; ++a) Mt[a] = srcc ? A.src.M[a] : 0.0;
  if (srcc) phi = A.src.phi[j];
  __syncthreads();

  // ---- forward recursion: a_1 .. a_{N-1} kept, qbar accumulated ----------------------------
  double qb[NV];
  if (act) {
#pragma unroll
    for (int v = 0; v < NV; ++v) qb[v] = base[j * NVP + v];
  }
#pragma unroll
  for (int k = 0; k < N; ++k) {
    if (act) {
      double R[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) R[v] = 0.0;
      ck_apply<N>(base + k * REC, j, Dr, cf, R);
      if (srcc) {
#pragma unroll
        for (int v = 3; v < NV; ++v) R[v] = fma(-Mt[v - 3] * phi, s_sk[k], R[v]);
      }
      const double f = dt * (1.0 / (k + 1));
      const double wk = 1.0 / (k + 2);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const double a = f * R[v];
        qb[v] = fma(wk, a, qb[v]);
        if (k + 1 < N) base[(k + 1) * REC + j * NVP + v] = a;
      }
    }
    __syncthreads();
  }
  // qbar -> P, lambda^{n+1} -> Q (coalesced)
  if (act) {
#pragma unroll
    for (int v = 0; v < NV; ++v) P[j * NVP + v] = qb[v];
  }
  for (int e = tid; e < ncb * NL; e += TPB) {
    const int s = e / NL, r = e - s * NL;
    smem[(size_t)s * NBUF * REC + (size_t)(N + 1) * REC + (r / NV) * NVP + r % NV] =
        J.lam[c0 * NL + e];
  }
  __syncthreads();

  // ---- adjoint of the volume term and of the face extrapolations ---------------------------
  double gm[3] = {0.0, 0.0, 0.0}, gM[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  double lam_j[NV], lq[NV];
  if (act) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      lam_j[v] = Q[j * NVP + v];
      lq[v] = 0.0;
    }
    ck_apply_T<N>(Q, j, DT, cf, lq);
#pragma unroll
    for (int v = 0; v < NV; ++v) lq[v] *= dt;
    ck_dmat<N>(P, j, Dr, ih, irho, lam_j, dt, gm);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int st = d == 0 ? 1 : (d == 1 ? n : n * n);
      const int jd = (j / st) % n;
      const int jp = (j % st) + (j / (st * n)) * st;
      const double* af = J.adjf + (c * 3 + d) * 2 * (long long)(NF * NV) + jp * NV;
      const double e0 = T.e0[jd], e1 = T.e1[jd];
#pragma unroll
      for (int v = 0; v < NV; ++v) lq[v] = fma(e0, af[v], fma(e1, af[NF * NV + v], lq[v]));
    }
    if (srcc) {
#pragma unroll
      for (int a = 0; a < 6; ++a) gM[a] = fma(dt * s_sbar, -phi * lam_j[3 + a], gM[a]);
    }
  }
  __syncthreads();  // P and Q are read above; mu_N goes into P
  double mu_c[NV];  // mu_{k+1} at this node
  if (act) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      mu_c[v] = lq[v] * (1.0 / (N + 1));
      P[j * NVP + v] = mu_c[v];
    }
  }
  __syncthreads();

  // ---- reverse Taylor recursion --------------------------------------------------------------
#pragma unroll
  for (int k = N - 1; k >= 0; --k) {
    const double* Yin = ((N - 1 - k) & 1) ? Q : P;  // mu_{k+1}
    double* Yout = ((N - 1 - k) & 1) ? P : Q;       // mu_k
    if (act) {
      const double f = dt * (1.0 / (k + 1));
      double Tt[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) Tt[v] = 0.0;
      ck_apply_T<N>(Yin, j, DT, cf, Tt);
      ck_dmat<N>(base + k * REC, j, Dr, ih, irho, mu_c, f, gm);
      if (srcc) {
#pragma unroll
        for (int a = 0; a < 6; ++a) gM[a] = fma(f * s_sk[k], -phi * mu_c[3 + a], gM[a]);
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        mu_c[v] = fma(f, Tt[v], lq[v] * (1.0 / (k + 1)));
        if (k > 0) Yout[j * NVP + v] = mu_c[v];
      }
    }
    if (k > 0) __syncthreads();
  }
  // lambda^n = lambda^{n+1} + mu_0 (+ dJ/du^n), staged in a_0 for a coalesced store
  bool bad = false;
  __syncthreads();  // every thread is done reading a_0 (the last level of the reverse sweep)
  if (act) {
#pragma unroll
    for (int v = 0; v < NV; ++v) base[j * NVP + v] = lam_j[v] + mu_c[v];
  }
  __syncthreads();
  for (int e = tid; e < ncb * NL; e += TPB) {
    const int s = e / NL, r = e - s * NL;
    double out = smem[(size_t)s * NBUF * REC + (r / NV) * NVP + r % NV];
    if (J.dJdu) out += J.dJdu[c0 * NL + e];
    J.lam[c0 * NL + e] = out;
    bad |= !isfinite(out);
  }
  if (bad) atomicOr(&A.dev->status, ST_NONFINITE);
  __syncthreads();

  // ---- gradients: per-node partial sums -> fixed-order sums per cell -------------------------
  // per-node values staged in a_1 (or P at order 1) of each cell: [9][NS] (3 material, 6 moment)
  double* red = base + (N > 1 ? REC : N * REC);
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
  if (act && j == 0) {
    double tot[3] = {s_sum[slot][0], s_sum[slot][1], s_sum[slot][2]};
    // the cell's faces: its left face (the cell is R there) and right face (the cell is L)
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
    if (srcc)
      for (int q = 0; q < 6; ++q) J.grad_M[q] += s_sum[slot][3 + q];
  }
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
    for (int d = 0; d < 3; ++d) {
      const long long nf = (long long)(a.g.n[d] + 1) * (a.g.ncells / a.g.n[d]);
      k_adj_riemann<3, N><<<(unsigned)((nf + 3) / 4), 128, 0, s>>>(a, j, t, d, offs[d]);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    const long long blocks = (a.g.ncells + C::CPB - 1) / C::CPB;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_adj_cell_ck<N><<<(unsigned)blocks, C::TPB, C::SMEM, s>>>(a, j, t, offs[1], offs[2]);
    return cudaGetLastError();
  }
};

}  // namespace ader
