// A-posteriori finite-volume subcell limiter (Sec. 3.5), FP64, for the Euler equations.
//
// Per step, after the unlimited ADER-DG step has written the candidate u* to u_next:
//   k_lim_detect  one block per cell: subcell averages P(u*), relaxed DMP against the min/max of
//                 the t^n representations of the cell and its face neighbours, positivity of
//                 density and pressure at nodes and subcells; writes the flags.
//   k_lim_compact one thread per cell: troubled cells compacted into the list by warp ballot (one
//                 atomic per warp, lanes at their prefix count).
//   k_lim_fv      persistent blocks over the troubled list: MUSCL-Hancock (minmod) + Rusanov on
//                 the (2N+1)^d subcells with a 2-subcell halo from the t^n representations of all
//                 neighbours, u_next = R(U_sub), the boundary subface fluxes saved per cell; if
//                 any result is not physically admissible, a second launch redoes every troubled
//                 cell with zero slopes (first-order fallback).
//   k_lim_fix     one block per cell: an untroubled face neighbour of a troubled cell replaces its
//                 DG flux on the shared face by the subface fluxes integrated against its test
//                 functions (exact conservation), then refreshes its representation.
// The t^n representation rep (subcell averages of every cell) and its per-variable min/max are
// double-buffered across steps.
#pragma once
#include <climits>
#include "kernels.cuh"

namespace ader {

// Hybrid status (Sec. 3.5): a detected cell keeps `persist` FV steps, the others count down;
// base = detected or still counting.
static __global__ void __launch_bounds__(256) k_lim_status(const uint8_t* __restrict__ flags,
                                                           uint8_t* __restrict__ status,
                                                           uint8_t* __restrict__ base,
                                                           long long ncells, int persist) {
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncells;
       c += (long long)gridDim.x * blockDim.x) {
    const bool det = flags[c] != 0;
    const int st = status[c];
    base[c] = (det || st > 0) ? 1 : 0;
    status[c] = (uint8_t)(det ? persist : (st > 0 ? st - 1 : 0));
  }
}

// The FV set of the hybrid step: the base cells and their face neighbours (the interface layer
// that computes with FV and projects to DG); neighbours across a periodic boundary wrap, a
// non-periodic boundary has none.
static __global__ void __launch_bounds__(256) k_lim_layer(const uint8_t* __restrict__ base,
                                                          uint8_t* __restrict__ flags,
                                                          const Geometry g) {
  const long long n0 = g.n[0], n1 = g.dim > 1 ? g.n[1] : 1;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < g.ncells;
       c += (long long)gridDim.x * blockDim.x) {
    const long long id[3] = {c % n0, (c / n0) % n1, c / (n0 * n1)};
    const long long stride[3] = {1, n0, n0 * n1};
    uint8_t f = base[c];
    for (int d = 0; d < g.dim; ++d) {
      const long long nd = g.n[d];
      for (int side = -1; side <= 1; side += 2) {
        long long k = id[d] + side;
        if (k < 0 || k >= nd) {
          if (g.bc[d][0] != BC_PERIODIC) continue;
          k = (k + nd) % nd;
        }
        f |= base[c + (k - id[d]) * stride[d]];
      }
    }
    flags[c] = f ? 1 : 0;
  }
}

template <int D, int N>
struct CfgL {
  static constexpr int n = N + 1, ns = 2 * N + 1, NV = D + 2;
  static constexpr int NN = ipow(n, D), NSS = ipow(ns, D), NSF = ipow(ns, D - 1);
  static constexpr int NH = ipow(ns + 4, D), NC = ipow(ns + 2, D);
  static constexpr int TPB = 128;
  // projection / reconstruction scratch: nodal values, two partial results, subcell values
  static constexpr int T1 = ipow(ns, D - 1) * n * NV;
  static constexpr int T2 = D == 3 ? n * ns * ns * NV : 0;
  static constexpr size_t SMEM_P = (size_t)(NN * NV + T1 + T2 + NSS * NV) * sizeof(double);
  static constexpr size_t SMEM_FV = (size_t)(NH * NV + NC * NV + (ns + 1) * NSF * NV) * sizeof(double);
};

// One axis of a sum-factorised tensor-product map: Y[o][q][i] = sum_p M[q][p] X[o][p][i] with
// M = P1 (PROJ) or R1.  One thread per (o, i) column holds the LIN inputs in registers; the
// loops over q and p are unrolled, so every matrix entry is a compile-time kernel-parameter
// operand shared by the warp.  Summation order over p is ascending.
template <int LIN, int LOUT, int OUTER, int INNER, bool PROJ>
__device__ __forceinline__ void contract_axis(const double* X, double* Y, const SubTables& S) {
  for (int it = threadIdx.x; it < OUTER * INNER; it += blockDim.x) {
    const int o = it / INNER, i = it - o * INNER;
    const double* x = X + o * (LIN * INNER) + i;
    double xv[LIN];
#pragma unroll
    for (int p = 0; p < LIN; ++p) xv[p] = x[p * INNER];
    double* y = Y + o * (LOUT * INNER) + i;
#pragma unroll
    for (int q = 0; q < LOUT; ++q) {
      double acc = 0.0;
#pragma unroll
      for (int p = 0; p < LIN; ++p) acc = fma(PROJ ? S.P1[q][p] : S.R1[q][p], xv[p], acc);
      y[q * INNER] = acc;
    }
  }
}

// sub[s][v] = sum over nodes of prod_e P1[s_e][a_e] u[a][v] (sum factorisation, x first).
// u: [NN][NV], out: [NSS][NV]; t1, t2 scratch.  All threads of the block participate.
template <int D, int N>
__device__ void project_P(const double* u, double* t1, double* t2, double* out,
                          const SubTables& S) {
  using L = CfgL<D, N>;
  constexpr int n = L::n, ns = L::ns, NV = L::NV;
  if constexpr (D == 2) {
    contract_axis<n, ns, n, NV, true>(u, t1, S);        // t1[b][sx][v]
    __syncthreads();
    contract_axis<n, ns, 1, ns * NV, true>(t1, out, S);  // out[sy][sx][v]
  } else {
    contract_axis<n, ns, n * n, NV, true>(u, t1, S);          // t1[z][b][sx][v]
    __syncthreads();
    contract_axis<n, ns, n, ns * NV, true>(t1, t2, S);        // t2[z][sy][sx][v]
    __syncthreads();
    contract_axis<n, ns, 1, ns * ns * NV, true>(t2, out, S);  // out[sz][sy][sx][v]
  }
  __syncthreads();
}

// u[a][v] = sum over subcells of prod_e R1[a_e][s_e] U[s][v].
template <int D, int N>
__device__ void reconstruct_R(const double* U, double* t1, double* t2, double* out,
                              const SubTables& S) {
  using L = CfgL<D, N>;
  constexpr int n = L::n, ns = L::ns, NV = L::NV;
  if constexpr (D == 2) {
    contract_axis<ns, n, ns, NV, false>(U, t1, S);       // t1[sy][a][v]
    __syncthreads();
    contract_axis<ns, n, 1, n * NV, false>(t1, out, S);  // out[b][a][v]
  } else {
    contract_axis<ns, n, ns * ns, NV, false>(U, t1, S);      // t1[sz][sy][a][v]
    __syncthreads();
    contract_axis<ns, n, ns, n * NV, false>(t1, t2, S);      // t2[sz][b][a][v]
    __syncthreads();
    contract_axis<ns, n, 1, n * n * NV, false>(t2, out, S);  // out[c][b][a][v]
  }
  __syncthreads();
}

// Order-preserving map of a double to a 64-bit integer (both zeros to 0, negative values to
// minus their magnitude bits); it is its own inverse.  For values that are not NaN,
// x <= y exactly when okey(x) <= okey(y), so the bound tests and the min / max of the
// limiter run on the integer pipes instead of the FP64 pipe.
__device__ __forceinline__ long long okey(double x) {
  const long long b = __double_as_longlong(x);
  return b >= 0 ? b : (long long)(0x8000000000000000ull - (unsigned long long)b);
}
__device__ __forceinline__ double okey_inv(long long k) {
  return __longlong_as_double(k >= 0 ? k : (long long)(0x8000000000000000ull - (unsigned long long)k));
}

// rho > 0 and p > 0 with every value finite.  For rho > 0 and gamma > 1, p > 0 is
// 2 E rho - |j|^2 > 0, which one fused multiply-add decides with the sign of E rho - |j|^2 / 2
// (the exact value is doubled before its single rounding); 2E by an exponent increment on the
// integer pipe (zero and subnormal E by an add).  Finiteness, the sign of rho and of the result
// are read from the bits.
template <int D>
__device__ __forceinline__ bool admissible(const double* q) {
  bool fin = true;
#pragma unroll
  for (int v = 0; v < D + 2; ++v) fin = fin && ((__double2hiint(q[v]) & 0x7ff00000) != 0x7ff00000);
  double j2 = 0.0;
#pragma unroll
  for (int i = 0; i < D; ++i) j2 = fma(q[1 + i], q[1 + i], j2);
  const long long eb = __double_as_longlong(q[D + 1]);
  const double e2 = (eb & 0x7ff0000000000000ll) != 0 ? __longlong_as_double(eb + (1ll << 52))
                                                      : q[D + 1] + q[D + 1];
  return fin && (__double_as_longlong(q[0]) > 0) &&
         (__double_as_longlong(fma(e2, q[0], -j2)) > 0);
}

// Physical admissibility with a floor: finite, density and pressure above `floor` (floor 0: the
// division-free positivity test above).
template <int D>
__device__ __forceinline__ bool admissible_f(const double* q, double floor, double gamma) {
  if (!(floor > 0.0)) return admissible<D>(q);
  bool fin = true;
#pragma unroll
  for (int v = 0; v < D + 2; ++v) fin = fin && ((__double2hiint(q[v]) & 0x7ff00000) != 0x7ff00000);
  double j2 = 0.0;
#pragma unroll
  for (int i = 0; i < D; ++i) j2 = fma(q[1 + i], q[1 + i], j2);
  const double p = (gamma - 1.0) * (q[D + 1] - 0.5 * j2 / q[0]);
  return fin && q[0] > floor && p > floor;
}


// Per-variable min / max of sub[NSS][NV] into mm[2][NV]; red: smem scratch [2][NV][32].
// Finite inputs give the same values as fmin / fmax (a zero comes out as +0).
template <int NSS, int NV>
__device__ void block_minmax(const double* sub, double* mm, long long* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int v = 0; v < NV; ++v) {
    long long lo = LLONG_MAX, hi = LLONG_MIN;
    for (int s = threadIdx.x; s < NSS; s += blockDim.x) {
      const long long k = okey(sub[s * NV + v]);
      lo = min(lo, k);
      hi = max(hi, k);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) {
      red[(0 * NV + v) * 32 + warp] = lo;
      red[(1 * NV + v) * 32 + warp] = hi;
    }
  }
  __syncthreads();
  if (threadIdx.x < 2 * NV) {
    const int k = threadIdx.x;
    long long r = red[k * 32];
    for (int w = 1; w < nw; ++w) r = (k < NV) ? min(r, red[k * 32 + w]) : max(r, red[k * 32 + w]);
    mm[k] = okey_inv(r);
  }
  __syncthreads();
}

template <int D>
__device__ __forceinline__ long long neighbor(const Geometry& g, long long c, int d, int side) {
  long long idx[3], rem = c;
  for (int e = 0; e < 3; ++e) {
    idx[e] = rem % g.n[e];
    rem /= g.n[e];
  }
  long long j = idx[d] + side;
  if (j < 0 || j >= g.n[d]) {
    if (g.bc[d][0] != BC_PERIODIC) return -1;
    j = (j + g.n[d]) % g.n[d];
  }
  idx[d] = j;
  return idx[0] + (long long)g.n[0] * (idx[1] + (long long)g.n[1] * idx[2]);
}

template <int D, int N>
__global__ void __launch_bounds__(128) k_lim_detect(const __grid_constant__ StepArgs A,
                                                    const __grid_constant__ LimArgs L,
                                                    const __grid_constant__ SubTables S) {
  using C = CfgL<D, N>;
  constexpr int NN = C::NN, NSS = C::NSS, NV = C::NV;
  extern __shared__ double sm[];
  double* us = sm;
  double* t1 = us + NN * NV;
  double* t2 = t1 + C::T1;
  double* sub = t2 + C::T2;
  __shared__ long long red[2 * NV * 32];
  __shared__ long long bk[2][NV];
  const long long c = blockIdx.x;
  if (L.status) {
    // hybrid status: a cell with FV steps left, or next to one, computes with FV in this step
    // and is not checked (its DG candidate may be built on skipped predictor data); the FV
    // recompute writes its representation
    bool known = L.status[c] != 0;
    for (int d = 0; d < D; ++d)
      for (int side = -1; side <= 1; side += 2) {
        const long long nb = neighbor<D>(A.g, c, d, side);
        if (nb >= 0 && L.status[nb] != 0) known = true;
      }
    if (known) {
      if (threadIdx.x == 0) L.flags[c] = 0;
      return;
    }
  }
  const double* u = A.u_next + c * (NN * NV);
  for (int e = threadIdx.x; e < NN * NV; e += blockDim.x) us[e] = u[e];
  if (threadIdx.x < NV) {
    const int v = threadIdx.x;
    double lo = L.mm[c * 2 * NV + v], hi = L.mm[c * 2 * NV + NV + v];
    for (int d = 0; d < D; ++d)
      for (int side = -1; side <= 1; side += 2) {
        const long long nb = neighbor<D>(A.g, c, d, side);
        if (nb >= 0) {
          lo = fmin(lo, L.mm[nb * 2 * NV + v]);
          hi = fmax(hi, L.mm[nb * 2 * NV + NV + v]);
        }
      }
    // DMP band [lo - delta, hi + delta] as ordered keys (a NaN bound admits nothing)
    const double delta = fmax(L.eps * (hi - lo), L.delta0);
    const double bl = lo - delta, bh = hi + delta;
    bk[0][v] = bl == bl ? okey(bl) : LLONG_MAX;
    bk[1][v] = bh == bh ? okey(bh) : LLONG_MIN;
  }
  __syncthreads();
  project_P<D, N>(us, t1, t2, sub, S);
  bool ok = true;
  for (int s = threadIdx.x; s < NSS; s += blockDim.x) {
    const double* q = sub + s * NV;
    ok = ok && admissible_f<D>(q, L.floor, A.p.gamma);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const long long k = okey(q[v]);
      ok = ok && (k >= bk[0][v]) && (k <= bk[1][v]);
    }
  }
  for (int j = threadIdx.x; j < NN; j += blockDim.x)
    ok = ok && admissible_f<D>(us + j * NV, L.floor, A.p.gamma);
  const bool all_ok = __syncthreads_and(ok) != 0;
  const bool troubled = L.force ? true : !all_ok;
  double* rn = L.rep_new + c * (NSS * NV);
  for (int e = threadIdx.x; e < NSS * NV; e += blockDim.x) rn[e] = sub[e];
  block_minmax<NSS, NV>(sub, L.mm_new + c * 2 * NV, red);
  if (threadIdx.x == 0) L.flags[c] = troubled ? 1 : 0;
}

// Troubled list by warp ballot: every lane votes with its cell's flag, lane 0 reserves the warp's
// slots with one atomic, each flagged lane writes its cell at base + (flagged lanes below it).
static __global__ void __launch_bounds__(256) k_lim_compact(const uint8_t* __restrict__ flags, int* list,
                                                     int* count, long long ncells) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool t = i < ncells && flags[i] != 0;
  const unsigned m = __ballot_sync(0xffffffffu, t);
  const int lane = threadIdx.x & 31;
  int base = 0;
  if (lane == 0 && m != 0u) base = atomicAdd(count, __popc(m));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (t) list[base + __popc(m & ((1u << lane) - 1u))] = (int)i;
}

// Halo value of subcell (hx, hy, hz) in [-2, ns+2)^D of cell c from the t^n representations,
// with the boundary conditions applied on the global subcell grid.
// idx: the cell's grid coordinates.
template <int D, int N>
__device__ __forceinline__ void halo_value(const Geometry& g, const double* rep, const int* idx,
                                           const int* h, double* out) {
  using C = CfgL<D, N>;
  constexpr int ns = C::ns, NV = C::NV, NSS = C::NSS;
  bool flip[3] = {false, false, false};
  int owner[3];
  int sidx[3] = {0, 0, 0};
  for (int d = 0; d < 3; ++d) {
    if (d >= D) {
      owner[d] = 0;
      continue;
    }
    const int Nd = g.n[d] * ns;
    int gs = idx[d] * ns + h[d];
    if (gs < 0) {
      if (g.bc[d][0] == BC_PERIODIC) gs += Nd;
      else {
        gs = -1 - gs;
        flip[d] = g.bc[d][0] == BC_WALL;
      }
    } else if (gs >= Nd) {
      if (g.bc[d][1] == BC_PERIODIC) gs -= Nd;
      else {
        gs = 2 * Nd - 1 - gs;
        flip[d] = g.bc[d][1] == BC_WALL;
      }
    }
    owner[d] = gs / ns;
    sidx[d] = gs - owner[d] * ns;
  }
  const long long oc = owner[0] + (long long)g.n[0] * (owner[1] + (long long)g.n[1] * owner[2]);
  const int s = D == 3 ? sidx[0] + ns * (sidx[1] + ns * sidx[2]) : sidx[0] + ns * sidx[1];
  const double* src = rep + (oc * NSS + s) * NV;
#pragma unroll
  for (int v = 0; v < NV; ++v) out[v] = src[v];
#pragma unroll
  for (int d = 0; d < D; ++d)
    if (flip[d]) out[1 + d] = -out[1 + d];
}

// minmod(a, b): the argument of smaller magnitude when a and b are nonzero with one sign, else 0,
// taken on the bits (sign test and magnitude compare on the integer pipes).  It differs from the
// product test a*b > 0 only where that product underflows to zero.
__device__ __forceinline__ double minmod(double a, double b) {
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  const unsigned long long ma = (unsigned long long)ia & 0x7fffffffffffffffull;
  const unsigned long long mb = (unsigned long long)ib & 0x7fffffffffffffffull;
  const unsigned long long m = ma < mb ? ma : mb;
  const bool take = ((ia ^ ib) >= 0) && (m != 0);
  return take ? __longlong_as_double((long long)(m | ((unsigned long long)ia & 0x8000000000000000ull))) : 0.0;
}

constexpr int FV_TPB = 256;

template <int D, int N>
__global__ void __launch_bounds__(FV_TPB) k_lim_fv(const __grid_constant__ StepArgs A,
                                                const __grid_constant__ LimArgs L,
                                                const __grid_constant__ SubTables S) {
  using C = CfgL<D, N>;
  using P = Euler<D>;
  constexpr int ns = C::ns, NV = C::NV, NSS = C::NSS, NSF = C::NSF, NN = C::NN;
  constexpr int W = ns + 4, WC = ns + 2;
  constexpr int NFC = (ns + 1) * NSF;   // subfaces of one direction
  extern __shared__ double sm[];
  double* H = sm;                  // halo [W^D][NV]
  double* INC = H + C::NH * NV;    // half-step increments of the core [WC^D][NV]
  double* FLX = INC + C::NC * NV;  // subface fluxes of one direction [NFC][NV]
  // after the flux stage: new averages over INC, reconstruction scratch over the halo
  double* UN = INC;
  double* t1 = H;
  double* t2 = t1 + C::T1;
  double* un = t2 + C::T2;         // reconstructed nodal values [NN][NV]
  static_assert(C::NC >= NSS && C::NH * NV >= C::T1 + C::T2 + NN * NV, "aliasing");
  __shared__ long long red[2 * NV * 32];
  const double dt = A.dev->dt;
  const int count = A.dev->n_troubled;
  // first-order pass (zero slopes): only when the MUSCL-Hancock pass of this step found an
  // inadmissible result, and then for every troubled cell (each subface keeps one flux)
  const bool fo = L.first_order != 0;
  if (fo && *(volatile const int*)&A.dev->fv_retry == 0) return;
  for (int it = blockIdx.x; it < count; it += gridDim.x) {
    const long long c = L.list[it];
    int cidx[3];
    {
      long long rem = c;
      for (int e = 0; e < 3; ++e) {
        cidx[e] = (int)(rem % A.g.n[e]);
        rem /= A.g.n[e];
      }
    }
    // halo
    for (int e = threadIdx.x; e < C::NH; e += blockDim.x) {
      int h[3] = {0, 0, 0};
      int r = e;
      for (int d = 0; d < D; ++d) {
        h[d] = r % W - 2;
        r /= W;
      }
      halo_value<D, N>(A.g, L.rep, cidx, h, H + e * NV);
    }
    __syncthreads();
    // half-step increments on the core [-1, ns] (order of directions as in the oracle)
    for (int e = threadIdx.x; e < C::NC; e += blockDim.x) {
      int h[3] = {0, 0, 0};
      int r = e;
      for (int d = 0; d < D; ++d) {
        h[d] = r % WC + 1;  // halo coordinate of the core cell
        r /= WC;
      }
      int hi = 0, st = 1;
      for (int d = 0; d < D; ++d) {
        hi += h[d] * st;
        st *= W;
      }
      const double* U = H + hi * NV;
      double inc[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) inc[v] = 0.0;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const int sd = d == 0 ? 1 : (d == 1 ? W : W * W);
        double Up[NV], Um[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const double sg = fo ? 0.0 : minmod(U[v] - U[v - sd * NV], U[v + sd * NV] - U[v]);
          Up[v] = U[v] + 0.5 * sg;
          Um[v] = U[v] - 0.5 * sg;
        }
        typename P::Aux ap, am;
        P::aux(Up, A.p, ap);
        P::aux(Um, A.p, am);
        double Fp[NV], Fm[NV];
        P::flux(Up, ap, A.p, d, Fp);
        P::flux(Um, am, A.p, d, Fm);
        const double dx = A.g.h[d] / ns;
        const double cf = dt / (2.0 * dx);
#pragma unroll
        for (int v = 0; v < NV; ++v) inc[v] = inc[v] - cf * (Fp[v] - Fm[v]);
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) INC[e * NV + v] = inc[v];
    }
    __syncthreads();
    // fluxes, one per subface, direction by direction (into FLX), then the
    // update of the owned interior subcells in registers (direction order as in the oracle)
    constexpr int KPT = (NSS + FV_TPB - 1) / FV_TPB;
    double Unew[KPT][NV];
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      const int e = threadIdx.x + k * FV_TPB;
      if (e < NSS) {
        int hi = 0, st = 1, r = e;
        for (int d = 0; d < D; ++d) {
          hi += (r % ns + 2) * st;
          r /= ns;
          st *= W;
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) Unew[k][v] = H[hi * NV + v];
      }
    }
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const int sd = d == 0 ? 1 : (d == 1 ? W : W * W);
      const int sdc = d == 0 ? 1 : (d == 1 ? WC : WC * WC);
      for (int f = threadIdx.x; f < NFC; f += FV_TPB) {
        const int i = f % (ns + 1);       // subface i lies between subcells i-1 and i along d
        int t = f / (ns + 1);             // transverse subcell index (lower direction fastest)
        int hL = 0, cL = 0, stw = 1, stc = 1;
        for (int e2 = 0; e2 < D; ++e2) {
          int se;
          if (e2 == d) {
            se = i - 1;
          } else {
            se = t % ns;
            t /= ns;
          }
          hL += (se + 2) * stw;
          cL += (se + 1) * stc;
          stw *= W;
          stc *= WC;
        }
        const int hR = hL + sd, cR = cL + sdc;
        double QL[NV], QR[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const double* UL = H + hL * NV;
          const double* UR = H + hR * NV;
          const double sL = fo ? 0.0 : minmod(UL[v] - UL[v - sd * NV], UL[v + sd * NV] - UL[v]);
          const double sR = fo ? 0.0 : minmod(UR[v] - UR[v - sd * NV], UR[v + sd * NV] - UR[v]);
          QL[v] = (UL[v] + 0.5 * sL) + INC[cL * NV + v];
          QR[v] = (UR[v] - 0.5 * sR) + INC[cR * NV + v];
        }
        typename P::Aux aL, aR;
        P::aux(QL, A.p, aL);
        P::aux(QR, A.p, aR);
        double FL[NV], FR[NV];
        P::flux(QL, aL, A.p, d, FL);
        P::flux(QR, aR, A.p, d, FR);
        const double sp = fmax(P::speed_aux(QL, aL, A.p, d), P::speed_aux(QR, aR, A.p, d));
        double fx[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          fx[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * sp * (QR[v] - QL[v]);
          FLX[f * NV + v] = fx[v];
        }
        const int tr = f / (ns + 1);
        double* bf = L.bflux + ((c * D + d) * 2) * (long long)(NSF * NV);
        if (i == 0)
#pragma unroll
          for (int v = 0; v < NV; ++v) bf[tr * NV + v] = fx[v];
        if (i == ns)
#pragma unroll
          for (int v = 0; v < NV; ++v) bf[NSF * NV + tr * NV + v] = fx[v];
      }
      __syncthreads();
      const double cf = dt / (A.g.h[d] / ns);
#pragma unroll
      for (int k = 0; k < KPT; ++k) {
        const int e = threadIdx.x + k * FV_TPB;
        if (e < NSS) {
          // subcell e: digit d gives i; transverse index from the other digits
          int r = e, sdg = 0, tr = 0, stt = 1;
          for (int e2 = 0; e2 < D; ++e2) {
            const int dg = r % ns;
            r /= ns;
            if (e2 == d) sdg = dg;
            else {
              tr += dg * stt;
              stt *= ns;
            }
          }
          const double* fl = FLX + (sdg + (ns + 1) * tr) * NV;
          const double* fr = fl + NV;
#pragma unroll
          for (int v = 0; v < NV; ++v) Unew[k][v] = Unew[k][v] + cf * (fl[v] - fr[v]);
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      const int e = threadIdx.x + k * FV_TPB;
      if (e < NSS) {
        if (!admissible_f<D>(Unew[k], L.floor, A.p.gamma)) {
          if (fo) atomicOr(&A.dev->status, ST_ADMISSIBLE);  // the fallback is not admissible
          else A.dev->fv_retry = 1;                         // redo the step first order
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) UN[e * NV + v] = Unew[k][v];
      }
    }
    __syncthreads();
    double* rn = L.rep_new + c * (NSS * NV);
    for (int e = threadIdx.x; e < NSS * NV; e += blockDim.x) rn[e] = UN[e];
    block_minmax<NSS, NV>(UN, L.mm_new + c * 2 * NV, red);
    reconstruct_R<D, N>(UN, t1, t2, un, S);
    double* uo = A.u_next + c * (NN * NV);
    for (int e = threadIdx.x; e < NN * NV; e += blockDim.x) uo[e] = un[e];
    __syncthreads();
  }
}

// Neighbour fix: for an untroubled cell with troubled face neighbours.
template <int D, int N>
__global__ void __launch_bounds__(128) k_lim_fix(const __grid_constant__ StepArgs A,
                                                 const __grid_constant__ LimArgs L,
                                                 const __grid_constant__ Tables T,
                                                 const __grid_constant__ SubTables S,
                                                 long long off1, long long off2) {
  using C = CfgL<D, N>;
  constexpr int n = C::n, ns = C::ns, NV = C::NV, NN = C::NN, NSS = C::NSS, NSF = C::NSF;
  constexpr int NF = ipow(n, D - 1);
  const long long c = blockIdx.x;
  if (L.flags[c]) return;
  long long nbs[3][2];
  bool any = false;
  for (int d = 0; d < D; ++d)
    for (int k = 0; k < 2; ++k) {
      const long long nb = neighbor<D>(A.g, c, d, k ? 1 : -1);
      nbs[d][k] = (nb >= 0 && L.flags[nb]) ? nb : -1;
      any = any || nbs[d][k] >= 0;
    }
  if (!any) return;  // uniform per block
  extern __shared__ double sm[];
  double* us = sm;
  double* t1 = us + NN * NV;
  double* t2 = t1 + C::T1;
  double* sub = t2 + C::T2;
  double* geff = sub + NSS * NV;  // [NF][NV]
  __shared__ long long red[2 * NV * 32];
  double* u = A.u_next + c * (NN * NV);
  for (int e = threadIdx.x; e < NN * NV; e += blockDim.x) us[e] = u[e];
  __syncthreads();
  const double dt = A.dev->dt;
  for (int d = 0; d < D; ++d) {
    for (int kk = 0; kk < 2; ++kk) {
      const int k = 1 - kk;  // right face first, then left (order of the oracle)
      const long long nb = nbs[d][k];
      if (nb < 0) continue;
      // subface fluxes of the troubled neighbour on the shared face (its opposite side)
      const double* f = L.bflux + ((nb * D + d) * 2 + (k ? 0 : 1)) * (long long)(NSF * NV);
      // G_eff[j][v] = prod over transverse axes (1/(ns w_je)) sum_s P1[s][je] f[s][v]
      for (int e = threadIdx.x; e < NF * NV; e += blockDim.x) {
        const int v = e % NV, jp = e / NV;
        const int j0 = jp % n, j1 = jp / n;
        double acc = 0.0;
        if constexpr (D == 2) {
          for (int s0 = 0; s0 < ns; ++s0) acc = fma(S.P1[s0][j0], f[s0 * NV + v], acc);
          acc = acc / ns / T.w[j0];
        } else {
          for (int s1 = 0; s1 < ns; ++s1) {
            double a0 = 0.0;
            for (int s0 = 0; s0 < ns; ++s0) a0 = fma(S.P1[s0][j0], f[(s1 * ns + s0) * NV + v], a0);
            acc = fma(S.P1[s1][j1], a0, acc);
          }
          acc = acc / ns / T.w[j0] / ns / T.w[j1];
        }
        geff[e] = acc;
      }
      __syncthreads();
      // DG flux on that face and the correction of the nodal values
      int id;
      const long long tr = FaceIdx::trans_of_cell(A.g, c, d, id);
      const int nd = A.g.n[d];
      int kf = k ? id + 1 : id;
      if (k && kf == nd && A.g.bc[d][1] == BC_PERIODIC) kf = 0;
      const long long off = d == 0 ? 0 : (d == 1 ? off1 : off2);
      const double* phi = A.phi + off + (kf + (long long)(nd + 1) * tr) * (NF * NV);
      const int st = d == 0 ? 1 : (d == 1 ? n : n * n);
      for (int e = threadIdx.x; e < NN * NV; e += blockDim.x) {
        const int v = e % NV, j = e / NV;
        const int jd = (j / st) % n;
        const int jp = (j % st) + (j / (st * n)) * st;
        const double g = geff[jp * NV + v] - phi[jp * NV + v];
        const double corr = k ? -dt / A.g.h[d] * T.c1[jd] * g : dt / A.g.h[d] * T.c0[jd] * g;
        us[e] = us[e] + corr;
      }
      __syncthreads();
    }
  }
  for (int e = threadIdx.x; e < NN * NV; e += blockDim.x) u[e] = us[e];
  project_P<D, N>(us, t1, t2, sub, S);
  double* rn = L.rep_new + c * (NSS * NV);
  for (int e = threadIdx.x; e < NSS * NV; e += blockDim.x) rn[e] = sub[e];
  block_minmax<NSS, NV>(sub, L.mm_new + c * 2 * NV, red);
}

// rep = P(u) for every cell (reset of the limiter history); flagged cells keep the given U_sub
// and get u = R(U_sub).
template <int D, int N>
__global__ void __launch_bounds__(128) k_lim_init(double* u, const double* Usub,
                                                  const uint8_t* flags, double* rep, double* mm,
                                                  const __grid_constant__ SubTables S) {
  using C = CfgL<D, N>;
  constexpr int NV = C::NV, NN = C::NN, NSS = C::NSS;
  extern __shared__ double sm[];
  double* us = sm;
  double* t1 = us + NN * NV;
  double* t2 = t1 + C::T1;
  double* sub = t2 + C::T2;
  __shared__ long long red[2 * NV * 32];
  const long long c = blockIdx.x;
  double* uc = u + c * (NN * NV);
  const bool fl = flags && flags[c];
  if (fl) {
    const double* U = Usub + c * (NSS * NV);
    for (int e = threadIdx.x; e < NSS * NV; e += blockDim.x) sub[e] = U[e];
    __syncthreads();
    reconstruct_R<D, N>(sub, t1, t2, us, S);
    for (int e = threadIdx.x; e < NN * NV; e += blockDim.x) uc[e] = us[e];
  } else {
    for (int e = threadIdx.x; e < NN * NV; e += blockDim.x) us[e] = uc[e];
    __syncthreads();
    project_P<D, N>(us, t1, t2, sub, S);
  }
  double* r = rep + c * (NSS * NV);
  for (int e = threadIdx.x; e < NSS * NV; e += blockDim.x) r[e] = sub[e];
  block_minmax<NSS, NV>(sub, mm + c * 2 * NV, red);
}

// ---- launchers -----------------------------------------------------------------------------
template <int D, int N>
struct LimLaunch {
  using C = CfgL<D, N>;
  static size_t smem_fix() { return C::SMEM_P + (size_t)ipow(N + 1, D - 1) * C::NV * sizeof(double); }
  static cudaError_t init(double* u, const double* Usub, const uint8_t* flags, double* rep,
                          double* mm, long long ncells, const SubTables& S, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
      cudaError_t e = cudaFuncSetAttribute(k_lim_init<D, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)C::SMEM_P);
      if (e != cudaSuccess) return e;
      attr = true;
    }
    k_lim_init<D, N><<<(unsigned)ncells, C::TPB, C::SMEM_P, s>>>(u, Usub, flags, rep, mm, S);
    return cudaGetLastError();
  }
  static cudaError_t step(const StepArgs& a, const LimArgs& l, const Tables& T, const SubTables& S,
                          cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
      cudaError_t e = cudaFuncSetAttribute(k_lim_detect<D, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)C::SMEM_P);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_lim_fv<D, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)C::SMEM_FV);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_lim_fix<D, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_fix());
      if (e != cudaSuccess) return e;
      attr = true;
    }
    const unsigned nc = (unsigned)a.g.ncells;
    k_lim_detect<D, N><<<nc, C::TPB, C::SMEM_P, s>>>(a, l, S);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (l.status) {  // hybrid status: widen the flags before the compaction
      const unsigned blocks = (unsigned)((a.g.ncells + 255) / 256);
      k_lim_status<<<blocks, 256, 0, s>>>(l.flags, l.status, l.base, a.g.ncells, l.persist);
      k_lim_layer<<<blocks, 256, 0, s>>>(l.base, l.flags, a.g);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    k_lim_compact<<<(unsigned)((a.g.ncells + 255) / 256), 256, 0, s>>>(l.flags, l.list,
                                                                         &a.dev->n_troubled, a.g.ncells);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_lim_fv<D, N><<<152 * 2, FV_TPB, C::SMEM_FV, s>>>(a, l, S);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    LimArgs lf = l;  // the first-order fallback (its blocks return unless a retry is flagged)
    lf.first_order = 1;
    k_lim_fv<D, N><<<152 * 2, FV_TPB, C::SMEM_FV, s>>>(a, lf, S);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    long long offs[3] = {0, 0, 0}, off = 0;
    const int nf = ipow(N + 1, D - 1);
    for (int d = 0; d < D; ++d) {
      offs[d] = off;
      off += (long long)(a.g.n[d] + 1) * (a.g.ncells / a.g.n[d]) * nf * C::NV;
    }
    k_lim_fix<D, N><<<nc, C::TPB, smem_fix(), s>>>(a, l, T, S, offs[1], offs[2]);
    return cudaGetLastError();
  }
};

}  // namespace ader
