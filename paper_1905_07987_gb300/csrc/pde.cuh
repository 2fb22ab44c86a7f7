// PDE terms of dQ/dt + div F(Q) + B(Q).grad Q = S(Q) (Eq. (1)) for the built-in systems.
// Each system mirrors the user functions of Table 2: flux, nonConservativeProduct (here as the
// single non-zero of each row of the cell-constant matrix B_d), eigenvalues (max |lambda|),
// boundaryValues (ghost states) and, for the limiter, isPhysicallyAdmissable.
#pragma once
#include "ader_internal.h"

namespace ader {

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }
__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }

// Scalar advection dq/dt + div(a q) = 0 (test system).
template <int D>
struct Advection {
  static constexpr int NV = 1;
  static constexpr bool CONS = true;
  static constexpr bool NCP = false;
  static constexpr bool NCPS = false;
  static constexpr bool LINEAR = true;
  static constexpr int DIM = D;
  struct Aux {};
  __device__ static void aux(const double*, const PdeParams&, Aux&) {}
  __device__ static void flux(const double* q, const Aux&, const PdeParams& p, int d, double* F) {
    F[0] = p.a[d] * q[0];
  }
  __device__ static double speed(const double*, const PdeParams& p, int d) { return fabs(p.a[d]); }
  __device__ static void mirror(double*, int) {}
  __device__ static void mirror_flux(double*, int) {}
};

// Compressible Euler equations (Eq. (8)), gamma-law pressure p = (gamma-1)(E - |j|^2/(2 rho)).
template <int D>
struct Euler {
  static constexpr int NV = D + 2;
  static constexpr bool CONS = true;
  static constexpr bool NCP = false;
  static constexpr bool NCPS = false;
  static constexpr bool LINEAR = false;
  static constexpr int DIM = D;
  struct Aux {
    double ir, p;
  };
  __device__ static void aux(const double* q, const PdeParams& pp, Aux& a) {
    a.ir = 1.0 / q[0];
    double j2 = 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i) j2 = fma(q[1 + i], q[1 + i], j2);
    a.p = (pp.gamma - 1.0) * fma(-0.5 * j2, a.ir, q[NV - 1]);
  }
  __device__ static void flux(const double* q, const Aux& a, const PdeParams&, int d, double* F) {
    const double vd = q[1 + d] * a.ir;
    F[0] = q[1 + d];
#pragma unroll
    for (int i = 0; i < D; ++i) F[1 + i] = q[1 + i] * vd;
    F[1 + d] += a.p;
    F[NV - 1] = (q[NV - 1] + a.p) * vd;
  }
  __device__ static double pressure(const double* q, double gamma) {
    double j2 = 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i) j2 = fma(q[1 + i], q[1 + i], j2);
    return (gamma - 1.0) * (q[NV - 1] - 0.5 * j2 / q[0]);
  }
  // |v_d| + c; a negative c^2 (non-admissible state, rejected by the limiter) counts as 0 so the
  // estimate stays finite; NaN propagates.
  __device__ static double speed(const double* q, const PdeParams& pp, int d) {
    const double ir = 1.0 / q[0];
    double j2 = 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i) j2 = fma(q[1 + i], q[1 + i], j2);
    const double p = (pp.gamma - 1.0) * (q[NV - 1] - 0.5 * j2 * ir);
    double c2 = pp.gamma * p * ir;
    if (c2 < 0.0) c2 = 0.0;
    return fabs(q[1 + d] * ir) + sqrt(c2);
  }
  // |v_d| + c from the aux values (1/rho, p) already computed for the flux
  __device__ static double speed_aux(const double* q, const Aux& a, const PdeParams& pp, int d) {
    double c2 = pp.gamma * a.p * a.ir;
    if (c2 < 0.0) c2 = 0.0;
    return fabs(q[1 + d] * a.ir) + sqrt(c2);
  }
  // max over directions of |v_d| + c with one division and one square root (FP64)
  __device__ static double speed_all(const double* q, const PdeParams& pp) {
    const double ir = 1.0 / q[0];
    double j2 = 0.0, vm = 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      j2 = fma(q[1 + i], q[1 + i], j2);
      vm = fmax(vm, fabs(q[1 + i]));
    }
    const double p = (pp.gamma - 1.0) * (q[NV - 1] - 0.5 * j2 * ir);
    double c2 = pp.gamma * p * ir;
    if (c2 < 0.0) c2 = 0.0;
    return vm * fabs(ir) + sqrt(c2);  // |v_d| = |j_d| / |rho|, as for a non-admissible rho < 0
  }
  __device__ static void mirror(double* q, int d) { q[1 + d] = -q[1 + d]; }
  // F_d of the mirrored state: all components but the normal momentum flux change sign.
  __device__ static void mirror_flux(double* F, int d) {
#pragma unroll
    for (int v = 0; v < NV; ++v)
      if (v != 1 + d) F[v] = -F[v];
  }
};

// Linear elasticity in velocity-stress form, Q = (v, sigma_xx, yy, zz, xy, xz, yz), material
// m = (rho, lambda, mu) per cell (Sec. 2.1).  Every term is non-conservative and each row of
// B_d has a single non-zero entry: row v gets coef * dQ[src]/dx_d.
struct Elastic {
  static constexpr int NV = 9;
  static constexpr bool CONS = false;
  static constexpr bool NCP = true;
  static constexpr bool NCPS = false;
  static constexpr bool LINEAR = true;
  static constexpr int DIM = 3;
  __host__ __device__ static constexpr int sig(int i, int j) {
    return i == j ? 3 + i : (i + j == 1 ? 6 : (i + j == 2 ? 7 : 8));
  }
  // Source variable of row v of B_d (-1: the row is zero).
  __host__ __device__ static constexpr int src(int d, int v) {
    return v < 3 ? sig(v, d)
                 : (v < 6 ? d
                          : (v == 6 ? (d == 0 ? 1 : (d == 1 ? 0 : -1))
                                    : (v == 7 ? (d == 0 ? 2 : (d == 2 ? 0 : -1))
                                              : (d == 1 ? 2 : (d == 2 ? 1 : -1)))));
  }
  // Coefficient of row v of B_d for material (rho, lambda, mu).
  __device__ static double coef(int d, int v, double rho, double lam, double mu) {
    if (v < 3) return -1.0 / rho;
    if (v < 6) return (v - 3 == d) ? -(lam + 2.0 * mu) : -lam;
    return -mu;
  }
  // Coefficient given 1/rho precomputed.
  __device__ static double coef_ir(int d, int v, double irho, double lam, double mu) {
    if (v < 3) return -irho;
    if (v < 6) return (v - 3 == d) ? -(lam + 2.0 * mu) : -lam;
    return -mu;
  }
  __device__ static double vp(double rho, double lam, double mu) {
    return sqrt((lam + 2.0 * mu) / rho);
  }
  // Wall boundaries are not offered for elastic contexts (rejected at creation).
  __device__ static void mirror(double*, int) {}
  __device__ static void mirror_flux(double*, int) {}
};

// Shallow water equations with bathymetry (Eq. (9), Sec. 2), Q = (h, hu, hv, b): the flux
// F_d = (h u_d, hu u_d, hv u_d, 0) and the state-dependent non-conservative product
// g h d(h + b)/dx_d on the momentum of direction d (the hydrostatic pressure and the bathymetry
// slope; b is a state variable the equations keep constant).  NCPS: B_d(Q) depends on the state.
struct ShallowWater {
  static constexpr int NV = 4;
  static constexpr bool CONS = true;
  static constexpr bool NCP = false;
  static constexpr bool NCPS = true;
  static constexpr bool LINEAR = false;
  static constexpr int DIM = 2;
  struct Aux {
    double ih;
  };
  __device__ static void aux(const double* q, const PdeParams&, Aux& a) { a.ih = 1.0 / q[0]; }
  __device__ static void flux(const double* q, const Aux& a, const PdeParams&, int d, double* F) {
    const double ud = q[1 + d] * a.ih;
    F[0] = q[1 + d];
    F[1] = q[1] * ud;
    F[2] = q[2] * ud;
    F[3] = 0.0;
  }
  // |u_d| + sqrt(g h): the largest |eigenvalue| of the direction-d system (NaN for h < 0)
  __device__ static double speed(const double* q, const PdeParams& pp, int d) {
    return fabs(q[1 + d] / q[0]) + sqrt(pp.grav * q[0]);
  }
  __device__ static double speed_all(const double* q, const PdeParams& pp) {
    const double ih = 1.0 / q[0];
    return fmax(fabs(q[1] * ih), fabs(q[2] * ih)) + sqrt(pp.grav * q[0]);
  }
  __device__ static void mirror(double* q, int d) { q[1 + d] = -q[1 + d]; }
  // F_d of the mirrored state: every component but the normal momentum flux changes sign
  __device__ static void mirror_flux(double* F, int d) {
#pragma unroll
    for (int v = 0; v < NV; ++v)
      if (v != 1 + d) F[v] = -F[v];
  }
};

}  // namespace ader
