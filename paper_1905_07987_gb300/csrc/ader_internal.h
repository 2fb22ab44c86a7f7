// Internal declarations shared by the host runtime (api.cu) and the kernel translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ader {

constexpr int MAXN = 7;   // nodes per direction supported (order <= 6)
constexpr int MAXNS = 13; // FV subcells per direction (2N+1)

// Boundary kinds (same values as ader_bc in include/ader.h).
constexpr int BC_PERIODIC = 0, BC_WALL = 1, BC_ABSORBING = 2;

// Error bits latched in DevScalars::status by kernels.
enum : int {
  ST_NONFINITE = 1,
  ST_ADMISSIBLE = 2,
  ST_TIMEOUT = 4,
  ST_SEISMO_FULL = 8,
};

// Device-resident scalars of the time loop.  dt and t never travel to the host during a run.
struct DevScalars {
  double t;                  // t^n
  double dt;                 // dt of the current / last step
  unsigned long long lam_bits;  // max signal speed of the state at t^n (bit pattern, >= 0)
  int status;                // latched error bits
  unsigned lam_lo_bits;      // mixed-form CFL: a lower bound of the max signal speed (binary32 bits)
  long long nstep;           // steps taken
  long long seismo_row;      // next seismogram row
  int n_troubled;            // troubled cells of the last step
  int fv_retry;              // limiter: a MUSCL-Hancock recompute of this step was inadmissible
};

// 1-D reference-element tables, passed by value as a kernel parameter (constant bank).
struct Tables {
  double D[MAXN][MAXN];   // D[i][m] = phi_m'(x_i)
  double Kw[MAXN][MAXN];  // K1^{-1} diag(w): predictor update q = u + dt Kw R
  double w[MAXN];         // Gauss-Legendre weights on [0,1]
  double x[MAXN];         // nodes
  double e0[MAXN], e1[MAXN];  // phi_m(0), phi_m(1)
  double c0[MAXN], c1[MAXN];  // e0/w, e1/w
  double pz[3], pw[3];        // 3-point Gauss-Legendre rule on [0,1] (path integral of B)
  double Vi[MAXN][MAXN];      // Vi[k][t]: coefficient of tau^k of the Lagrange polynomial of
                              // time node t (interpolant -> monomial coefficients)
  double cerk[3][MAXN];       // dense-output weights b1, b2 (= b3), b4 of the four-stage
                              // Runge-Kutta guess at the time nodes
};

// Single-precision and float-float copies of the tables for the mixed-precision predictor.
// A float-float value is hi + lo with hi = fl32(x), lo = fl32(x - hi).
struct TablesF {
  float Dh[MAXN][MAXN], Dl[MAXN][MAXN];    // strong derivative D
  float Wh[MAXN][MAXN], Wl[MAXN][MAXN];    // weak derivative Dw = c1 e1^T - c0 e0^T - D
  float Kw[MAXN][MAXN], Kwl[MAXN][MAXN];   // K1^{-1} diag(w) (hi, lo)
  float kw1[MAXN], kw1l[MAXN];             // row sums of Kw (hi, lo)
  float wk1h, wk1l;                        // sum_t w_t kw1[t]      (time average of the
  float wKh[MAXN], wKl[MAXN];              // sum_t w_t Kw[t][m]     time solve)
  float w[MAXN], wl[MAXN];
  float ihh[3], ihl[3];                    // 1/h_d (hi, lo)
  float g1h, g1l;                          // gamma - 1 (hi, lo)
  float e0h[MAXN], e0l[MAXN], e1h[MAXN], e1l[MAXN];
  float th[MAXN];                          // time nodes x_t
  float cerk[3][MAXN];                     // dense-output weights b1, b2 (= b3), b4 at x_t
};

// Subcell tables of the limiter (Sec. 3.5).
struct SubTables {
  double P1[MAXNS][MAXN];  // DG nodal values -> subcell averages
  double R1[MAXN][MAXNS];  // subcell averages -> DG (mean-preserving least squares)
  double Pf[MAXNS][MAXN];  // P1[s][m] / (w_m ns): subface flux -> nodal face flux weights
};

// Arguments of the limiter kernels (Sec. 3.5).
struct LimArgs {
  const double* rep;     // [C][NSS][NV] representation at t^n
  double* rep_new;       // [C][NSS][NV] representation at t^{n+1}
  const double* mm;      // [C][2][NV] min / max of rep
  double* mm_new;
  const uint8_t* flags_prev;  // [C] troubled at the previous step (unused by the kernels)
  uint8_t* flags;        // [C] recomputed with FV at this step (the troubled cells; with the
                         // hybrid status, the widened set)
  int* list;             // [C] troubled cells (first n_troubled entries)
  double* bflux;         // [C][D][2][NSF][NV] subface fluxes on the cell boundary
  int force;             // 1: every cell troubled (pure FV scheme)
  double delta0, eps;
  // hybrid ADER-DG / FV status (null: per-step limiter): FV steps each cell still has to take,
  // and the detected-or-counting set before the interface layer is added
  uint8_t* status;
  uint8_t* base;
  int persist;           // FV steps a detected cell keeps
  double floor;          // physical admissibility: density and pressure above floor (0: positive)
  int first_order;       // FV recompute with zero slopes (the first-order fallback pass)
};

// Arguments of the adjoint kernels of the linear elastic step.
struct AdjArgs {
  const double* u_n;     // forward state at t^n [C][NL]
  double* lam;           // in: lambda^{n+1}; out: lambda^n  [C][NL]
  const double* dJdu;    // optional dJ/du^n [C][NL]
  double* grad_mat;      // [C][3] accumulated
  double* grad_M;        // [6] accumulated
  double* adjf;          // [C][3][2][NF][NV] adjoint of the face extrapolations
  double* gface;         // [faces of all directions][2][3] material gradient of each face
  double* scratch;       // [gridDim][I-1][n][NL] forward Picard iterates
  long long scratch_per_block;
  double* lproj;         // [C][3][2][NF][NV] lambda's projections onto each cell's faces
                         // (Cauchy-Kowalevski adjoint; null otherwise)
};

// Ensemble of runs advanced together (one persistent launch per phase of the step for all runs):
// prefix offsets of the runs' cells and faces in the concatenated work lists, and the offset of
// each direction's fluxes in a run's flux buffer.
constexpr int ENS_MAXR = 64;
struct EnsTable {
  int nr;                              // runs
  int pblocks;                         // persistent blocks of the predictor (SMs x blocks per SM)
  long long cell0[ENS_MAXR + 1];       // first concatenated cell of run r; cell0[nr] = total
  long long face0[3][ENS_MAXR + 1];    // the same for the faces of direction d
  long long phioff[3][ENS_MAXR];       // run-local offset of direction d's fluxes
};

struct Geometry {
  int dim, order;
  int n[3];            // cells per direction
  long long ncells;
  double lo[3], h[3], inv_h[3];
  int bc[3][2];
};

struct PdeParams {
  double gamma;
  double a[3];
  double grav;         // gravitational acceleration (shallow water)
};

struct PointSrc {
  int cell;            // -1: none
  double M[6];
  double f0, t0;
  const double* phi;   // [n^dim]: Phi_j(xi0) / (W_j h^dim)
};

struct Receivers {
  int nrec;
  const int* cell;     // [nrec]
  const double* phi;   // [nrec][n^dim] basis values at the receiver
  double* seismo;      // [max_rows][nrec][3]
  long long max_rows;
};

// Arguments of one step's kernels.
struct StepArgs {
  Geometry g;
  PdeParams p;
  const double* u;     // state at t^n
  double* u_next;      // state at t^{n+1} (predictor writes u + volume terms, corrector adds faces)
  double* face;        // per cell, direction, side: time-averaged q (and flux) extrapolations
  double* phi;         // per direction and face: numerical fluxes
  const double* mat;   // [cells][3] or null
  DevScalars* dev;
  int iters;
  PointSrc src;
  double cw0[3][MAXN], cw1[3][MAXN];  // e0/(w h_d), e1/(w h_d): corrector face weights
  double dt_fixed;     // > 0: fixed dt
  double t_end;        // > 0: clip
  double cfl;
  // mixed form of the Euler step: FP64 wave speeds |v_d| + c of the face states
  // [cell][dir][side][face node], evaluated by the predictor and read by the Riemann solver (null:
  // the Riemann solver evaluates them)
  double* fspeed;
  // Euler: the CFL maximum through a binary32 filter with an error bound and FP64 evaluation of
  // the candidates (the same maximum as evaluating every node in FP64); 0: every node
  int cfl_filter;
  // 1: the FP64 Picard predictor starts from the continuous extension Runge-Kutta guess
  int cerk;
  // elastic: per face (directions concatenated) the wave speed max(vp_L, vp_R) and the nine
  // path-averaged coefficients of B_d, formed when the material is set (null: formed per step)
  const double* fmat;
  // hybrid limiter: the cells with FV steps left (nonzero) skip the predictor; their face
  // neighbours compute with FV too, so nothing kept reads their DG data (null: every cell)
  const uint8_t* skip;
};

// Per (pde, dim) kernel family; order dispatch happens inside.
struct Family {
  int nvar;
  bool conservative;   // has a flux F (face records carry Fbar)
  // launchers: return cudaError_t of the launch
  cudaError_t (*cfl)(const StepArgs&, cudaStream_t);
  cudaError_t (*predictor)(const StepArgs&, const Tables&, const TablesF&, int prec, cudaStream_t);
  cudaError_t (*riemann)(const StepArgs&, const Tables&, cudaStream_t);
  cudaError_t (*corrector)(const StepArgs&, const Tables&, cudaStream_t);
  size_t (*predictor_smem)(int order, int prec);
  // limiter (Euler only; null otherwise)
  cudaError_t (*lim_init)(int order, double* u, const double* Usub, const uint8_t* flags,
                          double* rep, double* mm, long long ncells, const SubTables& S,
                          cudaStream_t s);
  cudaError_t (*lim_step)(const StepArgs&, const LimArgs&, const Tables&, const SubTables&,
                          cudaStream_t);
  // adjoint of the linear elastic step (elastic only; null otherwise)
  cudaError_t (*adj_run)(const StepArgs&, const AdjArgs&, const Tables&, int blocks, cudaStream_t);
  long long (*adj_scratch_per_block)(int order, int iters);
  int (*adj_blocks_per_sm)(int order);
  // adjoint of the step with the Cauchy-Kowalevski predictor (prec 0: FP64; otherwise the
  // mixed-precision adjoint of a mixed forward step)
  cudaError_t (*adj_run_ck)(const StepArgs&, const AdjArgs&, const Tables&, const TablesF&,
                            int prec, cudaStream_t);
  // one step of every run of an ensemble (fixed dt, no limiter, no receivers); runs: the runs'
  // step arguments of this step in device memory; null when the family has no batched path
  cudaError_t (*ens_step)(const StepArgs* runs, const EnsTable& E, const Tables& t,
                          const TablesF& f, int prec, int order, cudaStream_t s);
  // Cauchy-Kowalevski predictor (linear systems; null otherwise): same outputs as `predictor`
  cudaError_t (*predictor_ck)(const StepArgs&, const Tables&, const TablesF&, int prec,
                              cudaStream_t);
  // numerical fluxes per face node and variable the Riemann kernel writes (2: the left and right
  // cells see different values, a path-conservative fluctuation); sizes the flux buffer
  int nphi;
  // one step of every run of an ensemble with the Cauchy-Kowalevski predictor (prec 0 FP64, 1
  // mixed; orders with one cell per predictor block); null when the family has no such path
  cudaError_t (*ens_step_ck)(const StepArgs* runs, const EnsTable& E, const Tables& t,
                             const TablesF& f, int prec, int order, cudaStream_t s);
  // `steps` steps of every run of an ensemble as one cooperative persistent launch with grid-wide
  // barriers (bar: device barrier state; limit: polls of a barrier wait before it gives up); null
  // when the family has no batched path
  cudaError_t (*ens_fused)(const StepArgs* runs, const EnsTable& E, const Tables& t,
                           const TablesF& f, int prec, int order, int steps, void* bar,
                           long long limit, int blocks_per_sm, cudaStream_t s);
};
cudaError_t launch_set_scalars(DevScalars* d, double t, double dt, cudaStream_t s);
cudaError_t launch_copy(double* dst, const double* src, long long n, cudaStream_t s);
cudaError_t launch_merge_status(DevScalars* src, DevScalars* dst, cudaStream_t s);
cudaError_t launch_seed_status(const uint8_t* flags, uint8_t* status, long long ncells,
                               int persist, cudaStream_t s);
// FV steps a detected cell keeps under the hybrid limiter status (limiter = 3)
constexpr int LIM_PERSIST = 2;
cudaError_t launch_sub(const double* a, const double* b, double* out, int n, cudaStream_t s);
cudaError_t launch_misfit(const double* a, const double* b, long long n, double scale, double* J,
                          cudaStream_t s);
cudaError_t launch_receivers_adjoint(const Receivers& r, const double* res, double scale,
                                     double* dJdu, int nodes, int nvar, cudaStream_t s);

// Elastic: the per-face material terms of the Riemann solver (StepArgs::fmat), 10 doubles per face
constexpr int FMAT = 10;
cudaError_t launch_face_material_elastic(const Geometry& g, const double* mat, const Tables& t,
                                         double* out, cudaStream_t s);

// orders of the tensor-core Cauchy-Kowalevski predictor (ADER_PREC_MIXED_TF32X3)
bool predictor_ck_tc_order_ok(int order);

const Family* family_advection2();
const Family* family_advection3();
const Family* family_euler2();
const Family* family_euler3();
const Family* family_elastic3();
const Family* family_swe2();
int limiter_max_order2();
int limiter_max_order3();

// Small kernels shared by all families (common.cu).
cudaError_t launch_dt_finalize(const StepArgs& a, cudaStream_t s);
cudaError_t launch_ens_dt(const StepArgs* runs, int nr, cudaStream_t s);
cudaError_t launch_ens_advance(const StepArgs* runs, int nr, cudaStream_t s);
cudaError_t launch_advance(const StepArgs& a, cudaStream_t s);
cudaError_t launch_advance_rec(const StepArgs& a, int receivers_on, cudaStream_t s);
cudaError_t launch_receivers(const StepArgs& a, const Receivers& r, int nodes, int nvar,
                             cudaStream_t s);

}  // namespace ader
