/*
 * ader.h - C ABI of the GB300 ADER-DG time-step library (libader.so).
 *
 * The library advances first-order hyperbolic systems
 *     dQ/dt + div F(Q) + B(Q) . grad Q = S(Q) + sum_i delta_i          (Eq. (1), Sec. 2)
 * on uniform Cartesian grids with the ADER-DG scheme of Sec. 3.3: per cell an element-local
 * space-time predictor (Eq. (5), fixed-point iteration from a constant or a continuous extension
 * Runge-Kutta guess, or the Cauchy-Kowalevski procedure for the linear elastic system), per face
 * a Rusanov numerical flux (with a path-conservative fluctuation for B(Q).grad Q), per cell the
 * corrector Eq. (6), the CFL time step Eq. (7) and, for the Euler equations, the a-posteriori FV
 * subcell limiter of Sec. 3.5.  PDE terms follow the user functions of Table 2 (flux, nonConservativeProduct,
 * pointSource, eigenvalues, boundaryValues, multiplyMaterialParameterMatrix,
 * isPhysicallyAdmissable), built in for three systems: scalar advection (tests), compressible
 * Euler (Eq. (8), gamma-law pressure of Sec. 6.1) and linear elasticity (Sec. 2.1).
 *
 * Conventions for every call:
 *  - All floating-point data are IEEE binary64 ("double").
 *  - State layout: q[cell][node][var], cell = i + nx*(j + ny*k), node = a + n*(b + n*c)
 *    (x fastest), n = order+1 Gauss-Legendre nodes per direction on each cell, nodes
 *    ascending in [0,1] (ader_reference_nodes returns them).
 *  - Pointers are owned by the caller.  The context copies what it needs; it never keeps a
 *    caller pointer except the seismogram buffer of ader_set_receivers.
 *  - "on_device" = 1: the pointer is CUDA device memory of the context's device, used in
 *    stream order on the context's stream; 0: host memory, the call synchronises the stream.
 *  - Calls are asynchronous on the context's stream unless stated otherwise.  Errors found on
 *    the device (non-finite state, inadmissible FV result, a device wait that gave up) are
 *    latched in a device status word and returned by the next synchronising call
 *    (ader_sync, ader_last_dt, ader_get_state with on_device = 0, ...).  No kernel traps.
 *  - A context is not thread-safe.  Calls before the state is set return ADER_ESTATE.
 */
#ifndef ADER_H
#define ADER_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ader_ctx ader_ctx;

typedef enum {
  ADER_OK = 0,
  ADER_EINVAL = 1,        /* bad argument (NULL pointer, size mismatch, out-of-range value) */
  ADER_ENOMEM = 2,        /* device or host allocation failed */
  ADER_ECUDA = 3,         /* a CUDA runtime call failed */
  ADER_ESTATE = 4,        /* call order: e.g. ader_step before ader_set_state */
  ADER_ENONFINITE = 5,    /* a non-finite value appeared in the state */
  ADER_EADMISSIBLE = 6,   /* the FV recompute of a troubled cell is not physically admissible */
  ADER_ETIMEOUT = 7,      /* a bounded device-side wait gave up */
  ADER_EUNSUPPORTED = 8   /* combination of PDE / dimension / order / option not built */
} ader_status;

/* Built-in systems: scalar advection (tests), compressible Euler (Eq. (8)), linear elasticity
 * (Sec. 2.1, 3-D), and the shallow water equations with bathymetry (Eq. (9), 2-D, FP64 Picard
 * predictor): Q = (h, hu, hv, b), flux (h u_d, hu u_d, hv u_d, 0) and the state-dependent
 * non-conservative product g h d(h + b)/dx_d on the momentum of direction d, taken node by node
 * in the predictor and as the path-conservative fluctuation along the straight segment between
 * the face states (3-point rule) at faces.  Shallow water has no limiter: a state whose depth
 * h falls to or below zero gives a non-finite wave speed sqrt(g h), which the CFL reduction of
 * a step with the CFL dt latches as ADER_ENONFINITE. */
typedef enum { ADER_PDE_ADVECTION = 0, ADER_PDE_EULER = 1, ADER_PDE_ELASTIC = 2,
               ADER_PDE_SWE = 3 } ader_pde;

/* Boundary kinds per face (Table 2 "boundaryValues"):
 *  PERIODIC  - wrap around (both faces of a direction must be periodic);
 *  WALL      - reflecting wall: mirror state with the normal momentum negated (Euler, shallow
 *              water);
 *  ABSORBING - zero exterior state for linear PDEs (advection, elastic), a transmissive copy of
 *              the interior state for Euler and shallow water; the exterior material is the
 *              interior one. */
typedef enum { ADER_BC_PERIODIC = 0, ADER_BC_WALL = 1, ADER_BC_ABSORBING = 2 } ader_bc;

/* Arithmetic of the step:
 *  FP64  - everything in binary64;
 *  MIXED - predictor iterations on the increment q - u^n in binary32 with float-float base
 *          terms, time averages and contractions.  Pressure / sound speed and eigenvalues, the
 *          Riemann flux, the corrector and the limiter stay binary64 (for Euler the face wave
 *          speeds are evaluated by the predictor, and the CFL maximum only on the nodes that a
 *          binary32 enclosure cannot rule out; dt equals the FP64 form's on the same state);
 *  MIXED_TF32X3 - the Cauchy-Kowalevski predictor of the elastic family (orders 1, 3, 5) with
 *          every contraction on the tensor cores (tcgen05.mma kind::tf32): the derivatives of the
 *          Taylor coefficients and the face extrapolation of the time average as products with
 *          the 1-D tables, operands split into TF32 hi + lo parts, three products (hi hi, lo hi,
 *          hi lo) accumulated in FP32, relative error about 2^-21 of sum |table| |operand| per
 *          contraction; the material combination and the Taylor recursion in binary32, the
 *          update u + dt vol in FP64.  The error is relative to the size of the wavefield, so the
 *          form suits solutions without a large constant background (the elastic wavefield from
 *          rest).  Other predictors, PDEs or orders: ADER_EUNSUPPORTED.
 * The value 2 (a BF16 x 3 split: 2^-16 per product, above the step-change bound the mixed forms
 * keep) is not built. */
typedef enum { ADER_PREC_FP64 = 0, ADER_PREC_MIXED = 1, ADER_PREC_MIXED_TF32X3 = 3 } ader_prec;

/* Space-time predictor of Sec. 3.3:
 *  PICARD - the element-local space-time system Eq. (5) solved by picard_iters fixed-point
 *           iterations (every PDE);
 *  CK     - the Cauchy-Kowalevski procedure of linear PDEs (Sec. 2, Sec. 3.3): the local Taylor
 *           series in time about t^n, cut after degree N, whose time derivatives are repeated
 *           applications of the spatial operator; a point source's time factor enters through
 *           its degree-N interpolant at the step's Gauss-Legendre time nodes.  Built for the
 *           3-D elastic family (others: ADER_EUNSUPPORTED), with ADER_PREC_FP64 and with
 *           ADER_PREC_MIXED (the O(1) base term L u and the first Taylor coefficient in
 *           float-float, the higher coefficients in binary32, the update u + dt vol in FP64).
 *           Differentiated (orders 1-5): the adjoint entry points take the FP64 adjoint of the
 *           Taylor recursion. */
typedef enum { ADER_PREDICTOR_PICARD = 0, ADER_PREDICTOR_CK = 1 } ader_predictor;

/* Initial guess of the Picard predictor (Sec. 5):
 *  CONSTANT - q^0 = u^n at every time node;
 *  CERK     - the dense output of the classical four-stage Runge-Kutta method on the cell-local
 *             ODE dq/dt = R(q), natural continuous extension of uniform order 3, evaluated at
 *             the time nodes; picard_iters iterations follow (full order needs max(0, N-3)).
 *             The Picard predictor only (else ADER_EUNSUPPORTED), FP64 or MIXED (MIXED: the
 *             stages on the increment u - u^n in binary32 like the iterations); not
 *             differentiated (the adjoint entry points reject it). */
typedef enum { ADER_GUESS_CONSTANT = 0, ADER_GUESS_CERK = 1 } ader_guess;

typedef struct {
  int dim;             /* 2 or 3 (elastic: 3) */
  int order;           /* polynomial order N >= 1 (n = N+1 nodes per direction) */
  int pde;             /* ader_pde */
  int n[3];            /* cells per direction (n[2] ignored for dim = 2) */
  double lo[3], hi[3]; /* domain box */
  int bc[3][2];        /* ader_bc for the low / high face of each direction */
  double cfl;          /* CFL_N of Eq. (7): dt = cfl / (dim (2N+1)) * min h / lambda_max */
  double gamma;        /* ratio of specific heats (Euler), e.g. 1.4 */
  double adv[3];       /* advection velocity (ADER_PDE_ADVECTION) */
  int picard_iters;    /* fixed number of predictor iterations; 0 => order + 1 */
  int limiter;         /* a-posteriori FV subcell limiter (Euler, order <= 4): 0 off, 1 on,
                          2 every cell troubled (the pure FV scheme, for tests), 3 hybrid
                          ADER-DG / FV status (Sec. 3.5): a troubled cell stays FV for two
                          more steps and its face neighbours also compute with FV; a cell
                          with FV steps left, or next to one, is not checked on a DG
                          candidate, and a cell with FV steps left skips the predictor; the
                          counts restart at ader_set_state, and the cells that
                          ader_set_subcell_state puts into the FV space start with two FV
                          steps to take */
  int precision;       /* ader_prec */
  int predictor;       /* ader_predictor (0 = Picard) */
  int initial_guess;   /* ader_guess (0 = constant in time) */
  double grav;         /* gravitational acceleration (ADER_PDE_SWE); <= 0 => 9.81 */
  double adm_floor;    /* limiter, physical admissibility (Table 2 isPhysicallyAdmissable): density
                          and pressure above adm_floor at every node and subcell (<= 0: positive).
                          A step whose MUSCL-Hancock recompute of a troubled cell is not
                          admissible is redone for all its troubled cells with the first-order
                          (zero-slope) scheme; if that is not admissible either, the next
                          synchronising call returns ADER_EADMISSIBLE */
} ader_config;

/* Create a context on the current CUDA device.  `cuda_stream` is a cudaStream_t (NULL = the
 * legacy default stream).  Allocates every device buffer the step needs (the state, the next
 * state, face data, face fluxes, limiter data).  *out is NULL on failure.  ADER_EUNSUPPORTED for
 * combinations the kernels do not cover, among them a predictor whose cell does not fit the
 * 227 KB of shared memory of a thread block (the 3-D Euler MIXED form at order 6). */
ader_status ader_create(const ader_config* cfg, void* cuda_stream, ader_ctx** out);

/* Release the context and its device buffers; NULL-safe.  Synchronises its stream. */
void ader_destroy(ader_ctx* ctx);

/* The library's n = order+1 Gauss-Legendre nodes x[n] (ascending in [0,1]) and weights w[n]
 * (sum 1), host arrays.  Either pointer may be NULL. */
ader_status ader_reference_nodes(int order, double* x, double* w);

/* The library's 1-D reference-element tables for order N (n = N+1), host arrays of n*n doubles,
 * row-major; any pointer may be NULL.  No device is needed.
 *  D[i][m]  = phi_m'(x_i), the collocation derivative on [0,1] (Sec. 3.3);
 *  Kw[k][l] = (K1^{-1} diag(w))[k][l] with K1[k][l] = e1[k] e1[l] - w[l] D[l][k]: the predictor's
 *             time solve q = u + dt Kw R(q) (Eq. (5), time integrated by parts);
 *  Vi[k][t] = coefficient of tau^k of the Lagrange polynomial of time node t: the monomial
 *             coefficients of an interpolant through the time nodes (the Cauchy-Kowalevski
 *             predictor's point-source factor).
 * ADER_EINVAL for an order outside 1..6. */
ader_status ader_reference_tables(int order, double* D, double* Kw, double* Vi);

/* Number of cells, nodes per cell (n^dim: the tensor-product Gauss-Legendre nodes of the nodal DG
 * basis of Sec. 3.3) and variables of the context (the components of Q in Eq. (1)). */
ader_status ader_sizes(const ader_ctx* ctx, int64_t* cells, int64_t* nodes_per_cell, int* nvar);

/* Copy the state in / out: the nodal values of the DG solution u_h of Sec. 3.3 (the unknowns the
 * corrector Eq. (6) updates), [cells][nodes][nvar]; `count` must equal
 * cells * nodes_per_cell * nvar.  Setting the state also resets the limiter history of Sec. 3.5
 * (no cell troubled at the previous step). */
ader_status ader_set_state(ader_ctx* ctx, const double* q, int64_t count, int on_device);
ader_status ader_get_state(ader_ctx* ctx, double* q, int64_t count, int on_device);

/* Advance n independent states held in host memory by one step each (Eq. (5)-(7) as ader_step):
 * h_in[i] (host, ndof doubles) is a state at the context's current time t, h_out[i] (host, ndof
 * doubles) receives the state after one step of it (dt, t_end as in ader_step; every state starts
 * at t).  The host-to-device copy of state i+1 and the device-to-host copy of result i-1 run on
 * two copy streams of the context while state i steps (pinned host memory lets them overlap the
 * step; pageable memory works but serialises); two state-sized device buffers are allocated on
 * the first call.  With the limiter each input's limiter data are initialised as by
 * ader_set_state; receivers, if set, record every state's step.  Synchronises; afterwards the
 * context holds the last result and its time.  Errors as ader_step (a failing step ends the
 * batch; its outputs and later ones are not written). */
ader_status ader_step_host_batch(ader_ctx* ctx, int n, const double* const* h_in,
                                 double* const* h_out, double dt, double t_end);

/* Per-cell material (rho, lambda, mu), [cells][3], for the elastic PDE.  Required before
 * stepping an elastic context. */
ader_status ader_set_material(ader_ctx* ctx, const double* mat, int on_device);

/* Moment-tensor point source (Eq. (1) delta term; Table 2 pointSource) at x0, adding
 * -M R(t) delta(x - x0) to the stress components (xx, yy, zz, xy, xz, yz), R the Ricker wavelet
 * (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2).  Elastic only.  x0 lies in the half-open
 * cell [x_k, x_{k+1}) (the last cell also owns the upper boundary). */
ader_status ader_set_point_source(ader_ctx* ctx, const double x0[3], const double M[6],
                                  double f0, double t0);

/* Receivers at nrec host points xyz[nrec][3]: after every ader_step the velocity
 * (v_x, v_y, v_z) of the new state at each receiver is written to
 * seismo[k][nrec][3] (device memory, capacity `max_steps` rows, k = steps since this call).
 * The caller keeps `seismo` alive while stepping.  Elastic only.  nrec = 0 removes them. */
ader_status ader_set_receivers(ader_ctx* ctx, int nrec, const double* xyz, double* seismo,
                               int64_t max_steps);

/* Simulation time (device-side).  ader_get_time synchronises. */
ader_status ader_set_time(ader_ctx* ctx, double t);
ader_status ader_get_time(ader_ctx* ctx, double* t);

/* One ADER-DG time step on the context's stream.  dt > 0: that step size; dt <= 0: the CFL
 * step of Eq. (7) computed on the device from the current state.  t_end > 0: the step is
 * clipped so that t does not pass t_end (a step at t >= t_end leaves the state unchanged);
 * t_end <= 0: no clipping.  Does not synchronise. */
ader_status ader_step(ader_ctx* ctx, double dt, double t_end);

/* Run `steps` steps (same dt / t_end meaning as ader_step) and synchronise. */
ader_status ader_run(ader_ctx* ctx, int steps, double dt, double t_end);

/* The dt used by the last step (host; synchronises). */
ader_status ader_last_dt(ader_ctx* ctx, double* dt);

/* Limiter history (ader_config.limiter != 0).  ader_set_state resets it: every cell's
 * representation at the current time becomes the subcell averages of its DG polynomial and no
 * cell counts as troubled.  ader_set_subcell_state then puts the cells with flags[c] != 0 into
 * the FV space, as at the start of a limited run along a discontinuity (Sec. 3.5): their
 * representation becomes U_sub[c] ([cells][(2N+1)^dim][nvar], subcell index x fastest; rows of
 * unflagged cells are ignored) and their DG state R(U_sub[c]).  ader_get_subcell_state returns the
 * current representation of every cell. */
ader_status ader_set_subcell_state(ader_ctx* ctx, const double* U_sub, const uint8_t* flags,
                                   int on_device);
ader_status ader_get_subcell_state(ader_ctx* ctx, double* U_sub, int on_device);

/* Cells recomputed with FV at the last step, [cells] bytes (1 = FV), and their count.  With
 * limiter = 1 these are the troubled cells (the a-posteriori detection); with limiter = 3 they
 * are the hybrid FV set: the troubled cells, the cells still counting their FV steps, and the
 * face neighbours of both (the interface layer). */
ader_status ader_get_flags(ader_ctx* ctx, uint8_t* flags, int on_device);
ader_status ader_troubled_count(ader_ctx* ctx, int64_t* count);

/* Synchronise the stream and return (then clear) the latched device status: a non-finite state
 * or time step (ADER_ENONFINITE, found by the CFL reduction of Eq. (7) or the adjoint), an
 * inadmissible FV recompute (ADER_EADMISSIBLE, Sec. 3.5), a bounded device wait that gave up
 * (ADER_ETIMEOUT), a full seismogram buffer (ADER_EINVAL). */
ader_status ader_sync(ader_ctx* ctx);

/* Global time stepping (Sec. 4: every cell advances with the same dt of Eq. (7)) without host
 * round trips: capture `steps` calls of ader_step(dt, t_end) into a CUDA graph and replay it
 * `replays` times
 * (steps * replays steps in total); the graph is kept and reused while (steps, dt, t_end) stay
 * the same.  Does not synchronise. */
ader_status ader_run_graph(ader_ctx* ctx, int steps, int replays, double dt, double t_end);

/* Adjoint of one linear-elastic step (elastic contexts, order <= 5, with the Picard predictor
 * from the constant guess or with the Cauchy-Kowalevski predictor; other predictor settings:
 * ADER_EUNSUPPORTED).  With a fixed dt the step u^{n+1} = A(m) u^n + b^n(M, m) is affine
 * (Eq. (5) predictor, or its Cauchy-Kowalevski form of Sec. 3.3, Rusanov faces, Eq. (6)
 * corrector, moment-tensor point source of Eq. (1)); this call maps lam = lambda^{n+1} to
 *     lambda^n = A(m)^T lambda^{n+1} + dJdu   (in place in `lam`)
 * and accumulates  grad_mat[c][0..2] += d/d(rho, lambda, mu)_c of (lambda^{n+1})^T u^{n+1}  and
 * grad_M[0..5] += d/dM of the same, evaluated at the forward state u_n = u^n with the step
 * starting at time t_n.  With the Picard predictor this is the adjoint of the FP64 step (a MIXED
 * context too).  With the Cauchy-Kowalevski predictor an FP64 context gets the adjoint of its
 * FP64 step, a MIXED or TF32X3 context a mixed-precision adjoint: the base term F + dt L^T lambda
 * in float-float, the level corrections dt L^T mu in binary32, lambda + mu_0 in FP64 (within a
 * few binary32 roundoffs, relative to the largest value, of the FP64 adjoint).  The wave speed max(vp_L, vp_R) of a face takes the left value at
 * ties.  The gradient sums are formed in a fixed order: repeated calls give identical bits.
 * All pointers are device memory of the context's device ([cells][nodes][9] for u_n, lam, dJdu;
 * [cells][3]; [6]); dJdu may be NULL.  Uses the context's material, point source and order; the
 * context's own state and time are not touched.  Stream-ordered, no synchronisation.  The first
 * call allocates its work buffers (ADER_ENOMEM if that fails).  A non-finite adjoint or material
 * gradient (for example from a non-finite u_n) is latched on the device and returned as
 * ADER_ENONFINITE by the next synchronising call (ader_sync). */
ader_status ader_adjoint_step(ader_ctx* ctx, double t_n, double dt, const double* u_n, double* lam,
                              const double* dJdu, double* grad_mat, double* grad_M);

/* Same result as ader_adjoint_step, but this call allocates no memory: its work buffers (the
 * forward Picard iterates kept per thread block (none with the Cauchy-Kowalevski predictor), the
 * face adjoints and the per-face material gradients) live in one fixed 64 MiB array of device memory that the library defines, so no
 * cudaMalloc, cudaFree or other allocating call is made.  It exists for callers that cannot
 * allocate device memory at the time of the call: for example code whose device memory is
 * owned by another allocator (a framework's memory pool that has reserved the GPU), processes
 * that run under a fixed memory budget, or loops that cannot afford the device-wide
 * synchronisation that cudaMalloc and cudaFree imply.  There is no counterpart in the paper.
 * Limits and behaviour:
 *  - The face adjoints (cells x 3 x 2 x n^2 x 9 doubles), the face gradients (6 doubles per
 *    face) and, with the Picard predictor, one iterate slab (order x (order+1) x n^3 x 9
 *    doubles), with the Cauchy-Kowalevski predictor lambda's projections onto the cells' faces
 *    (cells x 3 x 2 x n^2 x 9 doubles), must fit in 64 MiB;
 *    otherwise ADER_EINVAL and nothing runs.  Fewer thread blocks are used when the slabs of all
 *    of them do not fit.
 *  - The array is shared by every call on a device and keeps the contents of the last call
 *    (every location the kernels read is written first in the same call).  Calls whose work
 *    overlaps on the GPU (different streams or contexts on the same device) race on it and must
 *    be ordered by the caller.
 *  - The first call in each CUDA context looks up the array's device address
 *    (cudaGetSymbolAddress; the address is cached per context id, so a context created after a
 *    device reset gets its own); make that first call before any stream capture begins.
 *  - Device-side errors (a non-finite adjoint or gradient) are returned by the next ader_sync,
 *    as for ader_adjoint_step.
 *  - The context's face buffer (and, with the Picard predictor, its next-state buffer), allocated
 *    by ader_create, is overwritten, as in ader_adjoint_step. */
ader_status ader_adjoint_step_static(ader_ctx* ctx, double t_n, double dt, const double* u_n,
                                     double* lam, const double* dJdu, double* grad_mat,
                                     double* grad_M);

/* Transpose of the receiver read-out: dJdu[cell_r][j][v] += scale * res[r][v] * Phi_j(x_r) for the
 * velocity components v = 0..2 of every receiver r (res: device [nrec][3]; dJdu: device state-sized,
 * accumulated).  With res = seismogram - observation and scale = dt this is the derivative of the
 * misfit 1/2 dt sum |v(x_r) - obs|^2 with respect to the state that was recorded. */
ader_status ader_receivers_adjoint(ader_ctx* ctx, const double* res, double scale, double* dJdu);

/* Receiver misfit and its gradient by the adjoint method with checkpointing (elastic contexts
 * with receivers set).  Runs `steps` forward steps of fixed size dt from the device state u0 at
 * time t0, recording the receiver velocities after every step, and evaluates
 *     J = 1/2 dt sum_k sum_r |v_r(u^{k+1}) - obs[k][r]|^2      (obs: device [steps][nrec][3]).
 * If grad_mat or grad_M is non-NULL it then runs the adjoint sweep: the state of every k_ckpt-th
 * step is kept on the device, each segment is recomputed from its checkpoint, and
 * ader_adjoint_step is applied backwards (same predictors as ader_adjoint_step, else
 * ADER_EUNSUPPORTED), writing dJ/d(rho, lambda, mu) per cell to grad_mat
 * (device [cells][3], overwritten) and dJ/dM to grad_M (device [6], overwritten).  J is written
 * to host memory.  Allocates (steps/k_ckpt + k_ckpt + 1) states of work memory for the call.
 * Synchronises.  The context's state afterwards is unspecified (set it again before stepping). */
ader_status ader_misfit_gradient(ader_ctx* ctx, const double* u0, double t0, double dt, int steps,
                                 int k_ckpt, const double* obs, double* J, double* grad_mat,
                                 double* grad_M);

/* Per-phase device timing.  While enabled, every ader_step records CUDA events on the context's
 * stream around its phases: 0 CFL speed reduction, 1 dt finalisation, 2 predictor, 3 Riemann,
 * 4 corrector, 5 limiter, 6 receivers and time advance.  ader_phase_times synchronises, writes
 * the summed milliseconds of each phase over the recorded steps to ms[7], the number of recorded
 * steps to *steps, and clears the record.  Timing adds no synchronisation between steps. */
ader_status ader_enable_timing(ader_ctx* ctx, int on);
ader_status ader_phase_times(ader_ctx* ctx, double ms[7], int* steps);

/* Ensembles of independent runs (several solvers on one machine, Sec. 5.1; batching of uneven
 * grids).  Each run is an ordinary context (its own grid, order, PDE, material, source), created
 * from cfgs[i] on `cuda_stream`.  ader_ensemble_step advances every run by `steps` steps (same dt /
 * t_end meaning as ader_step, applied to each run): all runs' kernels are captured into one CUDA
 * graph of `steps_per_graph` steps, forked over `branches` streams inside the graph and joined,
 * and the graph is replayed (re-captured when the arguments change); a remainder of steps is
 * launched directly.  Not synchronising.  The per-run contexts are owned by the ensemble
 * (ader_ensemble_run); use them to set states, materials, sources and receivers and to read
 * results, but do not destroy them. */
typedef struct ader_ensemble ader_ensemble;
ader_status ader_ensemble_create(const ader_config* cfgs, int nruns, void* cuda_stream,
                                 ader_ensemble** out);
void ader_ensemble_destroy(ader_ensemble* ens);
ader_ctx* ader_ensemble_run(ader_ensemble* ens, int i);
ader_status ader_ensemble_step(ader_ensemble* ens, int steps, double dt, double t_end);
ader_status ader_ensemble_sync(ader_ensemble* ens);
/* Launch shape: steps_per_graph even and >= 2.  branches in [1, 16]: the runs' per-context kernels
 * on that many forked streams inside the graph.  branches = 0: one persistent launch per phase of
 * the step (dt, predictor, Riemann per direction, corrector, time advance) for all runs together,
 * blocks_per_sm (1..8) persistent predictor blocks per SM.  branches = -1: the steps_per_graph
 * steps of all runs as ONE cooperative persistent launch (every block resident), the phases of
 * each step separated by grid-wide barriers (see ader_ensemble_set_wait_limit), blocks_per_sm
 * blocks per SM (at most as many as fit).  Both persistent forms need runs of one PDE family with
 * such a path (elastic, order <= 5), one order, precision, cell size and gamma, a fixed dt, no
 * limiter and no receivers (otherwise the step falls back to one branch).  ADER_EINVAL for other
 * values. */
ader_status ader_ensemble_set_launch(ader_ensemble* ens, int branches, int steps_per_graph,
                                     int blocks_per_sm);
/* Polls of a grid-wide barrier wait of the fused launch before it gives up (default 2^24, about
 * 1.7 s): a block whose wait runs out latches ADER_ETIMEOUT in every run's status word and leaves,
 * the other blocks then run out at the same barrier, and the next synchronising call
 * (ader_ensemble_sync) returns ADER_ETIMEOUT; the barrier is reset before every launch, so the
 * ensemble stays usable (the states of that launch are not).  0 gives up at once (a test knob). */
ader_status ader_ensemble_set_wait_limit(ader_ensemble* ens, int64_t polls);
/* Autotuner: times every candidate launch shape with fixed dt > 0 on the current states (which it
 * restores) and keeps the fastest: branches in {1, 2, 4} and, when the runs allow it, the
 * persistent launches with 1 or 2 blocks per SM, each with steps_per_graph in {2, 4}.
 * best[3] = {branches (0: persistent), steps_per_graph, blocks_per_sm (0 unless persistent)};
 * *ms_per_step receives its time per step.  Synchronises. */
ader_status ader_ensemble_autotune(ader_ensemble* ens, double dt, int* best, double* ms_per_step);

/* Receiver misfit and its gradient for every run of an ensemble (batched adjoint: several
 * seeded elastic runs on uneven grids, each with its own material, source and receivers), the
 * runs' forward sweeps, segment recomputations and adjoint sweeps interleaved step by step on
 * forked streams.  Per run r the call computes what ader_misfit_gradient computes for that
 * context: u0[r] (device state at t0), obs[r] (device [steps][nrec_r][3]), J[r] (host), and, if
 * grad_mat / grad_M are non-NULL, grad_mat[r] (device [cells_r][3]) and grad_M[r] (device [6],
 * overwritten).  The forward steps use each run's own precision (the mixed predictor allowed);
 * the adjoint is that of the FP64 step at those states.  Runs are processed in groups whose work
 * memory ((steps/k_ckpt + k_ckpt + 1) states each) fits mem_budget bytes (<= 0: half of the free
 * device memory; a run that alone exceeds it is processed alone).  Requires material and
 * receivers on every run (ADER_ESTATE otherwise); each run with the Picard predictor from the
 * constant guess or with the Cauchy-Kowalevski predictor (ADER_EUNSUPPORTED otherwise).
 * Synchronises.  The runs' states afterwards are unspecified. */
ader_status ader_ensemble_misfit_gradient(ader_ensemble* ens, const double* const* u0, double t0,
                                          double dt, int steps, int k_ckpt,
                                          const double* const* obs, double* J,
                                          double* const* grad_mat, double* const* grad_M,
                                          int64_t mem_budget);

/* Human-readable name of a status. */
const char* ader_status_string(ader_status s);

#ifdef __cplusplus
}
#endif

#endif /* ADER_H */
