// Host runtime behind the C ABI of include/ader.h: context, reference-element tables, device
// buffers, the per-step kernel sequence and CUDA-graph replay.
#include <cmath>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/ader.h"
#include "ader_internal.h"

using namespace ader;

namespace {

// ---- reference element (host, FP64) ------------------------------------------------------
// Gauss-Legendre nodes and weights on [0,1] by the Golub-Welsch method: eigenvalues of the
// symmetric tridiagonal Jacobi matrix of the Legendre recurrence (off-diagonal
// k / sqrt(4k^2 - 1)), weights 2 v_0^2 from the normalised eigenvectors; eigen-decomposition by
// cyclic Jacobi rotations.
void gauss_legendre_gw(int n, double* x, double* w) {
  double A[MAXNS][MAXNS] = {};
  double V[MAXNS][MAXNS] = {};
  for (int i = 0; i < n; ++i) V[i][i] = 1.0;
  for (int k = 1; k < n; ++k) {
    const double b = k / std::sqrt(4.0 * k * k - 1.0);
    A[k - 1][k] = A[k][k - 1] = b;
  }
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += A[p][q] * A[p][q];
    if (off < 1e-34) break;
    for (int p = 0; p < n; ++p) {
      for (int q = p + 1; q < n; ++q) {
        if (std::fabs(A[p][q]) < 1e-300) continue;
        const double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // A <- A J
          const double akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - s * akq;
          A[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // A <- J^T A
          const double apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - s * aqk;
          A[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {  // V <- V J
          const double vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - s * vkq;
          V[k][q] = s * vkp + c * vkq;
        }
      }
    }
  }
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      if (A[idx[j]][idx[j]] < A[idx[i]][idx[i]]) std::swap(idx[i], idx[j]);
  for (int i = 0; i < n; ++i) {
    const int k = idx[i];
    x[i] = 0.5 * (A[k][k] + 1.0);
    w[i] = V[0][k] * V[0][k];  // 2 v0^2 on [-1,1], halved on [0,1]
  }
  if (n % 2 == 1) x[n / 2] = 0.5;  // exact middle node
}

// Barycentric weights 1 / prod_{k != m} (x_m - x_k).
void bary(int n, const double* x, double* lam) {
  for (int m = 0; m < n; ++m) {
    double p = 1.0;
    for (int k = 0; k < n; ++k)
      if (k != m) p *= (x[m] - x[k]);
    lam[m] = 1.0 / p;
  }
}

// Lagrange basis values at xi by the second barycentric formula.
void basis_at(int n, const double* x, double xi, double* phi) {
  double lam[MAXN];
  bary(n, x, lam);
  for (int m = 0; m < n; ++m)
    if (xi == x[m]) {
      for (int k = 0; k < n; ++k) phi[k] = (k == m) ? 1.0 : 0.0;
      return;
    }
  double den = 0.0;
  for (int m = 0; m < n; ++m) den += lam[m] / (xi - x[m]);
  for (int m = 0; m < n; ++m) phi[m] = lam[m] / (xi - x[m]) / den;
}

// Gauss-Jordan inverse with partial pivoting (n <= MAXN).
bool invert(int n, double (*a)[MAXN], double (*inv)[MAXN]) {
  double m[MAXN][2 * MAXN];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j) m[i][j] = j < n ? a[i][j] : (j - n == i ? 1.0 : 0.0);
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(m[r][c]) > std::fabs(m[piv][c])) piv = r;
    if (std::fabs(m[piv][c]) < 1e-300) return false;
    for (int j = 0; j < 2 * n; ++j) std::swap(m[c][j], m[piv][j]);
    const double d = m[c][c];
    for (int j = 0; j < 2 * n; ++j) m[c][j] /= d;
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = m[r][c];
      for (int j = 0; j < 2 * n; ++j) m[r][j] -= f * m[c][j];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) inv[i][j] = m[i][j + n];
  return true;
}

bool build_tables(int order, Tables& T) {
  std::memset(&T, 0, sizeof(T));
  const int n = order + 1;
  double x[MAXN], w[MAXN], lam[MAXN];
  gauss_legendre_gw(n, x, w);
  bary(n, x, lam);
  for (int i = 0; i < n; ++i) {
    double diag = 0.0;
    for (int m = 0; m < n; ++m) {
      if (m == i) continue;
      T.D[i][m] = (lam[m] / lam[i]) / (x[i] - x[m]);
      diag -= T.D[i][m];
    }
    T.D[i][i] = diag;
  }
  basis_at(n, x, 0.0, T.e0);
  basis_at(n, x, 1.0, T.e1);
  for (int i = 0; i < n; ++i) {
    T.w[i] = w[i];
    T.x[i] = x[i];
    T.c0[i] = T.e0[i] / w[i];
    T.c1[i] = T.e1[i] / w[i];
  }
  // K1[k][l] = e1[k] e1[l] - w[l] D[l][k];  Kw = K1^{-1} diag(w)
  double K1[MAXN][MAXN] = {}, Ki[MAXN][MAXN] = {};
  for (int k = 0; k < n; ++k)
    for (int l = 0; l < n; ++l) K1[k][l] = T.e1[k] * T.e1[l] - w[l] * T.D[l][k];
  if (!invert(n, K1, Ki)) return false;
  for (int k = 0; k < n; ++k)
    for (int l = 0; l < n; ++l) T.Kw[k][l] = Ki[k][l] * w[l];
  double pz[3], pw[3];
  gauss_legendre_gw(3, pz, pw);
  for (int i = 0; i < 3; ++i) {
    T.pz[i] = pz[i];
    T.pw[i] = pw[i];
  }
  // dense output of the four-stage Runge-Kutta guess at the time nodes (natural continuous
  // extension, uniform order 3)
  for (int t = 0; t < n; ++t) {
    const double th = x[t];
    T.cerk[0][t] = th - 1.5 * th * th + 2.0 * th * th * th / 3.0;
    T.cerk[1][t] = th * th - 2.0 * th * th * th / 3.0;
    T.cerk[2][t] = -0.5 * th * th + 2.0 * th * th * th / 3.0;
  }
  // monomial coefficients of the Lagrange polynomials of the time nodes, by expanding the
  // products prod_{m != t} (tau - x_m) / (x_t - x_m) one factor at a time
  for (int t = 0; t < n; ++t) {
    double p[MAXN] = {1.0};
    int deg = 0;
    for (int m = 0; m < n; ++m) {
      if (m == t) continue;
      const double den = x[t] - x[m];
      for (int k = deg + 1; k >= 0; --k)
        p[k] = ((k > 0 ? p[k - 1] : 0.0) - x[m] * (k <= deg ? p[k] : 0.0)) / den;
      ++deg;
    }
    for (int k = 0; k < n; ++k) T.Vi[k][t] = p[k];
  }
  return true;
}

void split_f(double x, float& h, float& l) {
  h = (float)x;
  l = (float)(x - (double)h);
}

void build_tables_f(int order, const Tables& T, TablesF& F) {
  std::memset(&F, 0, sizeof(F));
  const int n = order + 1;
  for (int i = 0; i < n; ++i) {
    double rs = 0.0;
    for (int m = 0; m < n; ++m) {
      split_f(T.D[i][m], F.Dh[i][m], F.Dl[i][m]);
      const double w = T.c1[i] * T.e1[m] - T.c0[i] * T.e0[m] - T.D[i][m];
      split_f(w, F.Wh[i][m], F.Wl[i][m]);
      split_f(T.Kw[i][m], F.Kw[i][m], F.Kwl[i][m]);
      rs += T.Kw[i][m];
    }
    split_f(rs, F.kw1[i], F.kw1l[i]);
    split_f(T.w[i], F.w[i], F.wl[i]);
    split_f(T.e0[i], F.e0h[i], F.e0l[i]);
    split_f(T.e1[i], F.e1h[i], F.e1l[i]);
  }
  // time averages of the time solve: qbar = dt (sum_t w_t kw1_t B0 + sum_m (sum_t w_t Kw[t][m]) R_m)
  double wk1 = 0.0;
  for (int t = 0; t < n; ++t)
    for (int m = 0; m < n; ++m) wk1 += T.w[t] * T.Kw[t][m];
  split_f(wk1, F.wk1h, F.wk1l);
  for (int t = 0; t < n; ++t) {
    F.th[t] = (float)T.x[t];
    for (int i = 0; i < 3; ++i) F.cerk[i][t] = (float)T.cerk[i][t];
  }
  for (int m = 0; m < n; ++m) {
    double a = 0.0;
    for (int t = 0; t < n; ++t) a += T.w[t] * T.Kw[t][m];
    split_f(a, F.wKh[m], F.wKl[m]);
  }
}

// Solve A x = b for several right-hand sides (Gauss-Jordan, partial pivoting); A is m x m.
bool solve_dense(int m, std::vector<double> A, std::vector<double>& B, int nrhs) {
  for (int c = 0; c < m; ++c) {
    int piv = c;
    for (int r = c + 1; r < m; ++r)
      if (std::fabs(A[r * m + c]) > std::fabs(A[piv * m + c])) piv = r;
    if (std::fabs(A[piv * m + c]) < 1e-300) return false;
    if (piv != c) {
      for (int j = 0; j < m; ++j) std::swap(A[c * m + j], A[piv * m + j]);
      for (int j = 0; j < nrhs; ++j) std::swap(B[c * nrhs + j], B[piv * nrhs + j]);
    }
    const double d = A[c * m + c];
    for (int j = 0; j < m; ++j) A[c * m + j] /= d;
    for (int j = 0; j < nrhs; ++j) B[c * nrhs + j] /= d;
    for (int r = 0; r < m; ++r) {
      if (r == c) continue;
      const double f = A[r * m + c];
      if (f == 0.0) continue;
      for (int j = 0; j < m; ++j) A[r * m + j] -= f * A[c * m + j];
      for (int j = 0; j < nrhs; ++j) B[r * nrhs + j] -= f * B[c * nrhs + j];
    }
  }
  return true;
}

// Subcell tables of the limiter (Sec. 3.5): P1[s][m] = mean of phi_m over subcell s, computed
// from the monomial coefficients of phi_m (inverse Vandermonde) and exact antiderivatives;
// R1 = the mean-preserving least-squares left inverse of P1 (KKT system).
bool build_subtables(int order, const Tables& T, SubTables& S) {
  std::memset(&S, 0, sizeof(S));
  const int n = order + 1, ns = 2 * order + 1;
  // coefficients: phi_m(x) = sum_k a[k][m] x^k  <=>  V a = I with V[i][k] = x_i^k
  std::vector<double> V(n * n), a(n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    double p = 1.0;
    for (int k = 0; k < n; ++k) {
      V[i * n + k] = p;
      p *= T.x[i];
    }
    a[i * n + i] = 1.0;
  }
  if (!solve_dense(n, V, a, n)) return false;
  for (int s = 0; s < ns; ++s) {
    const double lo = (double)s / ns, hi = (double)(s + 1) / ns;
    for (int m = 0; m < n; ++m) {
      double acc = 0.0, plo = lo, phi = hi;
      for (int k = 0; k < n; ++k) {
        acc += a[k * n + m] * (phi - plo) / (k + 1);
        plo *= lo;
        phi *= hi;
      }
      S.P1[s][m] = acc * ns;
    }
  }
  // KKT: [2 P1^T P1, w; w^T, 0] [R1; mu] = [2 P1^T; 1^T / ns]
  const int m = n + 1;
  std::vector<double> K(m * m, 0.0), B(m * ns, 0.0);
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) {
      double acc = 0.0;
      for (int s = 0; s < ns; ++s) acc += S.P1[s][i] * S.P1[s][j];
      K[i * m + j] = 2.0 * acc;
    }
    K[i * m + n] = T.w[i];
    K[n * m + i] = T.w[i];
    for (int s = 0; s < ns; ++s) B[i * ns + s] = 2.0 * S.P1[s][i];
  }
  for (int s = 0; s < ns; ++s) B[n * ns + s] = 1.0 / ns;
  if (!solve_dense(m, K, B, ns)) return false;
  for (int i = 0; i < n; ++i)
    for (int s = 0; s < ns; ++s) S.R1[i][s] = B[i * ns + s];
  return true;
}

const Family* pick_family(int pde, int dim) {
  if (pde == ADER_PDE_ADVECTION) return dim == 2 ? family_advection2() : family_advection3();
  if (pde == ADER_PDE_EULER) return dim == 2 ? family_euler2() : family_euler3();
  if (pde == ADER_PDE_ELASTIC && dim == 3) return family_elastic3();
  if (pde == ADER_PDE_SWE && dim == 2) return family_swe2();
  return nullptr;
}

}  // namespace

struct ader_ctx {
  ader_config cfg;
  cudaStream_t stream = nullptr;
  const Family* fam = nullptr;
  Geometry g{};
  PdeParams p{};
  Tables tab{};
  TablesF tabf{};
  SubTables sub{};
  // limiter state (Euler, limiter != 0): representations, their min/max, flags, troubled list
  double *rep = nullptr, *rep_new = nullptr, *mm = nullptr, *mm_new = nullptr, *bflux = nullptr;
  uint8_t* flags = nullptr;
  int* list = nullptr;
  uint8_t *lstatus = nullptr, *lbase = nullptr;  // hybrid status (limiter = 3)
  long long nss = 0;
  // adjoint work buffers (allocated on the first ader_adjoint_step)
  DevScalars* dev_adj = nullptr;
  double *adjf = nullptr, *gface = nullptr, *adj_scratch = nullptr;
  int adj_blocks = 0;
  long long adj_spb = 0;
  long long nodes = 0, nvar = 0, ndof = 0;
  int nf = 0;
  double* u = nullptr;
  double* u_next = nullptr;
  // ader_step_host_batch: staging state buffers (input, output), copy streams and their events
  double* hb_in = nullptr;
  double* hb_out = nullptr;
  cudaStream_t hb_cin = nullptr, hb_cout = nullptr;
  cudaEvent_t hb_ev[4] = {nullptr, nullptr, nullptr, nullptr};
  double* face = nullptr;
  double* phi = nullptr;
  double* fmat = nullptr;    // elastic: per-face material terms of the Riemann solver
  double* fspeed = nullptr;  // mixed Euler: face wave speeds evaluated by the predictor
  double* mat = nullptr;
  DevScalars* dev = nullptr;
  bool state_set = false, mat_set = false;
  PointSrc src{};
  double* src_phi = nullptr;
  Receivers rec{};
  int* rec_cell = nullptr;
  double* rec_phi = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaGraph_t graph = nullptr;
  int g_steps = 0;
  double g_dt = 0, g_tend = 0;
  double* g_u0 = nullptr;
  // per-phase timing
  bool timing = false;
  std::vector<cudaEvent_t> ev;  // 8 events per recorded step
  int ev_used = 0;              // recorded steps
};

static const int NPHASE = 7;

#define CUDA_OK(x)                      \
  do {                                  \
    cudaError_t _e = (x);               \
    if (_e != cudaSuccess) return ADER_ECUDA; \
  } while (0)

static ader_status latched(int bits) {
  if (bits & ST_NONFINITE) return ADER_ENONFINITE;
  if (bits & ST_ADMISSIBLE) return ADER_EADMISSIBLE;
  if (bits & ST_TIMEOUT) return ADER_ETIMEOUT;
  if (bits & ST_SEISMO_FULL) return ADER_EINVAL;
  return ADER_OK;
}

static void free_all(ader_ctx* c) {
  cudaFree(c->dev_adj);
  cudaFree(c->adjf);
  cudaFree(c->gface);
  cudaFree(c->adj_scratch);
  cudaFree(c->rep);
  cudaFree(c->rep_new);
  cudaFree(c->mm);
  cudaFree(c->mm_new);
  cudaFree(c->bflux);
  cudaFree(c->flags);
  cudaFree(c->lstatus);
  cudaFree(c->lbase);
  cudaFree(c->list);
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  c->ev.clear();
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->graph) cudaGraphDestroy(c->graph);
  cudaFree(c->u);
  cudaFree(c->u_next);
  cudaFree(c->face);
  cudaFree(c->phi);
  cudaFree(c->fmat);
  cudaFree(c->hb_in);
  cudaFree(c->hb_out);
  if (c->hb_cin) cudaStreamDestroy(c->hb_cin);
  if (c->hb_cout) cudaStreamDestroy(c->hb_cout);
  for (cudaEvent_t e : c->hb_ev)
    if (e) cudaEventDestroy(e);
  cudaFree(c->fspeed);
  cudaFree(c->mat);
  cudaFree(c->dev);
  cudaFree(c->src_phi);
  cudaFree(c->rec_cell);
  cudaFree(c->rec_phi);
}

// RAII list of device buffers for the checkpointed driver.
struct DevBufs {
  std::vector<void*> p;
  ~DevBufs() {
    for (void* q : p) cudaFree(q);
  }
  template <typename T>
  cudaError_t alloc(T** out, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T));
    if (e == cudaSuccess) p.push_back(q);
    *out = (T*)q;
    return e;
  }
};


extern "C" {

const char* ader_status_string(ader_status s) {
  switch (s) {
    case ADER_OK: return "ok";
    case ADER_EINVAL: return "invalid argument";
    case ADER_ENOMEM: return "out of memory";
    case ADER_ECUDA: return "CUDA error";
    case ADER_ESTATE: return "call order (state not set)";
    case ADER_ENONFINITE: return "non-finite value in the state";
    case ADER_EADMISSIBLE: return "FV recompute not physically admissible";
    case ADER_ETIMEOUT: return "device wait timed out";
    case ADER_EUNSUPPORTED: return "unsupported configuration";
  }
  return "unknown status";
}

ader_status ader_reference_nodes(int order, double* x, double* w) {
  if (order < 1 || order > MAXN - 1) return ADER_EINVAL;
  double xx[MAXN], ww[MAXN];
  gauss_legendre_gw(order + 1, xx, ww);
  for (int i = 0; i <= order; ++i) {
    if (x) x[i] = xx[i];
    if (w) w[i] = ww[i];
  }
  return ADER_OK;
}

ader_status ader_reference_tables(int order, double* D, double* Kw, double* Vi) {
  if (order < 1 || order > MAXN - 1) return ADER_EINVAL;
  Tables T;
  if (!build_tables(order, T)) return ADER_EINVAL;
  const int n = order + 1;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      if (D) D[i * n + j] = T.D[i][j];
      if (Kw) Kw[i * n + j] = T.Kw[i][j];
      if (Vi) Vi[i * n + j] = T.Vi[i][j];
    }
  return ADER_OK;
}

ader_status ader_create(const ader_config* cfg, void* stream, ader_ctx** out) {
  if (!out) return ADER_EINVAL;
  *out = nullptr;
  if (!cfg) return ADER_EINVAL;
  if (cfg->dim < 2 || cfg->dim > 3 || cfg->order < 1 || cfg->order > MAXN - 1) return ADER_EUNSUPPORTED;
  const Family* fam = pick_family(cfg->pde, cfg->dim);
  if (!fam) return ADER_EUNSUPPORTED;
  if (cfg->predictor != ADER_PREDICTOR_PICARD && cfg->predictor != ADER_PREDICTOR_CK) return ADER_EINVAL;
  if (cfg->precision != ADER_PREC_FP64 && cfg->precision != ADER_PREC_MIXED &&
      cfg->precision != ADER_PREC_MIXED_TF32X3)
    return ADER_EUNSUPPORTED;
  // the tensor-core form: the Cauchy-Kowalevski predictor of the elastic family, orders 1, 3, 5
  if (cfg->precision == ADER_PREC_MIXED_TF32X3 &&
      (cfg->predictor != ADER_PREDICTOR_CK || cfg->pde != ADER_PDE_ELASTIC ||
       !predictor_ck_tc_order_ok(cfg->order)))
    return ADER_EUNSUPPORTED;
  if (cfg->predictor == ADER_PREDICTOR_CK && (!fam->predictor_ck || cfg->limiter))
    return ADER_EUNSUPPORTED;
  if (cfg->initial_guess != ADER_GUESS_CONSTANT && cfg->initial_guess != ADER_GUESS_CERK)
    return ADER_EINVAL;
  if (cfg->initial_guess == ADER_GUESS_CERK && cfg->predictor != ADER_PREDICTOR_PICARD)
    return ADER_EUNSUPPORTED;
  // shallow water: FP64 Picard predictor from the constant guess
  if (cfg->pde == ADER_PDE_SWE &&
      (cfg->precision != ADER_PREC_FP64 || cfg->initial_guess != ADER_GUESS_CONSTANT))
    return ADER_EUNSUPPORTED;
  // the predictor keeps a cell in shared memory: at most 227 KB per block on sm_103a, less the
  // kernel's static tables (the 3-D Euler mixed form at order 6 does not fit)
  if (cfg->predictor == ADER_PREDICTOR_PICARD &&
      fam->predictor_smem(cfg->order, cfg->precision) > 232448 - 4096)
    return ADER_EUNSUPPORTED;
  if (cfg->limiter < 0 || cfg->limiter > 3) return ADER_EINVAL;
  if (cfg->limiter) {
    if (cfg->pde != ADER_PDE_EULER) return ADER_EUNSUPPORTED;
    if (cfg->order > (cfg->dim == 2 ? limiter_max_order2() : limiter_max_order3())) return ADER_EUNSUPPORTED;
  }
  if (!(cfg->cfl > 0.0)) return ADER_EINVAL;
  long long ncells = 1;
  for (int d = 0; d < cfg->dim; ++d) {
    if (cfg->n[d] < 1 || !(cfg->hi[d] > cfg->lo[d])) return ADER_EINVAL;
    for (int s = 0; s < 2; ++s)
      if (cfg->bc[d][s] < 0 || cfg->bc[d][s] > 2) return ADER_EINVAL;
    if ((cfg->bc[d][0] == ADER_BC_PERIODIC) != (cfg->bc[d][1] == ADER_BC_PERIODIC)) return ADER_EINVAL;
    if (cfg->pde != ADER_PDE_EULER && cfg->pde != ADER_PDE_SWE)
      for (int s = 0; s < 2; ++s)
        if (cfg->bc[d][s] == ADER_BC_WALL) return ADER_EUNSUPPORTED;
    ncells *= cfg->n[d];
  }
  ader_ctx* c = new (std::nothrow) ader_ctx();
  if (!c) return ADER_ENOMEM;
  c->cfg = *cfg;
  c->stream = (cudaStream_t)stream;
  c->fam = fam;
  Geometry& g = c->g;
  g.dim = cfg->dim;
  g.order = cfg->order;
  g.ncells = ncells;
  for (int d = 0; d < 3; ++d) {
    g.n[d] = d < cfg->dim ? cfg->n[d] : 1;
    g.lo[d] = d < cfg->dim ? cfg->lo[d] : 0.0;
    g.h[d] = d < cfg->dim ? (cfg->hi[d] - cfg->lo[d]) / cfg->n[d] : 1.0;
    g.inv_h[d] = 1.0 / g.h[d];
    g.bc[d][0] = d < cfg->dim ? cfg->bc[d][0] : 0;
    g.bc[d][1] = d < cfg->dim ? cfg->bc[d][1] : 0;
  }
  c->p.gamma = cfg->gamma > 0 ? cfg->gamma : 1.4;
  c->p.grav = cfg->grav > 0 ? cfg->grav : 9.81;
  for (int d = 0; d < 3; ++d) c->p.a[d] = cfg->adv[d];
  if (!build_tables(cfg->order, c->tab)) {
    delete c;
    return ADER_EINVAL;
  }
  build_tables_f(cfg->order, c->tab, c->tabf);
  for (int d = 0; d < 3; ++d) split_f(c->g.inv_h[d], c->tabf.ihh[d], c->tabf.ihl[d]);
  split_f(c->p.gamma - 1.0, c->tabf.g1h, c->tabf.g1l);
  const int n = cfg->order + 1;
  c->nodes = 1;
  for (int d = 0; d < cfg->dim; ++d) c->nodes *= n;
  c->nvar = fam->nvar;
  c->ndof = ncells * c->nodes * c->nvar;
  c->nf = (int)(c->nodes / n);
  const long long face_rec = (long long)c->nf * c->nvar * (fam->conservative ? 2 : 1);
  const int nphi = fam->nphi;  // as many fluxes per face node as the family's kernels write
  long long nphi_total = 0;
  for (int d = 0; d < cfg->dim; ++d)
    nphi_total += (long long)(g.n[d] + 1) * (ncells / g.n[d]) * nphi * c->nf * c->nvar;
  cudaError_t e = cudaSuccess;
  e = cudaMalloc(&c->u, c->ndof * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->u_next, c->ndof * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->face, ncells * cfg->dim * 2 * face_rec * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->phi, nphi_total * sizeof(double));
  if (e == cudaSuccess && cfg->precision == ADER_PREC_MIXED && cfg->pde == ADER_PDE_EULER)
    e = cudaMalloc(&c->fspeed, ncells * cfg->dim * 2 * c->nf * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->dev, sizeof(DevScalars));
  if (e == cudaSuccess && cfg->pde == ADER_PDE_ELASTIC) e = cudaMalloc(&c->mat, ncells * 3 * sizeof(double));
  if (cfg->limiter) {
    const int ns = 2 * cfg->order + 1;
    c->nss = 1;
    long long nsf = 1;
    for (int d = 0; d < cfg->dim; ++d) c->nss *= ns;
    for (int d = 1; d < cfg->dim; ++d) nsf *= ns;
    if (!build_subtables(cfg->order, c->tab, c->sub)) e = cudaErrorInvalidValue;
    const size_t nrep = (size_t)ncells * c->nss * c->nvar;
    if (e == cudaSuccess) e = cudaMalloc(&c->rep, nrep * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&c->rep_new, nrep * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&c->mm, ncells * 2 * c->nvar * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&c->mm_new, ncells * 2 * c->nvar * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&c->bflux, (size_t)ncells * cfg->dim * 2 * nsf * c->nvar * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&c->flags, ncells);
    if (e == cudaSuccess) e = cudaMalloc(&c->list, ncells * sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(c->flags, 0, ncells, c->stream);
    if (cfg->limiter == 3) {
      if (e == cudaSuccess) e = cudaMalloc(&c->lstatus, ncells);
      if (e == cudaSuccess) e = cudaMalloc(&c->lbase, ncells);
      if (e == cudaSuccess) e = cudaMemsetAsync(c->lstatus, 0, ncells, c->stream);
      // the cells with FV steps left skip the predictor: their face records and candidate hold
      // finite (unused) values from the start
      if (e == cudaSuccess)
        e = cudaMemsetAsync(c->face, 0, ncells * cfg->dim * 2 * face_rec * sizeof(double), c->stream);
      if (e == cudaSuccess) e = cudaMemsetAsync(c->u_next, 0, c->ndof * sizeof(double), c->stream);
      if (e == cudaSuccess && c->fspeed)
        e = cudaMemsetAsync(c->fspeed, 0, ncells * cfg->dim * 2 * c->nf * sizeof(double), c->stream);
    }
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_all(c);
    delete c;
    return e == cudaErrorMemoryAllocation ? ADER_ENOMEM : ADER_ECUDA;
  }
  e = cudaMemsetAsync(c->dev, 0, sizeof(DevScalars), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->phi, 0, nphi_total * sizeof(double), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    free_all(c);
    delete c;
    return ADER_ECUDA;
  }
  c->src.cell = -1;
  *out = c;
  return ADER_OK;
}

void ader_destroy(ader_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  free_all(c);
  delete c;
}

ader_status ader_sizes(const ader_ctx* c, int64_t* cells, int64_t* nodes, int* nvar) {
  if (!c) return ADER_EINVAL;
  if (cells) *cells = c->g.ncells;
  if (nodes) *nodes = c->nodes;
  if (nvar) *nvar = (int)c->nvar;
  return ADER_OK;
}

static ader_status copy(void* dst, const void* src, size_t bytes, cudaMemcpyKind kind,
                        cudaStream_t s, bool sync) {
  CUDA_OK(cudaMemcpyAsync(dst, src, bytes, kind, s));
  if (sync) CUDA_OK(cudaStreamSynchronize(s));
  return ADER_OK;
}

ader_status ader_set_state(ader_ctx* c, const double* q, int64_t count, int on_device) {
  if (!c || !q || count != c->ndof) return ADER_EINVAL;
  ader_status st = copy(c->u, q, count * sizeof(double),
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream,
                        !on_device);
  if (st != ADER_OK) return st;
  if (c->cfg.limiter) {
    CUDA_OK(c->fam->lim_init(c->cfg.order, c->u, nullptr, nullptr, c->rep, c->mm, c->g.ncells,
                             c->sub, c->stream));
    CUDA_OK(cudaMemsetAsync(c->flags, 0, c->g.ncells, c->stream));
    if (c->lstatus) CUDA_OK(cudaMemsetAsync(c->lstatus, 0, c->g.ncells, c->stream));
  }
  c->state_set = true;
  return ADER_OK;
}

ader_status ader_set_subcell_state(ader_ctx* c, const double* U_sub, const uint8_t* flags,
                                   int on_device) {
  if (!c || !U_sub || !flags) return ADER_EINVAL;
  if (!c->cfg.limiter) return ADER_EUNSUPPORTED;
  if (!c->state_set) return ADER_ESTATE;
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  ader_status st = copy(c->rep_new, U_sub, (size_t)c->g.ncells * c->nss * c->nvar * sizeof(double),
                        k, c->stream, false);
  if (st == ADER_OK) st = copy(c->flags, flags, c->g.ncells, k, c->stream, false);
  if (st != ADER_OK) return st;
  CUDA_OK(c->fam->lim_init(c->cfg.order, c->u, c->rep_new, c->flags, c->rep, c->mm, c->g.ncells,
                           c->sub, c->stream));
  // hybrid status: the cells put into the FV space stay FV for LIM_PERSIST steps
  if (c->lstatus)
    CUDA_OK(launch_seed_status(c->flags, c->lstatus, c->g.ncells, LIM_PERSIST, c->stream));
  if (!on_device) CUDA_OK(cudaStreamSynchronize(c->stream));
  return ADER_OK;
}

ader_status ader_get_subcell_state(ader_ctx* c, double* U_sub, int on_device) {
  if (!c || !U_sub) return ADER_EINVAL;
  if (!c->cfg.limiter) return ADER_EUNSUPPORTED;
  if (!c->state_set) return ADER_ESTATE;
  return copy(U_sub, c->rep, (size_t)c->g.ncells * c->nss * c->nvar * sizeof(double),
              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream, !on_device);
}

ader_status ader_get_state(ader_ctx* c, double* q, int64_t count, int on_device) {
  if (!c || !q || count != c->ndof) return ADER_EINVAL;
  if (!c->state_set) return ADER_ESTATE;
  return copy(q, c->u, count * sizeof(double),
              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream, !on_device);
}

static ader_status step_impl(ader_ctx* c, double dt, double t_end);

ader_status ader_step_host_batch(ader_ctx* c, int n, const double* const* h_in,
                                 double* const* h_out, double dt, double t_end) {
  if (!c || n < 1 || !h_in || !h_out) return ADER_EINVAL;
  for (int i = 0; i < n; ++i)
    if (!h_in[i] || !h_out[i]) return ADER_EINVAL;
  if (c->cfg.pde == ADER_PDE_ELASTIC && !c->mat_set) return ADER_ESTATE;
  const size_t bytes = (size_t)c->ndof * sizeof(double);
  if (!c->hb_in) {
    cudaError_t e = cudaMalloc(&c->hb_in, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&c->hb_out, bytes);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->hb_cin, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->hb_cout, cudaStreamNonBlocking);
    for (int k = 0; k < 4 && e == cudaSuccess; ++k)
      e = cudaEventCreateWithFlags(&c->hb_ev[k], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? ADER_ENOMEM : ADER_ECUDA;
    }
  }
  double t0 = 0.0;
  CUDA_OK(cudaMemcpyAsync(&t0, &c->dev->t, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_OK(cudaStreamSynchronize(c->stream));
  // events: 0 input landed in hb_in, 1 hb_in consumed (copied into the state), 2 result in
  // hb_out, 3 hb_out drained to the host
  cudaEvent_t in_ready = c->hb_ev[0], in_free = c->hb_ev[1], out_ready = c->hb_ev[2],
              out_free = c->hb_ev[3];
  CUDA_OK(cudaMemcpyAsync(c->hb_in, h_in[0], bytes, cudaMemcpyHostToDevice, c->hb_cin));
  CUDA_OK(cudaEventRecord(in_ready, c->hb_cin));
  ader_status st = ADER_OK;
  for (int i = 0; i < n && st == ADER_OK; ++i) {
    // the input into the state; the next input may then land in hb_in while this one steps
    CUDA_OK(cudaStreamWaitEvent(c->stream, in_ready, 0));
    CUDA_OK(launch_copy(c->u, c->hb_in, c->ndof, c->stream));
    CUDA_OK(cudaEventRecord(in_free, c->stream));
    if (i + 1 < n) {
      CUDA_OK(cudaStreamWaitEvent(c->hb_cin, in_free, 0));
      CUDA_OK(cudaMemcpyAsync(c->hb_in, h_in[i + 1], bytes, cudaMemcpyHostToDevice, c->hb_cin));
      CUDA_OK(cudaEventRecord(in_ready, c->hb_cin));
    }
    if (c->cfg.limiter) {
      CUDA_OK(c->fam->lim_init(c->cfg.order, c->u, nullptr, nullptr, c->rep, c->mm, c->g.ncells,
                               c->sub, c->stream));
      CUDA_OK(cudaMemsetAsync(c->flags, 0, c->g.ncells, c->stream));
      if (c->lstatus) CUDA_OK(cudaMemsetAsync(c->lstatus, 0, c->g.ncells, c->stream));
    }
    c->state_set = true;
    CUDA_OK(launch_set_scalars(c->dev, t0, 0.0, c->stream));
    st = step_impl(c, dt, t_end);
    if (st != ADER_OK) break;
    // the result into hb_out once the previous result has left it, then to the host
    if (i > 0) CUDA_OK(cudaStreamWaitEvent(c->stream, out_free, 0));
    CUDA_OK(launch_copy(c->hb_out, c->u, c->ndof, c->stream));
    CUDA_OK(cudaEventRecord(out_ready, c->stream));
    CUDA_OK(cudaStreamWaitEvent(c->hb_cout, out_ready, 0));
    CUDA_OK(cudaMemcpyAsync(h_out[i], c->hb_out, bytes, cudaMemcpyDeviceToHost, c->hb_cout));
    CUDA_OK(cudaEventRecord(out_free, c->hb_cout));
  }
  CUDA_OK(cudaStreamSynchronize(c->hb_cin));
  CUDA_OK(cudaStreamSynchronize(c->hb_cout));
  CUDA_OK(cudaStreamSynchronize(c->stream));
  if (st != ADER_OK) return st;
  return ader_sync(c);
}

ader_status ader_set_material(ader_ctx* c, const double* mat, int on_device) {
  if (!c || !mat) return ADER_EINVAL;
  if (c->cfg.pde != ADER_PDE_ELASTIC) return ADER_EUNSUPPORTED;
  if (!on_device) {
    for (long long i = 0; i < c->g.ncells; ++i)
      if (!(mat[3 * i] > 0) || !(mat[3 * i + 2] > 0) || !(mat[3 * i + 1] + 2 * mat[3 * i + 2] > 0))
        return ADER_EINVAL;
  }
  ader_status st = copy(c->mat, mat, c->g.ncells * 3 * sizeof(double),
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream,
                        !on_device);
  if (st != ADER_OK) return st;
  // the Riemann solver's per-face material terms (speed and path-averaged coefficients)
  if (!c->fmat) {
    long long nf = 0;
    for (int d = 0; d < 3; ++d) nf += (long long)(c->g.n[d] + 1) * (c->g.ncells / c->g.n[d]);
    const cudaError_t e = cudaMalloc(&c->fmat, (size_t)nf * FMAT * sizeof(double));
    if (e != cudaSuccess) {
      cudaGetLastError();
      c->fmat = nullptr;
      return e == cudaErrorMemoryAllocation ? ADER_ENOMEM : ADER_ECUDA;
    }
  }
  CUDA_OK(launch_face_material_elastic(c->g, c->mat, c->tab, c->fmat, c->stream));
  c->mat_set = true;
  return ADER_OK;
}

// Cell and reference coordinates of a point (half-open cells, last cell owns the upper face).
static long long locate(const ader_ctx* c, const double* x, double* xi) {
  long long cell = 0, stride = 1;
  for (int d = 0; d < c->g.dim; ++d) {
    const double s = (x[d] - c->g.lo[d]) / c->g.h[d];
    long long k = (long long)std::floor(s);
    if (k < 0) k = 0;
    if (k > c->g.n[d] - 1) k = c->g.n[d] - 1;
    xi[d] = s - (double)k;
    cell += k * stride;
    stride *= c->g.n[d];
  }
  return cell;
}

// Phi_j(xi) = prod_d phi_{j_d}(xi_d) for every node j (x fastest).
static void tensor_basis(const ader_ctx* c, const double* xi, double* out) {
  const int n = c->g.order + 1;
  double b[3][MAXN];
  for (int d = 0; d < c->g.dim; ++d) basis_at(n, c->tab.x, xi[d], b[d]);
  for (long long j = 0; j < c->nodes; ++j) {
    long long r = j;
    double v = 1.0;
    for (int d = 0; d < c->g.dim; ++d) {
      v *= b[d][r % n];
      r /= n;
    }
    out[j] = v;
  }
}

ader_status ader_set_point_source(ader_ctx* c, const double x0[3], const double M[6], double f0,
                                  double t0) {
  if (!c || !x0 || !M) return ADER_EINVAL;
  if (c->cfg.pde != ADER_PDE_ELASTIC) return ADER_EUNSUPPORTED;
  for (int d = 0; d < 3; ++d)
    if (!(x0[d] >= c->g.lo[d]) || !(x0[d] <= c->g.lo[d] + c->g.h[d] * c->g.n[d])) return ADER_EINVAL;
  double xi[3];
  const long long cell = locate(c, x0, xi);
  std::vector<double> phi(c->nodes);
  tensor_basis(c, xi, phi.data());
  const int n = c->g.order + 1;
  double vol = 1.0;
  for (int d = 0; d < c->g.dim; ++d) vol *= c->g.h[d];
  for (long long j = 0; j < c->nodes; ++j) {
    long long r = j;
    double W = 1.0;
    for (int d = 0; d < c->g.dim; ++d) {
      W *= c->tab.w[r % n];
      r /= n;
    }
    phi[j] /= (W * vol);
  }
  if (!c->src_phi) CUDA_OK(cudaMalloc(&c->src_phi, c->nodes * sizeof(double)));
  ader_status st = copy(c->src_phi, phi.data(), c->nodes * sizeof(double), cudaMemcpyHostToDevice,
                        c->stream, true);
  if (st != ADER_OK) return st;
  c->src.cell = (int)cell;
  for (int a = 0; a < 6; ++a) c->src.M[a] = M[a];
  c->src.f0 = f0;
  c->src.t0 = t0;
  c->src.phi = c->src_phi;
  return ADER_OK;
}

ader_status ader_set_receivers(ader_ctx* c, int nrec, const double* xyz, double* seismo,
                               int64_t max_steps) {
  if (!c || nrec < 0) return ADER_EINVAL;
  if (c->cfg.pde != ADER_PDE_ELASTIC) return ADER_EUNSUPPORTED;
  cudaFree(c->rec_cell);
  cudaFree(c->rec_phi);
  c->rec_cell = nullptr;
  c->rec_phi = nullptr;
  c->rec.nrec = 0;
  if (nrec == 0) return ADER_OK;
  if (!xyz || !seismo || max_steps < 1) return ADER_EINVAL;
  std::vector<int> cells(nrec);
  std::vector<double> phi((size_t)nrec * c->nodes);
  for (int r = 0; r < nrec; ++r) {
    double xi[3];
    cells[r] = (int)locate(c, xyz + 3 * r, xi);
    tensor_basis(c, xi, phi.data() + (size_t)r * c->nodes);
  }
  CUDA_OK(cudaMalloc(&c->rec_cell, nrec * sizeof(int)));
  CUDA_OK(cudaMalloc(&c->rec_phi, phi.size() * sizeof(double)));
  ader_status st = copy(c->rec_cell, cells.data(), nrec * sizeof(int), cudaMemcpyHostToDevice, c->stream, false);
  if (st == ADER_OK)
    st = copy(c->rec_phi, phi.data(), phi.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream, true);
  if (st != ADER_OK) return st;
  // restart the row counter
  long long zero = 0;
  st = copy(&c->dev->seismo_row, &zero, sizeof(long long), cudaMemcpyHostToDevice, c->stream, true);
  if (st != ADER_OK) return st;
  c->rec.nrec = nrec;
  c->rec.cell = c->rec_cell;
  c->rec.phi = c->rec_phi;
  c->rec.seismo = seismo;
  c->rec.max_rows = max_steps;
  return ADER_OK;
}

ader_status ader_set_time(ader_ctx* c, double t) {
  if (!c) return ADER_EINVAL;
  return copy(&c->dev->t, &t, sizeof(double), cudaMemcpyHostToDevice, c->stream, true);
}

ader_status ader_get_time(ader_ctx* c, double* t) {
  if (!c || !t) return ADER_EINVAL;
  return copy(t, &c->dev->t, sizeof(double), cudaMemcpyDeviceToHost, c->stream, true);
}

static StepArgs make_args(ader_ctx* c, double dt, double t_end) {
  StepArgs a{};
  a.g = c->g;
  a.p = c->p;
  a.u = c->u;
  a.u_next = c->u_next;
  a.face = c->face;
  a.phi = c->phi;
  a.mat = c->mat;
  a.fmat = c->mat_set ? c->fmat : nullptr;
  a.dev = c->dev;
  a.iters = c->cfg.picard_iters > 0 ? c->cfg.picard_iters : c->cfg.order + 1;
  a.cerk = c->cfg.initial_guess == ADER_GUESS_CERK ? 1 : 0;
  a.skip = c->cfg.limiter == 3 ? c->lstatus : nullptr;
  a.src = c->src;
  a.dt_fixed = dt > 0 ? dt : 0.0;
  a.t_end = t_end > 0 ? t_end : 0.0;
  a.cfl = c->cfg.cfl;
  for (int d = 0; d < 3; ++d)
    for (int m = 0; m < MAXN; ++m) {
      a.cw0[d][m] = c->tab.c0[m] * c->g.inv_h[d];
      a.cw1[d][m] = c->tab.c1[m] * c->g.inv_h[d];
    }
  return a;
}

// Event slot for phase boundary k of the step being recorded (nullptr when not timing).
static cudaEvent_t mark_event(ader_ctx* c, int k) {
  if (!c->timing) return nullptr;
  const size_t need = (size_t)(c->ev_used + 1) * (NPHASE + 1);
  while (c->ev.size() < need) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    c->ev.push_back(e);
  }
  return c->ev[(size_t)c->ev_used * (NPHASE + 1) + k];
}

static ader_status mark(ader_ctx* c, int k) {
  cudaEvent_t e = mark_event(c, k);
  if (e) CUDA_OK(cudaEventRecord(e, c->stream));
  return ADER_OK;
}

static ader_status step_impl(ader_ctx* c, double dt, double t_end) {
  StepArgs a = make_args(c, dt, t_end);
  a.fspeed = c->fspeed;  // mixed Euler step: face speeds evaluated by the predictor
  // the filtered CFL maximum pays off from ~2^18 nodes; below, the plain FP64 pass has less latency
  a.cfl_filter = (c->cfg.pde == ADER_PDE_EULER && c->g.ncells * c->nodes >= (1LL << 18)) ? 1 : 0;
  cudaStream_t s = c->stream;
  ader_status st;
  if ((st = mark(c, 0)) != ADER_OK) return st;
  if (!(dt > 0)) CUDA_OK(c->fam->cfl(a, s));
  if ((st = mark(c, 1)) != ADER_OK) return st;
  CUDA_OK(launch_dt_finalize(a, s));
  if ((st = mark(c, 2)) != ADER_OK) return st;
  if (c->cfg.predictor == ADER_PREDICTOR_CK) {
    CUDA_OK(c->fam->predictor_ck(a, c->tab, c->tabf, c->cfg.precision, s));
  } else {
    CUDA_OK(c->fam->predictor(a, c->tab, c->tabf, c->cfg.precision, s));
  }
  if ((st = mark(c, 3)) != ADER_OK) return st;
  CUDA_OK(c->fam->riemann(a, c->tab, s));
  if ((st = mark(c, 4)) != ADER_OK) return st;
  CUDA_OK(c->fam->corrector(a, c->tab, s));
  if ((st = mark(c, 5)) != ADER_OK) return st;
  if (c->cfg.limiter) {
    LimArgs l{c->rep, c->rep_new, c->mm, c->mm_new, nullptr, c->flags, c->list, c->bflux,
              c->cfg.limiter == 2 ? 1 : 0, 1e-4, 1e-3};
    if (c->cfg.limiter == 3) {
      l.status = c->lstatus;
      l.base = c->lbase;
      l.persist = LIM_PERSIST;
    }
    l.floor = c->cfg.adm_floor > 0.0 ? c->cfg.adm_floor : 0.0;
    l.first_order = 0;
    CUDA_OK(c->fam->lim_step(a, l, c->tab, c->sub, s));
    std::swap(c->rep, c->rep_new);
    std::swap(c->mm, c->mm_new);
  }
  if ((st = mark(c, 6)) != ADER_OK) return st;
  if (c->rec.nrec > 0) CUDA_OK(launch_receivers(a, c->rec, (int)c->nodes, (int)c->nvar, s));
  CUDA_OK(launch_advance_rec(a, c->rec.nrec > 0, s));
  if ((st = mark(c, 7)) != ADER_OK) return st;
  if (c->timing) c->ev_used++;
  std::swap(c->u, c->u_next);
  return ADER_OK;
}

ader_status ader_step(ader_ctx* c, double dt, double t_end) {
  if (!c) return ADER_EINVAL;
  if (!c->state_set) return ADER_ESTATE;
  if (c->cfg.pde == ADER_PDE_ELASTIC && !c->mat_set) return ADER_ESTATE;
  if (!(dt == dt) || !(t_end == t_end)) return ADER_EINVAL;
  return step_impl(c, dt, t_end);
}

ader_status ader_sync(ader_ctx* c) {
  if (!c) return ADER_EINVAL;
  CUDA_OK(cudaStreamSynchronize(c->stream));
  int bits = 0;
  CUDA_OK(cudaMemcpy(&bits, &c->dev->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (bits) {
    int zero = 0;
    CUDA_OK(cudaMemcpy(&c->dev->status, &zero, sizeof(int), cudaMemcpyHostToDevice));
  }
  return latched(bits);
}

ader_status ader_run(ader_ctx* c, int steps, double dt, double t_end) {
  if (!c || steps < 0) return ADER_EINVAL;
  for (int i = 0; i < steps; ++i) {
    ader_status st = ader_step(c, dt, t_end);
    if (st != ADER_OK) return st;
  }
  return ader_sync(c);
}

ader_status ader_last_dt(ader_ctx* c, double* dt) {
  if (!c || !dt) return ADER_EINVAL;
  ader_status st = copy(dt, &c->dev->dt, sizeof(double), cudaMemcpyDeviceToHost, c->stream, true);
  if (st != ADER_OK) return st;
  return ader_sync(c);
}

ader_status ader_get_flags(ader_ctx* c, uint8_t* flags, int on_device) {
  if (!c || !flags) return ADER_EINVAL;
  if (!c->cfg.limiter) {
    if (on_device) {
      CUDA_OK(cudaMemsetAsync(flags, 0, c->g.ncells, c->stream));
    } else {
      std::memset(flags, 0, c->g.ncells);
    }
    return ADER_OK;
  }
  return copy(flags, c->flags, c->g.ncells,
              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream, !on_device);
}

ader_status ader_troubled_count(ader_ctx* c, int64_t* count) {
  if (!c || !count) return ADER_EINVAL;
  int n = 0;
  if (c->cfg.limiter) {
    ader_status st = copy(&n, &c->dev->n_troubled, sizeof(int), cudaMemcpyDeviceToHost, c->stream, true);
    if (st != ADER_OK) return st;
  }
  *count = n;
  return ADER_OK;
}

// Whether the context's step has a hand-written adjoint: the elastic step, orders 1-5, with the
// Picard predictor from the constant guess or with the Cauchy-Kowalevski predictor.
static bool adjoint_supported(const ader_ctx* c) {
  if (c->cfg.pde != ADER_PDE_ELASTIC || c->cfg.order > 5) return false;
  if (c->cfg.predictor == ADER_PREDICTOR_CK) return c->fam->adj_run_ck != nullptr;
  return c->fam->adj_run && c->cfg.predictor == ADER_PREDICTOR_PICARD &&
         c->cfg.initial_guess == ADER_GUESS_CONSTANT;
}

ader_status ader_adjoint_step(ader_ctx* c, double t_n, double dt, const double* u_n, double* lam,
                              const double* dJdu, double* grad_mat, double* grad_M) {
  if (!c || !u_n || !lam || !grad_mat || !grad_M || !(dt > 0.0)) return ADER_EINVAL;
  if (!adjoint_supported(c)) return ADER_EUNSUPPORTED;
  if (!c->mat_set) return ADER_ESTATE;
  const bool ck = c->cfg.predictor == ADER_PREDICTOR_CK;
  const int iters = c->cfg.picard_iters > 0 ? c->cfg.picard_iters : c->cfg.order + 1;
  if (!c->dev_adj) {
    int dev = 0, sms = 0;
    CUDA_OK(cudaGetDevice(&dev));
    CUDA_OK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // the Cauchy-Kowalevski adjoint keeps its cell in shared memory: no iterate slabs
    c->adj_blocks = ck ? 0 : sms * c->fam->adj_blocks_per_sm(c->cfg.order);
    c->adj_spb = ck ? 0 : c->fam->adj_scratch_per_block(c->cfg.order, iters);
    long long nfaces = 0;
    for (int d = 0; d < 3; ++d) nfaces += (long long)(c->g.n[d] + 1) * (c->g.ncells / c->g.n[d]);
    cudaError_t e = cudaMalloc(&c->dev_adj, sizeof(DevScalars));
    if (e == cudaSuccess) e = cudaMalloc(&c->adjf, (size_t)c->g.ncells * 3 * 2 * c->nf * c->nvar * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&c->gface, (size_t)nfaces * 6 * sizeof(double));
    // Picard: the iterate slabs; Cauchy-Kowalevski: lambda's projections onto the cells' faces
    const size_t scratch = ck ? (size_t)c->g.ncells * 3 * 2 * c->nf * c->nvar
                              : (size_t)c->adj_blocks * c->adj_spb;
    if (e == cudaSuccess) e = cudaMalloc(&c->adj_scratch, scratch * sizeof(double));
    if (e != cudaSuccess) {
      cudaGetLastError();
      cudaFree(c->dev_adj);
      cudaFree(c->adjf);
      cudaFree(c->gface);
      cudaFree(c->adj_scratch);
      c->dev_adj = nullptr;
      c->adjf = c->gface = c->adj_scratch = nullptr;
      return e == cudaErrorMemoryAllocation ? ADER_ENOMEM : ADER_ECUDA;
    }
    CUDA_OK(cudaMemsetAsync(c->dev_adj, 0, sizeof(DevScalars), c->stream));
  }
  CUDA_OK(launch_set_scalars(c->dev_adj, t_n, dt, c->stream));
  StepArgs a = make_args(c, dt, 0.0);
  a.u = u_n;
  a.dev = c->dev_adj;
  a.iters = iters;
  if (ck) {
    // the adjoint kernels form the forward face data themselves
    AdjArgs j{u_n, lam, dJdu, grad_mat, grad_M, c->adjf, c->gface, nullptr, 0, c->adj_scratch};
    CUDA_OK(c->fam->adj_run_ck(a, j, c->tab, c->tabf, c->cfg.precision, c->stream));
  } else {
    // forward face data of the step from u^n (the predictor also writes the scratch next state)
    CUDA_OK(c->fam->predictor(a, c->tab, c->tabf, ADER_PREC_FP64, c->stream));
    AdjArgs j{u_n, lam, dJdu, grad_mat, grad_M, c->adjf, c->gface, c->adj_scratch, c->adj_spb};
    CUDA_OK(c->fam->adj_run(a, j, c->tab, c->adj_blocks, c->stream));
  }
  // errors latched by the adjoint kernels reach the context's status word (ader_sync)
  CUDA_OK(launch_merge_status(c->dev_adj, c->dev, c->stream));
  return ADER_OK;
}

}  // extern "C"

// ---- allocation-free adjoint step ---------------------------------------------------------
// Work memory of ader_adjoint_step_static lives in this fixed device array, which every GPU that
// loads the library keeps until the process exits.  Host code must not use the symbol itself as
// a device address: its device address is looked up once per device below.
namespace {
constexpr size_t kStaticScratchBytes = 64ull << 20;  // 64 MiB
constexpr int kMaxContexts = 64;
static __device__ __align__(256) unsigned char g_adj_static[kStaticScratchBytes];
std::mutex g_adj_static_mu;
// A symbol's device address belongs to one CUDA context: the addresses are cached per context,
// keyed by the driver's context id (unique for the life of the process, so a context created
// after a device reset gets a fresh entry).  Without the driver entry points the address is
// looked up on every call.
struct StaticAddr {
  unsigned long long ctx_id;
  void* addr;
};
StaticAddr g_adj_static_addr[kMaxContexts] = {};
int g_adj_static_n = 0;
typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);

bool current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_cur = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_cur = (CtxGetCurrentFn)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = (CtxGetIdFn)f;
  }
  if (!get_cur || !get_id) return false;
  void* ctx = nullptr;
  if (get_cur(&ctx) != 0 || !ctx) return false;
  return get_id(ctx, id) == 0;
}

// Device address of the static array in the current context (cudaGetSymbolAddress on the first
// call in a context).
cudaError_t static_array_address(void** out) {
  std::lock_guard<std::mutex> lock(g_adj_static_mu);
  unsigned long long id = 0;
  const bool have_id = current_context_id(&id);
  if (have_id)
    for (int i = 0; i < g_adj_static_n; ++i)
      if (g_adj_static_addr[i].ctx_id == id) {
        *out = g_adj_static_addr[i].addr;
        return cudaSuccess;
      }
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_adj_static);
  if (e != cudaSuccess) return e;
  if (!p) return cudaErrorInvalidSymbol;
  if (have_id) {
    const int slot = g_adj_static_n < kMaxContexts ? g_adj_static_n++ : (int)(id % kMaxContexts);
    g_adj_static_addr[slot] = {id, p};
  }
  *out = p;
  return cudaSuccess;
}

size_t round256(size_t b) { return (b + 255) & ~size_t(255); }
}  // namespace

extern "C" {

ader_status ader_adjoint_step_static(ader_ctx* c, double t_n, double dt, const double* u_n,
                                     double* lam, const double* dJdu, double* grad_mat,
                                     double* grad_M) {
  if (!c || !u_n || !lam || !grad_mat || !grad_M || !(dt > 0.0)) return ADER_EINVAL;
  if (!adjoint_supported(c)) return ADER_EUNSUPPORTED;
  if (!c->mat_set) return ADER_ESTATE;
  const bool ck = c->cfg.predictor == ADER_PREDICTOR_CK;
  int dev = 0;
  CUDA_OK(cudaGetDevice(&dev));
  void* base = nullptr;
  CUDA_OK(static_array_address(&base));
  // layout: device scalars | face adjoints | face material gradients | per-block iterate slabs
  // (Picard) or lambda's face projections (Cauchy-Kowalevski)
  const int iters = c->cfg.picard_iters > 0 ? c->cfg.picard_iters : c->cfg.order + 1;
  long long nfaces = 0;
  for (int d = 0; d < 3; ++d) nfaces += (long long)(c->g.n[d] + 1) * (c->g.ncells / c->g.n[d]);
  const size_t b_dev = round256(sizeof(DevScalars));
  const size_t b_adjf = round256((size_t)c->g.ncells * 3 * 2 * c->nf * c->nvar * sizeof(double));
  const size_t b_gface = round256((size_t)nfaces * 6 * sizeof(double));
  // Picard: one iterate slab per thread block; Cauchy-Kowalevski: lambda's face projections
  const long long spb = ck ? 0 : c->fam->adj_scratch_per_block(c->cfg.order, iters);
  const size_t b_slab = ck ? (size_t)c->g.ncells * 3 * 2 * c->nf * c->nvar * sizeof(double)
                           : (size_t)spb * sizeof(double);
  const size_t fixed = b_dev + b_adjf + b_gface;
  if (fixed + b_slab > kStaticScratchBytes) return ADER_EINVAL;  // grid too large for the array
  long long blocks = 0;
  if (!ck) {
    int sms = 0;
    CUDA_OK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    blocks = (long long)sms * c->fam->adj_blocks_per_sm(c->cfg.order);
    blocks = std::min<long long>(blocks, (long long)((kStaticScratchBytes - fixed) / b_slab));
  }
  unsigned char* p = (unsigned char*)base;
  DevScalars* dev_s = (DevScalars*)p;
  double* adjf = (double*)(p + b_dev);
  double* gface = (double*)(p + b_dev + b_adjf);
  double* slab = (double*)(p + fixed);
  CUDA_OK(cudaMemsetAsync(&dev_s->status, 0, sizeof(int), c->stream));
  CUDA_OK(launch_set_scalars(dev_s, t_n, dt, c->stream));
  StepArgs a = make_args(c, dt, 0.0);
  a.u = u_n;
  a.dev = dev_s;
  a.iters = iters;
  if (ck) {
    AdjArgs j{u_n, lam, dJdu, grad_mat, grad_M, adjf, gface, nullptr, 0, slab};
    CUDA_OK(c->fam->adj_run_ck(a, j, c->tab, c->tabf, c->cfg.precision, c->stream));
  } else {
    CUDA_OK(c->fam->predictor(a, c->tab, c->tabf, ADER_PREC_FP64, c->stream));
    AdjArgs j{u_n, lam, dJdu, grad_mat, grad_M, adjf, gface, slab, spb};
    CUDA_OK(c->fam->adj_run(a, j, c->tab, (int)blocks, c->stream));
  }
  // errors latched in the array's scalars reach the context's status word (ader_sync), and the
  // scalars start the next call clear
  CUDA_OK(launch_merge_status(dev_s, c->dev, c->stream));
  return ADER_OK;
}

ader_status ader_receivers_adjoint(ader_ctx* c, const double* res, double scale, double* dJdu) {
  if (!c || !res || !dJdu) return ADER_EINVAL;
  if (c->cfg.pde != ADER_PDE_ELASTIC) return ADER_EUNSUPPORTED;
  if (c->rec.nrec <= 0) return ADER_ESTATE;
  CUDA_OK(launch_receivers_adjoint(c->rec, res, scale, dJdu, (int)c->nodes, (int)c->nvar, c->stream));
  return ADER_OK;
}

}  // extern "C"

// Checkpointed gradient of the receiver misfit of one context, split into phases so that the
// ensemble form can interleave the phases of several runs (each on its own stream).  The
// single-context entry point runs the same phases in the same order.
struct MisfitJob {
  ader_ctx* c = nullptr;
  const double* u0 = nullptr;
  const double* obs = nullptr;
  double t0 = 0.0, dt = 0.0;
  int steps = 0, k = 1, nseg = 0, nrec = 0;
  double* gm = nullptr;   // caller's (or work) gradient buffers
  double* gM = nullptr;
  bool grads = false;
  DevBufs B;
  double *ckpt = nullptr, *seg = nullptr, *lam = nullptr, *seismo = nullptr, *res = nullptr,
         *Jd = nullptr;
  Receivers saved{};
  ader_status st = ADER_OK;

  // device bytes of the work buffers
  static size_t bytes(const ader_ctx* c, int steps, int k) {
    const size_t nd = (size_t)c->ndof;
    const int nseg = (steps + k - 1) / k;
    return (nd * (nseg + k + 1) + (size_t)steps * c->rec.nrec * 3 + (size_t)c->rec.nrec * 3 +
            1 + (size_t)c->g.ncells * 3 + 6) * sizeof(double);
  }
  ader_status alloc(double* grad_mat, double* grad_M) {
    const size_t nd = (size_t)c->ndof;
    nseg = (steps + k - 1) / k;
    nrec = c->rec.nrec;
    grads = grad_mat || grad_M;
    cudaError_t e = B.alloc(&ckpt, nd * nseg);
    if (e == cudaSuccess) e = B.alloc(&seg, nd * (size_t)k);
    if (e == cudaSuccess) e = B.alloc(&lam, nd);
    if (e == cudaSuccess) e = B.alloc(&seismo, (size_t)steps * nrec * 3);
    if (e == cudaSuccess) e = B.alloc(&res, (size_t)nrec * 3);
    if (e == cudaSuccess) e = B.alloc(&Jd, 1);
    gm = grad_mat;
    gM = grad_M;
    if (e == cudaSuccess && grads && !gm) e = B.alloc(&gm, (size_t)c->g.ncells * 3);
    if (e == cudaSuccess && grads && !gM) e = B.alloc(&gM, 6);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? ADER_ENOMEM : ADER_ECUDA;
    }
    return ADER_OK;
  }
  // ---- forward sweep with a checkpoint every k steps ---------------------------------------
  ader_status forward_begin() {
    saved = c->rec;
    c->rec.seismo = seismo;
    c->rec.max_rows = steps;
    long long zero = 0;
    CUDA_OK(cudaMemcpyAsync(&c->dev->seismo_row, &zero, sizeof(long long), cudaMemcpyHostToDevice,
                            c->stream));
    CUDA_OK(cudaMemcpyAsync(c->u, u0, (size_t)c->ndof * sizeof(double), cudaMemcpyDeviceToDevice,
                            c->stream));
    c->state_set = true;
    CUDA_OK(launch_set_scalars(c->dev, t0, dt, c->stream));
    return ADER_OK;
  }
  ader_status forward_step(int n) {
    const size_t nd = (size_t)c->ndof;
    if (n % k == 0)
      CUDA_OK(cudaMemcpyAsync(ckpt + (size_t)(n / k) * nd, c->u, nd * sizeof(double),
                              cudaMemcpyDeviceToDevice, c->stream));
    return step_impl(c, dt, 0.0);
  }
  ader_status forward_end(double* J) {
    CUDA_OK(launch_misfit(seismo, obs, (long long)steps * nrec * 3, dt, Jd, c->stream));
    CUDA_OK(cudaMemcpyAsync(J, Jd, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return ADER_OK;
  }
  // ---- backward sweep: recompute each segment from its checkpoint --------------------------
  ader_status backward_begin() {
    CUDA_OK(cudaMemsetAsync(gm, 0, (size_t)c->g.ncells * 3 * sizeof(double), c->stream));
    CUDA_OK(cudaMemsetAsync(gM, 0, 6 * sizeof(double), c->stream));
    CUDA_OK(cudaMemsetAsync(lam, 0, (size_t)c->ndof * sizeof(double), c->stream));
    c->rec.nrec = 0;  // no recording while recomputing
    return ADER_OK;
  }
  ader_status recompute_segment(int sg) {
    const size_t nd = (size_t)c->ndof;
    const int a = sg * k, b = std::min(a + k, steps);
    CUDA_OK(cudaMemcpyAsync(c->u, ckpt + (size_t)sg * nd, nd * sizeof(double),
                            cudaMemcpyDeviceToDevice, c->stream));
    CUDA_OK(launch_set_scalars(c->dev, t0 + a * dt, dt, c->stream));
    ader_status r = ADER_OK;
    for (int i = 0; i < b - a && r == ADER_OK; ++i) {
      CUDA_OK(cudaMemcpyAsync(seg + (size_t)i * nd, c->u, nd * sizeof(double),
                              cudaMemcpyDeviceToDevice, c->stream));
      if (i + 1 < b - a) r = step_impl(c, dt, 0.0);
    }
    return r;
  }
  // lambda += dt R^T (seismo[n-1] - obs[n-1]); then lambda <- A^T lambda, gradients
  ader_status adjoint_step(int sg, int n) {
    const size_t nd = (size_t)c->ndof;
    const int a = sg * k;
    CUDA_OK(launch_sub(seismo + (size_t)(n - 1) * nrec * 3, obs + (size_t)(n - 1) * nrec * 3, res,
                       nrec * 3, c->stream));
    CUDA_OK(launch_receivers_adjoint(saved, res, dt, lam, (int)c->nodes, (int)c->nvar, c->stream));
    return ader_adjoint_step(c, t0 + (n - 1) * dt, dt, seg + (size_t)(n - 1 - a) * nd, lam, nullptr,
                             gm, gM);
  }
  void restore() { c->rec = saved; }
};

extern "C" {

ader_status ader_misfit_gradient(ader_ctx* c, const double* u0, double t0, double dt, int steps,
                                 int k_ckpt, const double* obs, double* J, double* grad_mat,
                                 double* grad_M) {
  if (!c || !u0 || !obs || !J || steps < 1 || k_ckpt < 1 || !(dt > 0.0)) return ADER_EINVAL;
  if (!adjoint_supported(c)) return ADER_EUNSUPPORTED;
  if (!c->mat_set || c->rec.nrec <= 0) return ADER_ESTATE;
  MisfitJob j;
  j.c = c;
  j.u0 = u0;
  j.obs = obs;
  j.t0 = t0;
  j.dt = dt;
  j.steps = steps;
  j.k = k_ckpt;
  ader_status st = j.alloc(grad_mat, grad_M);
  if (st != ADER_OK) return st;
  st = j.forward_begin();
  for (int n = 0; n < steps && st == ADER_OK; ++n) st = j.forward_step(n);
  if (st == ADER_OK) st = j.forward_end(J);
  if (st == ADER_OK && j.grads) {
    st = j.backward_begin();
    for (int sg = j.nseg - 1; sg >= 0 && st == ADER_OK; --sg) {
      st = j.recompute_segment(sg);
      const int a = sg * j.k, b = std::min(a + j.k, steps);
      for (int n = b; n > a && st == ADER_OK; --n) st = j.adjoint_step(sg, n);
    }
  }
  j.restore();
  CUDA_OK(cudaStreamSynchronize(c->stream));
  if (st != ADER_OK) return st;
  return ader_sync(c);
}

}  // extern "C"

// ---- ensembles ------------------------------------------------------------------------------
struct ader_ensemble {
  std::vector<ader_ctx*> runs;
  cudaStream_t stream = nullptr;
  std::vector<cudaStream_t> branch;   // fork streams used inside the captured graph
  std::vector<cudaEvent_t> ev;        // fork / join events
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int g_steps = 0, g_branches = 0;
  double g_dt = 0.0, g_tend = 0.0;
  std::vector<double*> g_u0;
  int branches = 1;                   // chosen by the autotuner (or 1); 0: persistent launches
                                      // per phase; -1: one fused cooperative launch
  int steps_per_graph = 2;
  int bps = 1;                        // persistent predictor blocks per SM (branches <= 0)
  int g_bps = 0;
  StepArgs* d_runs = nullptr;         // run tables of the captured persistent steps
  size_t d_runs_n = 0;
  void* d_bar = nullptr;              // grid-barrier state of the fused launch
  long long wait_limit = 1ll << 24;   // polls of a grid-barrier wait (about 1.7 s with 100 ns
                                      // sleeps) before it gives up with ADER_ETIMEOUT
  long long g_limit = -1;
};

static void ens_free_graph(ader_ensemble* e) {
  // a replay may still read the graph and the device run tables: let it finish first
  if (!e->branch.empty()) cudaStreamSynchronize(e->branch[0]);
  cudaStreamSynchronize(e->stream);
  if (e->gexec) cudaGraphExecDestroy(e->gexec);
  if (e->graph) cudaGraphDestroy(e->graph);
  e->gexec = nullptr;
  e->graph = nullptr;
}

static ader_status ens_capture(ader_ensemble* e, int steps, double dt, double t_end, int nb) {
  ens_free_graph(e);
  while ((int)e->branch.size() < nb) {
    cudaStream_t s;
    CUDA_OK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    e->branch.push_back(s);
  }
  while (e->ev.size() < (size_t)(nb + 1)) {
    cudaEvent_t v;
    CUDA_OK(cudaEventCreateWithFlags(&v, cudaEventDisableTiming));
    e->ev.push_back(v);
  }
  cudaStream_t cap = e->branch[0];
  std::vector<cudaStream_t> saved(e->runs.size());
  for (size_t r = 0; r < e->runs.size(); ++r) saved[r] = e->runs[r]->stream;
  CUDA_OK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
  ader_status st = ADER_OK;
  // fork: branches 1..nb-1 wait on the start of the capture
  if (cudaEventRecord(e->ev[0], cap) != cudaSuccess) st = ADER_ECUDA;
  for (int b = 1; b < nb && st == ADER_OK; ++b)
    if (cudaStreamWaitEvent(e->branch[b], e->ev[0], 0) != cudaSuccess) st = ADER_ECUDA;
  for (size_t r = 0; r < e->runs.size() && st == ADER_OK; ++r) {
    ader_ctx* c = e->runs[r];
    c->stream = e->branch[r % nb];
    for (int k = 0; k < steps && st == ADER_OK; ++k) st = step_impl(c, dt, t_end);
  }
  // join
  for (int b = 1; b < nb && st == ADER_OK; ++b) {
    if (cudaEventRecord(e->ev[b], e->branch[b]) != cudaSuccess) st = ADER_ECUDA;
    else if (cudaStreamWaitEvent(cap, e->ev[b], 0) != cudaSuccess) st = ADER_ECUDA;
  }
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(cap, &g);
  for (size_t r = 0; r < e->runs.size(); ++r) e->runs[r]->stream = saved[r];
  if (st != ADER_OK || ce != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return st != ADER_OK ? st : ADER_ECUDA;
  }
  e->graph = g;
  CUDA_OK(cudaGraphInstantiate(&e->gexec, g, 0));
  e->g_steps = steps;
  e->g_branches = nb;
  e->g_dt = dt;
  e->g_tend = t_end;
  e->g_u0.clear();
  for (ader_ctx* c : e->runs) e->g_u0.push_back(c->u);
  return ADER_OK;
}

// The runs can be advanced by the persistent launches of their family: same family, order,
// precision, cell size and gamma (shared tables), fixed dt, no limiter, no receivers.
static bool ens_batchable(const ader_ensemble* e, double dt) {
  if (!(dt > 0.0) || e->runs.empty() || (int)e->runs.size() > ENS_MAXR) return false;
  const ader_ctx* a = e->runs[0];
  if (a->cfg.order > 5) return false;
  // Picard runs, or Cauchy-Kowalevski runs (FP64 or mixed) at the orders with one cell per block
  if (a->cfg.predictor == ADER_PREDICTOR_CK) {
    if (!a->fam->ens_step_ck || a->cfg.order < 4 || a->cfg.precision > ADER_PREC_MIXED)
      return false;
  } else if (!a->fam->ens_step) {
    return false;
  }
  for (const ader_ctx* c : e->runs) {
    if (c->fam != a->fam || c->cfg.order != a->cfg.order || c->cfg.precision != a->cfg.precision ||
        c->cfg.predictor != a->cfg.predictor ||
        c->cfg.limiter || c->rec.nrec > 0 || c->p.gamma != a->p.gamma)
      return false;
    for (int d = 0; d < 3; ++d)
      if (c->g.h[d] != a->g.h[d]) return false;
  }
  return true;
}

// Capture `steps` steps of every run as one persistent launch per phase: the run tables of each
// step (the runs' step arguments with that step's state buffers) go to device memory first.
static ader_status ens_capture_persistent(ader_ensemble* e, int steps, double dt, double t_end,
                                          int bps, bool fused) {
  ens_free_graph(e);
  const int nr = (int)e->runs.size();
  const size_t need = (size_t)steps * nr;
  if (e->d_runs_n < need) {
    cudaFree(e->d_runs);
    e->d_runs = nullptr;
    e->d_runs_n = 0;
    CUDA_OK(cudaMalloc(&e->d_runs, need * sizeof(StepArgs)));
    e->d_runs_n = need;
  }
  std::vector<StepArgs> h(need);
  for (int k = 0; k < steps; ++k)
    for (int r = 0; r < nr; ++r) {
      ader_ctx* c = e->runs[r];
      h[(size_t)k * nr + r] = make_args(c, dt, t_end);
      h[(size_t)k * nr + r].fspeed = c->fspeed;
      std::swap(c->u, c->u_next);  // as the step does
    }
  CUDA_OK(cudaMemcpy(e->d_runs, h.data(), need * sizeof(StepArgs), cudaMemcpyHostToDevice));
  EnsTable E{};
  E.nr = nr;
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  E.pblocks = sms * bps;
  const long long nphi = e->runs[0]->fam->nphi;
  for (int r = 0; r < nr; ++r) {
    const ader_ctx* c = e->runs[r];
    E.cell0[r + 1] = E.cell0[r] + c->g.ncells;
    long long off = 0;
    for (int d = 0; d < c->g.dim; ++d) {
      const long long nf = (long long)(c->g.n[d] + 1) * (c->g.ncells / c->g.n[d]);
      E.face0[d][r + 1] = E.face0[d][r] + nf;
      E.phioff[d][r] = off;
      off += nf * nphi * c->nf * c->nvar;
    }
  }
  cudaStream_t cap = e->branch[0];
  const ader_ctx* a = e->runs[0];
  if (fused && !e->d_bar) CUDA_OK(cudaMalloc(&e->d_bar, 64));
  CUDA_OK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
  cudaError_t ce = cudaSuccess;
  if (fused) {
    ce = a->fam->ens_fused(e->d_runs, E, a->tab, a->tabf, a->cfg.precision, a->cfg.order, steps,
                           e->d_bar, e->wait_limit, bps, cap);
  } else {
    const bool ck = a->cfg.predictor == ADER_PREDICTOR_CK;
    for (int k = 0; k < steps && ce == cudaSuccess; ++k)
      ce = (ck ? a->fam->ens_step_ck : a->fam->ens_step)(e->d_runs + (size_t)k * nr, E, a->tab,
                                                         a->tabf, a->cfg.precision, a->cfg.order,
                                                         cap);
  }
  cudaGraph_t g = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(cap, &g);
  if (ce != cudaSuccess || ee != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return ADER_ECUDA;
  }
  e->graph = g;
  CUDA_OK(cudaGraphInstantiate(&e->gexec, g, 0));
  e->g_steps = steps;
  e->g_branches = fused ? -1 : 0;
  e->g_bps = bps;
  e->g_limit = e->wait_limit;
  e->g_dt = dt;
  e->g_tend = t_end;
  e->g_u0.clear();
  for (ader_ctx* c : e->runs) e->g_u0.push_back(c->u);
  return ADER_OK;
}

extern "C" {

ader_status ader_ensemble_create(const ader_config* cfgs, int nruns, void* stream,
                                 ader_ensemble** out) {
  if (!out) return ADER_EINVAL;
  *out = nullptr;
  if (!cfgs || nruns < 1) return ADER_EINVAL;
  ader_ensemble* e = new (std::nothrow) ader_ensemble();
  if (!e) return ADER_ENOMEM;
  e->stream = (cudaStream_t)stream;
  for (int r = 0; r < nruns; ++r) {
    ader_ctx* c = nullptr;
    const ader_status st = ader_create(&cfgs[r], stream, &c);
    if (st != ADER_OK) {
      ader_ensemble_destroy(e);
      return st;
    }
    e->runs.push_back(c);
  }
  *out = e;
  return ADER_OK;
}

void ader_ensemble_destroy(ader_ensemble* e) {
  if (!e) return;
  ens_free_graph(e);
  cudaFree(e->d_runs);
  cudaFree(e->d_bar);
  for (ader_ctx* c : e->runs) ader_destroy(c);
  for (cudaStream_t s : e->branch) cudaStreamDestroy(s);
  for (cudaEvent_t v : e->ev) cudaEventDestroy(v);
  delete e;
}

ader_ctx* ader_ensemble_run(ader_ensemble* e, int i) {
  if (!e || i < 0 || i >= (int)e->runs.size()) return nullptr;
  return e->runs[i];
}

ader_status ader_ensemble_step(ader_ensemble* e, int steps, double dt, double t_end) {
  if (!e || steps < 1) return ADER_EINVAL;
  for (ader_ctx* c : e->runs) {
    if (!c->state_set) return ADER_ESTATE;
    if (c->cfg.pde == ADER_PDE_ELASTIC && !c->mat_set) return ADER_ESTATE;
    if (c->timing) return ADER_EINVAL;
  }
  // whole graphs of steps_per_graph (even) steps, the remainder one step at a time
  const int spg = e->steps_per_graph;
  const int ng = steps / spg, rest = steps % spg;
  if (ng > 0) {
    const bool fused = e->branches < 0 && ens_batchable(e, dt) && e->runs[0]->fam->ens_fused &&
                       e->runs[0]->cfg.predictor == ADER_PREDICTOR_PICARD;
    const bool persistent = (e->branches == 0 || fused) && ens_batchable(e, dt);
    const int nb = fused ? -1 : (persistent ? 0 : (e->branches > 0 ? e->branches : 1));
    bool same = e->gexec && e->g_steps == spg && e->g_dt == dt && e->g_tend == t_end &&
                e->g_branches == nb && (!persistent || e->g_bps == e->bps) &&
                (!fused || e->g_limit == e->wait_limit);
    for (size_t r = 0; same && r < e->runs.size(); ++r) same = e->g_u0[r] == e->runs[r]->u;
    if (!same) {
      if (e->branch.empty()) {  // the capture stream and the fork / join event
        cudaStream_t bs;
        CUDA_OK(cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking));
        e->branch.push_back(bs);
      }
      if (e->ev.empty()) {
        cudaEvent_t v;
        CUDA_OK(cudaEventCreateWithFlags(&v, cudaEventDisableTiming));
        e->ev.push_back(v);
      }
      const ader_status st = persistent ? ens_capture_persistent(e, spg, dt, t_end, e->bps, fused)
                                        : ens_capture(e, spg, dt, t_end, nb);
      if (st != ADER_OK) return st;
    }
    // order the replays after earlier work on the ensemble stream
    CUDA_OK(cudaEventRecord(e->ev[0], e->stream));
    CUDA_OK(cudaStreamWaitEvent(e->branch[0], e->ev[0], 0));
    for (int k = 0; k < ng; ++k) CUDA_OK(cudaGraphLaunch(e->gexec, e->branch[0]));
    CUDA_OK(cudaEventRecord(e->ev[0], e->branch[0]));
    CUDA_OK(cudaStreamWaitEvent(e->stream, e->ev[0], 0));
  }
  for (int k = 0; k < rest; ++k)
    for (ader_ctx* c : e->runs) {
      const ader_status st = step_impl(c, dt, t_end);
      if (st != ADER_OK) return st;
    }
  return ADER_OK;
}

ader_status ader_ensemble_sync(ader_ensemble* e) {
  if (!e) return ADER_EINVAL;
  ader_status first = ADER_OK;
  for (ader_ctx* c : e->runs) {
    const ader_status st = ader_sync(c);
    if (st != ADER_OK && first == ADER_OK) first = st;
  }
  return first;
}

ader_status ader_ensemble_set_launch(ader_ensemble* e, int branches, int steps_per_graph,
                                     int blocks_per_sm) {
  if (!e || branches < -1 || branches > 16 || steps_per_graph < 2 || steps_per_graph % 2)
    return ADER_EINVAL;
  if (branches <= 0 && (blocks_per_sm < 1 || blocks_per_sm > 8)) return ADER_EINVAL;
  e->branches = branches;
  e->steps_per_graph = steps_per_graph;
  if (branches <= 0) e->bps = blocks_per_sm;
  return ADER_OK;
}

ader_status ader_ensemble_set_wait_limit(ader_ensemble* e, int64_t polls) {
  if (!e || polls < 0) return ADER_EINVAL;
  e->wait_limit = polls;
  return ADER_OK;
}

// Time each (branches or persistent blocks per SM, steps per graph) candidate on the current
// states (restored afterwards) and keep the fastest.  best[0..2] receives the choice, ms_per_step
// its time.
ader_status ader_ensemble_autotune(ader_ensemble* e, double dt, int* best, double* ms_per_step) {
  if (!e || !(dt > 0.0)) return ADER_EINVAL;
  for (ader_ctx* c : e->runs)
    if (!c->state_set) return ADER_ESTATE;
  DevBufs B;
  std::vector<double*> save(e->runs.size());
  for (size_t r = 0; r < e->runs.size(); ++r) {
    if (B.alloc(&save[r], (size_t)e->runs[r]->ndof) != cudaSuccess) return ADER_ENOMEM;
    CUDA_OK(cudaMemcpyAsync(save[r], e->runs[r]->u, e->runs[r]->ndof * sizeof(double),
                            cudaMemcpyDeviceToDevice, e->stream));
  }
  // candidates: (branches, persistent blocks per SM); branches 0 = one persistent launch per
  // phase for all runs
  std::vector<std::pair<int, int>> cand = {{1, 1}, {2, 1}, {4, 1}};
  if (ens_batchable(e, dt)) {
    cand.push_back({0, 1});
    cand.push_back({0, 2});
    if (e->runs[0]->fam->ens_fused && e->runs[0]->cfg.predictor == ADER_PREDICTOR_PICARD) {
      cand.push_back({-1, 1});
      cand.push_back({-1, 2});
    }
  }
  const int cand_s[] = {2, 4};
  cudaEvent_t t0, t1;
  CUDA_OK(cudaEventCreate(&t0));
  CUDA_OK(cudaEventCreate(&t1));
  double best_ms = 1e300;
  int bb = 1, bs = 2, bp = 1;
  const int ob = e->branches, os = e->steps_per_graph, op = e->bps;
  for (const auto& cb : cand) {
    const int b = cb.first;
    if (b > (int)e->runs.size()) continue;
    for (int sp : cand_s) {
      e->branches = b;
      e->bps = cb.second;
      e->steps_per_graph = sp;
      ader_status st = ader_ensemble_step(e, sp, dt, 0.0);  // capture + warm-up
      if (st != ADER_OK) break;
      CUDA_OK(cudaEventRecord(t0, e->stream));
      st = ader_ensemble_step(e, sp, dt, 0.0);
      CUDA_OK(cudaEventRecord(t1, e->stream));
      CUDA_OK(cudaEventSynchronize(t1));
      float ms = 0.f;
      CUDA_OK(cudaEventElapsedTime(&ms, t0, t1));
      const double per = ms / sp;
      if (st == ADER_OK && per < best_ms) {
        best_ms = per;
        bb = b;
        bs = sp;
        bp = cb.second;
      }
      for (size_t r = 0; r < e->runs.size(); ++r)  // restore the states (even steps: same buffers)
        CUDA_OK(cudaMemcpyAsync(e->runs[r]->u, save[r], e->runs[r]->ndof * sizeof(double),
                                cudaMemcpyDeviceToDevice, e->stream));
    }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  CUDA_OK(cudaStreamSynchronize(e->stream));
  if (best_ms == 1e300) {
    e->branches = ob;
    e->steps_per_graph = os;
    e->bps = op;
    return ADER_ECUDA;
  }
  e->branches = bb;
  e->steps_per_graph = bs;
  e->bps = bp;
  if (best) {
    best[0] = bb;
    best[1] = bs;
    best[2] = bb <= 0 ? bp : 0;
  }
  if (ms_per_step) *ms_per_step = best_ms;
  return ADER_OK;
}

ader_status ader_ensemble_misfit_gradient(ader_ensemble* e, const double* const* u0, double t0,
                                          double dt, int steps, int k_ckpt,
                                          const double* const* obs, double* J,
                                          double* const* grad_mat, double* const* grad_M,
                                          int64_t mem_budget) {
  if (!e || !u0 || !obs || !J || steps < 1 || k_ckpt < 1 || !(dt > 0.0)) return ADER_EINVAL;
  const int nr = (int)e->runs.size();
  for (int r = 0; r < nr; ++r) {
    const ader_ctx* c = e->runs[r];
    if (!u0[r] || !obs[r]) return ADER_EINVAL;
    if (!adjoint_supported(c)) return ADER_EUNSUPPORTED;
    if (!c->mat_set || c->rec.nrec <= 0 || c->timing) return ADER_ESTATE;
  }
  size_t budget = (size_t)(mem_budget > 0 ? mem_budget : 0);
  if (!budget) {
    size_t fr = 0, tot = 0;
    CUDA_OK(cudaMemGetInfo(&fr, &tot));
    budget = fr / 2;
  }
  // forked streams: the runs of a group work concurrently, each on its own stream
  const int nb = std::min(nr, 16);
  while ((int)e->branch.size() < nb) {
    cudaStream_t bs;
    CUDA_OK(cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking));
    e->branch.push_back(bs);
  }
  while (e->ev.size() < (size_t)(nb + 1)) {
    cudaEvent_t v;
    CUDA_OK(cudaEventCreateWithFlags(&v, cudaEventDisableTiming));
    e->ev.push_back(v);
  }
  CUDA_OK(cudaEventRecord(e->ev[0], e->stream));
  for (int b = 0; b < nb; ++b) CUDA_OK(cudaStreamWaitEvent(e->branch[b], e->ev[0], 0));
  std::vector<cudaStream_t> saved(nr);
  for (int r = 0; r < nr; ++r) saved[r] = e->runs[r]->stream;
  ader_status st = ADER_OK;
  for (int g0 = 0; g0 < nr && st == ADER_OK;) {
    // the next group: as many runs as fit the budget (at least one)
    int g1 = g0;
    size_t used = 0;
    while (g1 < nr) {
      const size_t b = MisfitJob::bytes(e->runs[g1], steps, k_ckpt);
      if (g1 > g0 && used + b > budget) break;
      used += b;
      ++g1;
    }
    std::vector<std::unique_ptr<MisfitJob>> jobs;
    for (int r = g0; r < g1 && st == ADER_OK; ++r) {
      ader_ctx* c = e->runs[r];
      c->stream = e->branch[(r - g0) % nb];
      auto j = std::make_unique<MisfitJob>();
      j->c = c;
      j->u0 = u0[r];
      j->obs = obs[r];
      j->t0 = t0;
      j->dt = dt;
      j->steps = steps;
      j->k = k_ckpt;
      st = j->alloc(grad_mat ? grad_mat[r] : nullptr, grad_M ? grad_M[r] : nullptr);
      jobs.push_back(std::move(j));
    }
    // the phases of every run of the group, interleaved step by step
    for (auto& j : jobs)
      if (st == ADER_OK) st = j->forward_begin();
    for (int n = 0; n < steps && st == ADER_OK; ++n)
      for (auto& j : jobs)
        if (st == ADER_OK) st = j->forward_step(n);
    for (int r = g0; r < g1 && st == ADER_OK; ++r) st = jobs[r - g0]->forward_end(J + r);
    if (st == ADER_OK && jobs[0]->grads) {
      for (auto& j : jobs)
        if (st == ADER_OK) st = j->backward_begin();
      const int nseg = jobs[0]->nseg;
      for (int sg = nseg - 1; sg >= 0 && st == ADER_OK; --sg) {
        for (auto& j : jobs)
          if (st == ADER_OK) st = j->recompute_segment(sg);
        const int a = sg * k_ckpt, b = std::min(a + k_ckpt, steps);
        for (int n = b; n > a && st == ADER_OK; --n)
          for (auto& j : jobs)
            if (st == ADER_OK) st = j->adjoint_step(sg, n);
      }
    }
    for (auto& j : jobs) {
      j->restore();
      cudaStreamSynchronize(j->c->stream);
    }
    jobs.clear();  // frees the group's work buffers
    g0 = g1;
  }
  for (int r = 0; r < nr; ++r) e->runs[r]->stream = saved[r];
  // join the forked streams into the ensemble stream
  for (int b = 0; b < nb; ++b) {
    CUDA_OK(cudaEventRecord(e->ev[1 + b], e->branch[b]));
    CUDA_OK(cudaStreamWaitEvent(e->stream, e->ev[1 + b], 0));
  }
  CUDA_OK(cudaStreamSynchronize(e->stream));
  if (st != ADER_OK) return st;
  return ader_ensemble_sync(e);
}

ader_status ader_enable_timing(ader_ctx* c, int on) {
  if (!c) return ADER_EINVAL;
  c->timing = on != 0;
  c->ev_used = 0;
  return ADER_OK;
}

ader_status ader_phase_times(ader_ctx* c, double ms[7], int* steps) {
  if (!c || !ms) return ADER_EINVAL;
  CUDA_OK(cudaStreamSynchronize(c->stream));
  for (int k = 0; k < NPHASE; ++k) ms[k] = 0.0;
  for (int sidx = 0; sidx < c->ev_used; ++sidx) {
    for (int k = 0; k < NPHASE; ++k) {
      float t = 0.f;
      CUDA_OK(cudaEventElapsedTime(&t, c->ev[(size_t)sidx * (NPHASE + 1) + k],
                                   c->ev[(size_t)sidx * (NPHASE + 1) + k + 1]));
      ms[k] += t;
    }
  }
  if (steps) *steps = c->ev_used;
  c->ev_used = 0;
  return ADER_OK;
}

ader_status ader_run_graph(ader_ctx* c, int steps, int replays, double dt, double t_end) {
  if (!c || steps < 1 || replays < 0 || (steps % 2) != 0 || c->timing) return ADER_EINVAL;
  if (!c->state_set) return ADER_ESTATE;
  if (c->cfg.pde == ADER_PDE_ELASTIC && !c->mat_set) return ADER_ESTATE;
  if (!c->gexec || c->g_steps != steps || c->g_dt != dt || c->g_tend != t_end || c->g_u0 != c->u) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->gexec = nullptr;
    c->graph = nullptr;
    cudaStream_t cap = c->stream;
    bool own = false;
    if (cap == nullptr) {  // the legacy stream cannot be captured
      CUDA_OK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
      own = true;
      CUDA_OK(cudaStreamSynchronize(nullptr));
    }
    cudaStream_t saved = c->stream;
    c->stream = cap;
    double* u0 = c->u;
    CUDA_OK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    ader_status st = ADER_OK;
    for (int i = 0; i < steps && st == ADER_OK; ++i) st = step_impl(c, dt, t_end);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cap, &g);
    c->stream = saved;
    if (st != ADER_OK || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      if (own) cudaStreamDestroy(cap);
      c->u = u0;  // steps are even, but restore in case of a partial capture
      return st != ADER_OK ? st : ADER_ECUDA;
    }
    c->graph = g;
    CUDA_OK(cudaGraphInstantiate(&c->gexec, g, 0));
    if (own) cudaStreamDestroy(cap);
    c->g_steps = steps;
    c->g_dt = dt;
    c->g_tend = t_end;
    c->g_u0 = c->u;
  }
  for (int r = 0; r < replays; ++r) CUDA_OK(cudaGraphLaunch(c->gexec, c->stream));
  return ADER_OK;
}

}  // extern "C"
