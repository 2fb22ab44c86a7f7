// Small kernels shared by every kernel family: time-step finalisation (Eq. (7)), the time
// advance, and the receiver read-out.
#include "ader_internal.h"
#include "step_scalars.cuh"

namespace ader {

__global__ void k_dt_finalize(const __grid_constant__ StepArgs A) { dt_finalize_one(A); }

__global__ void k_advance(DevScalars* s, int receivers_on) { advance_one(s, receivers_on); }

// Ensemble: the same for every run (one thread per run).
__global__ void k_ens_dt(const StepArgs* __restrict__ runs, int nr) {
  if ((int)threadIdx.x < nr) dt_finalize_one(runs[threadIdx.x]);
}
__global__ void k_ens_advance(const StepArgs* __restrict__ runs, int nr) {
  if ((int)threadIdx.x < nr) advance_one(runs[threadIdx.x].dev, 0);
}

// One warp per receiver: v(x_r) = sum_j Phi_j(xi_r) u[cell_r][j][0..2].
__global__ void k_receivers(const double* __restrict__ u, DevScalars* s, Receivers r, int nodes,
                            int nvar) {
  const int lane = threadIdx.x & 31;
  const int rec = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (rec >= r.nrec) return;
  const long long row = s->seismo_row;
  if (row >= r.max_rows) {
    if (lane == 0) atomicOr(&s->status, ST_SEISMO_FULL);
    return;
  }
  const double* uc = u + (long long)r.cell[rec] * nodes * nvar;
  const double* ph = r.phi + (long long)rec * nodes;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  for (int j = lane; j < nodes; j += 32) {
    const double p = ph[j];
    a0 = fma(p, uc[j * nvar + 0], a0);
    a1 = fma(p, uc[j * nvar + 1], a1);
    a2 = fma(p, uc[j * nvar + 2], a2);
  }
  for (int o = 16; o > 0; o >>= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, o);
    a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
  }
  if (lane == 0) {
    double* out = r.seismo + (row * r.nrec + rec) * 3;
    out[0] = a0;
    out[1] = a1;
    out[2] = a2;
  }
}

__global__ void k_set_scalars(DevScalars* d, double t, double dt) {
  d->t = t;
  d->dt = dt;
}

// Move the error bits latched in `src` (the adjoint's scalars) into `dst` (the context's status
// word, which ader_sync reads) and clear them in `src`.
__global__ void k_merge_status(DevScalars* src, DevScalars* dst) {
  const int bits = src->status;
  if (bits) {
    atomicOr(&dst->status, bits);
    src->status = 0;
  }
}

// dJ/du[cell_r][j][v] += scale * res[r][v] * Phi_j(xi_r), receivers in order (deterministic: each
// thread owns one (node, component) slot).
__global__ void k_receivers_adjoint(Receivers r, const double* res, double scale, double* dJdu,
                                    int nodes, int nvar) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nodes * 3) return;
  const int j = e / 3, v = e % 3;
  for (int k = 0; k < r.nrec; ++k) {
    double* dst = dJdu + ((long long)r.cell[k] * nodes + j) * nvar + v;
    *dst = fma(scale * res[k * 3 + v], r.phi[(long long)k * nodes + j], *dst);
  }
}

// res = seismo_row - obs_row ([n] values)
__global__ void k_sub(const double* a, const double* b, double* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a[i] - b[i];
}

// J = 1/2 scale sum (a - b)^2 over n values (one block, fixed reduction order).
__global__ void k_misfit(const double* a, const double* b, long long n, double scale, double* J) {
  __shared__ double red[256];
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    const double r = a[i] - b[i];
    s = fma(r, r, s);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *J = 0.5 * scale * red[0];
}

cudaError_t launch_sub(const double* a, const double* b, double* out, int n, cudaStream_t s) {
  k_sub<<<(n + 127) / 128, 128, 0, s>>>(a, b, out, n);
  return cudaGetLastError();
}

cudaError_t launch_misfit(const double* a, const double* b, long long n, double scale, double* J,
                          cudaStream_t s) {
  k_misfit<<<1, 256, 0, s>>>(a, b, n, scale, J);
  return cudaGetLastError();
}

// Device-to-device copy of n doubles on the SMs (16-byte vectors; the copy engines stay free for
// host transfers running beside it).
__global__ void __launch_bounds__(256) k_copy(double* __restrict__ dst,
                                              const double* __restrict__ src, long long n) {
  const long long n2 = n / 2;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const double2* s2 = reinterpret_cast<const double2*>(src);
  double2* d2 = reinterpret_cast<double2*>(dst);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += stride)
    d2[i] = s2[i];
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) dst[n - 1] = src[n - 1];
}

cudaError_t launch_copy(double* dst, const double* src, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if ((((uintptr_t)dst) | ((uintptr_t)src)) & 15) {  // not 16-byte aligned: the runtime's copy
    return cudaMemcpyAsync(dst, src, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  }
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
      sms = 152;
  }
  const long long want = (n / 2 + 255) / 256;
  const long long blocks = want < (long long)sms * 8 ? (want > 0 ? want : 1) : (long long)sms * 8;
  k_copy<<<(unsigned)blocks, 256, 0, s>>>(dst, src, n);
  return cudaGetLastError();
}

cudaError_t launch_set_scalars(DevScalars* d, double t, double dt, cudaStream_t s) {
  k_set_scalars<<<1, 1, 0, s>>>(d, t, dt);
  return cudaGetLastError();
}

// Hybrid limiter status at the start of a run: cells put into the FV space along the initial
// discontinuity take `persist` FV steps, as if troubled at the initial time.
__global__ void k_seed_status(const uint8_t* __restrict__ flags, uint8_t* __restrict__ status,
                              long long ncells, int persist) {
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncells;
       c += (long long)gridDim.x * blockDim.x)
    if (flags[c]) status[c] = (uint8_t)persist;
}

cudaError_t launch_seed_status(const uint8_t* flags, uint8_t* status, long long ncells,
                               int persist, cudaStream_t s) {
  if (ncells <= 0) return cudaSuccess;
  const long long blocks = (ncells + 255) / 256;
  k_seed_status<<<(unsigned)(blocks < 65535 ? blocks : 65535), 256, 0, s>>>(flags, status, ncells,
                                                                            persist);
  return cudaGetLastError();
}

cudaError_t launch_merge_status(DevScalars* src, DevScalars* dst, cudaStream_t s) {
  k_merge_status<<<1, 1, 0, s>>>(src, dst);
  return cudaGetLastError();
}

cudaError_t launch_receivers_adjoint(const Receivers& r, const double* res, double scale,
                                     double* dJdu, int nodes, int nvar, cudaStream_t s) {
  if (r.nrec <= 0) return cudaSuccess;
  const int tot = nodes * 3;
  k_receivers_adjoint<<<(tot + 127) / 128, 128, 0, s>>>(r, res, scale, dJdu, nodes, nvar);
  return cudaGetLastError();
}

cudaError_t launch_dt_finalize(const StepArgs& a, cudaStream_t s) {
  k_dt_finalize<<<1, 1, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_ens_dt(const StepArgs* runs, int nr, cudaStream_t s) {
  k_ens_dt<<<1, ENS_MAXR, 0, s>>>(runs, nr);
  return cudaGetLastError();
}

cudaError_t launch_ens_advance(const StepArgs* runs, int nr, cudaStream_t s) {
  k_ens_advance<<<1, ENS_MAXR, 0, s>>>(runs, nr);
  return cudaGetLastError();
}

cudaError_t launch_advance_rec(const StepArgs& a, int receivers_on, cudaStream_t s) {
  k_advance<<<1, 1, 0, s>>>(a.dev, receivers_on);
  return cudaGetLastError();
}

cudaError_t launch_advance(const StepArgs& a, cudaStream_t s) { return launch_advance_rec(a, 0, s); }

cudaError_t launch_receivers(const StepArgs& a, const Receivers& r, int nodes, int nvar,
                             cudaStream_t s) {
  if (r.nrec <= 0) return cudaSuccess;
  const int wpb = 4;
  k_receivers<<<(r.nrec + wpb - 1) / wpb, 32 * wpb, 0, s>>>(a.u_next, a.dev, r, nodes, nvar);
  return cudaGetLastError();
}

}  // namespace ader
