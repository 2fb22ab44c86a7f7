// Arithmetic-pipe throughput of the GPU, measured the way the roofline denominators of the
// benchmark need them: every thread runs CHAINS independent fused multiply-add chains (enough
// independent work per warp to hide the pipe latency) for `iters` rounds, and the launch's
// CUDA-event time gives the FMA rate.  FP64 (DFMA) and binary32 (FFMA).  The chains' values
// stay finite and are written out, so no work is removed by the compiler.
#include <cuda_runtime.h>

namespace {
constexpr int CHAINS = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(T* sink, int iters, T a, T b) {
  T x[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += x[c];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
}  // namespace

extern "C" {

// Launch `blocks` x 256 threads, each with 8 chains of `iters` FMA (2 flops each) in FP64
// (fp64 = 1) or binary32; `sink` must hold blocks * 256 elements of that type (device memory).
// Returns the cudaError_t of the launch.  The multiplier 0.999 and addend 1e-3 keep each chain
// bounded.
int peaks_fma_launch(int fp64, void* sink, int blocks, int iters, void* stream) {
  if (blocks < 1 || iters < 1 || !sink) return (int)cudaErrorInvalidValue;
  cudaStream_t s = (cudaStream_t)stream;
  if (fp64)
    k_fma_chains<double><<<blocks, 256, 0, s>>>((double*)sink, iters, 0.999, 1e-3);
  else
    k_fma_chains<float><<<blocks, 256, 0, s>>>((float*)sink, iters, 0.999f, 1e-3f);
  return (int)cudaGetLastError();
}

// Flops of one launch: blocks x 256 threads x 8 chains x iters x 2.
double peaks_fma_flops(int blocks, int iters) {
  return (double)blocks * 256.0 * CHAINS * (double)iters * 2.0;
}

}  // extern "C"
