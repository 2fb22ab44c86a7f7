// Cauchy-Kowalevski predictor of the 3-D elastic family, orders 1-6, FP64 and mixed precision
// (the tensor-core form is in ck_tc_elastic3.cu).
#include "kernels_ck.cuh"

namespace ader {

cudaError_t predictor_ck_tc_elastic3(const StepArgs& a, const Tables& t, cudaStream_t s);

cudaError_t predictor_ck_elastic3(const StepArgs& a, const Tables& t, const TablesF& f, int prec,
                                  cudaStream_t s) {
  if (prec == 3) return predictor_ck_tc_elastic3(a, t, s);
  if (prec == 1) {
    switch (a.g.order) {
      case 1: return launch_predictor_ck_mixed_n<1>(a, t, f, s);
      case 2: return launch_predictor_ck_mixed_n<2>(a, t, f, s);
      case 3: return launch_predictor_ck_mixed_n<3>(a, t, f, s);
      case 4: return launch_predictor_ck_mixed_n<4>(a, t, f, s);
      case 5: return launch_predictor_ck_mixed_n<5>(a, t, f, s);
      case 6: return launch_predictor_ck_mixed_n<6>(a, t, f, s);
    }
    return cudaErrorInvalidValue;
  }
  switch (a.g.order) {
    case 1: return launch_predictor_ck_n<1>(a, t, s);
    case 2: return launch_predictor_ck_n<2>(a, t, s);
    case 3: return launch_predictor_ck_n<3>(a, t, s);
    case 4: return launch_predictor_ck_n<4>(a, t, s);
    case 5: return launch_predictor_ck_n<5>(a, t, s);
    case 6: return launch_predictor_ck_n<6>(a, t, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace ader
