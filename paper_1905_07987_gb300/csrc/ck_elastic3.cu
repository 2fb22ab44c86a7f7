// Cauchy-Kowalevski predictor of the 3-D elastic family, orders 1-6.
#include "kernels_ck.cuh"

namespace ader {

cudaError_t predictor_ck_elastic3(const StepArgs& a, const Tables& t, const TablesF&, int prec,
                                  cudaStream_t s) {
  if (prec != 0) return cudaErrorInvalidValue;
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
