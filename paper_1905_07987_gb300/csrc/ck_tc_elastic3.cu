// Cauchy-Kowalevski predictor of the 3-D elastic family on the tensor cores (TF32 split
// operands, ADER_PREC_MIXED_TF32X3), orders with an even number of nodes per direction.
#include "kernels_ck_tc.cuh"

namespace ader {

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link-time dependency on
// the driver library).
EncodeTiledFn tensor_map_encoder() {
  static EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return (EncodeTiledFn) nullptr;
    return (EncodeTiledFn)p;
  }();
  return fn;
}

bool predictor_ck_tc_order_ok(int order) { return order == 1 || order == 3 || order == 5; }

cudaError_t predictor_ck_tc_elastic3(const StepArgs& a, const Tables& t, cudaStream_t s) {
  switch (a.g.order) {
    case 1: return launch_predictor_ck_tc_n<1>(a, t, s);
    case 3: return launch_predictor_ck_tc_n<3>(a, t, s);
    case 5: return launch_predictor_ck_tc_n<5>(a, t, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace ader
