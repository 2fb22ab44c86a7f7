// Kernel family: shallow water equations with bathymetry in 2D (Eq. (9)), orders 1-6, FP64.
#include "kernels.cuh"

namespace ader {
const Family* family_swe2() { return FamilyImpl<ShallowWater, 2>::get(); }
}  // namespace ader
