// Kernel family: Elastic in 3D, orders 1-6.
#include "kernels.cuh"

namespace ader {
const Family* family_elastic3() { return FamilyImpl<Elastic, 3>::get(); }
}  // namespace ader
