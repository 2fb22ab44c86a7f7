// Kernel family: Euler<3> in 3D, orders 1-6.
#include "kernels.cuh"

namespace ader {
const Family* family_euler3() { return FamilyImpl<Euler<3>, 3>::get(); }
}  // namespace ader
