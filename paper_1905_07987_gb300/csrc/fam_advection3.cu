// Kernel family: Advection<3> in 3D, orders 1-6.
#include "kernels.cuh"

namespace ader {
const Family* family_advection3() { return FamilyImpl<Advection<3>, 3>::get(); }
}  // namespace ader
