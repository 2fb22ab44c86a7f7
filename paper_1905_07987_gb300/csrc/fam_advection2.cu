// Kernel family: Advection<2> in 2D, orders 1-6.
#include "kernels.cuh"

namespace ader {
const Family* family_advection2() { return FamilyImpl<Advection<2>, 2>::get(); }
}  // namespace ader
