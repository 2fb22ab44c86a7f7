// Kernel family: Euler<2> in 2D, orders 1-6.
#include "kernels.cuh"

namespace ader {
const Family* family_euler2() { return FamilyImpl<Euler<2>, 2>::get(); }
}  // namespace ader
