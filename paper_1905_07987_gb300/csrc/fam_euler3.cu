// Kernel family: Euler<3> in 3D, orders 1-6, with the a-posteriori subcell limiter (orders 1-4).
#include "kernels_limiter.cuh"

namespace ader {
namespace {
constexpr int LIM_MAX_ORDER = 4;

cudaError_t lim_init(int order, double* u, const double* Usub, const uint8_t* flags, double* rep,
                     double* mm, long long ncells, const SubTables& S, cudaStream_t s) {
  switch (order) {
    case 1: return LimLaunch<3, 1>::init(u, Usub, flags, rep, mm, ncells, S, s);
    case 2: return LimLaunch<3, 2>::init(u, Usub, flags, rep, mm, ncells, S, s);
    case 3: return LimLaunch<3, 3>::init(u, Usub, flags, rep, mm, ncells, S, s);
    case 4: return LimLaunch<3, 4>::init(u, Usub, flags, rep, mm, ncells, S, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t lim_step(const StepArgs& a, const LimArgs& l, const Tables& t, const SubTables& S,
                     cudaStream_t s) {
  switch (a.g.order) {
    case 1: return LimLaunch<3, 1>::step(a, l, t, S, s);
    case 2: return LimLaunch<3, 2>::step(a, l, t, S, s);
    case 3: return LimLaunch<3, 3>::step(a, l, t, S, s);
    case 4: return LimLaunch<3, 4>::step(a, l, t, S, s);
  }
  return cudaErrorInvalidValue;
}
}  // namespace

const Family* family_euler3() {
  static Family f = [] {
    Family g = *FamilyImpl<Euler<3>, 3>::get();
    g.lim_init = &lim_init;
    g.lim_step = &lim_step;
    return g;
  }();
  return &f;
}
int limiter_max_order3() { return LIM_MAX_ORDER; }
}  // namespace ader
