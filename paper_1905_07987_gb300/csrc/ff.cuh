// Float-float arithmetic on the FP32 pipe: a value is hi + lo, two binary32 numbers with
// |lo| <= ulp(hi)/2 (about 44 significant bits), combined by error-free transformations (exact
// products of the hi parts by FMA, two-sum for the additions).
#pragma once
#include <cuda_runtime.h>

namespace ader {

struct ff {
  float h, l;
};

__device__ __forceinline__ ff ff_split(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double ff_to_d(ff a) { return (double)a.h + (double)a.l; }

__device__ __forceinline__ ff ff_norm(float s, float e) {
  const float h = s + e;
  return {h, e - (h - s)};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const float s = a.h + b.h;
  const float bv = s - a.h;
  const float e = (a.h - (s - bv)) + (b.h - bv);
  return ff_norm(s, e + (a.l + b.l));
}
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, {-b.h, -b.l}); }
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return ff_norm(p, e);
}
__device__ __forceinline__ ff ff_mulf(ff a, float b) {
  const float p = a.h * b;
  float e = fmaf(a.h, b, -p);
  e = fmaf(a.l, b, e);
  return ff_norm(p, e);
}
// a / b: approximate binary32 quotient (2 ulp), float-float residual, one correction; the
// correction step restores float-float accuracy.
__device__ __forceinline__ ff ff_div(ff a, ff b) {
  const float q1 = __fdividef(a.h, b.h);
  const ff r = ff_sub(a, ff_mulf(b, q1));
  return ff_norm(q1, __fdividef(r.h, b.h));
}

// acc += (ah + al) * (bh + bl): exact product of the high parts by FMA, cross terms, two-sum.
__device__ __forceinline__ void ff_mac(ff& acc, float ah, float al, float bh, float bl) {
  const float p = ah * bh;
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  const float s = acc.h + p;
  const float bv = s - acc.h;
  const float err = (acc.h - (s - bv)) + (p - bv);
  acc.h = s;
  acc.l = acc.l + (err + e);
}

}  // namespace ader
