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

// Conversions on the integer pipe (bit operations only, no FP64 instruction), for kernels whose
// FP64 pipe is the bottleneck.
//
// x = hi + lo: hi keeps the leading 24 significant bits of x and lo the next 23 (both truncated,
// both with the sign of x), so |x - (hi + lo)| < 2^-46 |x| for 2^-80 <= |x| < 2^128.  Below:
// lo is 0 for |x| < 2^-80 (relative error < 2^-23, absolute < 2^-103) and |x| < 2^-126 gives
// (0, 0); |x| >= 2^128 and NaN give an infinite or NaN hi.
__device__ __forceinline__ ff ff_split_int(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned b1 = (unsigned)(b >> 32), b0 = (unsigned)b;
  const unsigned sign = b1 & 0x80000000u;
  const int e = (int)((b1 >> 20) & 0x7ffu);
  const unsigned mh = ((b1 & 0xfffffu) << 3) | (b0 >> 29);        // mantissa bits 51..29
  const unsigned ml = (b0 >> 6) & 0x7fffffu;                        // mantissa bits 28..6
  // ml 2^(e - 1069): (2^23 + ml) - 2^23 is exact, the scale is a power of two
  const float l = (__uint_as_float(0x4b000000u | ml) - 8388608.0f) *
                  __uint_as_float((unsigned)(e > 942 && e < 1197 ? e - 942 : 1) << 23);
  // special ranges by selects (no branches: a divergent path would split the warp's later
  // instructions)
  const unsigned nan = (e == 2047 && (b & 0xfffffffffffffull)) ? 0x400000u : 0u;
  const unsigned hb = e <= 896 ? sign
                               : (e >= 1151 ? (sign | 0x7f800000u | nan)
                                            : (sign | ((unsigned)(e - 896) << 23) | mh));
  const unsigned lb = (e <= 942 || e >= 1151) ? sign : (__float_as_uint(l) | sign);
  return {__uint_as_float(hb), __uint_as_float(lb)};
}

// Exact binary32 -> binary64 conversion (binary32 subnormals flush to a signed zero; infinities
// and NaN are kept); selects only.
__device__ __forceinline__ double f2d_int(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned s = u & 0x80000000u;
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned m = u & 0x7fffffu;
  const unsigned hn = s | ((e + 896u) << 20) | (m >> 3);
  const unsigned hs = s | 0x7ff00000u | (m ? 0x80000u : 0u) | (m >> 3);
  const unsigned hi = e == 0u ? s : (e == 255u ? hs : hn);
  const unsigned lo = (e == 0u || e == 255u) ? 0u : (m << 29);
  return __hiloint2double((int)hi, (int)lo);
}

}  // namespace ader
