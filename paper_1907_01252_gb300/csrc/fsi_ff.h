// Float-float arithmetic for FP64-accurate linear algebra on the FP32 pipe.
//
// A double d is carried as an unevaluated sum hi + lo of two floats
// (hi = fl32(d), lo = fl32(d - hi)), which holds d to a relative 2^-48 or
// better while it stays in the float range. Products and sums use the
// error-free transformations:
//   TwoSum (Knuth, The Art of Computer Programming vol. 2, 4.2.2): s + e = a + b
//     exactly, s = fl(a + b);
//   TwoProduct with a fused multiply-add: p + e = a b exactly, p = fl(a b),
//     e = fma(a, b, -p);
// and a dot product accumulates them in the manner of the compensated dot
// product Dot2 of Ogita, Rump and Oishi ("Accurate sum and dot product", SIAM
// J. Sci. Comput. 26, 2005): the running sum s carries the leading part and a
// compensation the sum of all rounding errors and low-order cross terms. Each
// term then contributes an error of order 2^-48 relative to the running sum.
#pragma once

#include <cmath>

#ifdef __CUDACC__
#define FSI_FF_HD __host__ __device__
#else
#define FSI_FF_HD
#endif

namespace fsiff {

struct ff {
  float hi, lo;
};

FSI_FF_HD inline ff split(double d) {
  const float hi = (float)d;
  return ff{hi, (float)(d - (double)hi)};
}

FSI_FF_HD inline double join(ff a) { return (double)a.hi + (double)a.lo; }

FSI_FF_HD inline float fma32(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return std::fma(a, b, c);
#endif
}

// s + e = a + b exactly (any ordering of |a|, |b|).
FSI_FF_HD inline void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bv = s - a;
  e = (a - (s - bv)) + (b - bv);
}

// Running dot product: s (leading part) and the compensation c + cc, itself
// kept as a float pair so that summing the rounding errors adds no error of
// its own at the 2^-48 level.
struct ffacc {
  float s = 0.0f, c = 0.0f, cc = 0.0f;
};

// acc += a x for float-float a and x: the leading product a.hi x.hi by
// TwoProduct; its rounding error, the error of adding it to s, and the two
// first-order cross terms go into the compensation (a.lo x.lo is below 2^-48
// relative and dropped).
FSI_FF_HD inline void fma_ff(ffacc& acc, ff a, ff x) {
  const float p = a.hi * x.hi;
  const float ep = fma32(a.hi, x.hi, -p);
  const float cross = fma32(a.hi, x.lo, a.lo * x.hi);
  float s, es, c, ec;
  two_sum(acc.s, p, s, es);
  acc.s = s;
  two_sum(acc.c, es + (ep + cross), c, ec);
  acc.c = c;
  acc.cc += ec;
}

FSI_FF_HD inline double result(const ffacc& acc) { return (double)acc.s + ((double)acc.c + (double)acc.cc); }

}  // namespace fsiff
