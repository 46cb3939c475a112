// Host build of the float-float dot product of the library (csrc/fsi_ff.h).
#include "../../paper_1907_01252_gb300/csrc/fsi_ff.h"

extern "C" double ff_dot_host(const double* a, const double* x, int n) {
  fsiff::ffacc acc;
  for (int i = 0; i < n; ++i) fsiff::fma_ff(acc, fsiff::split(a[i]), fsiff::split(x[i]));
  return fsiff::result(acc);
}

extern "C" double f64_dot_host(const double* a, const double* x, int n) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += a[i] * x[i];
  return s;
}
