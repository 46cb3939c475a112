// Host build of the float-float dot product of the library (csrc/fsi_ff.h).
#include "../../paper_1907_01252_gb300/csrc/fsi_ff.h"

extern "C" double ff_dot_host(const double* a, const double* x, int n) {
  fsiff::ffacc acc;
  for (int i = 0; i < n; ++i) fsiff::fma_ff(acc, fsiff::split(a[i]), fsiff::split(x[i]));
  return fsiff::result(acc);
}

// The same dot product as the warp-per-row product forms it: lane (c, e) of a row sums the terms
// whose index is e mod 5, and the five partial sums are merged as the shuffle tree does
// (e0 += e2, e1 += e3, e0 += e1, e0 += e4).
extern "C" double ff_dot5_host(const double* a, const double* x, int n) {
  fsiff::ffacc acc[5];
  for (int i = 0; i < n; ++i) fsiff::fma_ff(acc[i % 5], fsiff::split(a[i]), fsiff::split(x[i]));
  fsiff::merge(acc[0], acc[2]);
  fsiff::merge(acc[1], acc[3]);
  fsiff::merge(acc[0], acc[1]);
  fsiff::merge(acc[0], acc[4]);
  return fsiff::result(acc[0]);
}

extern "C" double f64_dot_host(const double* a, const double* x, int n) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += a[i] * x[i];
  return s;
}
