// Multigrid transfers between 3D hexahedral Q2 levels (the 3D counterpart of
// the 2D tensor-product transfers). Levels are coarsened by pairing cells
// inside each segment of each axis, so every level stays interface-fitted;
// with an odd cell count the last coarse cell of a segment spans one fine
// cell. Prolongation is Q2 interpolation of the coarse field at the fine
// nodes (a tensor product of 1D quadratic Lagrange weights), restriction its
// transpose, and the state of a coarse level is the fine Q2 field evaluated at
// the coarse nodes. Identity rows (Dirichlet, p = 0) are left out of both.
// Host tables plus __host__ __device__ per-entry functions (kernels and host
// checks compile the same code).
#pragma once

#include <algorithm>
#include <cmath>
#include <vector>

#include "fsi_mesh3d.h"

namespace fsi3 {

// Pair the cells of each segment: n cells -> (n + 1) / 2 (the 2D rule).
inline void coarsen_axis3(const std::vector<double>& v, const std::vector<int>& seg, std::vector<double>& vc,
                          std::vector<int>& segc) {
  vc.assign(1, v[0]);
  segc.clear();
  int off = 0;
  for (int n : seg) {
    for (int j = 2; j <= n; j += 2) vc.push_back(v[off + j]);
    if (n % 2) vc.push_back(v[off + n]);
    segc.push_back((n + 1) / 2);
    off += n;
  }
}

inline double lag2_3(int a, double s) {
  return a == 0 ? (1 - s) * (1 - 2 * s) : (a == 1 ? 4 * s * (1 - s) : s * (2 * s - 1));
}

// 1D Q2 interpolation from the cells with vertices vc to the points x:
// pidx/pw [points][3] (node of the vc grid, weight; -1 padded) and the
// transpose ridx/rw [vc nodes][7].
inline void interp_1d3(const std::vector<double>& vc, const std::vector<double>& x, std::vector<int>& pidx,
                       std::vector<double>& pw, std::vector<int>& ridx, std::vector<double>& rw) {
  const int nf = (int)x.size(), nc = 2 * ((int)vc.size() - 1) + 1;
  pidx.assign((size_t)nf * 3, -1);
  pw.assign((size_t)nf * 3, 0.0);
  std::vector<std::vector<std::pair<int, double>>> cols(nc);
  for (int i = 0; i < nf; ++i) {
    int cc = (int)(std::upper_bound(vc.begin(), vc.end(), x[i]) - vc.begin()) - 1;
    cc = std::max(0, std::min(cc, (int)vc.size() - 2));
    const double s = (x[i] - vc[cc]) / (vc[cc + 1] - vc[cc]);
    int e = 0;
    for (int a = 0; a < 3; ++a) {
      double w = lag2_3(a, s);
      if (std::fabs(w) < 1e-13) continue;
      if (std::fabs(w - 1.0) < 1e-13) w = 1.0;
      pidx[(size_t)i * 3 + e] = 2 * cc + a;
      pw[(size_t)i * 3 + e] = w;
      cols[2 * cc + a].push_back({i, w});
      ++e;
    }
  }
  ridx.assign((size_t)nc * 7, -1);
  rw.assign((size_t)nc * 7, 0.0);
  for (int I = 0; I < nc; ++I)
    for (size_t e = 0; e < cols[I].size() && e < 7; ++e) {
      ridx[(size_t)I * 7 + e] = cols[I][e].first;
      rw[(size_t)I * 7 + e] = cols[I][e].second;
    }
}

// Host tables of the transfer between a fine level F and the coarse level C.
struct Transfer3 {
  int nn_f[3], nn_c[3];
  std::vector<int> pidx[3], ridx[3], iidx[3];
  std::vector<double> pw[3], rw[3], iw[3];
};

// xv_*: vertex coordinates per axis; xn_*: Q2 node coordinates per axis.
inline void build_transfer3(Transfer3& T, const std::vector<double>* xv_c, const std::vector<double>* xn_c,
                            const std::vector<double>* xv_f, const std::vector<double>* xn_f) {
  std::vector<int> d0;
  std::vector<double> d1;
  for (int a = 0; a < 3; ++a) {
    T.nn_f[a] = (int)xn_f[a].size();
    T.nn_c[a] = (int)xn_c[a].size();
    interp_1d3(xv_c[a], xn_f[a], T.pidx[a], T.pw[a], T.ridx[a], T.rw[a]);   // coarse -> fine and its transpose
    interp_1d3(xv_f[a], xn_c[a], T.iidx[a], T.iw[a], d0, d1);               // fine field at the coarse nodes
  }
}

struct Transfer3View {
  int nn_f[3], nn_c[3];
  const int *pidx[3], *ridx[3], *iidx[3];
  const double *pw[3], *rw[3], *iw[3];
};

inline Transfer3View view(const Transfer3& T) {
  Transfer3View v;
  for (int a = 0; a < 3; ++a) {
    v.nn_f[a] = T.nn_f[a];
    v.nn_c[a] = T.nn_c[a];
    v.pidx[a] = T.pidx[a].data();
    v.ridx[a] = T.ridx[a].data();
    v.iidx[a] = T.iidx[a].data();
    v.pw[a] = T.pw[a].data();
    v.rw[a] = T.rw[a].data();
    v.iw[a] = T.iw[a].data();
  }
  return v;
}

// Prolongation of the coarse vector xc [coarse nodes][7] at fine row (node, c)
// (to be added to the fine correction; 0 on identity rows).
template <typename V>
FSI3M_HD inline V prolong3(const Transfer3View& T, const uint8_t* nflags_f, const V* xc, int node, int c) {
  if (identity_row3(nflags_f[node], c)) return V(0);
  const int i = node % T.nn_f[0], j = (node / T.nn_f[0]) % T.nn_f[1], k = node / (T.nn_f[0] * T.nn_f[1]);
  V acc = 0;
  for (int ez = 0; ez < 3; ++ez) {
    const int K = T.pidx[2][k * 3 + ez];
    if (K < 0) break;
    for (int ey = 0; ey < 3; ++ey) {
      const int J = T.pidx[1][j * 3 + ey];
      if (J < 0) break;
      for (int ex = 0; ex < 3; ++ex) {
        const int I = T.pidx[0][i * 3 + ex];
        if (I < 0) break;
        const V w = V(T.pw[2][k * 3 + ez] * T.pw[1][j * 3 + ey] * T.pw[0][i * 3 + ex]);
        acc += w * xc[((size_t)I + T.nn_c[0] * ((size_t)J + T.nn_c[1] * K)) * 7 + c];
      }
    }
  }
  return acc;
}

// Restriction of the fine residual rf [fine nodes][7] to coarse row (node, c):
// the transpose of prolong3 over the free rows of both levels.
template <typename V>
FSI3M_HD inline V restrict3(const Transfer3View& T, const uint8_t* nflags_f, const uint8_t* nflags_c, const V* rf,
                            int node, int c) {
  if (identity_row3(nflags_c[node], c)) return V(0);
  const int I = node % T.nn_c[0], J = (node / T.nn_c[0]) % T.nn_c[1], K = node / (T.nn_c[0] * T.nn_c[1]);
  V acc = 0;
  for (int ez = 0; ez < 7; ++ez) {
    const int k = T.ridx[2][K * 7 + ez];
    if (k < 0) break;
    for (int ey = 0; ey < 7; ++ey) {
      const int j = T.ridx[1][J * 7 + ey];
      if (j < 0) break;
      for (int ex = 0; ex < 7; ++ex) {
        const int i = T.ridx[0][I * 7 + ex];
        if (i < 0) break;
        const size_t fn = (size_t)i + T.nn_f[0] * ((size_t)j + T.nn_f[1] * k);
        if (identity_row3(nflags_f[fn], c)) continue;
        acc += V(T.rw[2][K * 7 + ez] * T.rw[1][J * 7 + ey] * T.rw[0][I * 7 + ex]) * rf[fn * 7 + c];
      }
    }
  }
  return acc;
}

// The fine state Uf [fine nodes][7] evaluated at coarse node `node`, component c.
FSI3M_HD inline double interp_state3(const Transfer3View& T, const double* Uf, int node, int c) {
  const int I = node % T.nn_c[0], J = (node / T.nn_c[0]) % T.nn_c[1], K = node / (T.nn_c[0] * T.nn_c[1]);
  double acc = 0.0;
  for (int ez = 0; ez < 3; ++ez) {
    const int k = T.iidx[2][K * 3 + ez];
    if (k < 0) break;
    for (int ey = 0; ey < 3; ++ey) {
      const int j = T.iidx[1][J * 3 + ey];
      if (j < 0) break;
      for (int ex = 0; ex < 3; ++ex) {
        const int i = T.iidx[0][I * 3 + ex];
        if (i < 0) break;
        acc += T.iw[2][K * 3 + ez] * T.iw[1][J * 3 + ey] * T.iw[0][I * 3 + ex] *
               Uf[((size_t)i + T.nn_f[0] * ((size_t)j + T.nn_f[1] * k)) * 7 + c];
      }
    }
  }
  return acc;
}

}  // namespace fsi3
