// Cell-wise Vanka smoother of the 3D path (the multigrid smoother of Sec. 3.2,
// on 27-node hexahedra). The local matrix of a cell is the global Jacobian
// restricted to the cell's 189 dofs. The full FP64 inverse (286 KB) does not fit
// one CTA's shared memory, so the local solve is a block elimination over the
// split of the cell's dofs into
//   part 1: velocity and pressure, index q * 27 + l (q = 0, 1, 2 velocity, 3 pressure),
//   part 2: displacement,          index (c - 3) * 27 + l,
// A = [A11 A12; A21 A22], S = A22 - A21 A11^{-1} A12:
//   y1 = A11^{-1} r1,  z2 = S^{-1} (r2 - A21 y1),  z1 = y1 - (A11^{-1} A12) z2.
// In cells flagged C3_U_DECOUPLED, A21 = 0 and A22 = diag(L_x, L_y, L_z):
//   z2 = L_q^{-1} r2 per component,  z1 = A11^{-1} (r1 - A12 z2).
// A11 and S are inverted by Gauss-Jordan with partial pivoting (108 x 108 and
// 81 x 81 in FP64 fit one CTA). The corrections of the cells are averaged per
// node and damped by omega, as in the 2D smoother.
//
// The per-cell routines are written once for a cooperative thread group
// (fsi_cta.h), so host checks execute the kernels' arithmetic.
//
// Stored inverse of a cell: VK3_SIZE elements (= 189^2), all column-major:
//   [VK3_O_A] A11^{-1}            108 x 108
//   [VK3_O_B] A11^{-1} A12 (coupled) or A12 (decoupled)       108 x 81
//   [VK3_O_C] A21 (coupled; unused when decoupled)            81 x 108
//   [VK3_O_S] S^{-1} (coupled) or L_q^{-1}, q = 0..2, 27 x 27 each (decoupled)
#pragma once

#include <cmath>

#include "fsi_cta.h"
#include "fsi_mesh3d.h"

namespace fsi3 {

constexpr int VK3_N1 = 108, VK3_N2 = 81;
constexpr int VK3_O_A = 0;
constexpr int VK3_O_B = VK3_O_A + VK3_N1 * VK3_N1;
constexpr int VK3_O_C = VK3_O_B + VK3_N1 * VK3_N2;
constexpr int VK3_O_S = VK3_O_C + VK3_N2 * VK3_N1;
constexpr int VK3_SIZE = VK3_O_S + VK3_N2 * VK3_N2;
static_assert(VK3_SIZE == 189 * 189, "block storage holds one dense local matrix");

// Shared scratch of the setup (elements of T, then ints).
constexpr int VK3_LD1 = VK3_N1 + 1, VK3_LD2 = VK3_N2 + 1;
constexpr int VK3_SH_M = 0;                                  // [108][109]: A11, later A21
constexpr int VK3_SH_B = VK3_SH_M + VK3_N1 * VK3_LD1;        // [108][81]:  P A12, later X
constexpr int VK3_SH_S = VK3_SH_B + VK3_N1 * VK3_N2;         // [81][82]:   S (or a 27 x 28 block), temp of X
constexpr int VK3_SH_COL = VK3_SH_S + VK3_N2 * VK3_LD2;      // [108]
constexpr int VK3_SH_T = VK3_SH_COL + VK3_N1 + 1;            // elements of T (one for the pivot inverse)
constexpr int VK3_SH_I = 2 * VK3_N1 + 2;                     // ints: perm1, perm2 (<= 108 each), pivot
template <typename T>
constexpr int vk3_setup_smem_bytes() {
  return VK3_SH_T * (int)sizeof(T) + VK3_SH_I * (int)sizeof(int);
}
// Shared scratch of the apply: r1, r2, y1, t2, z2, z1.
constexpr int VK3_AP_R1 = 0, VK3_AP_R2 = 108, VK3_AP_Y1 = 189, VK3_AP_T2 = 297, VK3_AP_Z2 = 378, VK3_AP_Z1 = 459;
constexpr int VK3_AP_T = 567;

// Local dof (l * 7 + c) of a part-1 / part-2 index.
FSI3M_HD inline int vk3_dof1(int i) {
  const int q = i / 27, l = i % 27;
  return l * 7 + (q < 3 ? q : 6);
}
FSI3M_HD inline int vk3_dof2(int i) { return (i % 27) * 7 + 3 + i / 27; }

// Entry (local dof a, local dof b) of the local matrix of `cell`: one slice's
// block values A[nnzb][7][7].
template <typename T>
FSI3M_HD inline T vk3_entry(const Mesh3View& m, const T* A, int cell, int a, int b) {
  const int blk = m.cell_blk[(size_t)cell * 729 + (a / 7) * 27 + b / 7];
  return A[(size_t)blk * 49 + (a % 7) * 7 + b % 7];
}

// Row of the largest |M[r][kk]|, r in [kk, n), the lowest such row on ties;
// -1 if that maximum is not positive. Written to *piv by thread 0 (a warp
// reduction on the device, a scan on the host: the same result).
template <class Cta, typename T>
FSI3M_HD inline void vk3_pivot(const Cta& cta, const T* M, int ld, int n, int kk, int* piv) {
#ifdef __CUDA_ARCH__
  if (cta.tid < 32) {
    T best = -1;
    int bi = kk;
    for (int r = kk + cta.tid; r < n; r += 32) {
      const T a = fabs(M[r * ld + kk]);
      if (a > best) {
        best = a;
        bi = r;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const T ob = __shfl_down_sync(0xffffffffu, best, o);
      const int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    if (cta.tid == 0) *piv = best > 0 ? bi : -1;
  }
#else
  if (cta.tid == 0) {
    T best = -1;
    int bi = kk;
    for (int r = kk; r < n; ++r) {
      const T a = std::fabs(M[r * ld + kk]);
      if (a > best) {
        best = a;
        bi = r;
      }
    }
    *piv = best > 0 ? bi : -1;
  }
#endif
}

// In-place Gauss-Jordan inversion of the n x n matrix M (row stride ld) with
// row exchanges: on return M[r][c] = (A^{-1})[r][perm[c]]. colk: n scratch
// elements; piv, pinv: one shared slot each. Returns false (in every thread)
// when a pivot column has no nonzero entry.
template <class Cta, typename T>
FSI3M_HD inline bool vk3_gauss_jordan(const Cta& cta, T* M, int ld, int n, int* perm, T* colk, int* piv, T* pinv) {
  for (int r = cta.tid; r < n; r += cta.nt) perm[r] = r;
  cta.sync();
  for (int kk = 0; kk < n; ++kk) {
    vk3_pivot(cta, M, ld, n, kk, piv);
    cta.sync();
    const int p = *piv;
    if (p < 0) return false;
    if (p != kk) {
      for (int c = cta.tid; c < n; c += cta.nt) {
        const T t = M[kk * ld + c];
        M[kk * ld + c] = M[p * ld + c];
        M[p * ld + c] = t;
      }
      if (cta.tid == 0) {
        const int t = perm[kk];
        perm[kk] = perm[p];
        perm[p] = t;
      }
    }
    cta.sync();
    if (cta.tid == 0) *pinv = T(1) / M[kk * ld + kk];
    cta.sync();
    const T d = *pinv;
    for (int c = cta.tid; c < n; c += cta.nt) M[kk * ld + c] = (c == kk) ? d : M[kk * ld + c] * d;
    for (int r = cta.tid; r < n; r += cta.nt) colk[r] = (r == kk) ? T(0) : M[r * ld + kk];
    cta.sync();
    for (int e = cta.tid; e < n * n; e += cta.nt) {
      const int r = e / n, c = e % n;
      if (r == kk) continue;
      const T f = colk[r];
      M[r * ld + c] = (c == kk) ? -f * d : M[r * ld + c] - f * M[kk * ld + c];
    }
    cta.sync();
  }
  return true;
}

// Block inverse of one cell (layout above) from one slice's Jacobian blocks A.
// sh: VK3_SH_T elements of T; ish: VK3_SH_I ints (shared memory on the device).
// Returns false if A11 or S (or an L_q) is singular.
template <class Cta, typename T>
FSI3M_HD inline bool vk3_setup_cell(const Cta& cta, const Mesh3View& m, const T* A, int cell, T* sh, int* ish,
                                    T* out) {
  T* M = sh + VK3_SH_M;
  T* B = sh + VK3_SH_B;
  T* Sm = sh + VK3_SH_S;
  T* colk = sh + VK3_SH_COL;
  T* pinv = colk + VK3_N1;
  int* perm1 = ish;
  int* perm2 = ish + VK3_N1;
  int* piv = ish + 2 * VK3_N1;
  const bool dec = m.cell_flags[cell] & C3_U_DECOUPLED;
  for (int e = cta.tid; e < VK3_N1 * VK3_N1; e += cta.nt) {
    const int i = e / VK3_N1, j = e % VK3_N1;
    M[i * VK3_LD1 + j] = vk3_entry(m, A, cell, vk3_dof1(i), vk3_dof1(j));
  }
  cta.sync();
  if (!vk3_gauss_jordan(cta, M, VK3_LD1, VK3_N1, perm1, colk, piv, pinv)) return false;
  for (int e = cta.tid; e < VK3_N1 * VK3_N1; e += cta.nt) {
    const int i = e / VK3_N1, j = e % VK3_N1;
    out[VK3_O_A + perm1[j] * VK3_N1 + i] = M[i * VK3_LD1 + j];
  }
  if (dec) {
    for (int e = cta.tid; e < VK3_N1 * VK3_N2; e += cta.nt) {   // A12, column-major
      const int j = e / VK3_N1, i = e % VK3_N1;
      out[VK3_O_B + e] = vk3_entry(m, A, cell, vk3_dof1(i), vk3_dof2(j));
    }
    for (int q = 0; q < 3; ++q) {
      for (int e = cta.tid; e < 27 * 27; e += cta.nt) {
        const int i = e / 27, j = e % 27;
        Sm[i * 28 + j] = vk3_entry(m, A, cell, vk3_dof2(q * 27 + i), vk3_dof2(q * 27 + j));
      }
      cta.sync();
      if (!vk3_gauss_jordan(cta, Sm, 28, 27, perm2, colk, piv, pinv)) return false;
      for (int e = cta.tid; e < 27 * 27; e += cta.nt) {
        const int i = e / 27, j = e % 27;
        out[VK3_O_S + q * 729 + perm2[j] * 27 + i] = Sm[i * 28 + j];
      }
      cta.sync();
    }
    return true;
  }
  // B = P A12 (rows in pivot order), then X = M B = A11^{-1} A12 column block by column block
  for (int e = cta.tid; e < VK3_N1 * VK3_N2; e += cta.nt) {
    const int k = e / VK3_N2, j = e % VK3_N2;
    B[e] = vk3_entry(m, A, cell, vk3_dof1(perm1[k]), vk3_dof2(j));
  }
  cta.sync();
  constexpr int kChunk = (VK3_N2 * VK3_LD2) / VK3_N1;   // columns of X per pass through the S scratch
  for (int j0 = 0; j0 < VK3_N2; j0 += kChunk) {
    const int nj = (VK3_N2 - j0 < kChunk) ? VK3_N2 - j0 : kChunk;
    for (int e = cta.tid; e < VK3_N1 * nj; e += cta.nt) {
      const int i = e / nj, j = j0 + e % nj;
      T acc = 0;
      for (int k = 0; k < VK3_N1; ++k) acc += M[i * VK3_LD1 + k] * B[k * VK3_N2 + j];
      Sm[e] = acc;
    }
    cta.sync();
    for (int e = cta.tid; e < VK3_N1 * nj; e += cta.nt) {
      const int i = e / nj, j = j0 + e % nj;
      B[i * VK3_N2 + j] = Sm[e];
      out[VK3_O_B + j * VK3_N1 + i] = Sm[e];
    }
    cta.sync();
  }
  // S = A22 - A21 X, with A21 in the M scratch
  for (int e = cta.tid; e < VK3_N2 * VK3_N1; e += cta.nt) {
    const int i = e / VK3_N1, k = e % VK3_N1;
    const T a = vk3_entry(m, A, cell, vk3_dof2(i), vk3_dof1(k));
    M[i * VK3_LD1 + k] = a;
    out[VK3_O_C + k * VK3_N2 + i] = a;
  }
  cta.sync();
  for (int e = cta.tid; e < VK3_N2 * VK3_N2; e += cta.nt) {
    const int i = e / VK3_N2, j = e % VK3_N2;
    T acc = vk3_entry(m, A, cell, vk3_dof2(i), vk3_dof2(j));
    for (int k = 0; k < VK3_N1; ++k) acc -= M[i * VK3_LD1 + k] * B[k * VK3_N2 + j];
    Sm[i * VK3_LD2 + j] = acc;
  }
  cta.sync();
  if (!vk3_gauss_jordan(cta, Sm, VK3_LD2, VK3_N2, perm2, colk, piv, pinv)) return false;
  for (int e = cta.tid; e < VK3_N2 * VK3_N2; e += cta.nt) {
    const int i = e / VK3_N2, j = e % VK3_N2;
    out[VK3_O_S + perm2[j] * VK3_N2 + i] = Sm[i * VK3_LD2 + j];
  }
  cta.sync();
  return true;
}

// Local correction z (local dof order l * 7 + c, written to z_out[189]) of one
// cell from its residual values r_loc[189] (local dof order), with the stored
// inverse inv. sh: VK3_AP_T elements of T.
template <class Cta, typename T>
FSI3M_HD inline void vk3_apply_cell(const Cta& cta, bool decoupled, const T* inv, const T* r_loc, T* sh, T* z_out) {
  T *r1 = sh + VK3_AP_R1, *r2 = sh + VK3_AP_R2, *y1 = sh + VK3_AP_Y1, *t2 = sh + VK3_AP_T2, *z2 = sh + VK3_AP_Z2,
    *z1 = sh + VK3_AP_Z1;
  for (int i = cta.tid; i < VK3_N1; i += cta.nt) r1[i] = r_loc[vk3_dof1(i)];
  for (int i = cta.tid; i < VK3_N2; i += cta.nt) r2[i] = r_loc[vk3_dof2(i)];
  cta.sync();
  if (decoupled) {
    for (int i = cta.tid; i < VK3_N2; i += cta.nt) {
      const int q = i / 27, ii = i % 27;
      const T* L = inv + VK3_O_S + q * 729;
      T acc = 0;
      for (int j = 0; j < 27; ++j) acc += L[j * 27 + ii] * r2[q * 27 + j];
      z2[i] = acc;
    }
    cta.sync();
    for (int i = cta.tid; i < VK3_N1; i += cta.nt) {
      T acc = r1[i];
      for (int j = 0; j < VK3_N2; ++j) acc -= inv[VK3_O_B + j * VK3_N1 + i] * z2[j];
      y1[i] = acc;
    }
    cta.sync();
    for (int i = cta.tid; i < VK3_N1; i += cta.nt) {
      T acc = 0;
      for (int j = 0; j < VK3_N1; ++j) acc += inv[VK3_O_A + j * VK3_N1 + i] * y1[j];
      z1[i] = acc;
    }
    cta.sync();
  } else {
    for (int i = cta.tid; i < VK3_N1; i += cta.nt) {
      T acc = 0;
      for (int j = 0; j < VK3_N1; ++j) acc += inv[VK3_O_A + j * VK3_N1 + i] * r1[j];
      y1[i] = acc;
    }
    cta.sync();
    for (int i = cta.tid; i < VK3_N2; i += cta.nt) {
      T acc = r2[i];
      for (int j = 0; j < VK3_N1; ++j) acc -= inv[VK3_O_C + j * VK3_N2 + i] * y1[j];
      t2[i] = acc;
    }
    cta.sync();
    for (int i = cta.tid; i < VK3_N2; i += cta.nt) {
      T acc = 0;
      for (int j = 0; j < VK3_N2; ++j) acc += inv[VK3_O_S + j * VK3_N2 + i] * t2[j];
      z2[i] = acc;
    }
    cta.sync();
    for (int i = cta.tid; i < VK3_N1; i += cta.nt) {
      T acc = y1[i];
      for (int j = 0; j < VK3_N2; ++j) acc -= inv[VK3_O_B + j * VK3_N1 + i] * z2[j];
      z1[i] = acc;
    }
    cta.sync();
  }
  for (int i = cta.tid; i < VK3_N1; i += cta.nt) z_out[vk3_dof1(i)] = z1[i];
  for (int i = cta.tid; i < VK3_N2; i += cta.nt) z_out[vk3_dof2(i)] = z2[i];
}

// Smoothed update of row (node, c): x += omega / (cells of the node) * (sum of
// the cells' corrections at the node), cells in ascending order. cellz:
// [cell][189] corrections of one slice.
template <typename T>
FSI3M_HD inline T vk3_gather(const Mesh3View& m, const T* cellz, double omega, int node, int c) {
  T acc = 0;
  int cnt = 0;
  for (int e = 0; e < 8; ++e) {
    const int code = m.node_cells[(size_t)node * 8 + e];
    if (code < 0) break;
    acc += cellz[(size_t)(code / 27) * 189 + (code % 27) * 7 + c];
    ++cnt;
  }
  return T(omega / cnt) * acc;
}

}  // namespace fsi3
