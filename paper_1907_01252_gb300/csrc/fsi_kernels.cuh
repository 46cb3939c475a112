// Device kernels of the batched ALE-FSI step: element residual and Jacobian,
// deterministic node/block gathers, block-sparse SpMV, Vanka smoother,
// multigrid transfers, coarsest dense inverse and FGMRES vector kernels.
//
// Every kernel takes the slice index from blockIdx.y (or a flattened index)
// and reads an `active` flag per slice: inactive slices do no work. No kernel
// uses atomics, so the result of a slice never depends on the other slices of
// the batch (a batched run is bit-for-bit the serial run of each slice).
#pragma once
#include <cstdint>

#include <cooperative_groups.h>

#include "fsi_element.cuh"
#include "fsi_tc.cuh"

// --------------------------------------------------------------------------
// Reference-cell tables (3 x 3 Gauss points, Q2 basis, q = q2*3 + q1,
// local node l = b*3 + a), filled from the host at set-up.
// --------------------------------------------------------------------------
__constant__ double c_phi[9][9];
__constant__ double c_dps[9][9];    // d/ds on the unit square
__constant__ double c_dpt[9][9];    // d/dt
__constant__ double c_wq[9];        // product weights on the unit square
__constant__ double c_phie[3][9];   // edge s = 1, t = Gauss points
__constant__ double c_dpse[3][9];
__constant__ double c_dpte[3][9];
__constant__ double c_we[3];
__constant__ double c_lps_ss[9][9]; // int grad_s kappa phi_i grad_s kappa phi_j over the unit square
__constant__ double c_lps_tt[9][9];

enum : uint8_t { NF_DIR_V = 1, NF_DIR_U = 2, NF_P_ID = 4, NF_IN_SOLID = 8, NF_INFLOW = 16 };
// CF_U_DECOUPLED: a fluid cell none of whose nodes touches the solid; its
// displacement rows (harmonic extension or Dirichlet) couple only to the same
// displacement component.
enum : uint8_t { CF_SOLID = 1, CF_OUTFLOW = 2, CF_U_DECOUPLED = 4 };

struct DevMesh {
  int nnx, nny, n_nodes, n_cells, nnzb;
  const int* cell_nodes;    // [n_cells][9]
  const double* cell_h;     // [n_cells][2]
  const uint8_t* cell_flags;
  const uint8_t* node_flags;
  const double* node_y;
  const int* node_cells;    // [n_nodes][4]: cell * 9 + local, ascending cell, -1 pad
  const int* rowptr;        // [n_nodes + 1]
  const int* colidx;        // [nnzb]
  const int* blk_row;       // [nnzb]
  const int* blk_src;       // [nnzb][4]: cell * 81 + li * 9 + lj, -1 pad
  const int* cell_blk;      // [n_cells][81]
  const int* spmv_rows;     // [n_nodes] rows ordered by block count (uniform warps)
};

// Whether cell contribution of test component c enters the row of a node.
__device__ inline bool row_takes(uint8_t cflags, uint8_t nflags, int c) {
  const bool solid = cflags & CF_SOLID;
  if (c < 2) return true;
  if (c < 4) return solid == bool(nflags & NF_IN_SOLID);
  return !solid;
}

__device__ inline bool is_identity_row(uint8_t nflags, int c) {
  if (c < 2) return nflags & NF_DIR_V;
  if (c < 4) return nflags & NF_DIR_U;
  return nflags & NF_P_ID;
}

__device__ inline double inflow_ramp(double t, double ramp_t) {
  return t < ramp_t ? 0.5 * (1.0 - cos(M_PI * t / ramp_t)) : 1.0;
}

// Dirichlet value of component c at a node (parabolic inflow, zero elsewhere).
__device__ inline double dirichlet_value(const Phys& P, uint8_t nflags, double y, int c, double t) {
  if (c == 0 && (nflags & NF_INFLOW) && (nflags & NF_DIR_V)) {
    double yy = y - P.y0;
    return inflow_ramp(t, P.ramp_t) * 1.5 * P.vbar * 4.0 * yy * (P.H - yy) / (P.H * P.H);
  }
  return 0.0;
}

// Gather the 9 x 5 nodal values of a cell.
__device__ inline void load_cell(const DevMesh& m, const double* U, int cell, double* Ue) {
  for (int l = 0; l < 9; ++l) {
    const double* src = U + (size_t)m.cell_nodes[cell * 9 + l] * 5;
    for (int c = 0; c < 5; ++c) Ue[l * 5 + c] = src[c];
  }
}

// alpha_K = alpha0 h_K^2 / (rho_f nu_f + rho_f |vbar_K| h_K), vbar_K the cell mean of v_{n-1}.
__device__ inline double lps_weight(const Phys& P, const double* Uo, double hx, double hy) {
  double mx = 0.0, my = 0.0, ws = 0.0;
  for (int q = 0; q < 9; ++q) {
    double vx = 0.0, vy = 0.0;
    for (int l = 0; l < 9; ++l) {
      vx += c_phi[q][l] * Uo[l * 5 + 0];
      vy += c_phi[q][l] * Uo[l * 5 + 1];
    }
    mx += c_wq[q] * vx;
    my += c_wq[q] * vy;
    ws += c_wq[q];
  }
  mx /= ws;
  my /= ws;
  double h = sqrt(hx * hx + hy * hy);
  return P.alpha0 * h * h / (P.rho_f * P.nu_f + P.rho_f * sqrt(mx * mx + my * my) * h);
}

// Values and gradients of all fields at volume quadrature point q.
__device__ inline void eval_qp(const double* Ue, const double* Uo, int q, double ihx, double ihy, QpIn& s) {
  double val[5] = {0, 0, 0, 0, 0}, gx[5] = {0, 0, 0, 0, 0}, gy[5] = {0, 0, 0, 0, 0};
  double valo[4] = {0, 0, 0, 0}, gxo[4] = {0, 0, 0, 0}, gyo[4] = {0, 0, 0, 0};
  for (int l = 0; l < 9; ++l) {
    const double ph = c_phi[q][l], ps = c_dps[q][l] * ihx, pt = c_dpt[q][l] * ihy;
    for (int c = 0; c < 5; ++c) {
      val[c] += ph * Ue[l * 5 + c];
      gx[c] += ps * Ue[l * 5 + c];
      gy[c] += pt * Ue[l * 5 + c];
    }
    for (int c = 0; c < 4; ++c) {
      valo[c] += ph * Uo[l * 5 + c];
      gxo[c] += ps * Uo[l * 5 + c];
      gyo[c] += pt * Uo[l * 5 + c];
    }
  }
  s.v[0] = val[0]; s.v[1] = val[1]; s.u[0] = val[2]; s.u[1] = val[3]; s.p = val[4];
  s.G = m2(gx[0], gy[0], gx[1], gy[1]);
  s.Hu = m2(gx[2], gy[2], gx[3], gy[3]);
  s.vo[0] = valo[0]; s.vo[1] = valo[1]; s.uo[0] = valo[2]; s.uo[1] = valo[3];
  s.Go = m2(gxo[0], gyo[0], gxo[1], gyo[1]);
  s.Huo = m2(gxo[2], gyo[2], gxo[3], gyo[3]);
}

__device__ inline void eval_edge_grad(const double* U, int q, double ihx, double ihy, M2& G, M2& Hu) {
  double gx[4] = {0, 0, 0, 0}, gy[4] = {0, 0, 0, 0};
  for (int l = 0; l < 9; ++l) {
    const double ps = c_dpse[q][l] * ihx, pt = c_dpte[q][l] * ihy;
    for (int c = 0; c < 4; ++c) {
      gx[c] += ps * U[l * 5 + c];
      gy[c] += pt * U[l * 5 + c];
    }
  }
  G = m2(gx[0], gy[0], gx[1], gy[1]);
  Hu = m2(gx[2], gy[2], gx[3], gy[3]);
}

// --------------------------------------------------------------------------
// Element residual: one thread per (slice, cell) -> cellbuf[s][cell][45].
// --------------------------------------------------------------------------
__global__ void k_cell_residual(DevMesh m, Phys P, const double* __restrict__ U, const double* __restrict__ Uold,
                                size_t stride, double k, double theta, const uint8_t* __restrict__ active,
                                double* __restrict__ cellbuf) {
  const int s = blockIdx.y;
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || cell >= m.n_cells) return;
  double Ue[45], Uo[45], R[45];
  load_cell(m, U + s * stride, cell, Ue);
  load_cell(m, Uold + s * stride, cell, Uo);
  const double hx = m.cell_h[cell * 2], hy = m.cell_h[cell * 2 + 1];
  const double ihx = 1.0 / hx, ihy = 1.0 / hy, area = hx * hy;
  const uint8_t cf = m.cell_flags[cell];
  const bool solid = cf & CF_SOLID;
  for (int i = 0; i < 45; ++i) R[i] = 0.0;
  for (int q = 0; q < 9; ++q) {
    QpIn st;
    QpDerived dd;
    eval_qp(Ue, Uo, q, ihx, ihy, st);
    derive(st, dd);
    double f[15];
    qp_flux(P, st, dd, solid, k, theta, f);
    const double w = c_wq[q] * area;
    for (int l = 0; l < 9; ++l) {
      const double b0 = w * c_phi[q][l], b1 = w * c_dps[q][l] * ihx, b2 = w * c_dpt[q][l] * ihy;
      for (int c = 0; c < 5; ++c) R[l * 5 + c] += b0 * f[c * 3] + b1 * f[c * 3 + 1] + b2 * f[c * 3 + 2];
    }
  }
  if (!solid) {
    const double a = lps_weight(P, Uo, hx, hy) * k;
    const double sx = hy * ihx, sy = hx * ihy;
    for (int i = 0; i < 9; ++i) {
      double acc = 0.0;
      for (int j = 0; j < 9; ++j) acc += (sx * c_lps_ss[i][j] + sy * c_lps_tt[i][j]) * Ue[j * 5 + 4];
      R[i * 5 + 4] += a * acc;
    }
    if (cf & CF_OUTFLOW) {
      for (int q = 0; q < 3; ++q) {
        M2 G, Hu, Go, Huo;
        eval_edge_grad(Ue, q, ihx, ihy, G, Hu);
        eval_edge_grad(Uo, q, ihx, ihy, Go, Huo);
        double e[2];
        edge_flux(P, G, Hu, Go, Huo, k, theta, e);
        const double w = c_we[q] * hy;
        for (int l = 0; l < 9; ++l) {
          R[l * 5 + 0] += w * c_phie[q][l] * e[0];
          R[l * 5 + 1] += w * c_phie[q][l] * e[1];
        }
      }
    }
  }
  double* out = cellbuf + ((size_t)s * m.n_cells + cell) * 45;
  for (int i = 0; i < 45; ++i) out[i] = R[i];
}

// Node gather of the residual in fixed cell order, identity rows last.
__global__ void k_gather_residual(DevMesh m, Phys P, const double* __restrict__ cellbuf, const double* __restrict__ U,
                                  size_t stride, const double* __restrict__ t_new, const uint8_t* __restrict__ active,
                                  double* __restrict__ R) {
  const int s = blockIdx.y;
  const int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || node >= m.n_nodes) return;
  const uint8_t nf = m.node_flags[node];
  double acc[5] = {0, 0, 0, 0, 0};
  for (int e = 0; e < 4; ++e) {
    const int code = m.node_cells[node * 4 + e];
    if (code < 0) break;
    const int cell = code / 9, l = code % 9;
    const uint8_t cf = m.cell_flags[cell];
    const double* src = cellbuf + ((size_t)s * m.n_cells + cell) * 45 + l * 5;
    for (int c = 0; c < 5; ++c)
      if (row_takes(cf, nf, c)) acc[c] += src[c];
  }
  const double* Un = U + s * stride + (size_t)node * 5;
  double* out = R + s * stride + (size_t)node * 5;
  for (int c = 0; c < 5; ++c) {
    if (is_identity_row(nf, c)) acc[c] = Un[c] - dirichlet_value(P, nf, m.node_y[node], c, t_new[s]);
    out[c] = acc[c];
  }
}

// Impose the Dirichlet data of time t[s] on a state.
__global__ void k_apply_dirichlet(DevMesh m, Phys P, double* __restrict__ U, size_t stride, const double* __restrict__ t,
                                  const uint8_t* __restrict__ active) {
  const int s = blockIdx.y;
  const int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || node >= m.n_nodes) return;
  const uint8_t nf = m.node_flags[node];
  double* x = U + s * stride + (size_t)node * 5;
  for (int c = 0; c < 4; ++c)
    if (is_identity_row(nf, c)) x[c] = dirichlet_value(P, nf, m.node_y[node], c, t[s]);
}

// --------------------------------------------------------------------------
// Element Jacobian: one CTA of 128 threads per (slice, cell).
// K[(i,ci),(j,cj)] = sum_q w_q sum_{a,b} B_a(i,q) D_q[(ci,a),(cj,b)] B_b(j,q)
// with D_q the linearised flux (15 test slots x 15 trial directions).
// --------------------------------------------------------------------------
constexpr int JAC_THREADS = 160;   // one round for the 9 x 15 tangent directions

// Field blocks (test component ci, trial component cj) of the element
// matrix that can be nonzero (the LPS pressure block is added separately).
__device__ inline bool jac_block_nonzero(bool solid, int ci, int cj) {
  if (!solid) {
    if (ci < 2) return true;                 // momentum: v, u, p
    if (ci < 4) return cj == ci;             // harmonic extension
    return cj < 4;                           // divergence: v, u
  }
  if (ci < 2) return cj == ci || cj == 2 || cj == 3;   // mass, elastic stress
  if (ci < 4) return cj == ci || cj == ci - 2;         // kinematic row
  return false;
}

// Old-state blocks (OLD = true: dR_n / dU_{n-1}, for the discrete adjoint):
// the t_{n-1} fields (v, u) enter every row but the divergence rows, which see
// the old state only through the stabilisation weight (added separately).
__device__ inline bool jac_old_block_nonzero(bool solid, int ci, int cj) {
  if (cj >= 4 || ci == 4) return false;
  if (!solid) return ci < 2 || cj == ci;
  if (ci < 2) return cj == ci || cj == 2 || cj == 3;
  return cj == ci || cj == ci - 2;
}

// Shared state of the element Jacobian's tangent stage (one CTA per cell and slice).
struct JacTangentShared {
  double sU[45], sUo[45];
  QpIn sq[9];
  QpDerived sd[9];
  double sD[9][15][15];     // [q][test slot][trial direction]
  double sDe[3][2][12];     // outflow edge: [q][momentum comp][trial direction (c<4)]
  double sAlpha;
  double sSp[9], sDalpha[2];   // OLD: S p per local node, d alpha / d vbar
};

// The tangent stage: the cell's states, the quadrature-point quantities, the
// 15 x 15 tangent D_q at every quadrature point (sD), the outflow-edge tangent
// (sDe) and the stabilisation weight; ends with a CTA barrier.
template <bool OLD>
__device__ __forceinline__ void jac_tangent(const DevMesh& m, const Phys& P, const double* __restrict__ U,
                                            const double* __restrict__ Uold, size_t stride, double k, double theta,
                                            double lps_scale, int s, int cell, JacTangentShared& sh) {
  double* sU = sh.sU;
  double* sUo = sh.sUo;
  QpIn* sq = sh.sq;
  QpDerived* sd = sh.sd;
  auto& sD = sh.sD;
  auto& sDe = sh.sDe;
  double& sAlpha = sh.sAlpha;
  double* sSp = sh.sSp;
  double* sDalpha = sh.sDalpha;
  const int tid = threadIdx.x;
  const double hx = m.cell_h[cell * 2], hy = m.cell_h[cell * 2 + 1];
  const double ihx = 1.0 / hx, ihy = 1.0 / hy;
  const uint8_t cf = m.cell_flags[cell];
  const bool solid = cf & CF_SOLID;
  const bool outflow = !solid && (cf & CF_OUTFLOW);
  if (tid < 45) {
    sU[tid] = U[s * stride + (size_t)m.cell_nodes[cell * 9 + tid / 5] * 5 + tid % 5];
    sUo[tid] = Uold[s * stride + (size_t)m.cell_nodes[cell * 9 + tid / 5] * 5 + tid % 5];
  }
  __syncthreads();
  if (tid < 9) {
    eval_qp(sU, sUo, tid, ihx, ihy, sq[tid]);
    derive(sq[tid], sd[tid]);
  }
  if (tid == 32 && !solid) sAlpha = lps_scale * lps_weight(P, sUo, hx, hy);
  if (OLD && !solid && tid >= 64 && tid < 73) {
    const int i = tid - 64;
    double acc = 0.0;
    for (int j = 0; j < 9; ++j) acc += (hy * ihx * c_lps_ss[i][j] + hx * ihy * c_lps_tt[i][j]) * sU[j * 5 + 4];
    sSp[i] = acc;
  }
  if (OLD && !solid && tid == 96) {
    // alpha = alpha0 h^2 / (rho nu + rho |vbar| h): derivative in the cell mean of v_{n-1}
    double mx = 0.0, my = 0.0, ws = 0.0;
    for (int q = 0; q < 9; ++q) {
      double vx = 0.0, vy = 0.0;
      for (int l = 0; l < 9; ++l) {
        vx += c_phi[q][l] * sUo[l * 5 + 0];
        vy += c_phi[q][l] * sUo[l * 5 + 1];
      }
      mx += c_wq[q] * vx;
      my += c_wq[q] * vy;
      ws += c_wq[q];
    }
    mx /= ws;
    my /= ws;
    const double sp = sqrt(mx * mx + my * my), h = sqrt(hx * hx + hy * hy);
    const double den = P.rho_f * P.nu_f + P.rho_f * sp * h;
    const double f = sp > 0.0 ? -lps_scale * P.alpha0 * h * h * P.rho_f * h / (den * den * sp) : 0.0;
    sDalpha[0] = f * mx;
    sDalpha[1] = f * my;
  }
  __syncthreads();
  for (int t = tid; t < 9 * 15; t += JAC_THREADS) {
    const int q = t / 15, dir = t % 15, cj = dir / 3, b = dir % 3;
    double dv[2] = {0, 0}, du[2] = {0, 0}, dp = 0.0;
    M2 dG = m2(0, 0, 0, 0), dH = m2(0, 0, 0, 0);
    // unit trial direction: value (b = 0) or x / y derivative (b = 1, 2) of component cj
    if (cj < 2) {
      if (b == 0) dv[cj] = 1.0;
      else if (cj == 0) { if (b == 1) dG.a = 1.0; else dG.b = 1.0; }
      else { if (b == 1) dG.c = 1.0; else dG.d = 1.0; }
    } else if (cj < 4) {
      const int c = cj - 2;
      if (b == 0) du[c] = 1.0;
      else if (c == 0) { if (b == 1) dH.a = 1.0; else dH.b = 1.0; }
      else { if (b == 1) dH.c = 1.0; else dH.d = 1.0; }
    } else {
      if (b == 0) dp = 1.0;
    }
    double out[15];
    if (OLD) qp_flux_lin_old(P, sq[q], sd[q], solid, k, theta, dv, dG, du, dH, out);
    else qp_flux_lin(P, sq[q], sd[q], solid, k, theta, dv, dG, du, dH, dp, out);
    for (int r = 0; r < 15; ++r) sD[q][r][dir] = out[r];
  }
  if (outflow) {
    for (int t = tid; t < 3 * 12; t += JAC_THREADS) {
      const int q = t / 12, dir = t % 12, cj = dir / 3, b = dir % 3;
      M2 G, Hu;
      eval_edge_grad(OLD ? sUo : sU, q, ihx, ihy, G, Hu);
      M2 dG = m2(0, 0, 0, 0), dH = m2(0, 0, 0, 0);
      double out[2] = {0, 0};
      if (b > 0) {
        M2& X = cj < 2 ? dG : dH;
        const int c = cj % 2;
        if (c == 0) { if (b == 1) X.a = 1.0; else X.b = 1.0; }
        else { if (b == 1) X.c = 1.0; else X.d = 1.0; }
        if (OLD) edge_flux_lin_old(P, G, Hu, dG, dH, k, theta, out);
        else edge_flux_lin(P, G, Hu, dG, dH, k, theta, out);
      }
      sDe[q][0][dir] = out[0];
      sDe[q][1][dir] = out[1];
    }
  }
  __syncthreads();
}

// TC: type of the B^T D B contraction and of the element matrices (double, or
// float for the FP32 linear solver); the tangent D is always computed in FP64.
template <bool OLD, typename TC = double>
__global__ void __launch_bounds__(JAC_THREADS, 4) k_cell_jacobian(DevMesh m, Phys P, const double* __restrict__ U,
                                                               const double* __restrict__ Uold, size_t stride,
                                                               double k, double theta, double lps_scale,
                                                               const uint8_t* __restrict__ active,
                                                               TC* __restrict__ Ke) {
  const int s = blockIdx.y;
  const int cell = blockIdx.x;
  if (!active[s]) return;
  __shared__ JacTangentShared sh;
  jac_tangent<OLD>(m, P, U, Uold, stride, k, theta, lps_scale, s, cell, sh);
  auto& sD = sh.sD;
  auto& sDe = sh.sDe;
  const double& sAlpha = sh.sAlpha;
  const double* sSp = sh.sSp;
  const double* sDalpha = sh.sDalpha;
  const int tid = threadIdx.x;
  const double hx = m.cell_h[cell * 2], hy = m.cell_h[cell * 2 + 1];
  const double ihx = 1.0 / hx, ihy = 1.0 / hy, area = hx * hy;
  const uint8_t cf = m.cell_flags[cell];
  const bool solid = cf & CF_SOLID;
  const bool outflow = !solid && (cf & CF_OUTFLOW);
  // Two-stage contraction over the field blocks (ci, cj) that the cell's
  // material couples, one quadrature point at a time:
  //   E[(ci,a)][(j,cj)] = w_q sum_b D_q[(ci,a)][(cj,b)] B_b(j,q)
  //   K[(i,ci)][(j,cj)] += sum_a B_a(i,q) E[(ci,a)][(j,cj)]
  // Work items run over the coupled blocks only (81 entries of K, 27 of E per
  // block), so warps carry no structurally zero entries; the remaining blocks
  // are zero or closed-form stabilisation terms, written separately.
  __shared__ TC sE[15][45];
  __shared__ TC sB[3][9];
  __shared__ unsigned char sBlk[25];
  __shared__ int sNb;
  if (tid == 0) {
    int nb = 0;
    for (int b = 0; b < 25; ++b)
      if (OLD ? jac_old_block_nonzero(solid, b / 5, b % 5) : jac_block_nonzero(solid, b / 5, b % 5))
        sBlk[nb++] = (unsigned char)b;
    sNb = nb;
  }
  __syncthreads();
  const int nK = sNb * 81, nE = sNb * 27;
  constexpr int PER = (16 * 81 + JAC_THREADS - 1) / JAC_THREADS;   // at most 16 coupled blocks
  TC acc[PER];
#pragma unroll
  for (int r = 0; r < PER; ++r) acc[r] = 0;
  for (int q = 0; q < 9; ++q) {
    const double wq = c_wq[q] * area;
    if (tid < 9) {
      sB[0][tid] = (TC)c_phi[q][tid];
      sB[1][tid] = (TC)(c_dps[q][tid] * ihx);
      sB[2][tid] = (TC)(c_dpt[q][tid] * ihy);
    }
    for (int f = tid; f < nE; f += JAC_THREADS) {
      const int blk = sBlk[f / 27], r = f % 27, a = r / 9, j = r % 9;
      const int ci = blk / 5, cj = blk % 5;
      const double* Dr = sD[q][ci * 3 + a] + cj * 3;
      sE[ci * 3 + a][j * 5 + cj] =
          (TC)(wq * (Dr[0] * c_phi[q][j] + Dr[1] * (c_dps[q][j] * ihx) + Dr[2] * (c_dpt[q][j] * ihy)));
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      const int e = tid + r * JAC_THREADS;
      if (e < nK) {
        const int blk = sBlk[e / 81], w = e % 81, i = w / 9, j = w % 9;
        const int ci = blk / 5, col = j * 5 + blk % 5;
        acc[r] += sB[0][i] * sE[ci * 3][col] + sB[1][i] * sE[ci * 3 + 1][col] + sB[2][i] * sE[ci * 3 + 2][col];
      }
    }
    __syncthreads();
  }
  TC* out = Ke + ((size_t)s * m.n_cells + cell) * 2025;
  // coupled blocks: the contraction, plus the outflow-edge term of the momentum rows
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    const int e = tid + r * JAC_THREADS;
    if (e >= nK) continue;
    const int blk = sBlk[e / 81], w = e % 81, i = w / 9, j = w % 9;
    const int ci = blk / 5, cj = blk % 5;
    double v = (double)acc[r];
    if (outflow && ci < 2 && cj < 4) {
      for (int q = 0; q < 3; ++q) {
        const double Bj[3] = {c_phie[q][j], c_dpse[q][j] * ihx, c_dpte[q][j] * ihy};
        const double* Drow = sDe[q][ci] + cj * 3;
        v += c_we[q] * hy * c_phie[q][i] * (Drow[0] * Bj[0] + Drow[1] * Bj[1] + Drow[2] * Bj[2]);
      }
    }
    out[(i * 5 + ci) * 45 + j * 5 + cj] = (TC)v;
  }
  // the other blocks: zero, the stabilisation block (fluid p-p), or, for the
  // old state, the derivative of the stabilisation weight (fluid p-v)
  for (int e = tid; e < 2025; e += JAC_THREADS) {
    const int row = e / 45, col = e % 45;
    const int i = row / 5, ci = row % 5, j = col / 5, cj = col % 5;
    if (OLD ? jac_old_block_nonzero(solid, ci, cj) : jac_block_nonzero(solid, ci, cj)) continue;
    double v = 0.0;
    if (!OLD && !solid && ci == 4 && cj == 4)
      v = k * sAlpha * (hy * ihx * c_lps_ss[i][j] + hx * ihy * c_lps_tt[i][j]);
    if (OLD && !solid && ci == 4 && cj < 2) {
      double mj = 0.0, ws = 0.0;   // d vbar / d v_{n-1} at local node j
      for (int q = 0; q < 9; ++q) {
        mj += c_wq[q] * c_phi[q][j];
        ws += c_wq[q];
      }
      v = k * sSp[i] * sDalpha[cj] * (mj / ws);
    }
    out[e] = (TC)v;
  }
}

// Block-sparse assembly: one thread per (slice, block, row component),
// fixed-order sum over the cells sharing both nodes, identity rows replaced.
// identity_value: 1 for dR/dU (identity rows), 0 for dR/dU_old (those rows do
// not depend on the old state).
template <typename T, typename TK = double>
__global__ void k_assemble_bsr(DevMesh m, const TK* __restrict__ Ke, const uint8_t* __restrict__ active,
                               T* __restrict__ A, double identity_value) {
  const int s = blockIdx.y;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || t >= m.nnzb * 5) return;
  const int b = t / 5, ci = t % 5;
  const int i = m.blk_row[b], j = m.colidx[b];
  const uint8_t nf = m.node_flags[i];
  double acc[5] = {0, 0, 0, 0, 0};
  if (is_identity_row(nf, ci)) {
    if (i == j) acc[ci] = identity_value;
  } else {
    for (int e = 0; e < 4; ++e) {
      const int code = m.blk_src[b * 4 + e];
      if (code < 0) break;
      const int cell = code / 81, li = (code / 9) % 9, lj = code % 9;
      if (!row_takes(m.cell_flags[cell], nf, ci)) continue;
      const TK* src = Ke + ((size_t)s * m.n_cells + cell) * 2025 + (li * 5 + ci) * 45 + lj * 5;
      for (int cj = 0; cj < 5; ++cj) acc[cj] += (double)src[cj];
    }
  }
  T* dst = A + ((size_t)s * m.nnzb + b) * 25 + ci * 5;
  for (int cj = 0; cj < 5; ++cj) dst[cj] = (T)acc[cj];
}

// --------------------------------------------------------------------------
// Block-sparse matrix-vector product, y = A x or y = b - A x.
// One thread per (slice, row dof).
// --------------------------------------------------------------------------
// rows: the node rows to compute (m.spmv_rows for all rows, visited in order
// of their block count so that a warp's rows have equal length, or the rows of
// one colour of the multiplicative smoother); the other rows of y are untouched.
template <typename T, bool RESIDUAL>
__global__ void k_bsr_spmv(DevMesh m, const T* __restrict__ A, const T* __restrict__ x,
                           const T* __restrict__ bvec, size_t stride, const uint8_t* __restrict__ active,
                           T* __restrict__ y, const int* __restrict__ rows, int nrows) {
  const int s = blockIdx.y;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || t >= nrows * 5) return;
  const int i = rows[t / 5], c = t % 5;
  const T* As = A + (size_t)s * m.nnzb * 25 + c * 5;
  const T* xs = x + s * stride;
  T acc = 0;
  const int b1 = m.rowptr[i + 1];
  for (int b = m.rowptr[i]; b < b1; ++b) {
    const T* blk = As + (size_t)b * 25;
    const T* xj = xs + (size_t)m.colidx[b] * 5;
    acc = fma(blk[0], xj[0], acc);
    acc = fma(blk[1], xj[1], acc);
    acc = fma(blk[2], xj[2], acc);
    acc = fma(blk[3], xj[3], acc);
    acc = fma(blk[4], xj[4], acc);
  }
  const size_t o = s * stride + (size_t)i * 5 + c;
  y[o] = RESIDUAL ? bvec[o] - acc : acc;
}

// --------------------------------------------------------------------------
// Vanka smoother: local 45 x 45 matrices A restricted to a cell's dofs,
// inverted by Gauss-Jordan with partial pivoting (one CTA per slice-cell),
// stored transposed: inv[s][cell][col][row].
// --------------------------------------------------------------------------
constexpr int VK_THREADS = 128;

template <typename T>
__global__ void __launch_bounds__(VK_THREADS) k_vanka_setup(DevMesh m, const T* __restrict__ A,
                                                            const uint8_t* __restrict__ active,
                                                            T* __restrict__ inv, int* __restrict__ status) {
  const int s = blockIdx.y;
  const int cell = blockIdx.x;
  if (!active[s]) return;
  __shared__ T M[45][46];
  __shared__ T colk[45];
  __shared__ int perm[45];
  __shared__ int piv;
  __shared__ T pinv;
  const int tid = threadIdx.x;
  const T* As = A + (size_t)s * m.nnzb * 25;
  for (int e = tid; e < 2025; e += VK_THREADS) {
    const int r = e / 45, c = e % 45;
    const int blk = m.cell_blk[cell * 81 + (r / 5) * 9 + c / 5];
    M[r][c] = As[(size_t)blk * 25 + (r % 5) * 5 + c % 5];
  }
  if (tid < 45) perm[tid] = tid;
  __syncthreads();
  // in-place Gauss-Jordan with partial (row) pivoting
  for (int kk = 0; kk < 45; ++kk) {
    if (tid < 32) {
      T best = -1;
      int bi = kk;
      for (int r = kk + tid; r < 45; r += 32) {
        const T a = fabs(M[r][kk]);
        if (a > best) { best = a; bi = r; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const T ob = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (tid == 0) {
        piv = (best > 0) ? bi : -1;
        if (best > 0 && bi != kk) { const int t = perm[kk]; perm[kk] = perm[bi]; perm[bi] = t; }
      }
    }
    __syncthreads();
    const int p = piv;
    if (p < 0) {
      if (tid == 0) status[s] = -6;
      return;
    }
    if (p != kk)
      for (int c = tid; c < 45; c += VK_THREADS) { const T t = M[kk][c]; M[kk][c] = M[p][c]; M[p][c] = t; }
    __syncthreads();
    if (tid == 0) pinv = T(1) / M[kk][kk];
    __syncthreads();
    const T d = pinv;
    for (int c = tid; c < 45; c += VK_THREADS) M[kk][c] = (c == kk) ? d : M[kk][c] * d;
    for (int r = tid; r < 45; r += VK_THREADS) colk[r] = (r == kk) ? T(0) : M[r][kk];
    __syncthreads();
    for (int e = tid; e < 2025; e += VK_THREADS) {
      const int r = e / 45, c = e % 45;
      if (r == kk) continue;
      const T f = colk[r];
      M[r][c] = (c == kk) ? -f * d : M[r][c] - f * M[kk][c];
    }
    __syncthreads();
  }
  // A^{-1}[r][perm[c]] = M[r][c]; stored transposed: inv[col][row]
  T* dst = inv + ((size_t)s * m.n_cells + cell) * 2025;
  for (int e = tid; e < 2025; e += VK_THREADS) {
    const int r = e / 45, c = e % 45;
    dst[perm[c] * 45 + r] = M[r][c];
  }
}

// z_cell = inv_cell * r_cell: one thread per (slice, cell, local row).
// cells: optional list of cells (one colour of the multiplicative smoother).
template <typename T>
__global__ void k_vanka_cell(DevMesh m, const T* __restrict__ inv, const T* __restrict__ r, size_t stride,
                             const uint8_t* __restrict__ active, T* __restrict__ cellbuf,
                             const int* __restrict__ cells, int ncells) {
  const int s = blockIdx.y;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || t >= ncells * 45) return;
  const int cell = cells ? cells[t / 45] : t / 45, row = t % 45;
  const T* Mi = inv + ((size_t)s * m.n_cells + cell) * 2025;
  const T* rs = r + s * stride;
  T acc = 0;
  for (int l = 0; l < 9; ++l) {
    const T* rl = rs + (size_t)m.cell_nodes[cell * 9 + l] * 5;
    for (int c = 0; c < 5; ++c) acc += Mi[(l * 5 + c) * 45 + row] * rl[c];
  }
  cellbuf[((size_t)s * m.n_cells + cell) * 45 + row] = acc;
}

// x += omega * (sum over the node's cells of z) / (number of cells).
// Vanka apply using the block structure of the local inverse: in cells
// flagged CF_U_DECOUPLED the displacement rows of the local matrix couple only
// to their own displacement component, so the displacement rows of the inverse
// vanish outside that 9 x 9 block and take 9 products instead of 45. A CTA
// takes VKS_CELLS cells: threads [0, 27 VKS_CELLS) the velocity and pressure
// rows, the rest the displacement rows, so that all warps but one do the same
// work. The cells' residual values are staged in shared memory.
constexpr int VKS_CELLS = 8;
constexpr int VKS_THREADS = 45 * VKS_CELLS;

template <typename T>
__global__ void __launch_bounds__(VKS_THREADS) k_vanka_cell_split(DevMesh m, const T* __restrict__ inv,
                                                                  const T* __restrict__ r, size_t stride,
                                                                  const uint8_t* __restrict__ active,
                                                                  T* __restrict__ cellbuf,
                                                                  const int* __restrict__ cells, int ncells) {
  const int s = blockIdx.y;
  if (!active[s]) return;
  const int c0 = blockIdx.x * VKS_CELLS;
  __shared__ T sr[VKS_CELLS][45];
  const int tid = threadIdx.x;
  const T* rs = r + s * stride;
  for (int e = tid; e < VKS_CELLS * 45; e += VKS_THREADS) {
    const int k = e / 45, col = e % 45;
    if (c0 + k < ncells) {
      const int cell = cells ? cells[c0 + k] : c0 + k;
      sr[k][col] = rs[(size_t)m.cell_nodes[cell * 9 + col / 5] * 5 + col % 5];
    }
  }
  __syncthreads();
  int k, row;
  bool urow;
  if (tid < 27 * VKS_CELLS) {   // velocity and pressure rows: components 0, 1, 4 of node f / 3
    k = tid / 27;
    const int f = tid % 27, c = f % 3;
    row = (f / 3) * 5 + (c == 2 ? 4 : c);
    urow = false;
  } else {                      // displacement rows: components 2, 3 of node g / 2
    const int u = tid - 27 * VKS_CELLS;
    k = u / 18;
    const int g = u % 18;
    row = (g / 2) * 5 + 2 + g % 2;
    urow = true;
  }
  if (c0 + k >= ncells) return;
  const int cell = cells ? cells[c0 + k] : c0 + k;
  const T* Mi = inv + ((size_t)s * m.n_cells + cell) * 2025;
  T acc = 0;
  if (urow && (m.cell_flags[cell] & CF_U_DECOUPLED)) {
    const int comp = row % 5;
    for (int l = 0; l < 9; ++l) acc += Mi[(l * 5 + comp) * 45 + row] * sr[k][l * 5 + comp];
  } else {
    for (int col = 0; col < 45; ++col) acc += Mi[col * 45 + row] * sr[k][col];
  }
  cellbuf[((size_t)s * m.n_cells + cell) * 45 + row] = acc;
}

template <typename T>
__global__ void k_vanka_gather(DevMesh m, const T* __restrict__ cellbuf, double omega, size_t stride,
                               const uint8_t* __restrict__ active, T* __restrict__ x) {
  const int s = blockIdx.y;
  const int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || node >= m.n_nodes) return;
  T acc[5] = {0, 0, 0, 0, 0};
  int cnt = 0;
  for (int e = 0; e < 4; ++e) {
    const int code = m.node_cells[node * 4 + e];
    if (code < 0) break;
    const T* src = cellbuf + ((size_t)s * m.n_cells + code / 9) * 45 + (code % 9) * 5;
    for (int c = 0; c < 5; ++c) acc[c] += src[c];
    ++cnt;
  }
  const T w = T(omega / cnt);
  T* xs = x + s * stride + (size_t)node * 5;
  for (int c = 0; c < 5; ++c) xs[c] += w * acc[c];
}

// Multiplicative (coloured) Vanka: cells of one colour share no node, so each
// node of the colour takes the correction of its one cell: x += omega z.
template <typename T>
__global__ void k_vanka_scatter(int n_cells, const int* __restrict__ nodes, const int* __restrict__ src, int nnodes,
                                const T* __restrict__ cellbuf, double omega, size_t stride,
                                const uint8_t* __restrict__ active, T* __restrict__ x) {
  const int s = blockIdx.y;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || t >= nnodes * 5) return;
  const int k = t / 5, c = t % 5;
  const int code = src[k];
  x[s * stride + (size_t)nodes[k] * 5 + c] += (T)omega * cellbuf[((size_t)s * n_cells + code / 9) * 45 + (code % 9) * 5 + c];
}

// --------------------------------------------------------------------------
// Multigrid transfers (tensor products of 1D Q2 interpolation tables).
// --------------------------------------------------------------------------
struct Transfer {
  int nnx_f, nny_f, nnx_c, nny_c;
  const int* px_idx;  const double* px_w;   // [nnx_f][3] coarse index / weight (-1 pad)
  const int* py_idx;  const double* py_w;   // [nny_f][3]
  const int* rx_idx;  const double* rx_w;   // [nnx_c][7] fine index / weight (-1 pad)
  const int* ry_idx;  const double* ry_w;   // [nny_c][7]
  const int* ix_idx;  const double* ix_w;   // [nnx_c][3] fine index / weight: fine field at coarse nodes
  const int* iy_idx;  const double* iy_w;   // [nny_c][3]
};

__device__ inline bool is_free(uint8_t nf, int c) { return !is_identity_row(nf, c); }

template <typename V>
__global__ void k_restrict(Transfer T, const uint8_t* __restrict__ nflags_f, const uint8_t* __restrict__ nflags_c,
                           const V* __restrict__ rf, size_t stride_f, size_t stride_c,
                           const uint8_t* __restrict__ active, V* __restrict__ rc) {
  const int s = blockIdx.y;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int n_c = T.nnx_c * T.nny_c;
  if (!active[s] || t >= n_c * 5) return;
  const int node = t / 5, c = t % 5;
  const int I = node % T.nnx_c, Jy = node / T.nnx_c;
  V acc = 0;
  if (is_free(nflags_c[node], c)) {
    const V* r = rf + s * stride_f;
    for (int ey = 0; ey < 7; ++ey) {
      const int j = T.ry_idx[Jy * 7 + ey];
      if (j < 0) break;
      const V wy = (V)T.ry_w[Jy * 7 + ey];
      for (int ex = 0; ex < 7; ++ex) {
        const int i = T.rx_idx[I * 7 + ex];
        if (i < 0) break;
        const int fn = j * T.nnx_f + i;
        if (is_free(nflags_f[fn], c)) acc += wy * (V)T.rx_w[I * 7 + ex] * r[(size_t)fn * 5 + c];
      }
    }
  }
  rc[s * stride_c + t] = acc;
}

template <typename V>
__global__ void k_prolong_add(Transfer T, const uint8_t* __restrict__ nflags_f, const V* __restrict__ xc,
                              size_t stride_f, size_t stride_c, const uint8_t* __restrict__ active,
                              V* __restrict__ xf) {
  const int s = blockIdx.y;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int n_f = T.nnx_f * T.nny_f;
  if (!active[s] || t >= n_f * 5) return;
  const int node = t / 5, c = t % 5;
  if (!is_free(nflags_f[node], c)) return;
  const int i = node % T.nnx_f, j = node / T.nnx_f;
  const V* x = xc + s * stride_c;
  V acc = 0;
  for (int ey = 0; ey < 3; ++ey) {
    const int J = T.py_idx[j * 3 + ey];
    if (J < 0) break;
    const V wy = (V)T.py_w[j * 3 + ey];
    for (int ex = 0; ex < 3; ++ex) {
      const int I = T.px_idx[i * 3 + ex];
      if (I < 0) break;
      acc += wy * (V)T.px_w[i * 3 + ex] * x[((size_t)J * T.nnx_c + I) * 5 + c];
    }
  }
  xf[s * stride_f + t] += acc;
}

// Coarse-level state: the fine Q2 field evaluated at the coarse nodes (the
// coarsened meshes need not be nested when a segment has an odd cell count).
__global__ void k_interp_state(Transfer T, const double* __restrict__ Uf, size_t stride_f, size_t stride_c,
                               const uint8_t* __restrict__ active, double* __restrict__ Uc) {
  const int s = blockIdx.y;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || t >= T.nnx_c * T.nny_c * 5) return;
  const int node = t / 5, c = t % 5;
  const int I = node % T.nnx_c, J = node / T.nnx_c;
  const double* u = Uf + s * stride_f;
  double acc = 0.0;
  for (int ey = 0; ey < 3; ++ey) {
    const int j = T.iy_idx[J * 3 + ey];
    if (j < 0) break;
    for (int ex = 0; ex < 3; ++ex) {
      const int i = T.ix_idx[I * 3 + ex];
      if (i < 0) break;
      acc += T.iy_w[J * 3 + ey] * T.ix_w[I * 3 + ex] * u[((size_t)j * T.nnx_f + i) * 5 + c];
    }
  }
  Uc[s * stride_c + t] = acc;
}

// --------------------------------------------------------------------------
// Coarsest level: dense matrix, Gauss-Jordan inverse (one CTA per slice),
// stored transposed, and its product.
// --------------------------------------------------------------------------
template <typename T>
__global__ void k_dense_from_bsr(DevMesh m, const T* __restrict__ A, const uint8_t* __restrict__ active,
                                 T* __restrict__ D) {
  const int s = blockIdx.y;
  const int n = m.n_nodes * 5;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || t >= n * n) return;
  const int r = t / n, c = t % n;
  const int i = r / 5, j = c / 5;
  T v = 0;
  for (int b = m.rowptr[i]; b < m.rowptr[i + 1]; ++b)
    if (m.colidx[b] == j) { v = A[((size_t)s * m.nnzb + b) * 25 + (r % 5) * 5 + c % 5]; break; }
  D[(size_t)s * n * n + t] = v;
}

constexpr int GJ_THREADS = 1024;

// In-place Gauss-Jordan inversion with partial pivoting of D[s] (n x n,
// row-major); the inverse is written transposed to inv[s].
// The same in-place Gauss-Jordan inversion on a thread-block cluster of
// GJC_CTAS CTAs per slice: CTA c keeps rows [c rows_per, (c + 1) rows_per) in
// shared memory; per pivot step the CTAs agree on the pivot (local maxima
// exchanged through distributed shared memory), every CTA copies the pivot row
// from its owner, the two rows are swapped, and each CTA eliminates its own
// rows. Pivot choice, scaling and elimination are those of k_dense_invert, so
// both kernels give the same inverse. Two cluster barriers per step; every
// CTA of a cluster takes the same branches, so all reach every barrier.
constexpr int GJC_CTAS = 8;
constexpr int GJC_THREADS = 256;

template <typename T>
__host__ __device__ inline size_t gjc_smem_bytes(int n) {
  const int rows_per = (n + GJC_CTAS - 1) / GJC_CTAS;
  return ((size_t)rows_per * n + 2 * (size_t)n + 2) * sizeof(T) + ((size_t)n + 2) * sizeof(int);
}

template <typename T>
__global__ void __launch_bounds__(GJC_THREADS) k_dense_invert_cluster(int n, const T* __restrict__ D,
                                                                      const uint8_t* __restrict__ active,
                                                                      T* __restrict__ inv, int* __restrict__ status) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int s = blockIdx.y;
  if (!active[s]) return;   // uniform over the cluster (one slice per cluster)
  const int rank = (int)cluster.block_rank();
  const int rows_per = (n + GJC_CTAS - 1) / GJC_CTAS;
  const int r0 = rank * rows_per, r1 = min(n, r0 + rows_per);
  extern __shared__ __align__(16) unsigned char gjc_raw[];
  T* rows = reinterpret_cast<T*>(gjc_raw);     // [rows_per][n], local row r - r0
  T* prow = rows + (size_t)rows_per * n;       // [n] pivot row (copy)
  T* tmp = prow + n;                           // [n] row kk, moving to row p
  T* cand_v = tmp + n;                         // [1] local pivot candidate
  int* cand_i = reinterpret_cast<int*>(cand_v + 2);   // [1]
  int* pr = cand_i + 2;                        // [n] row permutation
  __shared__ T red_v[GJC_THREADS / 32];
  __shared__ int red_i[GJC_THREADS / 32];
  const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
  const T* Ms = D + (size_t)s * n * n;
  for (int e = tid; e < (r1 - r0) * n; e += GJC_THREADS) rows[e] = Ms[(size_t)r0 * n + e];
  for (int r = tid; r < n; r += GJC_THREADS) pr[r] = r;
  __syncthreads();
  for (int kk = 0; kk < n; ++kk) {
    // local candidate among rows >= kk
    T best = -1;
    int bi = n;
    for (int r = max(kk, r0) + tid; r < r1; r += GJC_THREADS) {
      const T a = fabs(rows[(size_t)(r - r0) * n + kk]);
      if (a > best) { best = a; bi = r; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const T ob = __shfl_down_sync(0xffffffffu, best, o);
      const int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { red_v[warp] = best; red_i[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      T b = red_v[0];
      int ii = red_i[0];
      for (int w = 1; w < GJC_THREADS / 32; ++w)
        if (red_v[w] > b || (red_v[w] == b && red_i[w] < ii)) { b = red_v[w]; ii = red_i[w]; }
      cand_v[0] = b;
      cand_i[0] = ii;
    }
    cluster.sync();   // S1: candidates published; the previous step's writes are complete
    // the pivot: largest candidate, ties to the lowest row (computed alike in every CTA)
    T b = -1;
    int p = n;
    for (int c = 0; c < GJC_CTAS; ++c) {
      const T v = *cluster.map_shared_rank(cand_v, c);
      const int i = *cluster.map_shared_rank(cand_i, c);
      if (v > b || (v == b && i < p)) { b = v; p = i; }
    }
    if (!(b > 0)) {   // singular (same decision in every CTA)
      if (rank == 0 && tid == 0) status[s] = -6;
      cluster.sync();   // the candidates may still be read remotely
      return;
    }
    const int op = p / rows_per, ok = kk / rows_per;
    const T* rp = cluster.map_shared_rank(rows, op) + (size_t)(p - op * rows_per) * n;
    for (int c = tid; c < n; c += GJC_THREADS) prow[c] = rp[c];
    if (p != kk && rank == op) {   // the owner of row p takes row kk's content
      const T* rk = cluster.map_shared_rank(rows, ok) + (size_t)(kk - ok * rows_per) * n;
      for (int c = tid; c < n; c += GJC_THREADS) tmp[c] = rk[c];
    }
    if (p != kk && tid == 0) { const int t1 = pr[kk]; pr[kk] = pr[p]; pr[p] = t1; }
    cluster.sync();   // S2: every remote read of this step is done
    const T d = T(1) / prow[kk];
    __syncthreads();
    for (int c = tid; c < n; c += GJC_THREADS) prow[c] = (c == kk) ? d : prow[c] * d;
    if (p != kk && rank == op)
      for (int c = tid; c < n; c += GJC_THREADS) rows[(size_t)(p - r0) * n + c] = tmp[c];
    __syncthreads();
    if (rank == ok)
      for (int c = tid; c < n; c += GJC_THREADS) rows[(size_t)(kk - r0) * n + c] = prow[c];
    // eliminate column kk from every other local row, one warp per row (every
    // lane reads the row's factor before any lane overwrites column kk)
    for (int lr = warp; lr < r1 - r0; lr += GJC_THREADS / 32) {
      if (lr + r0 == kk) continue;
      T* row = rows + (size_t)lr * n;
      const T f = row[kk];
      __syncwarp();
      for (int c = lane; c < n; c += 32) row[c] = (c == kk) ? -f * d : row[c] - f * prow[c];
    }
    __syncthreads();
  }
  // undo the row permutation on the columns: inv[:, pr[c]] = M[:, c] (row-major)
  T* out = inv + (size_t)s * n * n;
  for (int e = tid; e < (r1 - r0) * n; e += GJC_THREADS) {
    const int lr = e / n, c = e % n;
    out[(size_t)(lr + r0) * n + pr[c]] = rows[e];
  }
  cluster.sync();   // no CTA leaves while another may still read its shared memory
}

template <typename T>
__global__ void __launch_bounds__(GJ_THREADS) k_dense_invert(int n, T* __restrict__ D, int* __restrict__ perm,
                                                             const uint8_t* __restrict__ active,
                                                             T* __restrict__ inv, int* __restrict__ status) {
  const int s = blockIdx.x;
  if (!active[s]) return;
  T* M = D + (size_t)s * n * n;
  int* pr = perm + (size_t)s * n;
  __shared__ T red_v[GJ_THREADS / 32];
  __shared__ int red_i[GJ_THREADS / 32];
  __shared__ int piv;
  __shared__ T pinv;
  extern __shared__ unsigned char colk_raw[];
  T* colk = reinterpret_cast<T*>(colk_raw);   // [n]
  const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
  for (int r = tid; r < n; r += GJ_THREADS) pr[r] = r;
  __syncthreads();
  for (int kk = 0; kk < n; ++kk) {
    T best = -1;
    int bi = kk;
    for (int r = kk + tid; r < n; r += GJ_THREADS) {
      const T a = fabs(M[(size_t)r * n + kk]);
      if (a > best) { best = a; bi = r; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const T ob = __shfl_down_sync(0xffffffffu, best, o);
      const int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { red_v[warp] = best; red_i[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      T b = red_v[0];
      int ii = red_i[0];
      for (int w = 1; w < GJ_THREADS / 32; ++w)
        if (red_v[w] > b || (red_v[w] == b && red_i[w] < ii)) { b = red_v[w]; ii = red_i[w]; }
      piv = (b > 0) ? ii : -1;
    }
    __syncthreads();
    const int p = piv;
    if (p < 0) {
      if (tid == 0) status[s] = -6;
      return;
    }
    if (p != kk) {
      for (int c = tid; c < n; c += GJ_THREADS) {
        const T t0 = M[(size_t)kk * n + c];
        M[(size_t)kk * n + c] = M[(size_t)p * n + c];
        M[(size_t)p * n + c] = t0;
      }
      if (tid == 0) { const int t1 = pr[kk]; pr[kk] = pr[p]; pr[p] = t1; }
    }
    __syncthreads();
    if (tid == 0) pinv = T(1) / M[(size_t)kk * n + kk];
    __syncthreads();
    const T d = pinv;
    // in-place Gauss-Jordan: column kk becomes the kk-th column of the inverse
    for (int c = tid; c < n; c += GJ_THREADS) M[(size_t)kk * n + c] = (c == kk) ? d : M[(size_t)kk * n + c] * d;
    for (int r = tid; r < n; r += GJ_THREADS) colk[r] = (r == kk) ? T(0) : M[(size_t)r * n + kk];
    __syncthreads();
    for (int e = tid; e < n * n; e += GJ_THREADS) {
      const int r = e / n, c = e % n;
      if (r == kk) continue;
      const T f = colk[r];
      if (c == kk) M[e] = -f * d;
      else M[e] -= f * M[(size_t)kk * n + c];
    }
    __syncthreads();
  }
  // undo the row permutation on the columns: inv[:, pr[c]] = M[:, c] (row-major)
  T* out = inv + (size_t)s * n * n;
  for (int e = tid; e < n * n; e += GJ_THREADS) {
    const int r = e / n, c = e % n;
    out[(size_t)r * n + pr[c]] = M[e];
  }
}

// y = inv x: one warp per (slice, row), lanes split the row.
template <typename T>
__global__ void k_dense_apply(int n, const T* __restrict__ inv, const T* __restrict__ x, size_t stride,
                              const uint8_t* __restrict__ active, T* __restrict__ y) {
  const int s = blockIdx.y;
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x % 32;
  if (!active[s] || r >= n) return;
  const T* M = inv + (size_t)s * n * n + (size_t)r * n;
  const T* xs = x + s * stride;
  T acc = 0;
  for (int c = lane; c < n; c += 32) acc = fma(M[c], xs[c], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) y[s * stride + r] = acc;
}

// --------------------------------------------------------------------------
// Discrete adjoint helpers.
// --------------------------------------------------------------------------
// Block transpose: At[bt[b]] = A[b]^T (the block pattern is symmetric).
__global__ void k_bsr_transpose(int nnzb, const int* __restrict__ bt, const double* __restrict__ A,
                                const uint8_t* __restrict__ active, double* __restrict__ At) {
  const int s = blockIdx.y;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || t >= nnzb * 25) return;
  const int b = t / 25, r = (t % 25) / 5, c = t % 5;
  At[((size_t)s * nnzb + bt[b]) * 25 + c * 5 + r] = A[((size_t)s * nnzb + b) * 25 + r * 5 + c];
}

// Cell contributions of dR/dmu_s (which = 0) or dR/dlambda_s (which = 1):
// k theta dP(F_n) + k (1 - theta) dP(F_{n-1}) tested with grad phi, solid cells.
__global__ void k_cell_dres_dlame(DevMesh m, const double* __restrict__ U, const double* __restrict__ Uold,
                                  size_t stride, double k, double theta, int which,
                                  const uint8_t* __restrict__ active, double* __restrict__ cellbuf) {
  const int s = blockIdx.y;
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || cell >= m.n_cells) return;
  double* out = cellbuf + ((size_t)s * m.n_cells + cell) * 45;
  for (int i = 0; i < 45; ++i) out[i] = 0.0;
  if (!(m.cell_flags[cell] & CF_SOLID)) return;
  double Ue[45], Uo[45];
  load_cell(m, U + s * stride, cell, Ue);
  load_cell(m, Uold + s * stride, cell, Uo);
  const double hx = m.cell_h[cell * 2], hy = m.cell_h[cell * 2 + 1];
  const double ihx = 1.0 / hx, ihy = 1.0 / hy, area = hx * hy;
  for (int q = 0; q < 9; ++q) {
    QpIn st;
    eval_qp(Ue, Uo, q, ihx, ihy, st);
    const M2 F = eye2() + st.Hu, Fo = eye2() + st.Huo;
    const M2 S = which == 0 ? (k * theta) * dpiola_dmu(F) + (k * (1.0 - theta)) * dpiola_dmu(Fo)
                            : (k * theta) * dpiola_dlambda(F) + (k * (1.0 - theta)) * dpiola_dlambda(Fo);
    const double w = c_wq[q] * area;
    for (int l = 0; l < 9; ++l) {
      const double b1 = w * c_dps[q][l] * ihx, b2 = w * c_dpt[q][l] * ihy;
      out[l * 5 + 0] += b1 * S.a + b2 * S.b;
      out[l * 5 + 1] += b1 * S.c + b2 * S.d;
    }
  }
}

// Node gather of cell contributions with the residual's row selection and
// zero on identity rows (derivatives of rows that do not depend on the input).
__global__ void k_gather_vector(DevMesh m, const double* __restrict__ cellbuf, size_t stride,
                                const uint8_t* __restrict__ active, double* __restrict__ R) {
  const int s = blockIdx.y;
  const int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || node >= m.n_nodes) return;
  const uint8_t nf = m.node_flags[node];
  double acc[5] = {0, 0, 0, 0, 0};
  for (int e = 0; e < 4; ++e) {
    const int code = m.node_cells[node * 4 + e];
    if (code < 0) break;
    const int cell = code / 9, l = code % 9;
    const double* src = cellbuf + ((size_t)s * m.n_cells + cell) * 45 + l * 5;
    for (int c = 0; c < 5; ++c)
      if (row_takes(m.cell_flags[cell], nf, c)) acc[c] += src[c];
  }
  for (int c = 0; c < 5; ++c) R[s * stride + (size_t)node * 5 + c] = is_identity_row(nf, c) ? 0.0 : acc[c];
}

// dR/dvbar: the inflow rows carry U - g(t), g proportional to vbar.
__global__ void k_dres_dvbar(DevMesh m, Phys P, const double* __restrict__ t, size_t stride,
                             const uint8_t* __restrict__ active, double* __restrict__ R) {
  const int s = blockIdx.y;
  const int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || node >= m.n_nodes) return;
  const uint8_t nf = m.node_flags[node];
  for (int c = 0; c < 5; ++c) {
    double v = 0.0;
    if (c == 0 && P.vbar != 0.0) v = -dirichlet_value(P, nf, m.node_y[node], 0, t[s]) / P.vbar;
    R[s * stride + (size_t)node * 5 + c] = v;
  }
}

// --------------------------------------------------------------------------
// Vector kernels for FGMRES and Newton (per slice, fixed reduction order).
// --------------------------------------------------------------------------
constexpr int RED_THREADS = 256;
constexpr int RED_CHUNK = 1024;   // rows per block: the partition depends on n only

// partial[s][blk][i] = sum over this block's rows of V[s][i][row] * w[s][row], i < nv.
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_dots_partial(int n, int nv, const T* __restrict__ V,
                                                              size_t vstride, size_t vslice,
                                                              const T* __restrict__ w, size_t wstride,
                                                              const uint8_t* __restrict__ active,
                                                              double* __restrict__ partial, int max_nv) {
  const int s = blockIdx.y;
  if (!active[s]) return;
  __shared__ double red[RED_THREADS / 32][64];
  const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
  const int r0 = blockIdx.x * RED_CHUNK;
  const int r1 = min(n, r0 + RED_CHUNK);
  const T* Vs = V + s * vslice;
  const T* ws = w + s * wstride;
  for (int i = 0; i < nv; ++i) {
    T acc = 0;
    const T* vi = Vs + i * vstride;
    for (int r = r0 + tid; r < r1; r += RED_THREADS) acc += vi[r] * ws[r];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) red[warp][i] = (double)acc;
  }
  __syncthreads();
  for (int i = tid; i < nv; i += RED_THREADS) {
    double acc = 0.0;
    for (int wv = 0; wv < RED_THREADS / 32; ++wv) acc += red[wv][i];
    partial[((size_t)s * gridDim.x + blockIdx.x) * max_nv + i] = acc;
  }
}

// out[s][i] = sum_blk partial[s][blk][i] (fixed order); optional sqrt.
__global__ void k_dots_finish(int nblk, int nv, const double* __restrict__ partial, int max_nv,
                              const uint8_t* __restrict__ active, double* __restrict__ out, int out_stride,
                              bool take_sqrt, bool accumulate) {
  const int s = blockIdx.x;
  const int i = threadIdx.x;
  if (!active[s] || i >= nv) return;
  double acc = 0.0;
  for (int b = 0; b < nblk; ++b) acc += partial[((size_t)s * nblk + b) * max_nv + i];
  if (take_sqrt) acc = sqrt(acc);
  if (accumulate) out[s * out_stride + i] += acc;
  else out[s * out_stride + i] = acc;
}

// w[s] -= sum_{i < nv} h[s][i] V[s][i]
template <typename T>
__global__ void k_sub_basis(int n, int nv, const T* __restrict__ V, size_t vstride, size_t vslice,
                            const double* __restrict__ h, int hstride, const uint8_t* __restrict__ active,
                            T* __restrict__ w, size_t wstride) {
  const int s = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || r >= n) return;
  const T* Vs = V + s * vslice;
  T acc = w[s * wstride + r];
  for (int i = 0; i < nv; ++i) acc -= (T)h[s * hstride + i] * Vs[i * vstride + r];
  w[s * wstride + r] = acc;
}

// y[s] = x[s] * scale[s] (scale = 1 / norm), or y = a * x when inv = false.
template <typename T>
__global__ void k_scale(int n, const T* __restrict__ x, size_t xstride, const double* __restrict__ sc, int sstride,
                        bool invert, const uint8_t* __restrict__ active, T* __restrict__ y, size_t ystride) {
  const int s = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || r >= n) return;
  const T a = (T)(invert ? 1.0 / sc[s * sstride] : sc[s * sstride]);
  y[s * ystride + r] = a * x[s * xstride + r];
}

// x[s] += sum_{i < nv[s]} y[s][i] Z[s][i]
template <typename T>
__global__ void k_add_basis(int n, const int* __restrict__ nv, const T* __restrict__ Z, size_t zstride,
                            size_t zslice, const double* __restrict__ y, int ystride,
                            const uint8_t* __restrict__ active, T* __restrict__ x, size_t xstride) {
  const int s = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || r >= n) return;
  const T* Zs = Z + s * zslice;
  T acc = x[s * xstride + r];
  for (int i = 0; i < nv[s]; ++i) acc += (T)y[s * ystride + i] * Zs[i * zstride + r];
  x[s * xstride + r] = acc;
}

// Arnoldi step j of FGMRES for each active slice (one thread per slice):
// store column j of the Hessenberg matrix, apply the previous Givens
// rotations, form a new one and update the residual estimate |g[j+1]|.
__global__ void k_givens(int S, int j, int m, const double* __restrict__ hcol, int hstride,
                         const double* __restrict__ hnorm, const uint8_t* __restrict__ active,
                         double* __restrict__ H, double* __restrict__ cs, double* __restrict__ sn,
                         double* __restrict__ g, double* __restrict__ resid) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S || !active[s]) return;
  double* Hs = H + (size_t)s * (m + 1) * m;
  for (int i = 0; i <= j; ++i) Hs[i * m + j] = hcol[s * hstride + i];
  Hs[(j + 1) * m + j] = hnorm[s];
  double* c = cs + (size_t)s * m;
  double* sv = sn + (size_t)s * m;
  for (int i = 0; i < j; ++i) {
    const double a = Hs[i * m + j], b = Hs[(i + 1) * m + j];
    Hs[i * m + j] = c[i] * a + sv[i] * b;
    Hs[(i + 1) * m + j] = -sv[i] * a + c[i] * b;
  }
  const double a = Hs[j * m + j], b = Hs[(j + 1) * m + j];
  const double r = hypot(a, b);
  const double cj = (r > 0.0) ? a / r : 1.0, sj = (r > 0.0) ? b / r : 0.0;
  c[j] = cj;
  sv[j] = sj;
  Hs[j * m + j] = r;
  Hs[(j + 1) * m + j] = 0.0;
  double* gs = g + (size_t)s * (m + 1);
  gs[j + 1] = -sj * gs[j];
  gs[j] = cj * gs[j];
  resid[s] = fabs(gs[j + 1]);
}

// Solve the triangular system H y = g of size nv[s] (one thread per slice).
__global__ void k_backsolve(int S, int m, const int* __restrict__ nv, const double* __restrict__ H,
                            const double* __restrict__ g, const uint8_t* __restrict__ active, double* __restrict__ y) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S || !active[s]) return;
  const int n = nv[s];
  const double* Hs = H + (size_t)s * (m + 1) * m;
  const double* gs = g + (size_t)s * (m + 1);
  double* ys = y + (size_t)s * m;
  for (int i = n - 1; i >= 0; --i) {
    double acc = gs[i];
    for (int k = i + 1; k < n; ++k) acc -= Hs[i * m + k] * ys[k];
    ys[i] = acc / Hs[i * m + i];
  }
}

// Start a restart cycle: g = (beta, 0, ...), V0 = r / beta.
__global__ void k_init_g(int S, int m, const double* __restrict__ beta, const uint8_t* __restrict__ active,
                         double* __restrict__ g) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S || !active[s]) return;
  double* gs = g + (size_t)s * (m + 1);
  gs[0] = beta[s];
  for (int i = 1; i <= m; ++i) gs[i] = 0.0;
}

// y = a x + b y, masked per slice.
template <typename TX, typename TY>
__global__ void k_axpby(int n, double a, const TX* __restrict__ x, size_t xstride, double b,
                        const uint8_t* __restrict__ active, TY* __restrict__ y, size_t ystride) {
  const int s = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || r >= n) return;
  if (b == 0.0) y[s * ystride + r] = (TY)(a * (double)x[s * xstride + r]);
  else y[s * ystride + r] = (TY)(a * (double)x[s * xstride + r] + b * (double)y[s * ystride + r]);
}

template <typename T>
__global__ void k_fill(int n, double v, const uint8_t* __restrict__ active, T* __restrict__ y, size_t ystride) {
  const int s = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || r >= n) return;
  y[s * ystride + r] = (T)v;
}

// Parareal correction U_next = F + (C_new - C_old) (this order, Sec. 3), with
// per-field partial sums of the squared increment and of the new state.
__global__ void __launch_bounds__(RED_THREADS) k_parareal_correct(int n, const double* __restrict__ Fv,
                                                                  const double* __restrict__ Cnew,
                                                                  const double* __restrict__ Cold,
                                                                  double* __restrict__ Unext,
                                                                  double* __restrict__ partial) {
  __shared__ double red[RED_THREADS / 32][6];
  const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
  double a[6] = {0, 0, 0, 0, 0, 0};   // |dv|^2, |du|^2, |dp|^2, |v|^2, |u|^2, |p|^2
  for (int r = blockIdx.x * blockDim.x + tid; r < n; r += gridDim.x * blockDim.x) {
    const double un = Fv[r] + (Cnew[r] - Cold[r]);
    const double d = un - Unext[r];
    const int c = r % 5;
    const int f = c < 2 ? 0 : (c < 4 ? 1 : 2);
    a[f] += d * d;
    a[3 + f] += un * un;
    Unext[r] = un;
  }
  for (int i = 0; i < 6; ++i) {
    double v = a[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][i] = v;
  }
  __syncthreads();
  if (tid < 6) {
    double v = 0.0;
    for (int w = 0; w < RED_THREADS / 32; ++w) v += red[w][tid];
    partial[blockIdx.x * 6 + tid] = v;
  }
}

// FP64 FMA throughput probe (the denominator of the FP64 rooflines, measured
// on the device in use): every thread runs eight independent FMA chains of
// `iters` steps, 16 * iters flops per thread. The result is written only when
// it equals a value no input produces, so the chains cannot be optimised away.
constexpr int FMA_PROBE_THREADS = 256;
__global__ void __launch_bounds__(FMA_PROBE_THREADS) k_fma_probe(int iters, double seed, double* sink) {
  const double m = 1.0 + 1e-15, b = 1e-17;
  double a0 = seed + threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6,
         a7 = a0 + 7;
#pragma unroll 8
  for (int i = 0; i < iters; ++i) {
    a0 = fma(a0, m, b);
    a1 = fma(a1, m, b);
    a2 = fma(a2, m, b);
    a3 = fma(a3, m, b);
    a4 = fma(a4, m, b);
    a5 = fma(a5, m, b);
    a6 = fma(a6, m, b);
    a7 = fma(a7, m, b);
  }
  const double sum = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
  if (sum == -seed - 1e300) sink[0] = sum;
}

// --------------------------------------------------------------------------
// Element Jacobian for FP32 element matrices (the FP32 linear solver of
// precision 1, the FP32 multigrid levels of precision 2), with the tangent in
// FP32 and the B^T D B contraction on the tensor cores. The matrices only
// feed the FP32 solver: the Newton residual, and with it J = det F of the
// discrete equations, stays FP64.
//   K[(i,ci)][(j,cj)] = sum_{q,a} B_a(i,q) E_q[(ci,a)][(j,cj)]
// is one product D = A B^T per cell with
//   A[m][kk] = s_a E_q[(ci,a)][(j,cj)],  m = ci*45 + j*5 + cj (225 rows, two tiles of 128),
//   B[i][kk] = reference-cell basis value (a = 0) or s / t derivative (a = 1, 2) of
//              node i at Gauss point q (9 rows, padded to 16), kk = q*3 + a (27, padded to 32),
// s_a = 1, 1/hx, 1/hy the reference-to-cell derivative factors, E_q = w_q D_q B_q
// and D[m][i] the entry K[(i,ci)][(j,cj)]. Both operands enter tcgen05.mma
// (kind::f16, M = 128, N = 16, K = 16) as three BF16 terms (FP32-level
// accuracy); the two M tiles are built one after the other in one buffer and
// accumulate in 32 FP32 columns of tensor memory. Blocks the material does
// not couple are exactly zero rows of A; the closed-form stabilisation block
// and the outflow-edge term are added as in k_cell_jacobian. When an MMA
// completion is not seen within the poll limit the element matrix is filled
// with NaN (the solve then stops with FSI_ENAN) and *status is set.
// --------------------------------------------------------------------------
// FP32 copies of the reference-element tables for the FP32 tangent. They sit in global memory and each CTA
// stages them in shared memory: the contraction reads them with a per-thread basis index, which constant
// memory would serialise (one constant-cache access per distinct address in a warp).
struct TabF {
  float phi[9][9], dps[9][9], dpt[9][9];   // [Gauss point][basis function]
  float wq[9];
  float phie[3][9], dpse[3][9], dpte[3][9];
  float we[3];
  float lss[9][9], ltt[9][9];               // the stabilisation integrals
};
__device__ TabF g_tabf;

// FP32 counterparts of eval_qp and lps_weight for the FP32 tangent.
__device__ inline void eval_qp_f32(const TabF& T, const float* Ue, const float* Uo, int q, float ihx, float ihy,
                                   QpInT<float>& s) {
  float val[5] = {0, 0, 0, 0, 0}, gx[5] = {0, 0, 0, 0, 0}, gy[5] = {0, 0, 0, 0, 0};
  float valo[4] = {0, 0, 0, 0}, gxo[4] = {0, 0, 0, 0}, gyo[4] = {0, 0, 0, 0};
  for (int l = 0; l < 9; ++l) {
    const float ph = T.phi[q][l], ps = T.dps[q][l] * ihx, pt = T.dpt[q][l] * ihy;
    for (int c = 0; c < 5; ++c) {
      val[c] += ph * Ue[l * 5 + c];
      gx[c] += ps * Ue[l * 5 + c];
      gy[c] += pt * Ue[l * 5 + c];
    }
    for (int c = 0; c < 4; ++c) {
      valo[c] += ph * Uo[l * 5 + c];
      gxo[c] += ps * Uo[l * 5 + c];
      gyo[c] += pt * Uo[l * 5 + c];
    }
  }
  s.v[0] = val[0]; s.v[1] = val[1]; s.u[0] = val[2]; s.u[1] = val[3]; s.p = val[4];
  s.G = M2T<float>{gx[0], gy[0], gx[1], gy[1]};
  s.Hu = M2T<float>{gx[2], gy[2], gx[3], gy[3]};
  s.vo[0] = valo[0]; s.vo[1] = valo[1]; s.uo[0] = valo[2]; s.uo[1] = valo[3];
  s.Go = M2T<float>{gxo[0], gyo[0], gxo[1], gyo[1]};
  s.Huo = M2T<float>{gxo[2], gyo[2], gxo[3], gyo[3]};
}

__device__ inline float lps_weight_f32(const TabF& T, const Phys& P, const float* Uo, float hx, float hy) {
  float mx = 0.f, my = 0.f, ws = 0.f;
  for (int q = 0; q < 9; ++q) {
    float vx = 0.f, vy = 0.f;
    for (int l = 0; l < 9; ++l) {
      vx += T.phi[q][l] * Uo[l * 5 + 0];
      vy += T.phi[q][l] * Uo[l * 5 + 1];
    }
    mx += T.wq[q] * vx;
    my += T.wq[q] * vy;
    ws += T.wq[q];
  }
  mx /= ws;
  my /= ws;
  const float h = sqrtf(hx * hx + hy * hy), rf = (float)P.rho_f;
  return (float)P.alpha0 * h * h / (rf * (float)P.nu_f + rf * sqrtf(mx * mx + my * my) * h);
}

constexpr int JTC_NS = 3;                          // BF16 terms per FP32 operand
constexpr int JTC_A_TERM = 128 * 32 * 2;           // bytes of one A term of one tile
constexpr int JTC_B_TERM = 16 * 32 * 2;
constexpr int JTC_SMEM = JTC_NS * (JTC_A_TERM + JTC_B_TERM) + 2048;   // operands + slack
static_assert(JAC_THREADS >= 128, "the tensor-memory read-back takes four warps");

// Shared state of the FP32 tangent stage.
struct JacTangentShared32 {
  float sU[45], sUo[45];
  QpInT<float> sq[9];
  QpDerivedT<float> sd[9];
  float sD[9][15][15];      // [q][test slot][trial direction]
  float sDe[3][2][12];      // outflow edge: [q][momentum comp][trial direction (c<4)]
  float sAlpha;
};

__global__ void __launch_bounds__(JAC_THREADS, 4) k_cell_jacobian_tc(DevMesh m, Phys P, const double* __restrict__ U,
                                                                    const double* __restrict__ Uold, size_t stride,
                                                                    double k, double theta, double lps_scale,
                                                                    const uint8_t* __restrict__ active,
                                                                    float* __restrict__ Ke, int* __restrict__ status) {
  const int s = blockIdx.y;
  const int cell = blockIdx.x;
  if (!active[s]) return;   // uniform over the CTA, before any tensor-memory allocation
  extern __shared__ __align__(1024) unsigned char jtc[];
  __shared__ JacTangentShared32 sh;
  __shared__ TabF T;
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tc::tmem_alloc(&tmem_base, 32);
  if (tid == 0) tc::mbar_init(&bar, 1);
  const float hx = (float)m.cell_h[cell * 2], hy = (float)m.cell_h[cell * 2 + 1];
  const float fihx = 1.f / hx, fihy = 1.f / hy, farea = hx * hy;
  const uint8_t cf = m.cell_flags[cell];
  const bool solid = cf & CF_SOLID;
  const bool outflow = !solid && (cf & CF_OUTFLOW);
  // ---- FP32 tangent: the cell's states in FP32, then the Gauss-point quantities ----
  if (tid < 45) {
    sh.sU[tid] = (float)U[s * stride + (size_t)m.cell_nodes[cell * 9 + tid / 5] * 5 + tid % 5];
    sh.sUo[tid] = (float)Uold[s * stride + (size_t)m.cell_nodes[cell * 9 + tid / 5] * 5 + tid % 5];
  }
  for (int i = tid; i < (int)(sizeof(TabF) / sizeof(float)); i += JAC_THREADS)
    reinterpret_cast<float*>(&T)[i] = reinterpret_cast<const float*>(&g_tabf)[i];
  __syncthreads();
  if (tid < 9) {
    eval_qp_f32(T, sh.sU, sh.sUo, tid, fihx, fihy, sh.sq[tid]);
    derive(sh.sq[tid], sh.sd[tid]);
  }
  if (tid == 32 && !solid) sh.sAlpha = (float)lps_scale * lps_weight_f32(T, P, sh.sUo, hx, hy);
  __syncthreads();
  const float fk = (float)k, fth = (float)theta;
  for (int t = tid; t < 9 * 15; t += JAC_THREADS) {
    const int q = t / 15, dir = t % 15, cj = dir / 3, b = dir % 3;
    float dv[2] = {0.f, 0.f}, du[2] = {0.f, 0.f}, dp = 0.f;
    M2T<float> dG{0.f, 0.f, 0.f, 0.f}, dH{0.f, 0.f, 0.f, 0.f};
    if (cj < 2) {
      if (b == 0) dv[cj] = 1.f;
      else if (cj == 0) { if (b == 1) dG.a = 1.f; else dG.b = 1.f; }
      else { if (b == 1) dG.c = 1.f; else dG.d = 1.f; }
    } else if (cj < 4) {
      const int c = cj - 2;
      if (b == 0) du[c] = 1.f;
      else if (c == 0) { if (b == 1) dH.a = 1.f; else dH.b = 1.f; }
      else { if (b == 1) dH.c = 1.f; else dH.d = 1.f; }
    } else {
      if (b == 0) dp = 1.f;
    }
    float out[15];
    qp_flux_lin(P, sh.sq[q], sh.sd[q], solid, fk, fth, dv, dG, du, dH, dp, out);
    for (int r = 0; r < 15; ++r) sh.sD[q][r][dir] = out[r];
  }
  if (outflow) {
    for (int t = tid; t < 3 * 12; t += JAC_THREADS) {
      const int q = t / 12, dir = t % 12, cj = dir / 3, b = dir % 3;
      float gx[4] = {0.f, 0.f, 0.f, 0.f}, gy[4] = {0.f, 0.f, 0.f, 0.f};
      for (int l = 0; l < 9; ++l) {
        const float ps = T.dpse[q][l] * fihx, pt = T.dpte[q][l] * fihy;
        for (int cc = 0; cc < 4; ++cc) {
          gx[cc] += ps * sh.sU[l * 5 + cc];
          gy[cc] += pt * sh.sU[l * 5 + cc];
        }
      }
      const M2T<float> Gf{gx[0], gy[0], gx[1], gy[1]};
      const M2T<float> Hf{gx[2], gy[2], gx[3], gy[3]};
      M2T<float> dG{0.f, 0.f, 0.f, 0.f}, dH{0.f, 0.f, 0.f, 0.f};
      float out[2] = {0.f, 0.f};
      if (b > 0) {
        M2T<float>& X = cj < 2 ? dG : dH;
        const int c = cj % 2;
        if (c == 0) { if (b == 1) X.a = 1.f; else X.b = 1.f; }
        else { if (b == 1) X.c = 1.f; else X.d = 1.f; }
        edge_flux_lin(P, Gf, Hf, dG, dH, fk, fth, out);
      }
      sh.sDe[q][0][dir] = out[0];
      sh.sDe[q][1][dir] = out[1];
    }
  }
  __syncthreads();
  // ---- the contraction on the tensor cores ----
  unsigned char* sA = jtc;                          // one tile: JTC_NS terms of 128 x 32
  unsigned char* sB = jtc + JTC_NS * JTC_A_TERM;
  const uint32_t tmem = tmem_base;
  bool ok = true;
  for (int tile = 0; tile < 2; ++tile) {
    // B (first tile only): 16 rows x 4 chunks of 8 K values; A: 128 rows x 4 chunks
    const int nitems = (tile == 0 ? 64 : 0) + 128 * 4;
    for (int item = tid; item < nitems; item += JAC_THREADS) {
      const bool isB = tile == 0 && item < 64;
      const int local = isB ? item / 4 : (item - (tile == 0 ? 64 : 0)) / 4, c = item % 4;
      float v[8];
      if (isB) {
#pragma unroll
        for (int x = 0; x < 8; ++x) {
          const int kk = c * 8 + x, q = kk / 3, a = kk % 3;
          v[x] = (local < 9 && kk < 27) ? (a == 0 ? T.phi[q][local] : (a == 1 ? T.dps[q][local] : T.dpt[q][local]))
                                        : 0.f;
        }
      } else {
        const int row = tile * 128 + local;
        const int ci = row / 45, j = (row / 5) % 9, cj = row % 5;
        const bool live = row < 225 && jac_block_nonzero(solid, ci, cj);
#pragma unroll
        for (int x = 0; x < 8; ++x) {
          const int kk = c * 8 + x, q = kk / 3, a = kk % 3;
          float e = 0.f;
          if (live && kk < 27) {
            const float* Dr = &sh.sD[q][ci * 3 + a][cj * 3];
            const float sa = a == 0 ? 1.f : (a == 1 ? fihx : fihy);
            e = sa * T.wq[q] * farea *
                (Dr[0] * T.phi[q][j] + Dr[1] * (T.dps[q][j] * fihx) + Dr[2] * (T.dpt[q][j] * fihy));
          }
          v[x] = e;
        }
      }
      uint32_t w[JTC_NS][4];
#pragma unroll
      for (int x = 0; x < 8; x += 2) {
        __nv_bfloat16 t0[JTC_NS], t1[JTC_NS];
        tc::split_bf16<JTC_NS>(v[x], t0);
        tc::split_bf16<JTC_NS>(v[x + 1], t1);
#pragma unroll
        for (int t = 0; t < JTC_NS; ++t)
          w[t][x / 2] = (uint32_t)__bfloat16_as_ushort(t0[t]) | ((uint32_t)__bfloat16_as_ushort(t1[t]) << 16);
      }
      const uint32_t off = tc::kmajor_offset(local, c * 8, 4);
#pragma unroll
      for (int t = 0; t < JTC_NS; ++t) {
        unsigned char* base = isB ? sB + t * JTC_B_TERM : sA + t * JTC_A_TERM;
        *reinterpret_cast<uint4*>(base + off) = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
      }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0) {
      constexpr uint32_t idesc = tc::idesc_bf16_f32(128, 16);
      int issued = 0;
      for (int ks = 0; ks < 2; ++ks)
        for (int p = 0; p < tc::SplitPairs<JTC_NS>::count; ++p) {
          const uint32_t a0 = tc::smem_u32(sA + tc::SplitPairs<JTC_NS>::a(p) * JTC_A_TERM) + ks * 256;
          const uint32_t b0 = tc::smem_u32(sB + tc::SplitPairs<JTC_NS>::b(p) * JTC_B_TERM) + ks * 256;
          tc::mma_bf16(tmem + tile * 16, tc::smem_desc(a0, 128, 512), tc::smem_desc(b0, 128, 512), idesc,
                       issued++ > 0);
        }
      tc::mma_commit(&bar);
    }
    __syncwarp();
    // the wait also frees the operand buffer for the next tile
    bool done = tc::mbar_wait(&bar, tile, tc::kMaxPolls);
    if (!done) done = tc::mbar_wait(&bar, tile, tc::kMaxPolls);   // the MMAs in flight get a second chance
    ok = __syncthreads_and(ok && done);                              // one outcome for the whole CTA
    tc::fence_after_sync();
    if (!ok) break;
  }
  if (!ok && tid == 0) atomicExch(status, 1);
  float* out = Ke + ((size_t)s * m.n_cells + cell) * 2025;
  if (warp < 4) {
    for (int tile = 0; tile < 2; ++tile) {
      float d[16];
      if (ok) tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + tile * 16, d);
      const int row = tile * 128 + warp * 32 + lane;
      if (row >= 225) continue;
      const int ci = row / 45, j = (row / 5) % 9, cj = row % 5;
      if (!jac_block_nonzero(solid, ci, cj)) continue;
      for (int i = 0; i < 9; ++i) {
        float v = ok ? d[i] : __int_as_float(0x7fc00000);
        if (outflow && ci < 2 && cj < 4) {
          for (int q = 0; q < 3; ++q) {
            const float Bj[3] = {T.phie[q][j], T.dpse[q][j] * fihx, T.dpte[q][j] * fihy};
            const float* Drow = sh.sDe[q][ci] + cj * 3;
            v += T.we[q] * hy * T.phie[q][i] * (Drow[0] * Bj[0] + Drow[1] * Bj[1] + Drow[2] * Bj[2]);
          }
        }
        out[(i * 5 + ci) * 45 + j * 5 + cj] = v;
      }
    }
  }
  // the other blocks: zero, or the stabilisation block (fluid p-p)
  for (int e = tid; e < 2025; e += JAC_THREADS) {
    const int row = e / 45, col = e % 45;
    const int i = row / 5, ci = row % 5, j = col / 5, cj = col % 5;
    if (jac_block_nonzero(solid, ci, cj)) continue;
    float v = 0.f;
    if (!solid && ci == 4 && cj == 4)
      v = fk * sh.sAlpha * (hy * fihx * T.lss[i][j] + hx * fihy * T.ltt[i][j]);
    out[e] = v;
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 32);
}

// --------------------------------------------------------------------------
// Float-float operator product for FP64 operators. GB300 runs FP64 at 1/64 of
// the FP32 rate, which caps the FP64 block-sparse product (one FMA per 8-byte
// value) below the HBM bandwidth. Here the blocks and the input vector are
// carried as float pairs hi + lo (the same 8 bytes per value, 2^-48 relative)
// and every row is accumulated with error-free FP32 transformations in the
// manner of the compensated dot product Dot2 (fsi_ff.h): about 19 FP32
// operations per term on the FP32 pipe, an accuracy of order 2^-48 relative
// to the sum of |a x|, close to that of the FP64 product.
// --------------------------------------------------------------------------
#include "fsi_ff.h"

// out[s][i] = (hi, lo) of x[s][i] for active slices
__global__ void k_to_ff(size_t n, const double* __restrict__ x, size_t xstride, const uint8_t* __restrict__ active,
                        float2* __restrict__ out, size_t ostride) {
  const int s = blockIdx.y;
  if (!active[s]) return;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const fsiff::ff v = fsiff::split(x[s * xstride + i]);
    out[s * ostride + i] = make_float2(v.hi, v.lo);
  }
}

template <bool RESIDUAL>
__global__ void k_bsr_spmv_ff(DevMesh m, const float2* __restrict__ A, const float2* __restrict__ x,
                              const double* __restrict__ bvec, size_t stride, const uint8_t* __restrict__ active,
                              double* __restrict__ y, const int* __restrict__ rows, int nrows) {
  const int s = blockIdx.y;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || t >= nrows * 5) return;
  const int i = rows[t / 5], c = t % 5;
  const float2* As = A + (size_t)s * m.nnzb * 25 + c * 5;
  const float2* xs = x + s * stride;
  fsiff::ffacc acc;
  const int b1 = m.rowptr[i + 1];
  for (int b = m.rowptr[i]; b < b1; ++b) {
    const float2* blk = As + (size_t)b * 25;
    const float2* xj = xs + (size_t)m.colidx[b] * 5;
#pragma unroll
    for (int e = 0; e < 5; ++e) {
      const float2 a = blk[e], v = xj[e];
      fsiff::fma_ff(acc, fsiff::ff{a.x, a.y}, fsiff::ff{v.x, v.y});
    }
  }
  const size_t o = s * stride + (size_t)i * 5 + c;
  const double r = fsiff::result(acc);
  y[o] = RESIDUAL ? bvec[o] - r : r;
}

// --------------------------------------------------------------------------
// Row-tile block product: a CTA takes ROWS consecutive node rows. Their blocks
// are one contiguous range of the slice's values, which the CTA brings into
// shared memory at once: the 16-byte aligned middle of the range by one bulk
// asynchronous copy (cp.async.bulk, completion counted on an mbarrier), the
// unaligned head and tail by plain loads. Thread (r, c) then sums component c
// of row r over the row's blocks in ascending order, five terms per block:
// the order of k_bsr_spmv and k_bsr_spmv_ff, so the tile size changes the work
// distribution, never a bit of the result. V is the stored value type (double,
// float, or float2 = an FP64 value as a float pair), Y the type of b and y.
// A bulk copy that does not complete within the poll limit (twice) sets
// *status and leaves NaN in the tile's outputs.
// --------------------------------------------------------------------------
template <typename V> struct SptAcc;
template <> struct SptAcc<double> {
  double a = 0.0;
  __device__ void add(double v, double x) { a = fma(v, x, a); }
  __device__ double value() const { return a; }
};
template <> struct SptAcc<float> {
  float a = 0.f;
  __device__ void add(float v, float x) { a = fmaf(v, x, a); }
  __device__ float value() const { return a; }
};
template <> struct SptAcc<float2> {
  fsiff::ffacc a;
  __device__ void add(float2 v, float2 x) { fsiff::fma_ff(a, fsiff::ff{v.x, v.y}, fsiff::ff{x.x, x.y}); }
  __device__ double value() const { return fsiff::result(a); }
};

// Blocks of the largest tile of ROWS consecutive rows (host side: shared-memory size).
inline int spmv_tile_max_blocks(const int* rowptr, int n_nodes, int rows) {
  int mx = 0;
  for (int r0 = 0; r0 < n_nodes; r0 += rows) {
    const int r1 = r0 + rows < n_nodes ? r0 + rows : n_nodes;
    mx = rowptr[r1] - rowptr[r0] > mx ? rowptr[r1] - rowptr[r0] : mx;
  }
  return mx;
}
// Dynamic shared memory of a tile of `blocks` blocks: the values plus 16 bytes of
// alignment slack (the staged range keeps the address modulo 16 of the source).
template <typename V> constexpr size_t spmv_tile_smem(int blocks) { return (size_t)blocks * 25 * sizeof(V) + 16; }

template <typename V, typename Y, bool RESIDUAL, int ROWS>
__global__ void __launch_bounds__(ROWS * 5) k_bsr_spmv_tile(DevMesh m, const V* __restrict__ A,
                                                            const V* __restrict__ x, const Y* __restrict__ bvec,
                                                            size_t stride, const uint8_t* __restrict__ active,
                                                            Y* __restrict__ y, int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char spt_raw[];
  __shared__ __align__(8) uint64_t bar;
  const int s = blockIdx.y;
  if (!active[s]) return;   // uniform over the CTA
  const int tid = threadIdx.x;
  const int r0 = blockIdx.x * ROWS;
  const int r1 = min(r0 + ROWS, m.n_nodes);
  const int B0 = m.rowptr[r0], B1 = m.rowptr[r1];
  const V* src = A + ((size_t)s * m.nnzb + B0) * 25;
  const int n_el = (B1 - B0) * 25;
  // sm[k] holds src[k]; sm starts at the same address modulo 16 as src
  const uint32_t mis = (uint32_t)(reinterpret_cast<uintptr_t>(src) & 15u);
  V* sm = reinterpret_cast<V*>(spt_raw + mis);
  const int k_a = min(n_el, (int)(((16u - mis) & 15u) / sizeof(V)));   // first 16-byte aligned element
  const int k_b = k_a + (int)((((size_t)(n_el - k_a) * sizeof(V)) / 16) * 16 / sizeof(V));
  const uint32_t bytes = (uint32_t)((size_t)(k_b - k_a) * sizeof(V));
  if (tid == 0 && bytes) tc::mbar_init(&bar, 1);
  __syncthreads();
  if (tid == 0 && bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(&bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            tc::smem_u32(sm + k_a)),
        "l"(src + k_a), "r"(bytes), "r"(tc::smem_u32(&bar))
        : "memory");
  }
  for (int k = tid; k < k_a; k += ROWS * 5) sm[k] = src[k];
  for (int k = k_b + tid; k < n_el; k += ROWS * 5) sm[k] = src[k];
  bool ok = true;
  if (bytes) {
    ok = tc::mbar_wait(&bar, 0, tc::kMaxPolls);
    if (!ok) ok = tc::mbar_wait(&bar, 0, tc::kMaxPolls);   // the copy in flight gets a second chance
  }
  ok = __syncthreads_and(ok);
  if (!ok && tid == 0) atomicExch(status, 1);
  const int r = r0 + tid / 5, c = tid % 5;
  if (r >= r1) return;
  const size_t o = s * stride + (size_t)r * 5 + c;
  if (!ok) {
    y[o] = (Y)__longlong_as_double(0x7ff8000000000000ll);
    return;
  }
  const V* xs = x + s * stride;
  SptAcc<V> acc;
  const int b1 = m.rowptr[r + 1];
  for (int b = m.rowptr[r]; b < b1; ++b) {
    const V* blk = sm + (b - B0) * 25 + c * 5;
    const V* xj = xs + (size_t)m.colidx[b] * 5;
#pragma unroll
    for (int e = 0; e < 5; ++e) acc.add(blk[e], xj[e]);
  }
  const Y v = (Y)acc.value();
  y[o] = RESIDUAL ? bvec[o] - v : v;
}
