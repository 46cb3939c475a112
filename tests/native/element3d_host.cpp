// Host build of the 3D element physics of the CUDA library (the same header the
// kernels compile), so tests can compare it with the FP64 oracle on the CPU.
#include <algorithm>
#include <vector>

#include "../../paper_1907_01252_gb300/csrc/fsi_element3d.cuh"

extern "C" int fsi3_cell_residual_host(const double* phys, const double* Ue, const double* Uo, const double* h,
                                       int solid, int outflow, double k, double theta, double alpha, double* Re) {
  static fsi3::Tables3 T;
  static bool ready = false;
  if (!ready) {
    fsi3::build_tables3(T);
    ready = true;
  }
  const fsi3::Phys3 P{phys[0], phys[1], phys[2], phys[3], phys[4]};
  fsi3::cell_residual3(P, T, Ue, Uo, h, solid != 0, outflow != 0, k, theta, alpha, Re);
  return 0;
}

extern "C" int fsi3_cell_jacobian_host(const double* phys, const double* Ue, const double* Uo, const double* h,
                                       int solid, int outflow, double k, double theta, double alpha, double* Ke) {
  static fsi3::Tables3 T;
  static bool ready = false;
  if (!ready) {
    fsi3::build_tables3(T);
    ready = true;
  }
  const fsi3::Phys3 P{phys[0], phys[1], phys[2], phys[3], phys[4]};
  fsi3::cell_jacobian3(P, T, Ue, Uo, h, solid != 0, outflow != 0, k, theta, alpha, Ke);
  return 0;
}

// The same cell residual by the cooperative routine the kernel runs (one host thread).
extern "C" int fsi3_cell_residual_cta_host(const double* phys, const double* Ue, const double* Uo, const double* h,
                                           int solid, int outflow, double k, double theta, double alpha,
                                           double* Re) {
  static fsi3::Tables3 T;
  static bool ready = false;
  if (!ready) {
    fsi3::build_tables3(T);
    ready = true;
  }
  const fsi3::Phys3 P{phys[0], phys[1], phys[2], phys[3], phys[4]};
  std::vector<double> sh(fsi3::CR3_TOTAL, -1.0);
  std::copy(Ue, Ue + 189, sh.begin() + fsi3::CR3_UE);
  std::copy(Uo, Uo + 189, sh.begin() + fsi3::CR3_UE + 189);
  for (int i = 0; i < 189; ++i) Re[i] = -7.0;
  fsi3::cell_residual3_cta(fsi3::HostCta{}, P, T, h, solid != 0, outflow != 0, k, theta, alpha, sh.data(), Re);
  return 0;
}

// The same element matrix by the cooperative routine the kernel runs (one host thread).
extern "C" int fsi3_cell_jacobian_cta_host(const double* phys, const double* Ue, const double* Uo, const double* h,
                                           int solid, int outflow, double k, double theta, double alpha,
                                           double* Ke) {
  static fsi3::Tables3 T;
  static bool ready = false;
  if (!ready) {
    fsi3::build_tables3(T);
    ready = true;
  }
  const fsi3::Phys3 P{phys[0], phys[1], phys[2], phys[3], phys[4]};
  std::vector<double> sh(fsi3::CJ3_TOTAL, -1.0);   // stale values must not matter
  std::copy(Ue, Ue + 189, sh.begin() + fsi3::CJ3_UE);
  std::copy(Uo, Uo + 189, sh.begin() + fsi3::CJ3_UE + 189);
  for (int i = 0; i < 189 * 189; ++i) Ke[i] = -7.0;   // every entry must be written
  fsi3::cell_jacobian3_cta(fsi3::HostCta{}, P, T, h, solid != 0, outflow != 0, k, theta, alpha, sh.data(), Ke);
  return 0;
}

#include "../../paper_1907_01252_gb300/csrc/fsi_mesh3d.h"

namespace {
fsi3::HostMesh3 make_mesh(const double* xb, const int* nxs, int nxseg, const double* yb, const int* nys, int nyseg,
                          const double* zb, const int* nzs, int nzseg, const double* box) {
  fsi3::HostMesh3 m;
  fsi3::build_mesh3(m, fsi3::axis_vertices3(xb, nxs, nxseg), fsi3::axis_vertices3(yb, nys, nyseg),
                    fsi3::axis_vertices3(zb, nzs, nzseg), box);
  return m;
}
fsi3::Mesh3View view(const fsi3::HostMesh3& m) {
  return fsi3::Mesh3View{m.nnx, m.nny, m.nnz, m.n_nodes, m.n_cells, m.yn.data(), m.zn.data(),
                         m.cell_flags.data(), m.node_flags.data(), m.node_cells.data(), m.y0, m.y1, m.z0, m.z1,
                         m.blk_row.data(), m.colidx.data(), m.blk_src.data(), m.cell_blk.data()};
}
}  // namespace

// Mesh tables: sizes_out = {n_nodes, n_cells, nnzb}; the arrays are filled when non-null.
extern "C" int fsi3_mesh_host(const double* xb, const int* nxs, int nxseg, const double* yb, const int* nys, int nyseg,
                              const double* zb, const int* nzs, int nzseg, const double* box, int* sizes_out,
                              int* cell_nodes_out, unsigned char* node_flags_out, unsigned char* cell_flags_out) {
  const fsi3::HostMesh3 m = make_mesh(xb, nxs, nxseg, yb, nys, nyseg, zb, nzs, nzseg, box);
  sizes_out[0] = m.n_nodes;
  sizes_out[1] = m.n_cells;
  sizes_out[2] = m.nnzb;
  if (cell_nodes_out) std::copy(m.cell_nodes.begin(), m.cell_nodes.end(), cell_nodes_out);
  if (node_flags_out) std::copy(m.node_flags.begin(), m.node_flags.end(), node_flags_out);
  if (cell_flags_out) std::copy(m.cell_flags.begin(), m.cell_flags.end(), cell_flags_out);
  return 0;
}

// The assembled step residual R[n_nodes][7] of one slice, computed the way the
// kernels do: per cell (stabilisation weight, the cooperative cell residual),
// then per row (fixed-order gather or identity row). mat = {rho_f, nu_f, rho_s, mu_s,
// lambda_s, vbar, ramp_t, alpha0}.
extern "C" int fsi3_residual_host(const double* xb, const int* nxs, int nxseg, const double* yb, const int* nys,
                                  int nyseg, const double* zb, const int* nzs, int nzseg, const double* box,
                                  const double* mat, const double* U, const double* Uo, double t_new, double k,
                                  double theta, double* R) {
  static fsi3::Tables3 T;
  static bool ready = false;
  if (!ready) {
    fsi3::build_tables3(T);
    ready = true;
  }
  const fsi3::HostMesh3 m = make_mesh(xb, nxs, nxseg, yb, nys, nyseg, zb, nzs, nzseg, box);
  const fsi3::Phys3 P{mat[0], mat[1], mat[2], mat[3], mat[4]};
  std::vector<double> Re((size_t)m.n_cells * 27 * 7), Ue(189), Uoe(189), sh(fsi3::CR3_TOTAL);
  for (int c = 0; c < m.n_cells; ++c) {
    for (int l = 0; l < 27; ++l)
      for (int f = 0; f < 7; ++f) {
        Ue[l * 7 + f] = U[(size_t)m.cell_nodes[(size_t)c * 27 + l] * 7 + f];
        Uoe[l * 7 + f] = Uo[(size_t)m.cell_nodes[(size_t)c * 27 + l] * 7 + f];
      }
    const double* h = &m.cell_h[(size_t)c * 3];
    const bool solid = m.cell_flags[c] & fsi3::C3_SOLID, outflow = m.cell_flags[c] & fsi3::C3_OUTFLOW;
    const double alpha = fsi3::stab_weight3(T, Uoe.data(), h, mat[7], mat[0], mat[1]);
    // the kernel's routine (cooperative), run by one host thread
    std::copy(Ue.begin(), Ue.end(), sh.begin() + fsi3::CR3_UE);
    std::copy(Uoe.begin(), Uoe.end(), sh.begin() + fsi3::CR3_UE + 189);
    fsi3::cell_residual3_cta(fsi3::HostCta{}, P, T, h, solid, outflow, k, theta, alpha, sh.data(),
                             &Re[(size_t)c * 189]);
  }
  const fsi3::Mesh3View v = view(m);
  for (int n = 0; n < m.n_nodes; ++n)
    for (int c = 0; c < 7; ++c) R[(size_t)n * 7 + c] = fsi3::gather3(v, Re.data(), U, n, c, t_new, mat[5], mat[6]);
  return 0;
}

// The assembled Jacobian of one slice in 7 x 7 blocks (row-major), computed the
// way the kernels do: element matrices per cell by the kernel's cooperative
// routine, then every block entry by the fixed-order gather. rowptr_out [n_nodes + 1], colidx_out [nnzb],
// vals_out [nnzb][49]; the sizes come from fsi3_mesh_host.
extern "C" int fsi3_jacobian_host(const double* xb, const int* nxs, int nxseg, const double* yb, const int* nys,
                                  int nyseg, const double* zb, const int* nzs, int nzseg, const double* box,
                                  const double* mat, const double* U, const double* Uo, double k, double theta,
                                  int* rowptr_out, int* colidx_out, double* vals_out) {
  static fsi3::Tables3 T;
  static bool ready = false;
  if (!ready) {
    fsi3::build_tables3(T);
    ready = true;
  }
  const fsi3::HostMesh3 m = make_mesh(xb, nxs, nxseg, yb, nys, nyseg, zb, nzs, nzseg, box);
  const fsi3::Phys3 P{mat[0], mat[1], mat[2], mat[3], mat[4]};
  std::vector<double> Ke((size_t)m.n_cells * 189 * 189), Ue(189), Uoe(189), sh(fsi3::CJ3_TOTAL);
  for (int c = 0; c < m.n_cells; ++c) {
    for (int l = 0; l < 27; ++l)
      for (int f = 0; f < 7; ++f) {
        Ue[l * 7 + f] = U[(size_t)m.cell_nodes[(size_t)c * 27 + l] * 7 + f];
        Uoe[l * 7 + f] = Uo[(size_t)m.cell_nodes[(size_t)c * 27 + l] * 7 + f];
      }
    const double* h = &m.cell_h[(size_t)c * 3];
    const bool solid = m.cell_flags[c] & fsi3::C3_SOLID, outflow = m.cell_flags[c] & fsi3::C3_OUTFLOW;
    const double alpha = fsi3::stab_weight3(T, Uoe.data(), h, mat[7], mat[0], mat[1]);
    // the kernel's routine (cooperative, sum-factorised), run by one host thread
    std::copy(Ue.begin(), Ue.end(), sh.begin() + fsi3::CJ3_UE);
    std::copy(Uoe.begin(), Uoe.end(), sh.begin() + fsi3::CJ3_UE + 189);
    fsi3::cell_jacobian3_cta(fsi3::HostCta{}, P, T, h, solid, outflow, k, theta, alpha, sh.data(),
                             &Ke[(size_t)c * 189 * 189]);
  }
  const fsi3::Mesh3View v = view(m);
  std::copy(m.rowptr.begin(), m.rowptr.end(), rowptr_out);
  std::copy(m.colidx.begin(), m.colidx.end(), colidx_out);
  for (int b = 0; b < m.nnzb; ++b)
    for (int r = 0; r < 7; ++r)
      for (int c = 0; c < 7; ++c) vals_out[(size_t)b * 49 + r * 7 + c] = fsi3::assemble3(v, Ke.data(), b, r, c);
  return 0;
}

#include "../../paper_1907_01252_gb300/csrc/fsi_mg3d.h"

// One multigrid transfer between the mesh and its coarsening, run in host loops
// over the per-entry functions the kernels will call. sizes_out = {nnx_f, nny_f,
// nnz_f, nnx_c, nny_c, nnz_c}; coords_out (optional) = fine x, y, z node
// coordinates then coarse ones; flags_out (optional) = fine then coarse node
// flags. mode 1: out[fine][7] = prolongation of in[coarse][7]; mode 2:
// out[coarse][7] = restriction of in[fine][7]; mode 3: out[coarse][7] = the fine
// state in[fine][7] evaluated at the coarse nodes; mode 0: sizes only.
extern "C" int fsi3_transfer_host(const double* xb, const int* nxs, int nxseg, const double* yb, const int* nys,
                                  int nyseg, const double* zb, const int* nzs, int nzseg, const double* box, int mode,
                                  const double* in, double* out, int* sizes_out, double* coords_out,
                                  unsigned char* flags_out) {
  std::vector<double> vf[3] = {fsi3::axis_vertices3(xb, nxs, nxseg), fsi3::axis_vertices3(yb, nys, nyseg),
                               fsi3::axis_vertices3(zb, nzs, nzseg)};
  const std::vector<int> segf[3] = {std::vector<int>(nxs, nxs + nxseg), std::vector<int>(nys, nys + nyseg),
                                    std::vector<int>(nzs, nzs + nzseg)};
  std::vector<double> vc[3];
  std::vector<int> segc[3];
  for (int a = 0; a < 3; ++a) fsi3::coarsen_axis3(vf[a], segf[a], vc[a], segc[a]);
  fsi3::HostMesh3 F, Cm;
  fsi3::build_mesh3(F, vf[0], vf[1], vf[2], box);
  fsi3::build_mesh3(Cm, vc[0], vc[1], vc[2], box);
  const std::vector<double> xf[3] = {F.xn, F.yn, F.zn}, xc[3] = {Cm.xn, Cm.yn, Cm.zn};
  fsi3::Transfer3 T;
  fsi3::build_transfer3(T, vc, xc, vf, xf);
  for (int a = 0; a < 3; ++a) {
    sizes_out[a] = T.nn_f[a];
    sizes_out[3 + a] = T.nn_c[a];
  }
  if (coords_out) {
    for (int a = 0; a < 3; ++a) coords_out = std::copy(xf[a].begin(), xf[a].end(), coords_out);
    for (int a = 0; a < 3; ++a) coords_out = std::copy(xc[a].begin(), xc[a].end(), coords_out);
  }
  if (flags_out) {
    flags_out = std::copy(F.node_flags.begin(), F.node_flags.end(), flags_out);
    std::copy(Cm.node_flags.begin(), Cm.node_flags.end(), flags_out);
  }
  const fsi3::Transfer3View v = fsi3::view(T);
  if (mode == 1)
    for (int n = 0; n < F.n_nodes; ++n)
      for (int c = 0; c < 7; ++c) out[(size_t)n * 7 + c] = fsi3::prolong3(v, F.node_flags.data(), in, n, c);
  else if (mode == 2)
    for (int n = 0; n < Cm.n_nodes; ++n)
      for (int c = 0; c < 7; ++c)
        out[(size_t)n * 7 + c] = fsi3::restrict3(v, F.node_flags.data(), Cm.node_flags.data(), in, n, c);
  else if (mode == 3)
    for (int n = 0; n < Cm.n_nodes; ++n)
      for (int c = 0; c < 7; ++c) out[(size_t)n * 7 + c] = fsi3::interp_state3(v, in, n, c);
  return 0;
}

#include "../../paper_1907_01252_gb300/csrc/fsi_vanka3.h"

namespace {
template <typename T>
int vanka_cells(const fsi3::HostMesh3& m, const double* A, const double* r, double* zc) {
  const fsi3::Mesh3View v = view(m);
  std::vector<T> At(A, A + (size_t)m.nnzb * 49), inv(fsi3::VK3_SIZE), sh(fsi3::VK3_SH_T), ap(fsi3::VK3_AP_T),
      rl(189), z(189);
  std::vector<int> ish(fsi3::VK3_SH_I);
  const fsi3::HostCta cta;
  for (int c = 0; c < m.n_cells; ++c) {
    if (!fsi3::vk3_setup_cell(cta, v, At.data(), c, sh.data(), ish.data(), inv.data())) return -(c + 1);
    for (int l = 0; l < 27; ++l)
      for (int f = 0; f < 7; ++f) rl[l * 7 + f] = (T)r[(size_t)m.cell_nodes[(size_t)c * 27 + l] * 7 + f];
    fsi3::vk3_apply_cell(cta, (m.cell_flags[c] & fsi3::C3_U_DECOUPLED) != 0, inv.data(), rl.data(), ap.data(),
                         z.data());
    for (int e = 0; e < 189; ++e) zc[(size_t)c * 189 + e] = (double)z[e];
  }
  return 0;
}
}  // namespace

// Vanka local solves of every cell of one slice: zc[cell][189] = (local matrix)^{-1}
// (local residual) in local dof order, computed by the block elimination in T =
// double (precision 0) or float (precision 1) from the Jacobian blocks A[nnzb][49]
// (the mesh's own pattern) and the residual r[n_nodes][7]. x_out (optional):
// the damped node average omega / cnt * (sum of the cells' corrections).
// cell_flags_out (optional): the cell flags. Returns -(cell + 1) on a singular block.
extern "C" int fsi3_vanka_host(const double* xb, const int* nxs, int nxseg, const double* yb, const int* nys,
                               int nyseg, const double* zb, const int* nzs, int nzseg, const double* box,
                               const double* A, const double* r, int precision, double omega, double* zc,
                               double* x_out, unsigned char* cell_flags_out) {
  const fsi3::HostMesh3 m = make_mesh(xb, nxs, nxseg, yb, nys, nyseg, zb, nzs, nzseg, box);
  const int rc = precision ? vanka_cells<float>(m, A, r, zc) : vanka_cells<double>(m, A, r, zc);
  if (rc) return rc;
  if (cell_flags_out) std::copy(m.cell_flags.begin(), m.cell_flags.end(), cell_flags_out);
  if (x_out) {
    const fsi3::Mesh3View v = view(m);
    for (int n = 0; n < m.n_nodes; ++n)
      for (int c = 0; c < 7; ++c) x_out[(size_t)n * 7 + c] = fsi3::vk3_gather(v, zc, omega, n, c);
  }
  return 0;
}

// The tangent at every Gauss point in all 28 unit directions, by the general
// routine and by the unit-direction routine: Dg, Du [27][28 directions][28 outputs].
extern "C" int fsi3_tangents_host(const double* phys, const double* Ue, const double* Uo, const double* h, int solid,
                                  double k, double theta, double* Dg, double* Du) {
  static fsi3::Tables3 T;
  static bool ready = false;
  if (!ready) {
    fsi3::build_tables3(T);
    ready = true;
  }
  const fsi3::Phys3 P{phys[0], phys[1], phys[2], phys[3], phys[4]};
  for (int q = 0; q < 27; ++q) {
    const fsi3::Qp3 x = fsi3::qp_state3(T, Ue, Uo, h, q);
    fsi3::Qp3Lin L;
    fsi3::qp_lin_prepare3(P, x, solid != 0, L);
    for (int dir = 0; dir < 28; ++dir) {
      const int cj = dir / 4, b = dir % 4;
      double dv[3] = {0, 0, 0}, du[3] = {0, 0, 0}, dp = 0.0;
      fsi3::M3 dG{}, dH{};
      if (cj < 3) {
        if (b == 0) dv[cj] = 1.0;
        else dG.m[cj][b - 1] = 1.0;
      } else if (cj < 6) {
        if (b == 0) du[cj - 3] = 1.0;
        else dH.m[cj - 3][b - 1] = 1.0;
      } else if (b == 0) {
        dp = 1.0;
      }
      fsi3::qp_flux3_lin_prepared(P, x, L, solid != 0, k, theta, dv, dG, du, dH, dp, Dg + (q * 28 + dir) * 28);
      fsi3::qp_flux3_lin_unit(P, x, L, solid != 0, k, theta, cj, b, Du + (q * 28 + dir) * 28);
    }
  }
  return 0;
}
