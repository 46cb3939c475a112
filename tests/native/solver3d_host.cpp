// Host run of one 3D theta step, organised the way the library's solver is:
// Newton on the FP64 residual; each correction by FGMRES(m) with classical
// Gram-Schmidt twice, right-preconditioned by one multigrid V-cycle over the
// coarsened hierarchy (block Vanka smoother, Q2 transfers, a dense LU solve on
// the coarsest level). Every per-entry step (cell residual and Jacobian, row
// gathers, transfers, local Vanka solves, node averages) is the library's 3D
// header code; only the loops around them are written here.
#include <cstdio>
#include <numeric>
#include <string>

#include "../../paper_1907_01252_gb300/csrc/fsi_element3d.cuh"
#include "../../paper_1907_01252_gb300/csrc/fsi_mesh3d.h"
#include "../../paper_1907_01252_gb300/csrc/fsi_mg3d.h"
#include "../../paper_1907_01252_gb300/csrc/fsi_vanka3.h"

namespace {

int g_verbose = 0;

struct Params {
  double newton_tol;
  int newton_maxit, restart, gmres_maxit;
  double gmres_rtol, gmres_rtol_first, newton_eta;
  int coarsest_max_dofs, smooth;
  double omega, coarse_lps;
  int smoother;   // 0 additive (node averages), 1 multiplicative over the 8 cell colours
  int coarse_sweeps;   // 0: dense LU on the coarsest level; > 0: that many smoother sweeps there
  int reuse;           // 2: keep the hierarchy of the first Newton iterate; 0: rebuild it every iteration
};

fsi3::Mesh3View make_view(const fsi3::HostMesh3& m) {
  return fsi3::Mesh3View{m.nnx, m.nny, m.nnz, m.n_nodes, m.n_cells, m.yn.data(), m.zn.data(),
                         m.cell_flags.data(), m.node_flags.data(), m.node_cells.data(), m.y0, m.y1, m.z0, m.z1,
                         m.blk_row.data(), m.colidx.data(), m.blk_src.data(), m.cell_blk.data()};
}

template <typename TM>
struct Level {
  fsi3::HostMesh3 h;
  std::vector<double> xv[3];
  std::vector<int> seg[3];
  fsi3::Transfer3 T;   // from the next finer level (l >= 1)
  size_t n = 0;
  std::vector<double> U, Uo;
  std::vector<TM> A, inv, r, b, x, cz;
  std::vector<double> LU;   // coarsest
  std::vector<int> piv;
  bool coarsest = false;
};

const fsi3::Tables3& tables() {
  static fsi3::Tables3 T;
  static bool ready = false;
  if (!ready) {
    fsi3::build_tables3(T);
    ready = true;
  }
  return T;
}

void gather_cell(const fsi3::HostMesh3& m, const double* U, int c, double* Ue) {
  for (int l = 0; l < 27; ++l)
    for (int f = 0; f < 7; ++f) Ue[l * 7 + f] = U[(size_t)m.cell_nodes[(size_t)c * 27 + l] * 7 + f];
}

void residual(const fsi3::HostMesh3& m, const double* mat, const double* U, const double* Uo, double t, double k,
              double theta, double* R) {
  const fsi3::Tables3& T = tables();
  const fsi3::Phys3 P{mat[0], mat[1], mat[2], mat[3], mat[4]};
  std::vector<double> Re((size_t)m.n_cells * 189), Ue(189), Uoe(189);
  for (int c = 0; c < m.n_cells; ++c) {
    gather_cell(m, U, c, Ue.data());
    gather_cell(m, Uo, c, Uoe.data());
    const double* h = &m.cell_h[(size_t)c * 3];
    const double alpha = fsi3::stab_weight3(T, Uoe.data(), h, mat[7], mat[0], mat[1]);
    fsi3::cell_residual3(P, T, Ue.data(), Uoe.data(), h, m.cell_flags[c] & fsi3::C3_SOLID,
                         m.cell_flags[c] & fsi3::C3_OUTFLOW, k, theta, alpha, &Re[(size_t)c * 189]);
  }
  const fsi3::Mesh3View v = make_view(m);
  for (int n = 0; n < m.n_nodes; ++n)
    for (int c = 0; c < 7; ++c) R[(size_t)n * 7 + c] = fsi3::gather3(v, Re.data(), U, n, c, t, mat[5], mat[6]);
}

// Jacobian blocks A[nnzb][49]; lps scales the stabilisation weight (coarse levels).
void jacobian(const fsi3::HostMesh3& m, const double* mat, const double* U, const double* Uo, double k, double theta,
              double lps, std::vector<double>& A) {
  const fsi3::Tables3& T = tables();
  const fsi3::Phys3 P{mat[0], mat[1], mat[2], mat[3], mat[4]};
  std::vector<double> Ke((size_t)m.n_cells * 189 * 189), Ue(189), Uoe(189);
  for (int c = 0; c < m.n_cells; ++c) {
    gather_cell(m, U, c, Ue.data());
    gather_cell(m, Uo, c, Uoe.data());
    const double* h = &m.cell_h[(size_t)c * 3];
    const double alpha = lps * fsi3::stab_weight3(T, Uoe.data(), h, mat[7], mat[0], mat[1]);
    fsi3::cell_jacobian3(P, T, Ue.data(), Uoe.data(), h, m.cell_flags[c] & fsi3::C3_SOLID,
                         m.cell_flags[c] & fsi3::C3_OUTFLOW, k, theta, alpha, &Ke[(size_t)c * 189 * 189]);
  }
  const fsi3::Mesh3View v = make_view(m);
  A.assign((size_t)m.nnzb * 49, 0.0);
  for (int b = 0; b < m.nnzb; ++b)
    for (int r = 0; r < 7; ++r)
      for (int c = 0; c < 7; ++c) A[(size_t)b * 49 + r * 7 + c] = fsi3::assemble3(v, Ke.data(), b, r, c);
}

// y = b - A x (or y = A x when b is null).
template <typename T>
void spmv(const fsi3::HostMesh3& m, const T* A, const T* x, const T* b, T* y) {
  for (int n = 0; n < m.n_nodes; ++n)
    for (int r = 0; r < 7; ++r) {
      T acc = 0;
      for (int e = m.rowptr[n]; e < m.rowptr[n + 1]; ++e) {
        const T* blk = A + (size_t)e * 49 + r * 7;
        const T* xj = x + (size_t)m.colidx[e] * 7;
        for (int c = 0; c < 7; ++c) acc += blk[c] * xj[c];
      }
      y[(size_t)n * 7 + r] = b ? b[(size_t)n * 7 + r] - acc : acc;
    }
}

// Dense LU with partial pivoting of the assembled coarsest matrix (row-major).
bool dense_lu(const fsi3::HostMesh3& m, const std::vector<double>& A, std::vector<double>& LU, std::vector<int>& piv) {
  const int n = m.n_nodes * 7;
  LU.assign((size_t)n * n, 0.0);
  for (int i = 0; i < m.n_nodes; ++i)
    for (int e = m.rowptr[i]; e < m.rowptr[i + 1]; ++e)
      for (int r = 0; r < 7; ++r)
        for (int c = 0; c < 7; ++c) LU[(size_t)(i * 7 + r) * n + m.colidx[e] * 7 + c] = A[(size_t)e * 49 + r * 7 + c];
  piv.resize(n);
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(LU[(size_t)i * n + k]) > std::fabs(LU[(size_t)p * n + k])) p = i;
    if (!(std::fabs(LU[(size_t)p * n + k]) > 0.0)) return false;
    piv[k] = p;
    if (p != k)
      for (int j = 0; j < n; ++j) std::swap(LU[(size_t)k * n + j], LU[(size_t)p * n + j]);
    const double d = 1.0 / LU[(size_t)k * n + k];
    for (int i = k + 1; i < n; ++i) {
      double* ri = &LU[(size_t)i * n];
      const double f = (ri[k] *= d);
      if (f == 0.0) continue;
      const double* rk = &LU[(size_t)k * n];
      for (int j = k + 1; j < n; ++j) ri[j] -= f * rk[j];
    }
  }
  return true;
}

void lu_solve(const std::vector<double>& LU, const std::vector<int>& piv, std::vector<double>& x) {
  const int n = (int)piv.size();
  for (int k = 0; k < n; ++k) std::swap(x[k], x[piv[k]]);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) x[i] -= LU[(size_t)i * n + j] * x[j];
  for (int i = n - 1; i >= 0; --i) {
    for (int j = i + 1; j < n; ++j) x[i] -= LU[(size_t)i * n + j] * x[j];
    x[i] /= LU[(size_t)i * n + i];
  }
}

template <typename TM>
struct Solver {
  const double* mat;
  Params prm;
  std::vector<Level<TM>> lev;
  std::vector<double> A64;   // the fine Jacobian, FP64 (the Krylov operator)
  int gmres_its = 0;

  // Levels: pair cells per segment until the dofs fit coarsest_max_dofs or no axis coarsens.
  void build_levels(const double* const* br, const int* const* seg, const int* nseg, const double* box) {
    lev.emplace_back();
    for (int a = 0; a < 3; ++a) {
      lev[0].xv[a] = fsi3::axis_vertices3(br[a], seg[a], nseg[a]);
      lev[0].seg[a].assign(seg[a], seg[a] + nseg[a]);
    }
    fsi3::build_mesh3(lev[0].h, lev[0].xv[0], lev[0].xv[1], lev[0].xv[2], box);
    while ((size_t)lev.back().h.n_nodes * 7 > (size_t)prm.coarsest_max_dofs) {
      Level<TM> c;
      bool changed = false;
      for (int a = 0; a < 3; ++a) {
        fsi3::coarsen_axis3(lev.back().xv[a], lev.back().seg[a], c.xv[a], c.seg[a]);
        changed |= c.xv[a].size() != lev.back().xv[a].size();
      }
      if (!changed) break;
      fsi3::build_mesh3(c.h, c.xv[0], c.xv[1], c.xv[2], box);
      const Level<TM>& f = lev.back();
      const std::vector<double> xf[3] = {f.h.xn, f.h.yn, f.h.zn}, xc[3] = {c.h.xn, c.h.yn, c.h.zn};
      fsi3::build_transfer3(c.T, c.xv, xc, f.xv, xf);
      lev.push_back(std::move(c));
    }
    for (auto& L : lev) {
      L.n = (size_t)L.h.n_nodes * 7;
      L.r.resize(L.n);
      L.b.resize(L.n);
      L.x.resize(L.n);
      L.cz.resize((size_t)L.h.n_cells * 189);
    }
    lev.back().coarsest = true;
  }

  // Hierarchy from the Newton iterate: states on the coarse levels, operators, smoother and coarsest factors.
  int setup(const double* U, const double* Uo, double k, double theta) {
    lev[0].U.assign(U, U + lev[0].n);
    lev[0].Uo.assign(Uo, Uo + lev[0].n);
    double lps = 1.0;
    for (size_t l = 0; l < lev.size(); ++l) {
      Level<TM>& L = lev[l];
      if (l > 0) {
        const fsi3::Transfer3View tv = fsi3::view(L.T);
        L.U.resize(L.n);
        L.Uo.resize(L.n);
        for (int n = 0; n < L.h.n_nodes; ++n)
          for (int c = 0; c < 7; ++c) {
            L.U[(size_t)n * 7 + c] = fsi3::interp_state3(tv, lev[l - 1].U.data(), n, c);
            L.Uo[(size_t)n * 7 + c] = fsi3::interp_state3(tv, lev[l - 1].Uo.data(), n, c);
          }
        lps *= prm.coarse_lps;
      }
      std::vector<double> A;
      jacobian(L.h, mat, L.U.data(), L.Uo.data(), k, theta, lps, A);
      if (l == 0) A64 = A;
      L.A.assign(A.begin(), A.end());
      if (L.coarsest && prm.coarse_sweeps == 0) {
        std::vector<double> At(L.A.begin(), L.A.end());   // the factors of the preconditioner's operator
        if (!dense_lu(L.h, At, L.LU, L.piv)) return -1;
      } else {
        const fsi3::Mesh3View v = make_view(L.h);
        L.inv.resize((size_t)L.h.n_cells * fsi3::VK3_SIZE);
        std::vector<TM> sh(fsi3::VK3_SH_T);
        std::vector<int> ish(fsi3::VK3_SH_I);
        for (int c = 0; c < L.h.n_cells; ++c)
          if (!fsi3::vk3_setup_cell(fsi3::HostCta{}, v, L.A.data(), c, sh.data(), ish.data(),
                                    &L.inv[(size_t)c * fsi3::VK3_SIZE]))
            return -2;
      }
    }
    return 0;
  }

  // Multiplicative sweep: the cells of one colour (parities of the cell indices)
  // share no node, so each takes its full damped correction; the residual is
  // refreshed between colours.
  void smooth_colours(Level<TM>& L, const TM* b) {
    std::vector<TM> rl(189), ap(fsi3::VK3_AP_T), z(189);
    for (int col = 0; col < 8; ++col) {
      spmv(L.h, L.A.data(), L.x.data(), b, L.r.data());
      for (int c = 0; c < L.h.n_cells; ++c) {
        const int cx = c % L.h.nx, cy = (c / L.h.nx) % L.h.ny, cz = c / (L.h.nx * L.h.ny);
        if ((cx & 1) + 2 * (cy & 1) + 4 * (cz & 1) != col) continue;
        const int* cn = &L.h.cell_nodes[(size_t)c * 27];
        for (int l = 0; l < 27; ++l)
          for (int f = 0; f < 7; ++f) rl[l * 7 + f] = L.r[(size_t)cn[l] * 7 + f];
        fsi3::vk3_apply_cell(fsi3::HostCta{}, (L.h.cell_flags[c] & fsi3::C3_U_DECOUPLED) != 0,
                             &L.inv[(size_t)c * fsi3::VK3_SIZE], rl.data(), ap.data(), z.data());
        for (int l = 0; l < 27; ++l)
          for (int f = 0; f < 7; ++f) L.x[(size_t)cn[l] * 7 + f] += (TM)prm.omega * z[l * 7 + f];
      }
    }
  }

  void smooth(Level<TM>& L, const TM* b, bool first) {
    if (prm.smoother == 1) return smooth_colours(L, b);
    const TM* rr = b;
    if (!first) {
      spmv(L.h, L.A.data(), L.x.data(), b, L.r.data());
      rr = L.r.data();
    }
    std::vector<TM> rl(189), ap(fsi3::VK3_AP_T);
    for (int c = 0; c < L.h.n_cells; ++c) {
      for (int l = 0; l < 27; ++l)
        for (int f = 0; f < 7; ++f) rl[l * 7 + f] = rr[(size_t)L.h.cell_nodes[(size_t)c * 27 + l] * 7 + f];
      fsi3::vk3_apply_cell(fsi3::HostCta{}, (L.h.cell_flags[c] & fsi3::C3_U_DECOUPLED) != 0,
                           &L.inv[(size_t)c * fsi3::VK3_SIZE], rl.data(), ap.data(), &L.cz[(size_t)c * 189]);
    }
    const fsi3::Mesh3View v = make_view(L.h);
    for (int n = 0; n < L.h.n_nodes; ++n)
      for (int c = 0; c < 7; ++c) L.x[(size_t)n * 7 + c] += fsi3::vk3_gather(v, L.cz.data(), prm.omega, n, c);
  }

  // L.x = V-cycle applied to b (b may alias L.b).
  void vcycle(size_t l, const TM* b) {
    Level<TM>& L = lev[l];
    if (L.coarsest && prm.coarse_sweeps > 0) {
      std::fill(L.x.begin(), L.x.end(), TM(0));
      for (int i = 0; i < prm.coarse_sweeps; ++i) smooth(L, b, i == 0);
      return;
    }
    if (L.coarsest) {
      std::vector<double> t(b, b + L.n);
      lu_solve(L.LU, L.piv, t);
      for (size_t i = 0; i < L.n; ++i) L.x[i] = (TM)t[i];
      return;
    }
    std::fill(L.x.begin(), L.x.end(), TM(0));
    for (int i = 0; i < prm.smooth; ++i) smooth(L, b, i == 0);
    Level<TM>& C = lev[l + 1];
    const fsi3::Transfer3View tv = fsi3::view(C.T);
    spmv(L.h, L.A.data(), L.x.data(), b, L.r.data());
    for (int n = 0; n < C.h.n_nodes; ++n)
      for (int c = 0; c < 7; ++c)
        C.b[(size_t)n * 7 + c] = fsi3::restrict3(tv, L.h.node_flags.data(), C.h.node_flags.data(), L.r.data(), n, c);
    vcycle(l + 1, C.b.data());
    for (int n = 0; n < L.h.n_nodes; ++n)
      for (int c = 0; c < 7; ++c) L.x[(size_t)n * 7 + c] += fsi3::prolong3(tv, L.h.node_flags.data(), C.x.data(), n, c);
    for (int i = 0; i < prm.smooth; ++i) smooth(L, b, false);
  }

  static double dot(const std::vector<double>& a, const std::vector<double>& b) {
    return std::inner_product(a.begin(), a.end(), b.begin(), 0.0);
  }

  // FGMRES(m) for A64 x = b, x0 = 0; stop at ||b - A x|| <= max(rtol ||b||, abs_target).
  int fgmres(const std::vector<double>& b, std::vector<double>& x, double rtol, double abs_target) {
    const size_t n = b.size();
    const int m = prm.restart;
    x.assign(n, 0.0);
    const double bnorm = std::sqrt(dot(b, b));
    if (!(bnorm > 0.0)) return 0;
    const double target = std::max(rtol * bnorm, abs_target);
    std::vector<std::vector<double>> V(m + 1, std::vector<double>(n)), Z(m, std::vector<double>(n));
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), r(n), w(n), h(m + 1), h2(m + 1);
    int total = 0;
    while (true) {
      spmv(lev[0].h, A64.data(), x.data(), b.data(), r.data());
      const double beta = std::sqrt(dot(r, r));
      if (beta <= target) return 0;
      if (total >= prm.gmres_maxit) return -3;
      for (size_t i = 0; i < n; ++i) V[0][i] = r[i] / beta;
      std::fill(g.begin(), g.end(), 0.0);
      g[0] = beta;
      int j = 0;
      bool done = false;
      for (; j < m && total < prm.gmres_maxit; ++j) {
        ++total;
        ++gmres_its;
        std::vector<TM> vin(V[j].begin(), V[j].end());
        vcycle(0, vin.data());
        for (size_t i = 0; i < n; ++i) Z[j][i] = (double)lev[0].x[i];
        spmv<double>(lev[0].h, A64.data(), Z[j].data(), nullptr, w.data());
        for (int pass = 0; pass < 2; ++pass) {   // classical Gram-Schmidt, twice
          for (int i = 0; i <= j; ++i) h2[i] = dot(V[i], w);
          for (int i = 0; i <= j; ++i)
            for (size_t e = 0; e < n; ++e) w[e] -= h2[i] * V[i][e];
          for (int i = 0; i <= j; ++i) h[i] = pass ? h[i] + h2[i] : h2[i];
        }
        h[j + 1] = std::sqrt(dot(w, w));
        for (size_t e = 0; e < n; ++e) V[j + 1][e] = w[e] / h[j + 1];
        for (int i = 0; i < j; ++i) {   // earlier rotations
          const double a = h[i], c = h[i + 1];
          h[i] = cs[i] * a + sn[i] * c;
          h[i + 1] = -sn[i] * a + cs[i] * c;
        }
        const double den = std::hypot(h[j], h[j + 1]);
        cs[j] = h[j] / den;
        sn[j] = h[j + 1] / den;
        h[j] = den;
        h[j + 1] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = h[i];
        if (std::fabs(g[j + 1]) <= target) {
          ++j;
          done = true;
          break;
        }
      }
      std::vector<double> y(j);
      for (int i = j - 1; i >= 0; --i) {
        double acc = g[i];
        for (int q = i + 1; q < j; ++q) acc -= H[(size_t)i * m + q] * y[q];
        y[i] = acc / H[(size_t)i * m + i];
      }
      for (int i = 0; i < j; ++i)
        for (size_t e = 0; e < n; ++e) x[e] += y[i] * Z[i][e];
      if (done) {
        spmv(lev[0].h, A64.data(), x.data(), b.data(), r.data());
        if (std::sqrt(dot(r, r)) <= 1.01 * target) return 0;
      }
    }
  }
};

template <typename TM>
int theta_step(const double* const* br, const int* const* seg, const int* nseg, const double* box, const double* mat,
               const Params& prm, const double* Uold, double t_new, double k, double theta, double* Unew, int* stats) {
  Solver<TM> S{mat, prm, {}, {}, 0};
  S.build_levels(br, seg, nseg, box);
  const fsi3::HostMesh3& m = S.lev[0].h;
  const size_t n = S.lev[0].n;
  const fsi3::Mesh3View v = make_view(m);
  std::vector<double> U(Uold, Uold + n), R(n), b(n), x;
  for (int node = 0; node < m.n_nodes; ++node)
    for (int c = 0; c < 6; ++c)
      if (fsi3::identity_row3(m.node_flags[node], c)) U[(size_t)node * 7 + c] = fsi3::dirichlet3(v, node, c, t_new, mat[5], mat[6]);
  double r0 = 0.0;
  int it = 0;
  for (;; ++it) {
    residual(m, mat, U.data(), Uold, t_new, k, theta, R.data());
    const double nr = std::sqrt(Solver<TM>::dot(R, R));
    if (!std::isfinite(nr)) return -5;
    if (it == 0) r0 = nr;
    if (it >= 1 && nr <= prm.newton_tol * std::max(r0, 1.0)) break;
    if (it >= prm.newton_maxit) return -4;
    double rtol = prm.gmres_rtol, target = 0.0;
    if (prm.newton_eta > 0.0) {
      rtol = it == 0 ? std::max(prm.gmres_rtol, prm.gmres_rtol_first) : prm.gmres_rtol;
      if (it > 0) target = std::min(1e-2 * nr, prm.newton_eta * prm.newton_tol * std::max(r0, 1.0));
    }
    if (it == 0 || prm.reuse < 2) {
      const int rc = S.setup(U.data(), Uold, k, theta);   // with reuse 2 the first iterate's hierarchy is kept
      if (rc) return rc;
    } else {
      std::vector<double> A;   // exact Jacobian for the Krylov operator
      jacobian(m, mat, U.data(), Uold, k, theta, 1.0, A);
      S.A64 = A;
    }
    for (size_t i = 0; i < n; ++i) b[i] = -R[i];
    const int before = S.gmres_its;
    const int rc = S.fgmres(b, x, rtol, target);
    if (g_verbose)
      std::fprintf(stderr, "newton %d |R| %.3e rtol %.1e target %.3e fgmres %d rc %d\n", it, nr, rtol, target,
                   S.gmres_its - before, rc);
    if (rc) return rc;
    for (size_t i = 0; i < n; ++i) U[i] += x[i];
  }
  std::copy(U.begin(), U.end(), Unew);
  stats[0] = it;
  stats[1] = S.gmres_its;
  stats[2] = (int)S.lev.size();
  stats[3] = (int)S.lev.back().n;
  return 0;
}

}  // namespace

// One theta step t_new - k -> t_new of the 3D problem, solved as above. mat =
// {rho_f, nu_f, rho_s, mu_s, lambda_s, vbar, ramp_t, alpha0}; prm = {newton_tol,
// newton_maxit, gmres_restart, gmres_maxit, gmres_rtol, gmres_rtol_first,
// newton_eta, mg_coarsest_max_dofs, mg_smooth, mg_omega, mg_coarse_lps, mg_smoother, mg_coarse_sweeps,
// mg_reuse} (14 entries).
// precision 0: FP64 multigrid, 1: FP32 multigrid (FGMRES in FP64 either way).
// stats = {Newton iterations, FGMRES iterations, levels, coarsest dofs}.
// Returns 0, or -1/-2 singular coarsest/Vanka block, -3 FGMRES limit,
// -4 Newton limit, -5 non-finite residual.
extern "C" int fsi3_theta_step_host(const double* xb, const int* nxs, int nxseg, const double* yb, const int* nys,
                                    int nyseg, const double* zb, const int* nzs, int nzseg, const double* box,
                                    const double* mat, const double* prm_in, int precision, const double* Uold,
                                    double t_new, double k, double theta, double* Unew, int* stats) {
  const Params prm{prm_in[0], (int)prm_in[1], (int)prm_in[2], (int)prm_in[3], prm_in[4], prm_in[5],
                   prm_in[6], (int)prm_in[7], (int)prm_in[8], prm_in[9], prm_in[10], (int)prm_in[11],
                   (int)prm_in[12], (int)prm_in[13]};
  const double* br[3] = {xb, yb, zb};
  const int* seg[3] = {nxs, nys, nzs};
  const int nseg[3] = {nxseg, nyseg, nzseg};
  return precision ? theta_step<float>(br, seg, nseg, box, mat, prm, Uold, t_new, k, theta, Unew, stats)
                   : theta_step<double>(br, seg, nseg, box, mat, prm, Uold, t_new, k, theta, Unew, stats);
}

// Per-Newton-iteration lines on stderr (for experiments).
extern "C" void fsi3_host_verbose(int on) { g_verbose = on; }
