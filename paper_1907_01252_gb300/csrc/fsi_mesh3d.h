// Host-side tables of the 3D interface-fitted hexahedral Q2 mesh, and the
// per-node pieces of the 3D residual assembly written as __host__ __device__
// functions (the same code serves the CUDA kernels and host-side checks).
//
// Mesh (Sec. 2.2: the mesh resolves the interface): the channel is cut by
// break points on each axis into segments of uniform cells; cells whose centre
// lies in the solid box are solid. Q2 node grid (2nx+1) x (2ny+1) x (2nz+1),
// node id i + nnx (j + nny k) (x fastest); cell id cx + nx (cy + ny cz);
// local node a + 3 b + 9 c. Unknowns per node (v_x, v_y, v_z, u_x, u_y, u_z, p).
//
// Row rules of the assembled step residual (the same readings as in 2D):
//   momentum rows: all cells; velocity Dirichlet rows (inflow, lateral walls)
//     carry v - g(t);
//   displacement rows: nodes in the closure of the solid take the kinematic row
//     of solid cells, other nodes the harmonic row of fluid cells; u = 0 on the
//     whole outer boundary (identity rows u);
//   pressure rows: nodes touching a fluid cell take the divergence and
//     stabilisation rows of fluid cells; other pressure dofs carry p = 0.
// Inflow: v_x = s(t) 36 vbar (y - y0)(y1 - y)(z - z0)(z1 - z) / ((y1 - y0)^2 (z1 - z0)^2),
// s(t) = (1 - cos(pi t / ramp_t)) / 2 for t < ramp_t, else 1.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#ifdef __CUDACC__
#define FSI3M_HD __host__ __device__
#else
#define FSI3M_HD
#endif

namespace fsi3 {

enum : uint8_t { N3_DIR_V = 1, N3_DIR_U = 2, N3_P_ID = 4, N3_IN_SOLID = 8, N3_INFLOW = 16 };
// C3_U_DECOUPLED: a fluid cell none of whose nodes lies in the closure of the
// solid; its displacement rows are harmonic-extension or identity rows, which
// couple each displacement component only to itself.
enum : uint8_t { C3_SOLID = 1, C3_OUTFLOW = 2, C3_U_DECOUPLED = 4 };

struct HostMesh3 {
  int nx = 0, ny = 0, nz = 0, nnx = 0, nny = 0, nnz = 0, n_nodes = 0, n_cells = 0, nnzb = 0;
  std::vector<double> xn, yn, zn;     // node coordinates per axis
  std::vector<int> cell_nodes;        // [cell][27]
  std::vector<double> cell_h;         // [cell][3]
  std::vector<uint8_t> cell_flags, node_flags;
  std::vector<int> node_cells;        // [node][8]: cell * 27 + local, ascending cells, -1 padded
  std::vector<int> rowptr, colidx;    // node block pattern (nodes sharing a cell)
  std::vector<int> blk_row;           // [nnzb] row node of each block
  std::vector<int> blk_src;           // [nnzb][8]: cell * 729 + li * 27 + lj, ascending cells, -1 padded
  std::vector<int> cell_blk;          // [cell][27][27]: block of (local row node, local column node)
  double y0 = 0, y1 = 0, z0 = 0, z1 = 0;
};

inline std::vector<double> axis_vertices3(const double* br, const int* seg, int nseg) {
  std::vector<double> v{br[0]};
  for (int s = 0; s < nseg; ++s)
    for (int i = 1; i <= seg[s]; ++i) v.push_back(br[s] + (br[s + 1] - br[s]) * i / seg[s]);
  return v;
}

// box: {x0, x1, y0, y1, z0, z1} of the solid, or nullptr.
inline void build_mesh3(HostMesh3& m, const std::vector<double>& xv, const std::vector<double>& yv,
                        const std::vector<double>& zv, const double* box) {
  m.nx = (int)xv.size() - 1;
  m.ny = (int)yv.size() - 1;
  m.nz = (int)zv.size() - 1;
  m.nnx = 2 * m.nx + 1;
  m.nny = 2 * m.ny + 1;
  m.nnz = 2 * m.nz + 1;
  m.n_nodes = m.nnx * m.nny * m.nnz;
  m.n_cells = m.nx * m.ny * m.nz;
  auto nodes = [](const std::vector<double>& v) {
    std::vector<double> n(2 * (v.size() - 1) + 1);
    for (size_t i = 0; i + 1 < v.size(); ++i) {
      n[2 * i] = v[i];
      n[2 * i + 1] = 0.5 * (v[i] + v[i + 1]);
    }
    n.back() = v.back();
    return n;
  };
  m.xn = nodes(xv);
  m.yn = nodes(yv);
  m.zn = nodes(zv);
  m.y0 = yv.front();
  m.y1 = yv.back();
  m.z0 = zv.front();
  m.z1 = zv.back();
  m.cell_nodes.assign((size_t)m.n_cells * 27, 0);
  m.cell_h.assign((size_t)m.n_cells * 3, 0.0);
  m.cell_flags.assign(m.n_cells, 0);
  std::vector<char> in_solid(m.n_nodes, 0), in_fluid(m.n_nodes, 0);
  for (int cz = 0; cz < m.nz; ++cz)
    for (int cy = 0; cy < m.ny; ++cy)
      for (int cx = 0; cx < m.nx; ++cx) {
        const int c = cx + m.nx * (cy + m.ny * cz);
        for (int l = 0; l < 27; ++l) {
          const int a = l % 3, b = (l / 3) % 3, cc = l / 9;
          m.cell_nodes[(size_t)c * 27 + l] = (2 * cx + a) + m.nnx * ((2 * cy + b) + m.nny * (2 * cz + cc));
        }
        m.cell_h[c * 3] = xv[cx + 1] - xv[cx];
        m.cell_h[c * 3 + 1] = yv[cy + 1] - yv[cy];
        m.cell_h[c * 3 + 2] = zv[cz + 1] - zv[cz];
        const double xc = 0.5 * (xv[cx] + xv[cx + 1]), yc = 0.5 * (yv[cy] + yv[cy + 1]), zc = 0.5 * (zv[cz] + zv[cz + 1]);
        const bool solid = box && xc > box[0] && xc < box[1] && yc > box[2] && yc < box[3] && zc > box[4] && zc < box[5];
        m.cell_flags[c] = (solid ? C3_SOLID : 0) | (cx == m.nx - 1 ? C3_OUTFLOW : 0);
        for (int l = 0; l < 27; ++l) (solid ? in_solid : in_fluid)[m.cell_nodes[(size_t)c * 27 + l]] = 1;
      }
  m.node_flags.assign(m.n_nodes, 0);
  for (int k = 0; k < m.nnz; ++k)
    for (int j = 0; j < m.nny; ++j)
      for (int i = 0; i < m.nnx; ++i) {
        const int n = i + m.nnx * (j + m.nny * k);
        uint8_t f = 0;
        const bool wall = j == 0 || j == m.nny - 1 || k == 0 || k == m.nnz - 1;
        if (i == 0 || wall) f |= N3_DIR_V;
        if (i == 0 || i == m.nnx - 1 || wall) f |= N3_DIR_U;
        if (i == 0) f |= N3_INFLOW;
        if (in_solid[n]) f |= N3_IN_SOLID;
        if (!in_fluid[n]) f |= N3_P_ID;
        m.node_flags[n] = f;
      }
  for (int c = 0; c < m.n_cells; ++c) {
    bool dec = !(m.cell_flags[c] & C3_SOLID);
    for (int l = 0; l < 27 && dec; ++l) dec = !(m.node_flags[m.cell_nodes[(size_t)c * 27 + l]] & N3_IN_SOLID);
    if (dec) m.cell_flags[c] |= C3_U_DECOUPLED;
  }
  m.node_cells.assign((size_t)m.n_nodes * 8, -1);
  std::vector<int> cnt(m.n_nodes, 0);
  for (int c = 0; c < m.n_cells; ++c)
    for (int l = 0; l < 27; ++l) {
      const int n = m.cell_nodes[(size_t)c * 27 + l];
      m.node_cells[(size_t)n * 8 + cnt[n]++] = c * 27 + l;
    }
  std::vector<std::vector<int>> rows(m.n_nodes);
  for (int c = 0; c < m.n_cells; ++c)
    for (int li = 0; li < 27; ++li)
      for (int lj = 0; lj < 27; ++lj)
        rows[m.cell_nodes[(size_t)c * 27 + li]].push_back(m.cell_nodes[(size_t)c * 27 + lj]);
  m.rowptr.assign(m.n_nodes + 1, 0);
  m.colidx.clear();
  for (int n = 0; n < m.n_nodes; ++n) {
    auto& r = rows[n];
    std::sort(r.begin(), r.end());
    r.erase(std::unique(r.begin(), r.end()), r.end());
    m.colidx.insert(m.colidx.end(), r.begin(), r.end());
    m.rowptr[n + 1] = (int)m.colidx.size();
  }
  m.nnzb = (int)m.colidx.size();
  m.blk_row.assign(m.nnzb, 0);
  for (int n = 0; n < m.n_nodes; ++n)
    for (int b = m.rowptr[n]; b < m.rowptr[n + 1]; ++b) m.blk_row[b] = n;
  m.blk_src.assign((size_t)m.nnzb * 8, -1);
  m.cell_blk.assign((size_t)m.n_cells * 729, -1);
  std::vector<int> bcnt(m.nnzb, 0);
  for (int c = 0; c < m.n_cells; ++c)
    for (int li = 0; li < 27; ++li)
      for (int lj = 0; lj < 27; ++lj) {
        const int ni = m.cell_nodes[(size_t)c * 27 + li], nj = m.cell_nodes[(size_t)c * 27 + lj];
        const int b = (int)(std::lower_bound(m.colidx.begin() + m.rowptr[ni], m.colidx.begin() + m.rowptr[ni + 1], nj) -
                            m.colidx.begin());
        m.blk_src[(size_t)b * 8 + bcnt[b]++] = c * 729 + li * 27 + lj;
        m.cell_blk[(size_t)c * 729 + li * 27 + lj] = b;
      }
}

// Read-only view of the tables, as the kernels see them (device or host pointers).
struct Mesh3View {
  int nnx, nny, nnz, n_nodes, n_cells;
  const double *yn, *zn;
  const uint8_t *cell_flags, *node_flags;
  const int* node_cells;
  double y0, y1, z0, z1;
  const int *blk_row, *colidx, *blk_src;
  const int* cell_blk;
};

FSI3M_HD inline double inflow_ramp3(double t, double ramp_t) {
  return t < ramp_t ? 0.5 * (1.0 - cos(3.14159265358979323846 * t / ramp_t)) : 1.0;
}

// Boundary value of component c at node n and time t (zero except the inflow v_x).
FSI3M_HD inline double dirichlet3(const Mesh3View& m, int n, int c, double t, double vbar, double ramp_t) {
  if (c != 0 || !(m.node_flags[n] & N3_INFLOW)) return 0.0;
  const int j = (n / m.nnx) % m.nny, k = n / (m.nnx * m.nny);
  const double y = m.yn[j], z = m.zn[k];
  const double Ly = m.y1 - m.y0, Lz = m.z1 - m.z0;
  return inflow_ramp3(t, ramp_t) * 36.0 * vbar * (y - m.y0) * (m.y1 - y) * (z - m.z0) * (m.z1 - z) / (Ly * Ly * Lz * Lz);
}

FSI3M_HD inline bool identity_row3(uint8_t nf, int c) {
  if (c < 3) return nf & N3_DIR_V;
  if (c < 6) return nf & N3_DIR_U;
  return nf & N3_P_ID;
}

// Whether a cell's contribution enters row (node, c) (the row rules above).
FSI3M_HD inline bool row_takes3(uint8_t cf, uint8_t nf, int c) {
  const bool solid = cf & C3_SOLID;
  if (c < 3) return true;
  if (c < 6) return solid == bool(nf & N3_IN_SOLID);
  return !solid;
}

// Residual row (n, c) of one slice: the cell contributions Re[cell][27][7] in
// ascending cell order, or the identity row U - g(t) (p for the pressure).
FSI3M_HD inline double gather3(const Mesh3View& m, const double* Re, const double* U, int n, int c, double t,
                               double vbar, double ramp_t) {
  const uint8_t nf = m.node_flags[n];
  if (identity_row3(nf, c)) return U[(size_t)n * 7 + c] - dirichlet3(m, n, c, t, vbar, ramp_t);
  double acc = 0.0;
  for (int e = 0; e < 8; ++e) {
    const int code = m.node_cells[(size_t)n * 8 + e];
    if (code < 0) break;
    const int cell = code / 27, l = code % 27;
    if (row_takes3(m.cell_flags[cell], nf, c)) acc += Re[((size_t)cell * 27 + l) * 7 + c];
  }
  return acc;
}

// Entry (r, c) of Jacobian block b of one slice: the element matrices
// Ke[cell][189][189] of the cells sharing the block's two nodes, in ascending
// cell order, under the row rules; identity rows hold the unit diagonal.
FSI3M_HD inline double assemble3(const Mesh3View& m, const double* Ke, int b, int r, int c) {
  const int i = m.blk_row[b], j = m.colidx[b];
  const uint8_t nf = m.node_flags[i];
  if (identity_row3(nf, r)) return (i == j && r == c) ? 1.0 : 0.0;
  double acc = 0.0;
  for (int e = 0; e < 8; ++e) {
    const int code = m.blk_src[(size_t)b * 8 + e];
    if (code < 0) break;
    const int cell = code / 729, li = (code / 27) % 27, lj = code % 27;
    if (row_takes3(m.cell_flags[cell], nf, r)) acc += Ke[(size_t)cell * 189 * 189 + (size_t)(li * 7 + r) * 189 + lj * 7 + c];
  }
  return acc;
}

}  // namespace fsi3
