// GB300 library for Parareal time stepping of monolithic ALE fluid-structure
// interaction: host side (mesh hierarchy, tables, workspace, drivers, C ABI).
//
// The method follows Margenberg & Richter, "Parallel time-stepping for
// fluid-structure interactions": the ALE-FSI system of Sec. 2 discretised with
// equal-order Q2 elements and the shifted Crank-Nicolson step of Sec. 2.3; the
// Parareal iteration of Sec. 3. The paper leaves the linear solver open (it
// cites monolithic multigrid solvers); here every Newton step is solved by
// FGMRES preconditioned with a geometric multigrid V-cycle whose smoother is
// the cell-wise Vanka (local 45 x 45 solves) block smoother, coarse operators
// by rediscretisation on interface-fitted coarsened meshes.
//
// All slices of a batch advance together; every kernel works per slice with
// fixed reduction orders, so the result of a slice does not depend on the
// batch it ran in.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <condition_variable>
#include <system_error>
#include <thread>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/fsi.h"
#include "fsi_internal.h"
#include "fsi_mesh3d.h"
#include "fsi_kernels.cuh"

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define CK(call)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return fail(FSI_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));                  \
  } while (0)

#define TRY(call)                 \
  do {                            \
    int rc_ = (call);             \
    if (rc_ != FSI_OK) return rc_; \
  } while (0)

inline unsigned nblk(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

thread_local int g_nact = 0;   // active slices of the current launch sequence (work accounting only)

template <typename V>
int count_active(const V& v) {
  int n = 0;
  for (auto a : v) n += a != 0;
  return n;
}

// ---------------------------------------------------------------------------
// Host mesh of one multigrid level.
// ---------------------------------------------------------------------------
struct HostMesh {
  std::vector<double> xv, yv;   // vertices
  std::vector<int> xseg, yseg;  // cells per segment
  int nx = 0, ny = 0, nnx = 0, nny = 0, n_nodes = 0, n_cells = 0, nnzb = 0;
  std::vector<double> xn, yn;
  std::vector<int> cell_nodes;
  std::vector<double> cell_h;
  std::vector<uint8_t> cell_flags, node_flags;
  std::vector<double> node_y;
  std::vector<int> node_cells, rowptr, colidx, blk_row, blk_src, cell_blk, spmv_rows, blk_t;
  // multiplicative smoother: colour (cx%2 + 2 cy%2) -> its cells, its nodes and
  // the (cell, local node) each of those nodes belongs to
  std::vector<int> col_cells[4], col_nodes[4], col_src[4];
};

std::vector<double> axis_vertices(const std::vector<double>& breaks, const std::vector<int>& counts) {
  std::vector<double> v{breaks[0]};
  for (size_t s = 0; s < counts.size(); ++s)
    for (int i = 1; i <= counts[s]; ++i)
      v.push_back(i == counts[s] ? breaks[s + 1] : breaks[s] + (breaks[s + 1] - breaks[s]) * i / counts[s]);
  return v;
}

void build_mesh(HostMesh& m, bool has_solid, const double box[4]) {
  m.nx = (int)m.xv.size() - 1;
  m.ny = (int)m.yv.size() - 1;
  m.nnx = 2 * m.nx + 1;
  m.nny = 2 * m.ny + 1;
  m.n_nodes = m.nnx * m.nny;
  m.n_cells = m.nx * m.ny;
  m.xn.assign(m.nnx, 0.0);
  m.yn.assign(m.nny, 0.0);
  for (int i = 0; i <= m.nx; ++i) m.xn[2 * i] = m.xv[i];
  for (int i = 0; i < m.nx; ++i) m.xn[2 * i + 1] = 0.5 * (m.xv[i] + m.xv[i + 1]);
  for (int j = 0; j <= m.ny; ++j) m.yn[2 * j] = m.yv[j];
  for (int j = 0; j < m.ny; ++j) m.yn[2 * j + 1] = 0.5 * (m.yv[j] + m.yv[j + 1]);
  m.cell_nodes.assign(m.n_cells * 9, 0);
  m.cell_h.assign(m.n_cells * 2, 0.0);
  m.cell_flags.assign(m.n_cells, 0);
  std::vector<char> in_solid(m.n_nodes, 0), in_fluid(m.n_nodes, 0);
  for (int cy = 0; cy < m.ny; ++cy)
    for (int cx = 0; cx < m.nx; ++cx) {
      const int c = cy * m.nx + cx;
      for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a) m.cell_nodes[c * 9 + b * 3 + a] = (2 * cy + b) * m.nnx + 2 * cx + a;
      m.cell_h[c * 2] = m.xv[cx + 1] - m.xv[cx];
      m.cell_h[c * 2 + 1] = m.yv[cy + 1] - m.yv[cy];
      const double xc = 0.5 * (m.xv[cx] + m.xv[cx + 1]), yc = 0.5 * (m.yv[cy] + m.yv[cy + 1]);
      const bool solid = has_solid && xc > box[0] && xc < box[1] && yc > box[2] && yc < box[3];
      m.cell_flags[c] = (solid ? CF_SOLID : 0) | (cx == m.nx - 1 ? CF_OUTFLOW : 0);
      for (int l = 0; l < 9; ++l) (solid ? in_solid : in_fluid)[m.cell_nodes[c * 9 + l]] = 1;
    }
  m.node_flags.assign(m.n_nodes, 0);
  m.node_y.assign(m.n_nodes, 0.0);
  for (int j = 0; j < m.nny; ++j)
    for (int i = 0; i < m.nnx; ++i) {
      const int n = j * m.nnx + i;
      uint8_t f = 0;
      const bool wall = (j == 0 || j == m.nny - 1);
      if (i == 0 || wall) f |= NF_DIR_V;
      if (i == 0 || i == m.nnx - 1 || wall) f |= NF_DIR_U;
      if (i == 0) f |= NF_INFLOW;
      if (in_solid[n]) f |= NF_IN_SOLID;
      if (!in_fluid[n]) f |= NF_P_ID;
      m.node_flags[n] = f;
      m.node_y[n] = m.yn[j];
    }
  for (int c = 0; c < m.n_cells; ++c) {
    bool dec = !(m.cell_flags[c] & CF_SOLID);
    for (int l = 0; l < 9 && dec; ++l) dec = !(m.node_flags[m.cell_nodes[c * 9 + l]] & NF_IN_SOLID);
    if (dec) m.cell_flags[c] |= CF_U_DECOUPLED;
  }
  // node -> (cell, local) in ascending cell order
  m.node_cells.assign(m.n_nodes * 4, -1);
  std::vector<int> cnt(m.n_nodes, 0);
  for (int c = 0; c < m.n_cells; ++c)
    for (int l = 0; l < 9; ++l) {
      const int n = m.cell_nodes[c * 9 + l];
      m.node_cells[n * 4 + cnt[n]++] = c * 9 + l;
    }
  // block pattern: nodes sharing a cell
  std::vector<std::vector<int>> rows(m.n_nodes);
  for (int c = 0; c < m.n_cells; ++c)
    for (int li = 0; li < 9; ++li)
      for (int lj = 0; lj < 9; ++lj) rows[m.cell_nodes[c * 9 + li]].push_back(m.cell_nodes[c * 9 + lj]);
  m.rowptr.assign(m.n_nodes + 1, 0);
  m.colidx.clear();
  m.blk_row.clear();
  for (int n = 0; n < m.n_nodes; ++n) {
    auto& r = rows[n];
    std::sort(r.begin(), r.end());
    r.erase(std::unique(r.begin(), r.end()), r.end());
    for (int j : r) {
      m.colidx.push_back(j);
      m.blk_row.push_back(n);
    }
    m.rowptr[n + 1] = (int)m.colidx.size();
  }
  m.nnzb = (int)m.colidx.size();
  for (int k = 0; k < 4; ++k) {
    m.col_cells[k].clear();
    m.col_nodes[k].clear();
    m.col_src[k].clear();
  }
  for (int cy = 0; cy < m.ny; ++cy)
    for (int cx = 0; cx < m.nx; ++cx) {
      const int c = cy * m.nx + cx, k = (cx % 2) + 2 * (cy % 2);
      m.col_cells[k].push_back(c);
      for (int l = 0; l < 9; ++l) {
        m.col_nodes[k].push_back(m.cell_nodes[c * 9 + l]);
        m.col_src[k].push_back(c * 9 + l);
      }
    }
  m.blk_t.assign(m.nnzb, -1);
  for (int b = 0; b < m.nnzb; ++b) {
    const int i = m.blk_row[b], j = m.colidx[b];
    auto beg = m.colidx.begin() + m.rowptr[j], end = m.colidx.begin() + m.rowptr[j + 1];
    m.blk_t[b] = (int)(std::lower_bound(beg, end, i) - m.colidx.begin());
  }
  m.spmv_rows.resize(m.n_nodes);
  for (int n = 0; n < m.n_nodes; ++n) m.spmv_rows[n] = n;
  std::stable_sort(m.spmv_rows.begin(), m.spmv_rows.end(), [&](int a, int b) {
    return m.rowptr[a + 1] - m.rowptr[a] > m.rowptr[b + 1] - m.rowptr[b];
  });
  m.blk_src.assign((size_t)m.nnzb * 4, -1);
  m.cell_blk.assign(m.n_cells * 81, -1);
  std::vector<int> bcnt(m.nnzb, 0);
  for (int c = 0; c < m.n_cells; ++c)
    for (int li = 0; li < 9; ++li)
      for (int lj = 0; lj < 9; ++lj) {
        const int i = m.cell_nodes[c * 9 + li], j = m.cell_nodes[c * 9 + lj];
        auto beg = m.colidx.begin() + m.rowptr[i], end = m.colidx.begin() + m.rowptr[i + 1];
        const int b = (int)(std::lower_bound(beg, end, j) - m.colidx.begin());
        m.cell_blk[c * 81 + li * 9 + lj] = b;
        m.blk_src[(size_t)b * 4 + bcnt[b]++] = c * 81 + li * 9 + lj;
      }
}

// Coarsen one axis: pair cells inside each segment, keep the break points.
void coarsen_axis(const std::vector<double>& v, const std::vector<int>& seg, std::vector<double>& vc,
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

double lag2(int a, double s) {
  if (a == 0) return (1 - s) * (1 - 2 * s);
  if (a == 1) return 4 * s * (1 - s);
  return s * (2 * s - 1);
}

// 1D Q2 interpolation from coarse vertices vc to the Q2 nodes of fine vertices vf.
void prolong_1d(const std::vector<double>& vc, const std::vector<double>& xf, std::vector<int>& pidx,
                std::vector<double>& pw, std::vector<int>& ridx, std::vector<double>& rw) {
  const int nf = (int)xf.size(), nc = 2 * ((int)vc.size() - 1) + 1;
  pidx.assign(nf * 3, -1);
  pw.assign(nf * 3, 0.0);
  std::vector<std::vector<std::pair<int, double>>> cols(nc);
  for (int i = 0; i < nf; ++i) {
    const double x = xf[i];
    int cc = (int)(std::upper_bound(vc.begin(), vc.end(), x) - vc.begin()) - 1;
    cc = std::max(0, std::min(cc, (int)vc.size() - 2));
    const double s = (x - vc[cc]) / (vc[cc + 1] - vc[cc]);
    int e = 0;
    for (int a = 0; a < 3; ++a) {
      double w = lag2(a, s);
      if (std::fabs(w) < 1e-13) continue;
      if (std::fabs(w - 1.0) < 1e-13) w = 1.0;
      pidx[i * 3 + e] = 2 * cc + a;
      pw[i * 3 + e] = w;
      cols[2 * cc + a].push_back({i, w});
      ++e;
    }
  }
  ridx.assign(nc * 7, -1);
  rw.assign(nc * 7, 0.0);
  for (int I = 0; I < nc; ++I)
    for (size_t e = 0; e < cols[I].size() && e < 7; ++e) {
      ridx[I * 7 + e] = cols[I][e].first;
      rw[I * 7 + e] = cols[I][e].second;
    }
}

// ---------------------------------------------------------------------------
// Device level: tables, transfer from the next finer level, workspace.
// ---------------------------------------------------------------------------
constexpr int kSptRows[4] = {8, 16, 32, 64};   // tile heights of the row-tile block product
constexpr size_t kSptMaxSmem = 200 * 1024;     // largest staged tile (bytes)

struct Level {
  HostMesh h;
  DevMesh dm{};
  const int *col_cells[4] = {}, *col_nodes[4] = {}, *col_src[4] = {};
  const int* blk_t = nullptr;   // index of the transposed block
  Transfer T{};          // coarse = this level, fine = previous level (level >= 1)
  size_t n = 0;          // dofs
  std::vector<void*> owned;
  double *U = nullptr, *Uold = nullptr;       // injected states (level >= 1)
  double *KV = nullptr;                       // Vanka inverses (coarse levels: element matrices first)
  double *Ke = nullptr;                       // level 0: element matrices (kept apart from KV)
  double *A = nullptr;                        // block-sparse values
  double *cellbuf = nullptr, *r = nullptr, *x = nullptr, *b = nullptr;
  double *D = nullptr, *Dinv = nullptr;       // coarsest only
  float* A32 = nullptr;                       // level 0, mixed precision: the preconditioner's FP32 copy
  float2* Aff = nullptr;                      // FP64 operator as float pairs (float-float product)
  float2* xff = nullptr;                      // input vector of that product, as float pairs
  const void* aff_of = nullptr;               // the FP64 values Aff currently holds (nullptr: none)
  int* perm = nullptr;
  bool coarsest = false;
  // row-tile block product: blocks of the largest tile for each tile height of
  // kSptRows, and the tuned variant per value type (FP64, FP32, float pair) and
  // batch-size class (-1 not tuned yet, 0 the row-list kernel, t > 0 tile kSptRows[t - 1])
  int spt_blocks[4] = {};
  signed char spt_choice[3][4] = {{-1, -1, -1, -1}, {-1, -1, -1, -1}, {-1, -1, -1, -1}};
  int* async_status = nullptr;   // set when a bulk copy into shared memory did not complete
};

}  // namespace

namespace {

// ---------------------------------------------------------------------------
// Launch accounting: every kernel launch of the library goes through LAUNCH,
// which counts it and, when timing is enabled for its id, brackets it with
// CUDA events on the launching stream. Counters are process-wide atomics;
// timing records are kept under a mutex, so contexts driven by different host
// threads (the batch runner) can be counted and timed together.
// ---------------------------------------------------------------------------
enum KernelId {
  KI_ADD_BASIS,
  KI_APPLY_DIRICHLET,
  KI_ASSEMBLE_BSR,
  KI_AXPBY,
  KI_BACKSOLVE,
  KI_BSR_SPMV,
  KI_CELL_JACOBIAN,
  KI_CELL_RESIDUAL,
  KI_DENSE_APPLY,
  KI_DENSE_FROM_BSR,
  KI_DENSE_INVERT,
  KI_DOTS_FINISH,
  KI_DOTS_PARTIAL,
  KI_FILL,
  KI_GATHER_RESIDUAL,
  KI_GIVENS,
  KI_INIT_G,
  KI_INTERP_STATE,
  KI_PARAREAL_CORRECT,
  KI_PROLONG_ADD,
  KI_RESTRICT,
  KI_SCALE,
  KI_SUB_BASIS,
  KI_VANKA_CELL,
  KI_VANKA_GATHER,
  KI_VANKA_SETUP,
  KI_VANKA_SCATTER,
  KI_BSR_TRANSPOSE,
  KI_CELL_JACOBIAN_OLD,
  KI_CELL_DRES_DLAME,
  KI_GATHER_VECTOR,
  KI_DRES_DVBAR,
  KI_CELL_JACOBIAN_TC,
  KI_BSR_SPMV_FF,
  KI_TO_FF,
  KI_COUNT
};
const char* const kKernelNames[] = {"k_add_basis", "k_apply_dirichlet", "k_assemble_bsr", "k_axpby", "k_backsolve", "k_bsr_spmv", "k_cell_jacobian", "k_cell_residual", "k_dense_apply", "k_dense_from_bsr", "k_dense_invert", "k_dots_finish", "k_dots_partial", "k_fill", "k_gather_residual", "k_givens", "k_init_g", "k_interp_state", "k_parareal_correct", "k_prolong_add", "k_restrict", "k_scale", "k_sub_basis", "k_vanka_cell", "k_vanka_gather", "k_vanka_setup", "k_vanka_scatter", "k_bsr_transpose", "k_cell_jacobian_old", "k_cell_dres_dlame", "k_gather_vector", "k_dres_dvbar", "k_cell_jacobian_tc", "k_bsr_spmv_ff", "k_to_ff"};

struct Profiler {
  std::atomic<unsigned long long> mask{0};
  std::atomic<long long> launches[KI_COUNT] = {};
  std::atomic<long long> total{0};
  std::mutex mu;   // guards the members below
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<int> rec_id;
  std::vector<size_t> rec_ev;   // first of the record's two pool events
  std::vector<double> rec_work;
  std::vector<double> rec_bytes;
  // launches replayed inside CUDA graphs: summed after every replay
  double gms[KI_COUNT] = {}, gwork[KI_COUNT] = {}, gbytes[KI_COUNT] = {};
  long long gcnt[KI_COUNT] = {};
  std::atomic<unsigned> epoch{1};   // bumped by fsi_profile_enable: graphs captured earlier are re-captured
};
Profiler g_prof;
thread_local double g_pending_work = 0.0;   // algorithmic flops of the launch being issued
thread_local double g_pending_bytes = 0.0;  // algorithmic DRAM bytes of the launch being issued

// A timed launch recorded while a CUDA graph is being captured.
struct CapRec {
  int id;
  size_t ev;
  double work_per_slice;
  double bytes_per_slice;
};
struct Capture {
  bool on = false;
  int n_act = 1;
  std::vector<CapRec> recs;
  long long launches[KI_COUNT] = {};
};
thread_local Capture g_cap;

void prof_grow_pool_locked(size_t need) {
  while (g_prof.used + need > g_prof.pool.size()) {
    for (int i = 0; i < 256; ++i) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      g_prof.pool.push_back(e);
    }
  }
}

// Inside a stream capture a plain event record only orders streams; the
// external flag makes it an event-record node that replays can be timed by.
inline void prof_record(cudaEvent_t e, cudaStream_t st) {
  if (g_cap.on)
    cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
  else
    cudaEventRecord(e, st);
}

void prof_grow_pool(size_t need) {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  prof_grow_pool_locked(need);
}

constexpr size_t kNoEvent = ~size_t(0);

// Counts the launch; when its id is timed, reserves an event pair, records the
// first event and returns its index (kNoEvent otherwise).
inline size_t prof_pre(int id, cudaStream_t st) {
  if (g_cap.on) {
    g_cap.launches[id]++;
  } else {
    g_prof.launches[id].fetch_add(1, std::memory_order_relaxed);
    g_prof.total.fetch_add(1, std::memory_order_relaxed);
  }
  if (!(g_prof.mask.load(std::memory_order_relaxed) >> id & 1ull)) return kNoEvent;
  std::lock_guard<std::mutex> lk(g_prof.mu);
  prof_grow_pool_locked(2);
  const size_t ev = g_prof.used;
  g_prof.used += 2;
  prof_record(g_prof.pool[ev], st);
  return ev;
}
inline void prof_post(int id, size_t ev, cudaStream_t st) {
  if (ev == kNoEvent) return;
  std::lock_guard<std::mutex> lk(g_prof.mu);
  prof_record(g_prof.pool[ev + 1], st);
  if (g_cap.on) {
    g_cap.recs.push_back({id, ev, g_pending_work / std::max(1, g_cap.n_act),
                          g_pending_bytes / std::max(1, g_cap.n_act)});
  } else {
    g_prof.rec_id.push_back(id);
    g_prof.rec_ev.push_back(ev);
    g_prof.rec_work.push_back(g_pending_work);
    g_prof.rec_bytes.push_back(g_pending_bytes);
  }
}

// LAUNCH_W also records the algorithmic FP64 flops of the launch.
#define LAUNCH_W(work, id, kern, grid, block, smem, st, ...) \
  do {                                                       \
    g_pending_work = (work);                                 \
    LAUNCH(id, kern, grid, block, smem, st, __VA_ARGS__);    \
    g_pending_work = 0.0;                                    \
  } while (0)

// LAUNCH_WB records the flops and the algorithmic DRAM bytes (the data the
// launch must move at least once) of the launch.
#define LAUNCH_WB(work, bytes, id, kern, grid, block, smem, st, ...) \
  do {                                                               \
    g_pending_bytes = (bytes);                                       \
    LAUNCH_W(work, id, kern, grid, block, smem, st, __VA_ARGS__);    \
    g_pending_bytes = 0.0;                                           \
  } while (0)

#define LAUNCH(id, kern, grid, block, smem, st, ...) \
  do {                                               \
    const size_t ev_ = prof_pre(id, st);             \
    kern<<<grid, block, smem, st>>>(__VA_ARGS__);    \
    prof_post(id, ev_, st);                          \
  } while (0)

}  // namespace

struct fsi_ctx {
  fsi_params prm{};
  Phys P{};
  std::vector<Level> lev;
  int S = 0;            // max batch
  size_t n = 0;         // fine dofs
  int m = 0;            // FGMRES restart
  std::vector<void*> owned;
  double *Uit = nullptr, *Uold = nullptr, *R = nullptr, *dU = nullptr, *w = nullptr;
  double *V = nullptr, *Z = nullptr;
  double *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr;
  double *hcol = nullptr, *hcol2 = nullptr, *scal = nullptr, *resid = nullptr, *partial = nullptr;
  int *nv = nullptr, *status = nullptr;
  int* tc_status = nullptr;   // set by the tensor-core element Jacobian when an MMA completion was not seen
  uint8_t *active = nullptr, *active2 = nullptr;
  double* t_dev = nullptr;
  float *p_in = nullptr, *p_out = nullptr;   // FP32 preconditioner input / output (mixed precision)
  int n_act = 0;        // slices set in `active` (host mirror, for work accounting)
  int tip = -1;         // node at the top centre of the solid box (adjoint functional)
  // CUDA graphs of one FGMRES iteration for small batches, keyed by
  // (scalar sizes and transposition, batch, Krylov index); captured on an internal stream
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    unsigned epoch = 0;
    std::vector<CapRec> recs;
    long long launches[KI_COUNT] = {};
  };
  std::map<std::tuple<int, int, int>, Graph> graphs;
  cudaStream_t cap_stream = nullptr;
  // adjoint workspace (one slice)
  double *adj_ck = nullptr, *adj_sb = nullptr, *adj_vec = nullptr, *adj_B = nullptr, *adj_Bt = nullptr;
  size_t adj_ck_len = 0, adj_sb_len = 0;
  // Parareal workspace
  double *Cold = nullptr, *Fv = nullptr, *Cnew = nullptr, *ppart = nullptr;
  int red_blocks = 0;
  int pr_iter = -1;     // last completed iteration of the context's Parareal run (-1: none to continue)
  // pipelined Parareal: the sweeps run in a single-slice context of the same
  // mesh on their own stream; Uin holds the fine inputs of two iterations
  std::vector<double> mesh_xb, mesh_yb;
  std::vector<int> mesh_nx, mesh_ny;
  fsi_mesh mesh_desc{};
  fsi_ctx* sweep = nullptr;
  bool transposed = false;   // the multigrid hierarchy holds transposed operators (adjoint solves)
  // per-slice outcome: the last FGMRES solve's code per slice (0, FSI_ENAN, FSI_EGMRES), and the
  // index of the call's first slice within the caller's batch (fsi_stats.slice_status)
  std::vector<int> slice_code;
  int slice_offset = 0;
  cudaStream_t sweep_stream = nullptr;
  double* Uin = nullptr;
};

namespace {

template <typename T>
int dalloc(std::vector<void*>& own, T** p, size_t count) {
  void* q = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T));
  if (e != cudaSuccess) return fail(FSI_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  own.push_back(q);
  *p = (T*)q;
  return FSI_OK;
}

template <typename T>
int upload(std::vector<void*>& own, const T** p, const std::vector<T>& v) {
  T* q;
  TRY(dalloc(own, &q, v.size()));
  if (!v.empty()) CK(cudaMemcpy(q, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  *p = q;
  return FSI_OK;
}

int setup_level(Level& L, int S, bool coarsest, bool need_state, bool ff) {
  HostMesh& h = L.h;
  DevMesh& d = L.dm;
  d.nnx = h.nnx;
  d.nny = h.nny;
  d.n_nodes = h.n_nodes;
  d.n_cells = h.n_cells;
  d.nnzb = h.nnzb;
  TRY(upload(L.owned, &d.cell_nodes, h.cell_nodes));
  TRY(upload(L.owned, &d.cell_h, h.cell_h));
  TRY(upload(L.owned, &d.cell_flags, h.cell_flags));
  TRY(upload(L.owned, &d.node_flags, h.node_flags));
  TRY(upload(L.owned, &d.node_y, h.node_y));
  TRY(upload(L.owned, &d.node_cells, h.node_cells));
  TRY(upload(L.owned, &d.rowptr, h.rowptr));
  TRY(upload(L.owned, &d.colidx, h.colidx));
  TRY(upload(L.owned, &d.blk_row, h.blk_row));
  TRY(upload(L.owned, &d.blk_src, h.blk_src));
  TRY(upload(L.owned, &d.cell_blk, h.cell_blk));
  TRY(upload(L.owned, &d.spmv_rows, h.spmv_rows));
  for (int t = 0; t < 4; ++t) L.spt_blocks[t] = spmv_tile_max_blocks(h.rowptr.data(), h.n_nodes, kSptRows[t]);
  TRY(upload(L.owned, &L.blk_t, h.blk_t));
  for (int k = 0; k < 4; ++k) {
    TRY(upload(L.owned, &L.col_cells[k], h.col_cells[k]));
    TRY(upload(L.owned, &L.col_nodes[k], h.col_nodes[k]));
    TRY(upload(L.owned, &L.col_src[k], h.col_src[k]));
  }
  L.n = (size_t)h.n_nodes * 5;
  L.coarsest = coarsest;
  if (need_state) {
    TRY(dalloc(L.owned, &L.U, S * L.n));
    TRY(dalloc(L.owned, &L.Uold, S * L.n));
  }
  TRY(dalloc(L.owned, &L.KV, (size_t)S * h.n_cells * 2025));
  if (!need_state) TRY(dalloc(L.owned, &L.Ke, (size_t)S * h.n_cells * 2025));
  else L.Ke = L.KV;
  TRY(dalloc(L.owned, &L.A, (size_t)S * h.nnzb * 25));
  if (ff) {
    TRY(dalloc(L.owned, &L.Aff, (size_t)S * h.nnzb * 25));
    TRY(dalloc(L.owned, &L.xff, (size_t)S * h.n_nodes * 5));
  }
  if (!need_state) TRY(dalloc(L.owned, &L.A32, (size_t)S * h.nnzb * 25));
  TRY(dalloc(L.owned, &L.cellbuf, (size_t)S * h.n_cells * 45));
  TRY(dalloc(L.owned, &L.r, S * L.n));
  TRY(dalloc(L.owned, &L.x, S * L.n));
  TRY(dalloc(L.owned, &L.b, S * L.n));
  if (coarsest) {
    TRY(dalloc(L.owned, &L.D, (size_t)S * L.n * L.n));
    TRY(dalloc(L.owned, &L.Dinv, (size_t)S * L.n * L.n));
    TRY(dalloc(L.owned, &L.perm, (size_t)S * L.n));
  }
  return FSI_OK;
}

int setup_transfer(Level& C, const Level& F) {
  std::vector<int> pxi, pyi, rxi, ryi, ixi, iyi, d0;
  std::vector<double> pxw, pyw, rxw, ryw, ixw, iyw, d1;
  prolong_1d(C.h.xv, F.h.xn, pxi, pxw, rxi, rxw);   // coarse -> fine nodes and its transpose
  prolong_1d(C.h.yv, F.h.yn, pyi, pyw, ryi, ryw);
  prolong_1d(F.h.xv, C.h.xn, ixi, ixw, d0, d1);     // fine field at the coarse nodes
  prolong_1d(F.h.yv, C.h.yn, iyi, iyw, d0, d1);
  Transfer& T = C.T;
  T.nnx_f = F.h.nnx;
  T.nny_f = F.h.nny;
  T.nnx_c = C.h.nnx;
  T.nny_c = C.h.nny;
  TRY(upload(C.owned, &T.px_idx, pxi));
  TRY(upload(C.owned, &T.px_w, pxw));
  TRY(upload(C.owned, &T.py_idx, pyi));
  TRY(upload(C.owned, &T.py_w, pyw));
  TRY(upload(C.owned, &T.rx_idx, rxi));
  TRY(upload(C.owned, &T.rx_w, rxw));
  TRY(upload(C.owned, &T.ry_idx, ryi));
  TRY(upload(C.owned, &T.ry_w, ryw));
  TRY(upload(C.owned, &T.ix_idx, ixi));
  TRY(upload(C.owned, &T.ix_w, ixw));
  TRY(upload(C.owned, &T.iy_idx, iyi));
  TRY(upload(C.owned, &T.iy_w, iyw));
  return FSI_OK;
}

// Reference-cell tables: 3-point Gauss rule on [0, 1], Q2 basis, Q1 vertex
// projection for the local projection stabilisation.
int upload_tables_once();

// The basis tables live in constant memory: uploaded once per device and
// process (contexts set up from several host threads share them).
int upload_tables() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  CK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  if (dev >= 0 && dev < 64 && done[dev]) return FSI_OK;
  TRY(upload_tables_once());
  CK(cudaStreamSynchronize(cudaStreamLegacy));
  if (dev >= 0 && dev < 64) done[dev] = true;
  return FSI_OK;
}

int upload_tables_once() {
  const double gp[3] = {0.5 - std::sqrt(0.15), 0.5, 0.5 + std::sqrt(0.15)};
  const double gw[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
  auto L = [](int a, double s) { return lag2(a, s); };
  auto dL = [](int a, double s) { return a == 0 ? 4 * s - 3 : (a == 1 ? 4 - 8 * s : 4 * s - 1); };
  double phi[9][9], dps[9][9], dpt[9][9], wq[9], phie[3][9], dpse[3][9], dpte[3][9];
  for (int q2 = 0; q2 < 3; ++q2)
    for (int q1 = 0; q1 < 3; ++q1) {
      const int q = q2 * 3 + q1;
      wq[q] = gw[q1] * gw[q2];
      for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a) {
          const int l = b * 3 + a;
          phi[q][l] = L(a, gp[q1]) * L(b, gp[q2]);
          dps[q][l] = dL(a, gp[q1]) * L(b, gp[q2]);
          dpt[q][l] = L(a, gp[q1]) * dL(b, gp[q2]);
        }
    }
  for (int q = 0; q < 3; ++q)
    for (int b = 0; b < 3; ++b)
      for (int a = 0; a < 3; ++a) {
        const int l = b * 3 + a;
        phie[q][l] = L(a, 1.0) * L(b, gp[q]);
        dpse[q][l] = dL(a, 1.0) * L(b, gp[q]);
        dpte[q][l] = L(a, 1.0) * dL(b, gp[q]);
      }
  // kappa(phi_l) = phi_l - pi1(phi_l); pi1 phi_l = Q1 vertex function for vertex nodes
  double kss[9][9] = {}, ktt[9][9] = {};
  for (int q = 0; q < 9; ++q) {
    const double s = gp[q % 3], t = gp[q / 3];
    double gs[9], gt[9];
    for (int l = 0; l < 9; ++l) {
      const int a = l % 3, b = l / 3;
      gs[l] = dps[q][l];
      gt[l] = dpt[q][l];
      if (a != 1 && b != 1) {
        const double Ns = a == 0 ? 1 - s : s, Nt = b == 0 ? 1 - t : t;
        const double dNs = a == 0 ? -1.0 : 1.0, dNt = b == 0 ? -1.0 : 1.0;
        gs[l] -= dNs * Nt;
        gt[l] -= Ns * dNt;
      }
    }
    for (int i = 0; i < 9; ++i)
      for (int j = 0; j < 9; ++j) {
        kss[i][j] += wq[q] * gs[i] * gs[j];
        ktt[i][j] += wq[q] * gt[i] * gt[j];
      }
  }
  CK(cudaMemcpyToSymbol(c_phi, phi, sizeof(phi)));
  CK(cudaMemcpyToSymbol(c_dps, dps, sizeof(dps)));
  CK(cudaMemcpyToSymbol(c_dpt, dpt, sizeof(dpt)));
  CK(cudaMemcpyToSymbol(c_wq, wq, sizeof(wq)));
  CK(cudaMemcpyToSymbol(c_phie, phie, sizeof(phie)));
  CK(cudaMemcpyToSymbol(c_dpse, dpse, sizeof(dpse)));
  CK(cudaMemcpyToSymbol(c_dpte, dpte, sizeof(dpte)));
  CK(cudaMemcpyToSymbol(c_we, gw, sizeof(gw)));
  CK(cudaMemcpyToSymbol(c_lps_ss, kss, sizeof(kss)));
  CK(cudaMemcpyToSymbol(c_lps_tt, ktt, sizeof(ktt)));
  TabF tf;
  for (int q = 0; q < 9; ++q) {
    tf.wq[q] = (float)wq[q];
    for (int l = 0; l < 9; ++l) {
      tf.phi[q][l] = (float)phi[q][l];
      tf.dps[q][l] = (float)dps[q][l];
      tf.dpt[q][l] = (float)dpt[q][l];
      tf.lss[q][l] = (float)kss[q][l];
      tf.ltt[q][l] = (float)ktt[q][l];
    }
  }
  for (int q = 0; q < 3; ++q) {
    tf.we[q] = (float)gw[q];
    for (int l = 0; l < 9; ++l) {
      tf.phie[q][l] = (float)phie[q][l];
      tf.dpse[q][l] = (float)dpse[q][l];
      tf.dpte[q][l] = (float)dpte[q][l];
    }
  }
  CK(cudaMemcpyToSymbol(g_tabf, &tf, sizeof(tf)));
  return FSI_OK;
}



// ---------------------------------------------------------------------------
// Batched building blocks
// ---------------------------------------------------------------------------
int launch_check() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(FSI_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return FSI_OK;
}

int residual(fsi_ctx* c, Level& L, int S, const double* U, const double* Uold, double k, double theta,
             const uint8_t* act, double* R, cudaStream_t st) {
  LAUNCH(KI_CELL_RESIDUAL, k_cell_residual, (dim3(nblk(L.h.n_cells, 128), S)), 128, 0, st, L.dm, c->P, U, Uold, L.n, k, theta, act, L.cellbuf);
  LAUNCH(KI_GATHER_RESIDUAL, k_gather_residual, (dim3(nblk(L.h.n_nodes, 128), S)), 128, 0, st, L.dm, c->P, L.cellbuf, U, L.n, c->t_dev, act, R);
  return launch_check();
}

// Mixed precision: FP64 Krylov solver with an FP32 multigrid preconditioner.
template <typename T>
bool mixed(const fsi_ctx* c) {
  return sizeof(T) == sizeof(float) && c->prm.precision == 2;
}

// lps_scale = 1 on the finest level (the discretisation); coarse levels of the
// preconditioner scale the stabilisation weight down (see mg_coarse_lps).
// The tangent is FP64; the element contraction, the element matrices and the
// assembled values are in T.
template <typename T>
int jacobian(fsi_ctx* c, Level& L, int S, const double* U, const double* Uold, double k, double theta,
             const uint8_t* act, T* A, cudaStream_t st, double lps_scale = 1.0) {
  if (sizeof(T) == sizeof(float) && c->prm.tc_contraction) {
    // FP32 element matrices: the contraction on the tensor cores
    CK(cudaFuncSetAttribute((const void*)k_cell_jacobian_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, JTC_SMEM));
    LAUNCH_W(2.0 * 9 * (2025 + 675) * 3 * L.h.n_cells * (double)c->n_act, KI_CELL_JACOBIAN_TC, k_cell_jacobian_tc, (dim3(L.h.n_cells, S)), JAC_THREADS, JTC_SMEM, st, L.dm, c->P, U, Uold, L.n, k, theta, lps_scale, act, reinterpret_cast<float*>(L.Ke), c->tc_status);
    LAUNCH(KI_ASSEMBLE_BSR, (k_assemble_bsr<T, T>), (dim3(nblk((size_t)L.h.nnzb * 5, 128), S)), 128, 0, st, L.dm, reinterpret_cast<const T*>(L.Ke), act, A, 1.0);
    if ((const void*)A == (const void*)L.A) L.aff_of = nullptr;
    return launch_check();
  }
  LAUNCH_W(2.0 * 9 * (2025 + 675) * 3 * L.h.n_cells * (double)c->n_act, KI_CELL_JACOBIAN, (k_cell_jacobian<false, T>), (dim3(L.h.n_cells, S)), JAC_THREADS, 0, st, L.dm, c->P, U, Uold, L.n, k, theta, lps_scale, act, reinterpret_cast<T*>(L.Ke));
  LAUNCH(KI_ASSEMBLE_BSR, (k_assemble_bsr<T, T>), (dim3(nblk((size_t)L.h.nnzb * 5, 128), S)), 128, 0, st, L.dm, reinterpret_cast<const T*>(L.Ke), act, A, 1.0);
  if ((const void*)A == (const void*)L.A) {
    L.aff_of = nullptr;
    if (sizeof(T) == sizeof(double) && L.Aff) {   // the float-pair copy for the operator products
      const size_t cnt = (size_t)L.h.nnzb * 25;
      LAUNCH_WB(3.0 * cnt * c->n_act, 16.0 * cnt * c->n_act, KI_TO_FF, k_to_ff, (dim3(nblk(cnt, 256), S)), 256, 0, st, cnt, reinterpret_cast<const double*>(A), cnt, act, L.Aff, cnt);
      L.aff_of = A;
    }
  }
  return launch_check();
}

// The dynamic shared-memory limit of a kernel is one setting per kernel and device,
// shared by every context and host thread: it is only ever raised (to the largest
// size launched so far), never set to a launch's own size, which a launch or a
// captured graph of another thread could exceed. (Setting it is not a stream
// operation, so it may also happen while a stream is being captured.)
void raise_smem_limit(const void* fn, size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> limit;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = limit[{fn, dev}];
  if (smem <= cur) return;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess) cur = smem;
  else (void)cudaGetLastError();   // the launch then reports the error
}

// One launch of the row-tile product with tile index t (1..4) or, for t = 0,
// the row-list kernel of the same value type (bit-identical results).
template <typename V, typename Y, bool RES, int ROWS>
void spt_launch(Level& L, int S, const V* A, const V* x, const Y* b, const uint8_t* act, Y* y, cudaStream_t st,
                double work, double bytes, int ki, int t) {
  const size_t smem = spmv_tile_smem<V>(L.spt_blocks[t - 1]);
  if (smem > 48 * 1024) {   // both forms (y = A x and y = b - A x) share the tuned choice
    raise_smem_limit(reinterpret_cast<const void*>(k_bsr_spmv_tile<V, Y, false, ROWS>), smem);
    raise_smem_limit(reinterpret_cast<const void*>(k_bsr_spmv_tile<V, Y, true, ROWS>), smem);
  }
  LAUNCH_WB(work, bytes, ki, (k_bsr_spmv_tile<V, Y, RES, ROWS>), (dim3(nblk(L.h.n_nodes, ROWS), S)), ROWS * 5, smem, st,
            L.dm, A, x, b, L.n, act, y, L.async_status);
}

template <typename V, typename Y, bool RES>
void spt_run(Level& L, int S, const V* A, const V* x, const Y* b, const uint8_t* act, Y* y, cudaStream_t st,
             double work, double bytes, int ki, int t) {
  const int* rows = L.dm.spmv_rows;
  const int nrows = L.h.n_nodes;
  switch (t) {
    case 0:
      if constexpr (std::is_same<V, float2>::value)
        LAUNCH_WB(work, bytes, ki, k_bsr_spmv_ff<RES>, (dim3(nblk((size_t)nrows * 5, 128), S)), 128, 0, st, L.dm, A, x, b,
                  L.n, act, y, rows, nrows);
      else
        LAUNCH_WB(work, bytes, ki, (k_bsr_spmv<V, RES>), (dim3(nblk((size_t)nrows * 5, 128), S)), 128, 0, st, L.dm, A, x,
                  b, L.n, act, y, rows, nrows);
      break;
    case 1: spt_launch<V, Y, RES, 8>(L, S, A, x, b, act, y, st, work, bytes, ki, t); break;
    case 2: spt_launch<V, Y, RES, 16>(L, S, A, x, b, act, y, st, work, bytes, ki, t); break;
    case 3: spt_launch<V, Y, RES, 32>(L, S, A, x, b, act, y, st, work, bytes, ki, t); break;
    default: spt_launch<V, Y, RES, 64>(L, S, A, x, b, act, y, st, work, bytes, ki, t); break;
  }
}

// The product over all rows, in the variant tuned for this level, value type and
// batch-size class. The first call of a class that is not inside a stream capture
// (and whose output overlaps neither input) times every variant whose tile fits
// in shared memory, three launches each, and keeps the fastest; all variants give
// the same bits, so the choice never changes a result.
template <typename V, typename Y, bool RES>
int spt_product(Level& L, int S, const V* A, const V* x, const Y* b, const uint8_t* act, Y* y, cudaStream_t st,
                double work, double bytes, int ki) {
  const int type = std::is_same<V, double>::value ? 0 : std::is_same<V, float>::value ? 1 : 2;
  const int cls = S <= 1 ? 0 : S <= 4 ? 1 : S <= 16 ? 2 : 3;
  signed char& choice = L.spt_choice[type][cls];
  auto fits = [&](int t) { return t == 0 || spmv_tile_smem<V>(L.spt_blocks[t - 1]) <= kSptMaxSmem; };
  if (choice < 0) {
    const bool aliased = (const void*)y == (const void*)x || (RES && (const void*)y == (const void*)b);
    if (g_cap.on || aliased) {   // no timing here: the row-list kernel, untuned
      spt_run<V, Y, RES>(L, S, A, x, b, act, y, st, work, bytes, ki, 0);
      return launch_check();
    }
    cudaEvent_t ev[2];
    CK(cudaEventCreate(&ev[0]));
    CK(cudaEventCreate(&ev[1]));
    float best = 0.0f;
    int best_t = 0;
    for (int t = 0; t <= 4; ++t) {
      if (!fits(t)) continue;
      spt_run<V, Y, RES>(L, S, A, x, b, act, y, st, work, bytes, ki, t);   // warm-up
      cudaEventRecord(ev[0], st);
      for (int r = 0; r < 2; ++r) spt_run<V, Y, RES>(L, S, A, x, b, act, y, st, work, bytes, ki, t);
      cudaEventRecord(ev[1], st);
      TRY(launch_check());
      CK(cudaEventSynchronize(ev[1]));
      float ms = 0.0f;
      CK(cudaEventElapsedTime(&ms, ev[0], ev[1]));
      if (t == 0 || ms < best) best = ms, best_t = t;
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    choice = (signed char)best_t;
    if (std::getenv("FSI_TRACE_TUNE"))
      std::fprintf(stderr, "[fsi tune] level n=%zu type %d class %d: variant %d (%.3f ms per launch)\n", L.n, type,
                   cls, best_t, best / 2.0f);
    return FSI_OK;   // y holds the product of the last timed launch
  }
  spt_run<V, Y, RES>(L, S, A, x, b, act, y, st, work, bytes, ki, choice);
  return launch_check();
}

template <typename T, bool RES>
int spmv(Level& L, int S, const T* A, const T* x, const T* b, const uint8_t* act, T* y, cudaStream_t st,
         const int* rows = nullptr, int nrows = -1) {
  const bool all_rows = !rows;
  if (!rows) {
    rows = L.dm.spmv_rows;
    nrows = L.h.n_nodes;
  }
  const double blocks = nrows == L.h.n_nodes ? (double)L.h.nnzb : (double)L.h.nnzb * nrows / L.h.n_nodes;
  // per active slice: the blocks, x, y (and b); once per launch: the row list, row pointers and column indices
  const double bytes = (double)g_nact * sizeof(T) * (25.0 * blocks + (double)L.n + (RES ? 10.0 : 5.0) * nrows) +
                       4.0 * (blocks + 2.0 * nrows + 1.0);
  const double work = 50.0 * blocks * (double)g_nact;
  if (sizeof(T) == sizeof(double) && L.Aff && L.aff_of == (const void*)A) {
    // the FP64 operator as float pairs: x to float pairs, then the compensated FP32 product
    LAUNCH_WB(3.0 * (double)L.n * g_nact, 16.0 * (double)L.n * g_nact, KI_TO_FF, k_to_ff, (dim3(nblk(L.n, 256), S)), 256, 0, st, L.n, reinterpret_cast<const double*>(x), L.n, act, L.xff, L.n);
    if (all_rows)
      return spt_product<float2, double, RES>(L, S, L.Aff, L.xff, reinterpret_cast<const double*>(b), act,
                                              reinterpret_cast<double*>(y), st, work, bytes, KI_BSR_SPMV_FF);
    LAUNCH_WB(work, bytes, KI_BSR_SPMV_FF, k_bsr_spmv_ff<RES>, (dim3(nblk((size_t)nrows * 5, 128), S)), 128, 0, st, L.dm, L.Aff, L.xff, reinterpret_cast<const double*>(b), L.n, act, reinterpret_cast<double*>(y), rows, nrows);
    return launch_check();
  }
  if (all_rows) return spt_product<T, T, RES>(L, S, A, x, b, act, y, st, work, bytes, KI_BSR_SPMV);
  LAUNCH_WB(work, bytes, KI_BSR_SPMV, (k_bsr_spmv<T, RES>), (dim3(nblk((size_t)nrows * 5, 128), S)), 128, 0, st, L.dm, A, x, b, L.n, act, y, rows, nrows);
  return launch_check();
}

// Norms or dot products with fixed reduction order: out[s*ostride + i] = V_i . w
template <typename T>
int dots(fsi_ctx* c, int S, size_t n, int nv, const T* V, size_t vstride, size_t vslice, const T* w,
         size_t wstride, const uint8_t* act, double* out, int ostride, bool take_sqrt, cudaStream_t st) {
  const int nb = (int)nblk(n, RED_CHUNK);
  LAUNCH_W(2.0 * nv * (double)n * c->n_act, KI_DOTS_PARTIAL, k_dots_partial<T>, (dim3(nb, S)), RED_THREADS, 0, st, (int)n, nv, V, vstride, vslice, w, wstride, act, c->partial, 64);
  LAUNCH(KI_DOTS_FINISH, k_dots_finish, (S), 64, 0, st, nb, nv, c->partial, 64, act, out, ostride, take_sqrt, false);
  return launch_check();
}

// Multigrid setup for the Newton iterate U (level 0) and old state Uold; the
// preconditioner's matrices and inverses are stored in T.
// Inverse of S dense n x n matrices (the coarsest multigrid level): on a
// thread-block cluster when its rows fit in the cluster's shared memory, else
// on one CTA per slice with the matrix in global memory. D is overwritten.
template <typename T>
int dense_invert(int S, int n, T* D, int* perm, const uint8_t* act, T* inv, int* status, cudaStream_t st,
                 int force_single = 0) {
  const size_t smem = gjc_smem_bytes<T>(n);
  if (!force_single && smem <= 200 * 1024) {
    CK(cudaFuncSetAttribute((const void*)k_dense_invert_cluster<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)smem));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(GJC_CTAS, S);
    cfg.blockDim = dim3(GJC_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = GJC_CTAS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const size_t ev = prof_pre(KI_DENSE_INVERT, st);
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_dense_invert_cluster<T>, n, (const T*)D, act, inv, status);
    prof_post(KI_DENSE_INVERT, ev, st);
    if (e != cudaSuccess) return fail(FSI_ECUDA, std::string("cluster launch: ") + cudaGetErrorString(e));
    return launch_check();
  }
  LAUNCH(KI_DENSE_INVERT, k_dense_invert<T>, (S), GJ_THREADS, n * sizeof(T), st, n, D, perm, act, inv, status);
  return launch_check();
}

template <typename T>
int mg_setup(fsi_ctx* c, int S, const double* U, const double* Uold, double k, double theta, const uint8_t* act,
             cudaStream_t st, bool keep_coarsest = false, bool transpose = false) {
  const int NL = (int)c->lev.size();
  c->transposed = transpose;
  const double* Ul = U;
  const double* Uol = Uold;
  for (int l = 0; l < NL; ++l) {
    Level& L = c->lev[l];
    if (l > 0) {
      const Level& F = c->lev[l - 1];
      LAUNCH(KI_INTERP_STATE, k_interp_state, (dim3(nblk(L.n, 128), S)), 128, 0, st, L.T, Ul, F.n, L.n, act, L.U);
      LAUNCH(KI_INTERP_STATE, k_interp_state, (dim3(nblk(L.n, 128), S)), 128, 0, st, L.T, Uol, F.n, L.n, act, L.Uold);
      Ul = L.U;
      Uol = L.Uold;
    }
    T* A = reinterpret_cast<T*>(L.A);
    if (l == 0 && mixed<T>(c)) {
      // FP64 operator for the Krylov solver, FP32 copy for the preconditioner
      TRY(jacobian<double>(c, L, S, Ul, Uol, k, theta, act, L.A, st));
      LAUNCH(KI_ASSEMBLE_BSR, (k_assemble_bsr<float, double>), (dim3(nblk((size_t)L.h.nnzb * 5, 128), S)), 128, 0, st, L.dm, L.Ke, act, L.A32, 1.0);
      A = reinterpret_cast<T*>(L.A32);
    } else {
      TRY(jacobian<T>(c, L, S, Ul, Uol, k, theta, act, A, st, std::pow(c->prm.mg_coarse_lps, l)));
    }
    if (transpose) {   // the hierarchy of the transposed operator (adjoint solves, FP64 only)
      double* Ad = reinterpret_cast<double*>(A);
      LAUNCH(KI_BSR_TRANSPOSE, k_bsr_transpose, (dim3(nblk((size_t)L.h.nnzb * 25, 256), S)), 256, 0, st, L.h.nnzb, L.blk_t, Ad, act, L.Ke);
      CK(cudaMemcpyAsync(Ad, L.Ke, (size_t)S * L.h.nnzb * 25 * sizeof(double), cudaMemcpyDeviceToDevice, st));
      L.aff_of = nullptr;   // the float pairs hold the untransposed operator
    }
    if (L.coarsest) {
      if (keep_coarsest) continue;   // inverse of an earlier Newton iteration of this step
      const int n = (int)L.n;
      T* D = reinterpret_cast<T*>(L.D);
      LAUNCH(KI_DENSE_FROM_BSR, k_dense_from_bsr<T>, (dim3(nblk((size_t)n * n, 256), S)), 256, 0, st, L.dm, A, act, D);
      TRY(dense_invert<T>(S, n, D, L.perm, act, reinterpret_cast<T*>(L.Dinv), c->status, st));
    } else {
      LAUNCH_W(2.0 * 45 * 45 * 45 * L.h.n_cells * (double)c->n_act, KI_VANKA_SETUP, k_vanka_setup<T>, (dim3(L.h.n_cells, S)), VK_THREADS, 0, st, L.dm, A, act, reinterpret_cast<T*>(L.KV), c->status);
    }
    TRY(launch_check());
  }
  return FSI_OK;
}

// x = M_l^{-1} b : one V-cycle with Vanka smoothing, x is overwritten.
template <typename T>
int vcycle(fsi_ctx* c, int l, int S, const T* b, T* x, const uint8_t* act, cudaStream_t st) {
  Level& L = c->lev[l];
  const T* A = (l == 0 && mixed<T>(c)) ? reinterpret_cast<const T*>(L.A32) : reinterpret_cast<const T*>(L.A);
  T* r = reinterpret_cast<T*>(L.r);
  T* cellbuf = reinterpret_cast<T*>(L.cellbuf);
  if (L.coarsest) {
    LAUNCH(KI_DENSE_APPLY, k_dense_apply<T>, (dim3(nblk(L.n * 32, 256), S)), 256, 0, st, (int)L.n, reinterpret_cast<const T*>(L.Dinv), b, L.n, act, x);
    return launch_check();
  }
  const int nu = c->prm.mg_smooth;
  const double om = c->prm.mg_omega;
  LAUNCH(KI_FILL, k_fill<T>, (dim3(nblk(L.n, 256), S)), 256, 0, st, (int)L.n, 0.0, act, x, L.n);
  auto smooth = [&](bool first) -> int {
    if (c->prm.mg_smoother == 1) {
      // multiplicative: colour by colour, residual only on the colour's nodes
      for (int k = 0; k < 4; ++k) {
        const int nn = (int)L.h.col_nodes[k].size(), nc = (int)L.h.col_cells[k].size();
        if (nc == 0) continue;
        const T* rr = b;
        if (!(first && k == 0)) {
          TRY((spmv<T, true>(L, S, A, x, b, act, r, st, L.col_nodes[k], nn)));
          rr = r;
        }
        if (c->transposed)   // transposed operators lack the displacement-row structure
          LAUNCH_W(2.0 * 2025 * nc * (double)c->n_act, KI_VANKA_CELL, k_vanka_cell<T>, (dim3(nblk((size_t)nc * 45, 128), S)), 128, 0, st, L.dm, reinterpret_cast<const T*>(L.KV), rr, L.n, act, cellbuf, L.col_cells[k], nc);
        else
        LAUNCH_W(2.0 * 2025 * nc * (double)c->n_act, KI_VANKA_CELL, k_vanka_cell_split<T>, (dim3(nblk((size_t)nc, VKS_CELLS), S)), VKS_THREADS, 0, st, L.dm, reinterpret_cast<const T*>(L.KV), rr, L.n, act, cellbuf, L.col_cells[k], nc);
        LAUNCH(KI_VANKA_SCATTER, k_vanka_scatter<T>, (dim3(nblk((size_t)nn * 5, 128), S)), 128, 0, st, L.h.n_cells, L.col_nodes[k], L.col_src[k], nn, cellbuf, om, L.n, act, x);
      }
      return launch_check();
    }
    const T* rr = b;
    if (!first) {
      TRY((spmv<T, true>(L, S, A, x, b, act, r, st)));
      rr = r;
    }
    if (c->transposed)   // transposed operators lack the displacement-row structure
      LAUNCH_W(2.0 * 2025 * L.h.n_cells * (double)c->n_act, KI_VANKA_CELL, k_vanka_cell<T>, (dim3(nblk((size_t)L.h.n_cells * 45, 128), S)), 128, 0, st, L.dm, reinterpret_cast<const T*>(L.KV), rr, L.n, act, cellbuf, (const int*)nullptr, L.h.n_cells);
    else
    LAUNCH_W(2.0 * 2025 * L.h.n_cells * (double)c->n_act, KI_VANKA_CELL, k_vanka_cell_split<T>, (dim3(nblk((size_t)L.h.n_cells, VKS_CELLS), S)), VKS_THREADS, 0, st, L.dm, reinterpret_cast<const T*>(L.KV), rr, L.n, act, cellbuf, (const int*)nullptr, L.h.n_cells);
    LAUNCH(KI_VANKA_GATHER, k_vanka_gather<T>, (dim3(nblk(L.h.n_nodes, 128), S)), 128, 0, st, L.dm, cellbuf, om, L.n, act, x);
    return launch_check();
  };
  for (int i = 0; i < nu; ++i) TRY(smooth(i == 0));
  Level& C = c->lev[l + 1];
  T* Cb = reinterpret_cast<T*>(C.b);
  T* Cx = reinterpret_cast<T*>(C.x);
  TRY((spmv<T, true>(L, S, A, x, b, act, r, st)));
  LAUNCH(KI_RESTRICT, k_restrict<T>, (dim3(nblk(C.n, 128), S)), 128, 0, st, C.T, L.dm.node_flags, C.dm.node_flags, r, L.n, C.n, act, Cb);
  TRY(launch_check());
  TRY(vcycle<T>(c, l + 1, S, Cb, Cx, act, st));
  LAUNCH(KI_PROLONG_ADD, k_prolong_add<T>, (dim3(nblk(L.n, 128), S)), 128, 0, st, C.T, L.dm.node_flags, Cx, L.n, C.n, act, x);
  TRY(launch_check());
  for (int i = 0; i < nu; ++i) TRY(smooth(false));
  return FSI_OK;
}

// FGMRES(m) with multigrid right preconditioning: solve A x = b per active
// slice to ||b - A x|| <= rtol ||b||, vectors and operator in T (the
// Hessenberg matrix and the rotations are kept in FP64). x is overwritten.
// abs_target (optional, host [S]): stop a slice once ||b - A x|| <= max(abs_target[s], rtol ||b||).
// Tunes, ahead of a graph capture, the block products that an Arnoldi step of
// FGMRES will launch (the Krylov operator in T, each multigrid level's operator in
// TP) for this batch-size class: inside the capture no variant can be timed. Runs
// on scratch vectors (the preconditioner's input and output, each level's x and
// r), so it needs the level operators assembled and nothing else.
template <typename T, typename TP>
int spt_pretune(fsi_ctx* c, int S, cudaStream_t st) {
  const int cls = S <= 1 ? 0 : S <= 4 ? 1 : S <= 16 ? 2 : 3;
  auto type_of = [](size_t bytes) { return bytes == sizeof(float) ? 1 : 0; };
  for (size_t l = 0; l < c->lev.size(); ++l) {
    Level& L = c->lev[l];
    if (L.coarsest) break;
    const double work = 50.0 * L.h.nnzb * (double)c->n_act;
    if (sizeof(T) == sizeof(double) && L.Aff && L.aff_of == (const void*)L.A && L.spt_choice[2][cls] < 0) {
      const double bytes = (double)c->n_act * 8.0 * (25.0 * L.h.nnzb + 2.0 * L.n);   // float-pair products
      TRY((spt_product<float2, double, false>(L, S, L.Aff, L.xff, nullptr, c->active, reinterpret_cast<double*>(L.r),
                                              st, work, bytes, KI_BSR_SPMV_FF)));
    }
    if (l == 0 && L.spt_choice[type_of(sizeof(T))][cls] < 0) {
      const double bytes = (double)c->n_act * sizeof(T) * (25.0 * L.h.nnzb + 2.0 * L.n);
      TRY((spt_product<T, T, false>(L, S, reinterpret_cast<const T*>(L.A), reinterpret_cast<const T*>(c->dU), nullptr,
                                    c->active, reinterpret_cast<T*>(c->R), st, work, bytes, KI_BSR_SPMV)));
    }
    if (L.spt_choice[type_of(sizeof(TP))][cls] < 0) {
      const TP* A = (l == 0 && mixed<TP>(c)) ? reinterpret_cast<const TP*>(L.A32) : reinterpret_cast<const TP*>(L.A);
      const TP* xin = l == 0 ? reinterpret_cast<const TP*>(c->dU) : reinterpret_cast<const TP*>(L.x);
      const double bytes = (double)c->n_act * sizeof(TP) * (25.0 * L.h.nnzb + 2.0 * L.n);
      TRY((spt_product<TP, TP, false>(L, S, A, xin, nullptr, c->active, reinterpret_cast<TP*>(L.r), st, work, bytes,
                                      KI_BSR_SPMV)));
    }
  }
  return FSI_OK;
}

template <typename T, typename TP = T>
int fgmres(fsi_ctx* c, int S, const T* b, T* x, const uint8_t* act_in, double rtol, fsi_stats* stats,
           cudaStream_t st, const double* abs_target = nullptr) {
  Level& L = c->lev[0];
  const size_t n = L.n;
  const int m = c->m;
  const size_t vsl = (size_t)(m + 1) * n, zsl = (size_t)m * n;
  const T* A = reinterpret_cast<const T*>(L.A);
  T* V = reinterpret_cast<T*>(c->V);
  T* Z = reinterpret_cast<T*>(c->Z);
  T* w = reinterpret_cast<T*>(c->w);
  T* vin = reinterpret_cast<T*>(c->dU);
  T* vout = reinterpret_cast<T*>(c->R);
  std::vector<uint8_t> act(S), act2(S);
  std::vector<double> bnorm(S), res(S);
  std::vector<int> its(S, 0), nvh(S, 0);
  CK(cudaMemcpyAsync(act.data(), act_in, S, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(c->active, act_in, S, cudaMemcpyDeviceToDevice, st));
  LAUNCH(KI_FILL, k_fill<T>, (dim3(nblk(n, 256), S)), 256, 0, st, (int)n, 0.0, c->active, x, n);
  TRY(dots<T>(c, S, n, 1, b, 0, n, b, n, c->active, c->scal, 1, true, st));
  CK(cudaMemcpyAsync(bnorm.data(), c->scal, S * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  int status = FSI_OK;
  // the caller's mask, restored on exit (the cycles below narrow c->active)
  const std::vector<uint8_t> act_entry = act;
  c->slice_code.assign(S, 0);
  for (int s = 0; s < S; ++s)
    if (act[s] && !(bnorm[s] > 0.0)) {
      if (!std::isfinite(bnorm[s])) status = c->slice_code[s] = FSI_ENAN;
      act[s] = 0;
    }
  auto any = [&]() { return std::any_of(act.begin(), act.end(), [](uint8_t a) { return a != 0; }); };
  bool first_cycle = true;
  if (S <= c->prm.graph_max_batch && any()) {
    CK(cudaMemcpyAsync(c->active, act.data(), S, cudaMemcpyHostToDevice, st));
    c->n_act = g_nact = count_active(act);
    TRY((spt_pretune<T, TP>(c, S, st)));
  }
  while (any()) {
    CK(cudaMemcpyAsync(c->active, act.data(), S, cudaMemcpyHostToDevice, st));
    c->n_act = g_nact = count_active(act);
    // r = b - A x  (x = 0 in the first cycle)
    if (first_cycle) {
      CK(cudaMemcpy2DAsync(V, vsl * sizeof(T), b, n * sizeof(T), n * sizeof(T), S, cudaMemcpyDeviceToDevice, st));
    } else {
      // V[s][0] = b - A x for active slices (strided output through w)
      TRY((spmv<T, true>(L, S, A, x, b, c->active, w, st)));
      CK(cudaMemcpy2DAsync(V, vsl * sizeof(T), w, n * sizeof(T), n * sizeof(T), S, cudaMemcpyDeviceToDevice, st));
    }
    first_cycle = false;
    TRY(dots<T>(c, S, n, 1, V, 0, vsl, V, vsl, c->active, c->scal, 1, true, st));
    LAUNCH(KI_INIT_G, k_init_g, (nblk(S, 64)), 64, 0, st, S, m, c->scal, c->active, c->g);
    LAUNCH(KI_SCALE, k_scale<T>, (dim3(nblk(n, 256), S)), 256, 0, st, (int)n, V, vsl, c->scal, 1, true, c->active, V, vsl);
    TRY(launch_check());
    std::vector<uint8_t> cyc = act;   // slices still inside this cycle
    for (int j = 0; j < m; ++j) {
      CK(cudaMemcpyAsync(c->active, cyc.data(), S, cudaMemcpyHostToDevice, st));
      c->n_act = g_nact = count_active(cyc);
      T* Vj = V + (size_t)j * n;
      T* Zj = Z + (size_t)j * n;
      // one Arnoldi step: device work only, so that it can be a CUDA graph
      auto body = [&](cudaStream_t s2) -> int {
        // Z_j = M^{-1} V_j (the V-cycle works on contiguous [S][n] buffers)
        CK(cudaMemcpy2DAsync(vin, n * sizeof(T), Vj, vsl * sizeof(T), n * sizeof(T), S, cudaMemcpyDeviceToDevice, s2));
        if (sizeof(TP) == sizeof(T)) {
          TRY(vcycle<TP>(c, 0, S, reinterpret_cast<const TP*>(vin), reinterpret_cast<TP*>(vout), c->active, s2));
        } else {   // preconditioner in TP: convert in and out
          TP* pin = reinterpret_cast<TP*>(c->p_in);
          TP* pout = reinterpret_cast<TP*>(c->p_out);
          LAUNCH(KI_AXPBY, (k_axpby<T, TP>), (dim3(nblk(n, 256), S)), 256, 0, s2, (int)n, 1.0, vin, n, 0.0, c->active, pin, n);
          TRY(vcycle<TP>(c, 0, S, pin, pout, c->active, s2));
          LAUNCH(KI_AXPBY, (k_axpby<TP, T>), (dim3(nblk(n, 256), S)), 256, 0, s2, (int)n, 1.0, pout, n, 0.0, c->active, vout, n);
        }
        CK(cudaMemcpy2DAsync(Zj, zsl * sizeof(T), vout, n * sizeof(T), n * sizeof(T), S, cudaMemcpyDeviceToDevice, s2));
        // w = A Z_j
        TRY((spmv<T, false>(L, S, A, vout, nullptr, c->active, w, s2)));
        // classical Gram-Schmidt, twice
        TRY(dots<T>(c, S, n, j + 1, V, n, vsl, w, n, c->active, c->hcol, m + 1, false, s2));
        LAUNCH_W(2.0 * (j + 1) * (double)n * c->n_act, KI_SUB_BASIS, k_sub_basis<T>, (dim3(nblk(n, 256), S)), 256, 0, s2, (int)n, j + 1, V, n, vsl, c->hcol, m + 1, c->active, w, n);
        TRY(dots<T>(c, S, n, j + 1, V, n, vsl, w, n, c->active, c->hcol2, m + 1, false, s2));
        LAUNCH_W(2.0 * (j + 1) * (double)n * c->n_act, KI_SUB_BASIS, k_sub_basis<T>, (dim3(nblk(n, 256), S)), 256, 0, s2, (int)n, j + 1, V, n, vsl, c->hcol2, m + 1, c->active, w, n);
        LAUNCH(KI_AXPBY, (k_axpby<double, double>), (dim3(1, S)), 64, 0, s2, j + 1, 1.0, c->hcol2, m + 1, 1.0, c->active, c->hcol, m + 1);
        TRY(dots<T>(c, S, n, 1, w, 0, n, w, n, c->active, c->scal, 1, true, s2));
        LAUNCH(KI_SCALE, k_scale<T>, (dim3(nblk(n, 256), S)), 256, 0, s2, (int)n, w, n, c->scal, 1, true, c->active, V + (size_t)(j + 1) * n, vsl);
        LAUNCH(KI_GIVENS, k_givens, (nblk(S, 64)), 64, 0, s2, S, j, m, c->hcol, m + 1, c->scal, c->active, c->H, c->cs, c->sn, c->g, c->resid);
        return launch_check();
      };
      fsi_ctx::Graph* replayed = nullptr;
      if (S <= c->prm.graph_max_batch) {
        // the kernels a graph holds depend on the scalar types and on whether the
        // operators are transposed (structured or generic Vanka apply)
        fsi_ctx::Graph& ge =
            c->graphs[std::make_tuple((int)(sizeof(T) * 16 + sizeof(TP)) * 2 + (c->transposed ? 1 : 0), S, j)];
        if (!ge.exec || ge.epoch != g_prof.epoch) {
          if (ge.exec) {
            cudaGraphExecDestroy(ge.exec);
            ge.exec = nullptr;
          }
          if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
          if (g_prof.mask) prof_grow_pool(4096);
          g_cap = Capture{};
          g_cap.on = true;
          g_cap.n_act = c->n_act;
          CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
          const int rc = body(c->cap_stream);
          cudaGraph_t graph = nullptr;
          const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
          g_cap.on = false;
          if (rc != FSI_OK || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return rc != FSI_OK ? rc : fail(FSI_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
          }
          const cudaError_t ei = cudaGraphInstantiate(&ge.exec, graph, 0);
          cudaGraphDestroy(graph);
          if (ei != cudaSuccess) return fail(FSI_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
          ge.epoch = g_prof.epoch;
          ge.recs = g_cap.recs;
          for (int id = 0; id < KI_COUNT; ++id) ge.launches[id] = g_cap.launches[id];
        }
        CK(cudaGraphLaunch(ge.exec, st));
        for (int id = 0; id < KI_COUNT; ++id) {
          g_prof.launches[id] += ge.launches[id];
          g_prof.total += ge.launches[id];
        }
        replayed = &ge;
      } else {
        TRY(body(st));
      }
      CK(cudaMemcpyAsync(res.data(), c->resid, S * sizeof(double), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (replayed && !replayed->recs.empty()) {   // timed kernels inside the graph, read before the next replay
        std::lock_guard<std::mutex> lk(g_prof.mu);
        for (const CapRec& r : replayed->recs) {
          float e = 0.f;
          if (cudaEventElapsedTime(&e, g_prof.pool[r.ev], g_prof.pool[r.ev + 1]) != cudaSuccess) {
            (void)cudaGetLastError();   // timing is best effort: never fails the solve
            continue;
          }
          g_prof.gms[r.id] += e;
          g_prof.gwork[r.id] += r.work_per_slice * c->n_act;
          g_prof.gbytes[r.id] += r.bytes_per_slice * c->n_act;
          g_prof.gcnt[r.id] += 1;
        }
      }
      std::vector<uint8_t> fin(S, 0);
      bool any_fin = false, any_left = false;
      for (int s = 0; s < S; ++s) {
        if (!cyc[s]) continue;
        ++its[s];
        const bool conv = res[s] <= std::max(rtol * bnorm[s], abs_target ? abs_target[s] : 0.0);
        const bool bad = !std::isfinite(res[s]);
        if (conv || bad || j == m - 1 || its[s] >= c->prm.gmres_maxit) {
          fin[s] = 1;
          nvh[s] = j + 1;
          cyc[s] = 0;
          any_fin = true;
          if (conv || bad || its[s] >= c->prm.gmres_maxit) {
            act[s] = 0;
            if (bad) status = c->slice_code[s] = FSI_ENAN;
            else if (!conv) status = c->slice_code[s] = FSI_EGMRES;
          }
        } else {
          any_left = true;
        }
      }
      if (any_fin) {
        CK(cudaMemcpyAsync(c->active2, fin.data(), S, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(c->nv, nvh.data(), S * sizeof(int), cudaMemcpyHostToDevice, st));
        LAUNCH(KI_BACKSOLVE, k_backsolve, (nblk(S, 64)), 64, 0, st, S, m, c->nv, c->H, c->g, c->active2, c->y);
        LAUNCH(KI_ADD_BASIS, k_add_basis<T>, (dim3(nblk(n, 256), S)), 256, 0, st, (int)n, c->nv, Z, n, zsl, c->y, m, c->active2, x, n);
        TRY(launch_check());
      }
      if (!any_left) break;
    }
  }
  if (stats) {
    for (int s = 0; s < S; ++s) {
      stats->gmres_iters += its[s];
      stats->max_gmres = std::max(stats->max_gmres, its[s]);
    }
  }
  CK(cudaMemcpyAsync(c->active, act_entry.data(), S, cudaMemcpyHostToDevice, st));
  c->n_act = g_nact = count_active(act_entry);
  return status;
}

// Newton correction for the active slices: build (or update) the
// preconditioner and solve J delta = -R with the linear solver in T; the
// result is added to the FP64 iterate.
template <typename T, typename TP = T>
int newton_correction(fsi_ctx* c, int S, double k, double theta, int it, int reuse, bool hierarchy_valid,
                      double rtol, fsi_stats* stats, cudaStream_t st, const double* abs_target) {
  Level& L = c->lev[0];
  const size_t n = L.n;
  T* b = reinterpret_cast<T*>(L.b);
  T* x = reinterpret_cast<T*>(L.x);
  const bool keep_all = (it == 0) ? hierarchy_valid : reuse >= 2;
  if (keep_all)  // exact Jacobian for the Krylov operator; the multigrid hierarchy is kept
    TRY(jacobian<T>(c, L, S, c->Uit, c->Uold, k, theta, c->active, reinterpret_cast<T*>(L.A), st));
  else
    TRY(mg_setup<TP>(c, S, c->Uit, c->Uold, k, theta, c->active, st, it > 0 && reuse == 1));
  // right-hand side -R in T (R itself is scratch inside the solver)
  LAUNCH(KI_AXPBY, (k_axpby<double, T>), (dim3(nblk(n, 256), S)), 256, 0, st, (int)n, -1.0, c->R, n, 0.0, c->active, b, n);
  TRY(launch_check());
  const int rc = fgmres<T, TP>(c, S, b, x, c->active, rtol, stats, st, abs_target);
  if (rc != FSI_OK && rc != FSI_EGMRES) return rc;
  LAUNCH(KI_AXPBY, (k_axpby<T, double>), (dim3(nblk(n, 256), S)), 256, 0, st, (int)n, 1.0, x, n, 1.0, c->active, c->Uit, n);
  TRY(launch_check());
  return rc;
}

// FSI_TRACE_NEWTON set in the environment: the residual history of every slice
// whose step fails, and every FGMRES solve that stops at its limit, go to stderr.
bool trace_newton() {
  static const bool on = std::getenv("FSI_TRACE_NEWTON") != nullptr;
  return on;
}
void trace_slice(const char* path, int s, double t_old, double k, int code, const std::vector<double>& h) {
  std::fprintf(stderr, "[fsi trace] %s slice %d t=%.6g k=%.6g status %d, Newton residuals:", path, s, t_old + k, k,
               code);
  for (double x : h) std::fprintf(stderr, " %.3e", x);
  std::fprintf(stderr, "\n");
}

// One theta step for S slices (Newton + FGMRES/multigrid).
// reuse: what the preconditioner keeps across Newton iterations (see mg_reuse);
// hierarchy_valid: the multigrid hierarchy of an earlier step of the same
// propagator call may serve the first Newton iteration too.
int theta_step(fsi_ctx* c, int S, const double* U_old, const double* t_old, double k, double theta, double* U_new,
               fsi_stats* stats, cudaStream_t st, int reuse, bool hierarchy_valid) {
  if (S < 1 || S > c->S) return fail(FSI_EINVAL, "batch size outside 1..max_batch");
  Level& L = c->lev[0];
  const size_t n = L.n;
  std::vector<double> tn(S);
  for (int s = 0; s < S; ++s) tn[s] = t_old[s] + k;
  CK(cudaMemcpyAsync(c->t_dev, tn.data(), S * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(c->Uold, U_old, S * n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(c->Uit, U_old, S * n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  std::vector<uint8_t> act(S, 1);
  std::vector<int> st_h(S, 0);
  CK(cudaMemcpyAsync(c->active, act.data(), S, cudaMemcpyHostToDevice, st));
  c->n_act = g_nact = count_active(act);
  CK(cudaMemcpyAsync(c->status, st_h.data(), S * sizeof(int), cudaMemcpyHostToDevice, st));
  LAUNCH(KI_APPLY_DIRICHLET, k_apply_dirichlet, (dim3(nblk(L.h.n_nodes, 128), S)), 128, 0, st, L.dm, c->P, c->Uit, n, c->t_dev, c->active);
  TRY(launch_check());
  std::vector<double> r0(S, 0.0), nr(S);
  std::vector<int> nit(S, 0), why(S, 0);   // why: first failure code per slice
  // gmiss: an FGMRES solve of the slice stopped at its iteration limit. Its correction is
  // still applied (inexact Newton); the slice fails only if Newton then fails (FSI_EGMRES)
  std::vector<uint8_t> gmiss(S, 0);
  // slices whose last solve stopped at its limit: their multigrid hierarchy is rebuilt at the
  // current iterate before the next solve (the other slices keep theirs, so the batch stays bitwise solo)
  std::vector<uint8_t> rebuild(S, 0);
  const bool trace = trace_newton();
  std::vector<std::vector<double>> hist(trace ? S : 0);
  int status = FSI_OK;
  for (int it = 0;; ++it) {
    CK(cudaMemcpyAsync(c->active, act.data(), S, cudaMemcpyHostToDevice, st));
    c->n_act = g_nact = count_active(act);
    TRY(residual(c, L, S, c->Uit, c->Uold, k, theta, c->active, c->R, st));
    TRY(dots<double>(c, S, n, 1, c->R, 0, n, c->R, n, c->active, c->scal, 1, true, st));
    CK(cudaMemcpyAsync(nr.data(), c->scal, S * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    bool any = false;
    for (int s = 0; s < S; ++s) {
      if (!act[s]) continue;
      if (!std::isfinite(nr[s])) {
        status = why[s] = FSI_ENAN;
        act[s] = 0;
        continue;
      }
      if (it == 0) r0[s] = nr[s];
      if (trace) hist[s].push_back(nr[s]);
      if (it >= 1 && nr[s] <= c->prm.newton_tol * std::max(r0[s], 1.0)) {
        act[s] = 0;
        continue;
      }
      if (it >= c->prm.newton_maxit) {
        if (!why[s]) why[s] = gmiss[s] ? FSI_EGMRES : FSI_ENEWTON;
        if (status == FSI_OK) status = why[s];
        if (trace) trace_slice("2D", s, t_old[s], k, why[s], hist[s]);
        act[s] = 0;
        continue;
      }
      nit[s] = it + 1;
      any = true;
    }
    if (!any) break;
    CK(cudaMemcpyAsync(c->active, act.data(), S, cudaMemcpyHostToDevice, st));
    c->n_act = g_nact = count_active(act);
    // Inexact Newton forcing terms, per slice from its own residual history: the
    // first correction is solved to gmres_rtol_first, later ones until the
    // linearised residual is newton_eta times the Newton target (never looser
    // than 1e-2, never tighter than gmres_rtol).
    std::vector<double> target(S, 0.0);
    double rtol_now = c->prm.gmres_rtol;
    if (c->prm.newton_eta > 0.0) {
      rtol_now = it == 0 ? std::max(c->prm.gmres_rtol, c->prm.gmres_rtol_first) : c->prm.gmres_rtol;
      if (it > 0)
        for (int s = 0; s < S; ++s)
          target[s] = std::min(1e-2 * nr[s], c->prm.newton_eta * c->prm.newton_tol * std::max(r0[s], 1.0));
    }
    // FP64 throughout, or the FP32 linear solver inside the FP64 Newton loop
    // (FP32 cannot reach FP64 tolerances: its relative tolerance is >= 1e-6)
    int rc;
    if (std::any_of(rebuild.begin(), rebuild.end(), [](uint8_t v) { return v != 0; })) {
      std::vector<uint8_t> mask(S);
      for (int s = 0; s < S; ++s) mask[s] = act[s] && rebuild[s];
      CK(cudaMemcpyAsync(c->active2, mask.data(), S, cudaMemcpyHostToDevice, st));
      c->n_act = g_nact = count_active(mask);
      if (c->prm.precision == 0) TRY(mg_setup<double>(c, S, c->Uit, c->Uold, k, theta, c->active2, st));
      else TRY(mg_setup<float>(c, S, c->Uit, c->Uold, k, theta, c->active2, st));
      c->n_act = g_nact = count_active(act);
      std::fill(rebuild.begin(), rebuild.end(), 0);
    }
    if (c->prm.precision == 1)        // all-FP32 linear solver (inner tolerance >= 1e-6)
      rc = newton_correction<float>(c, S, k, theta, it, reuse, hierarchy_valid, std::max(rtol_now, 1e-6),
                                    stats, st, target.data());
    else if (c->prm.precision == 2)   // FP64 FGMRES, FP32 multigrid preconditioner
      rc = newton_correction<double, float>(c, S, k, theta, it, reuse, hierarchy_valid, rtol_now, stats, st,
                                            target.data());
    else
      rc = newton_correction<double>(c, S, k, theta, it, reuse, hierarchy_valid, rtol_now, stats, st,
                                     target.data());
    CK(cudaMemcpyAsync(st_h.data(), c->status, S * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int s = 0; s < S; ++s) {
      if (act[s] && st_h[s] != 0) {
        status = why[s] = FSI_EJAC;
        act[s] = 0;
      }
      const int code = (int)c->slice_code.size() == S ? c->slice_code[s] : 0;
      if (act[s] && code == FSI_EGMRES) {
        gmiss[s] = 1;
        rebuild[s] = 1;
        if (trace) std::fprintf(stderr, "[fsi trace] 2D slice %d t=%.6g Newton it %d: FGMRES at its limit\n", s,
                                t_old[s] + k, it);
      } else if (act[s] && !why[s] && code) {
        why[s] = code;
      }
    }
    if (rc != FSI_OK && rc != FSI_EGMRES) return fail(rc, "linear solve failed: " + g_err);
  }
  CK(cudaMemcpyAsync(U_new, c->Uit, S * n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (stats) {
    for (int s = 0; s < S; ++s) {
      stats->newton_iters += nit[s];
      stats->max_newton = std::max(stats->max_newton, nit[s]);
      const int idx = c->slice_offset + s;
      if (stats->slice_status && idx < stats->slice_status_len && !stats->slice_status[idx])
        stats->slice_status[idx] = why[s];
    }
    stats->status = status;
  }
  if (status != FSI_OK) {
    char buf[128];
    snprintf(buf, sizeof buf, "theta step failed with status %d", status);
    return fail(status, buf);
  }
  return FSI_OK;
}

int propagate(fsi_ctx* c, int S, const double* U0, const double* t0, double* U1, int m, bool fine, fsi_stats* stats,
              cudaStream_t st) {
  const double dt = c->prm.T / c->prm.n_slices;
  const double k = dt / m;
  const double theta = fine ? 0.5 + c->prm.theta0 * k : 1.0;
  std::vector<double> t(t0, t0 + S);
  const double* src = U0;
  const int every = std::max(1, c->prm.mg_rebuild_every);
  for (int j = 0; j < m; ++j) {
    if (fine)
      TRY(theta_step(c, S, src, t.data(), k, theta, U1, stats, st, c->prm.mg_reuse, j % every != 0));
    else
      TRY(theta_step(c, S, src, t.data(), k, theta, U1, stats, st, std::min(c->prm.mg_reuse, 1), false));
    for (double& x : t) x += k;
    src = U1;
  }
  if (m == 0 && U1 != U0)
    CK(cudaMemcpyAsync(U1, U0, S * c->n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  return FSI_OK;
}

// Batches of at most max_batch slices.
int propagate_chunked(fsi_ctx* c, int S, const double* U0, const double* t0, double* U1, bool fine, fsi_stats* stats,
                      cudaStream_t st) {
  const int m = fine ? c->prm.m_fine : c->prm.m_coarse;
  const int base = c->slice_offset;
  for (int s0 = 0; s0 < S; s0 += c->S) {
    const int b = std::min(c->S, S - s0);
    c->slice_offset = base + s0;
    const int rc = propagate(c, b, U0 + (size_t)s0 * c->n, t0 + s0, U1 + (size_t)s0 * c->n, m, fine, stats, st);
    c->slice_offset = base;
    if (rc != FSI_OK) return rc;
  }
  return FSI_OK;
}

int validate_mesh(const fsi_mesh* mesh) {
  if (!mesh) return fail(FSI_EINVAL, "null mesh");
  if (mesh->n_xseg < 1 || mesh->n_yseg < 1 || !mesh->x_breaks || !mesh->y_breaks || !mesh->nx_seg || !mesh->ny_seg)
    return fail(FSI_EINVAL, "empty mesh");
  for (int i = 0; i < mesh->n_xseg; ++i)
    if (mesh->nx_seg[i] < 1 || !(mesh->x_breaks[i + 1] > mesh->x_breaks[i])) return fail(FSI_EINVAL, "bad x segments");
  for (int i = 0; i < mesh->n_yseg; ++i)
    if (mesh->ny_seg[i] < 1 || !(mesh->y_breaks[i + 1] > mesh->y_breaks[i])) return fail(FSI_EINVAL, "bad y segments");
  return FSI_OK;
}

// The finest level of the mesh hierarchy (host tables only).
void finest_mesh(const fsi_mesh* mesh, HostMesh& h0) {
  const double box[4] = {mesh->solid_x0, mesh->solid_x1, mesh->solid_y0, mesh->solid_y1};
  std::vector<double> xb(mesh->x_breaks, mesh->x_breaks + mesh->n_xseg + 1);
  std::vector<double> yb(mesh->y_breaks, mesh->y_breaks + mesh->n_yseg + 1);
  h0.xseg.assign(mesh->nx_seg, mesh->nx_seg + mesh->n_xseg);
  h0.yseg.assign(mesh->ny_seg, mesh->ny_seg + mesh->n_yseg);
  h0.xv = axis_vertices(xb, h0.xseg);
  h0.yv = axis_vertices(yb, h0.yseg);
  build_mesh(h0, mesh->has_solid != 0, box);
}

int validate(const fsi_mesh* mesh, const fsi_params* p) {
  if (!p) return fail(FSI_EINVAL, "null params");
  TRY(validate_mesh(mesh));
  if (p->max_batch < 1 || p->n_slices < 1 || p->m_fine < 1 || p->m_coarse < 1 || !(p->T > 0))
    return fail(FSI_EINVAL, "bad time or batch parameters");
  if (p->gmres_restart < 1 || p->gmres_restart > 63 || p->gmres_maxit < 1 || p->newton_maxit < 1)
    return fail(FSI_EINVAL, "bad solver parameters (restart must be 1..63)");
  if (p->precision < 0 || p->precision > 2) return fail(FSI_EINVAL, "precision must be 0, 1 or 2");
  if (!(p->gmres_rtol > 0.0 && p->gmres_rtol < 1.0)) return fail(FSI_EINVAL, "gmres_rtol must lie in (0, 1)");
  if (!(p->newton_eta >= 0.0 && p->newton_eta < 1.0)) return fail(FSI_EINVAL, "newton_eta must lie in [0, 1)");
  if (p->pipeline_chunk < 0) return fail(FSI_EINVAL, "pipeline_chunk must be >= 0");
  if (p->newton_eta > 0.0 && !(p->gmres_rtol_first > 0.0 && p->gmres_rtol_first < 1.0))
    return fail(FSI_EINVAL, "gmres_rtol_first must lie in (0, 1)");
  if (p->mg_smoother != 0 && p->mg_smoother != 1) return fail(FSI_EINVAL, "mg_smoother must be 0 or 1");
  if (p->mg_smooth < 1 || !(p->mg_omega > 0) || p->mg_coarsest_max_dofs < 5 || !(p->mg_coarse_lps > 0))
    return fail(FSI_EINVAL, "bad multigrid parameters");
  return FSI_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Discrete adjoint of the fine trajectory (one slice).
// ---------------------------------------------------------------------------
int tip_u(fsi_ctx* c, const double* U, double out[2], cudaStream_t st) {
  CK(cudaMemcpyAsync(out, U + (size_t)c->tip * 5 + 2, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return FSI_OK;
}

int adjoint_impl(fsi_ctx* c, const double* U0, double t0, int M, double* J_out, double* grad, fsi_stats* stats,
                 cudaStream_t st) {
  if (c->tip < 0) return fail(FSI_EINVAL, "no mesh node at the top centre of the solid (adjoint functional)");
  if (M < 1) return fail(FSI_EINVAL, "n_steps must be >= 1");
  if (c->prm.precision != 0) return fail(FSI_EINVAL, "the adjoint runs in FP64 (precision 0)");
  Level& L = c->lev[0];
  const size_t n = c->n;
  const int m = c->prm.m_fine;
  const double k = c->prm.T / c->prm.n_slices / m;
  const double theta = 0.5 + c->prm.theta0 * k;
  const int nslice = (M + m - 1) / m;
  const size_t ck_len = (size_t)(nslice + 1) * n, sb_len = (size_t)(m + 1) * n;
  if (c->adj_ck_len < ck_len) {
    if (c->adj_ck) cudaFree(c->adj_ck);
    c->adj_ck = nullptr;
    CK(cudaMalloc(&c->adj_ck, ck_len * sizeof(double)));
    c->adj_ck_len = ck_len;
  }
  if (!c->adj_sb) {
    CK(cudaMalloc(&c->adj_sb, sb_len * sizeof(double)));
    CK(cudaMalloc(&c->adj_vec, 6 * n * sizeof(double)));
    CK(cudaMalloc(&c->adj_B, (size_t)L.h.nnzb * 25 * sizeof(double)));
    CK(cudaMalloc(&c->adj_Bt, (size_t)L.h.nnzb * 25 * sizeof(double)));
    c->adj_sb_len = sb_len;
  }
  double *lam = c->adj_vec, *lamn = lam + n, *rhs = lam + 2 * n, *rhs2 = lam + 3 * n, *dR = lam + 4 * n,
         *Unext = lam + 5 * n;
  std::vector<double> w(M + 1, k);
  w[0] = w[M] = 0.5 * k;
  // forward sweep, checkpoints at slice boundaries
  double u[2];
  CK(cudaMemcpyAsync(c->adj_ck, U0, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(c->adj_sb, U0, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  TRY(tip_u(c, U0, u, st));
  double J = w[0] * (u[0] * u[0] + u[1] * u[1]);
  double* cur = c->adj_sb;
  for (int step = 1; step <= M; ++step) {
    const double told = t0 + (step - 1) * k;
    TRY(theta_step(c, 1, cur, &told, k, theta, cur, stats, st, 1, false));
    TRY(tip_u(c, cur, u, st));
    J += w[step] * (u[0] * u[0] + u[1] * u[1]);
    if (step % m == 0 || step == M)
      CK(cudaMemcpyAsync(c->adj_ck + (size_t)((step + m - 1) / m) * n, cur, n * sizeof(double),
                         cudaMemcpyDeviceToDevice, st));
  }
  // backward sweep: recompute each slice from its checkpoint, then adjoint steps
  double g[3] = {0, 0, 0};
  bool have_next = false;
  std::vector<uint8_t> one(1, 1);
  for (int sl = nslice - 1; sl >= 0; --sl) {
    const int s0 = sl * m, s1 = std::min(M, s0 + m);   // steps s0+1 .. s1
    CK(cudaMemcpyAsync(c->adj_sb, c->adj_ck + (size_t)sl * n, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    for (int j = 1; j <= s1 - s0; ++j) {
      const double told = t0 + (s0 + j - 1) * k;
      TRY(theta_step(c, 1, c->adj_sb + (size_t)(j - 1) * n, &told, k, theta, c->adj_sb + (size_t)j * n, stats, st, 1,
                     false));
    }
    for (int nn = s1; nn > s0; --nn) {
      const double* Un = c->adj_sb + (size_t)(nn - s0) * n;
      const double* Um = c->adj_sb + (size_t)(nn - s0 - 1) * n;
      CK(cudaMemcpyAsync(c->active, one.data(), 1, cudaMemcpyHostToDevice, st));
      c->n_act = g_nact = 1;
      // rhs = -w_n dg/dU_n - (dR_{n+1}/dU_n)^T lam_{n+1}
      TRY(tip_u(c, Un, u, st));
      CK(cudaMemsetAsync(rhs, 0, n * sizeof(double), st));
      const double gtip[2] = {-w[nn] * 2.0 * u[0], -w[nn] * 2.0 * u[1]};
      CK(cudaMemcpyAsync(rhs + (size_t)c->tip * 5 + 2, gtip, 2 * sizeof(double), cudaMemcpyHostToDevice, st));
      if (have_next) {
        const double* Up = nn < s1 ? c->adj_sb + (size_t)(nn - s0 + 1) * n : Unext;
        LAUNCH(KI_CELL_JACOBIAN_OLD, k_cell_jacobian<true>, (dim3(L.h.n_cells, 1)), JAC_THREADS, 0, st, L.dm, c->P, Up, Un, L.n, k, theta, 1.0, c->active, L.Ke);
        LAUNCH(KI_ASSEMBLE_BSR, k_assemble_bsr<double>, (dim3(nblk((size_t)L.h.nnzb * 5, 128), 1)), 128, 0, st, L.dm, L.Ke, c->active, c->adj_B, 0.0);
        LAUNCH(KI_BSR_TRANSPOSE, k_bsr_transpose, (dim3(nblk((size_t)L.h.nnzb * 25, 256), 1)), 256, 0, st, L.h.nnzb, L.blk_t, c->adj_B, c->active, c->adj_Bt);
        TRY((spmv<double, true>(L, 1, c->adj_Bt, lamn, rhs, c->active, rhs2, st)));
        CK(cudaMemcpyAsync(rhs, rhs2, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
      }
      // (dR_n/dU_n)^T lam_n = rhs with the transposed multigrid hierarchy
      TRY(mg_setup<double>(c, 1, Un, Um, k, theta, c->active, st, false, true));
      CK(cudaMemcpyAsync(L.b, rhs, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
      int rc = fgmres<double>(c, 1, L.b, L.x, c->active, c->prm.gmres_rtol, stats, st);
      if (rc != FSI_OK) return fail(rc, "adjoint linear solve failed");
      CK(cudaMemcpyAsync(lam, L.x, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
      // dJ/dp += lam^T dR_n/dp
      CK(cudaMemcpyAsync(c->active, one.data(), 1, cudaMemcpyHostToDevice, st));
      const double tn = t0 + nn * k;
      CK(cudaMemcpyAsync(c->t_dev, &tn, sizeof(double), cudaMemcpyHostToDevice, st));
      for (int which = 0; which < 3; ++which) {
        if (which < 2) {
          LAUNCH(KI_CELL_DRES_DLAME, k_cell_dres_dlame, (dim3(nblk(L.h.n_cells, 128), 1)), 128, 0, st, L.dm, Un, Um, L.n, k, theta, which, c->active, L.cellbuf);
          LAUNCH(KI_GATHER_VECTOR, k_gather_vector, (dim3(nblk(L.h.n_nodes, 128), 1)), 128, 0, st, L.dm, L.cellbuf, L.n, c->active, dR);
        } else {
          LAUNCH(KI_DRES_DVBAR, k_dres_dvbar, (dim3(nblk(L.h.n_nodes, 128), 1)), 128, 0, st, L.dm, c->P, c->t_dev, L.n, c->active, dR);
        }
        TRY(dots<double>(c, 1, n, 1, dR, 0, n, lam, n, c->active, c->scal, 1, false, st));
        double d = 0.0;
        CK(cudaMemcpyAsync(&d, c->scal, sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        g[which] += d;
      }
      CK(cudaMemcpyAsync(lamn, lam, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
      have_next = true;
    }
    CK(cudaMemcpyAsync(Unext, c->adj_sb + n, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  *J_out = J;
  for (int i = 0; i < 3; ++i) grad[i] = g[i];
  return FSI_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free residual: its scratch lives in one file-scope device array.
// Layout (doubles): [0, 32) slice flags as bytes, [32, 32 + kNaMaxSlices)
// per-slice times, then the per-cell contributions [S][cells][45].
// ---------------------------------------------------------------------------
constexpr size_t kNaDoubles = size_t(1) << 21;          // 16 MiB per device
constexpr int kNaMaxSlices = 256;
constexpr size_t kNaCellOffset = 32 + kNaMaxSlices;     // 2304 bytes: 256-byte aligned
static __device__ __align__(256) double g_na_scratch[kNaDoubles];

namespace {

constexpr int kNaMaxDevices = 64;
double* g_na_ptr[kNaMaxDevices] = {};
std::mutex g_na_mutex;

// Device address of the scratch array on the current device, looked up once
// per device (with that device current) and cached.
int na_scratch(double** out) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNaMaxDevices) return fail(FSI_EINVAL, "device index beyond the supported range");
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    CK(cudaGetSymbolAddress(&p, g_na_scratch));
    g_na_ptr[dev] = (double*)p;
  }
  *out = g_na_ptr[dev];
  return FSI_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
namespace {

// Parareal correction of slice i (Eq. parareal:iteration, evaluated as
// F + (C_new - C_old)): U[i+1] = Fv[i] + Cn - Cold[i]; folds the slice's
// relative increments of v, u, p into inc.
int correct_slice(fsi_ctx* c, int i, const double* Cn, double* U, double inc[3], cudaStream_t st) {
  const size_t n = c->n;
  const int nrb = c->red_blocks;
  LAUNCH(KI_PARAREAL_CORRECT, k_parareal_correct, (nrb), RED_THREADS, 0, st, (int)n, c->Fv + (size_t)i * n, Cn,
         c->Cold + (size_t)i * n, U + (size_t)(i + 1) * n, c->ppart);
  TRY(launch_check());
  std::vector<double> part(nrb * 6);
  CK(cudaMemcpyAsync(part.data(), c->ppart, part.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  double a[6] = {0, 0, 0, 0, 0, 0};
  for (int b = 0; b < nrb; ++b)
    for (int f = 0; f < 6; ++f) a[f] += part[b * 6 + f];
  for (int f = 0; f < 3; ++f) {
    const double rel = a[3 + f] > 0 ? std::sqrt(a[f] / a[3 + f]) : std::sqrt(a[f]);
    if (!std::isfinite(rel)) return fail(FSI_EDIVERGE, "Parareal increment is not finite");
    inc[f] = std::max(inc[f], rel);
  }
  return FSI_OK;
}

// slot: the iteration's index among those of the current call (history row)
void record_iteration(fsi_parareal_stats& loc, int it, const double inc[3], int slot) {
  loc.increment_v = inc[0];
  loc.increment_u = inc[1];
  loc.increment_p = inc[2];
  if (loc.history && slot < loc.history_len)
    for (int f = 0; f < 3; ++f) loc.history[slot * 3 + f] = inc[f];
  loc.iterations = it;
}

// Parareal workspace, allocated on first use, all or nothing: Cold and Fv
// [N][n], Cnew [n], and the per-block partial sums of the increments.
int parareal_workspace(fsi_ctx* c) {
  if (c->Cold) return FSI_OK;
  const size_t N = (size_t)c->prm.n_slices, n = c->n;
  const int nrb = 152;
  double *cold = nullptr, *fv = nullptr, *cnew = nullptr, *ppart = nullptr;
  std::vector<void*> got;
  if (dalloc(got, &cold, N * n) || dalloc(got, &fv, N * n) || dalloc(got, &cnew, n) ||
      dalloc(got, &ppart, (size_t)nrb * 6)) {
    for (void* p : got) cudaFree(p);
    return FSI_ENOMEM;
  }
  c->owned.insert(c->owned.end(), got.begin(), got.end());
  c->red_blocks = nrb;
  c->Fv = fv;
  c->Cnew = cnew;
  c->ppart = ppart;
  c->Cold = cold;   // last: a non-null Cold means the whole workspace exists
  return FSI_OK;
}

// The predictor sweep U[i+1] = C(U[i]) (iteration 0); keeps C(U[i]) in Cold.
int parareal_predictor(fsi_ctx* c, double* U, fsi_parareal_stats& loc, cudaStream_t st) {
  const int N = c->prm.n_slices;
  const size_t n = c->n;
  const double dt = c->prm.T / N;
  for (int i = 0; i < N; ++i) {
    const double t = i * dt;
    TRY(propagate_chunked(c, 1, U + (size_t)i * n, &t, c->Cold + (size_t)i * n, false, &loc.coarse, st));
    CK(cudaMemcpyAsync(U + (size_t)(i + 1) * n, c->Cold + (size_t)i * n, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    loc.coarse_steps += c->prm.m_coarse;
  }
  return FSI_OK;
}

// Iteration it >= 1 of the run: the fine solves of every slice not yet exact
// (slices it-1 .. N-1, batched), then the corrected coarse sweep with the
// correction of each slice; inc receives the iteration's largest relative
// boundary increments of v, u and p.
int parareal_one(fsi_ctx* c, double* U, int it, fsi_parareal_stats& loc, double inc[3], cudaStream_t st) {
  const int N = c->prm.n_slices;
  const size_t n = c->n;
  const double dt = c->prm.T / N;
  const int first = it - 1;
  const int S = N - first;
  std::vector<double> t(S);
  for (int i = 0; i < S; ++i) t[i] = (first + i) * dt;
  TRY(propagate_chunked(c, S, U + (size_t)first * n, t.data(), c->Fv + (size_t)first * n, true, &loc.fine, st));
  loc.fine_steps += (long long)S * c->prm.m_fine;
  inc[0] = inc[1] = inc[2] = 0.0;
  for (int i = first; i < N; ++i) {
    const double* Cn;
    if (i == first) {
      Cn = c->Cold + (size_t)i * n;   // unchanged input: C(U_i^it) - C(U_i^(it-1)) = 0 exactly
    } else {
      const double ti = i * dt;
      TRY(propagate_chunked(c, 1, U + (size_t)i * n, &ti, c->Cnew, false, &loc.coarse, st));
      loc.coarse_steps += c->prm.m_coarse;
      Cn = c->Cnew;
    }
    TRY(correct_slice(c, i, Cn, U, inc, st));
    if (i != first)
      CK(cudaMemcpyAsync(c->Cold + (size_t)i * n, c->Cnew, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  return FSI_OK;
}

// Iterations it0 .. min(it_end, N) of the serial schedule; stops early once
// the largest increment is <= tol. c->pr_iter follows the completed iterations.
int parareal_iterations(fsi_ctx* c, double* U, int it0, int it_end, double tol, fsi_parareal_stats& loc,
                        cudaStream_t st) {
  const int N = c->prm.n_slices;
  for (int it = it0; it <= it_end && it <= N; ++it) {
    double inc[3];
    c->pr_iter = -1;   // Cold and U are mid-update until the iteration completes
    TRY(parareal_one(c, U, it, loc, inc, st));
    c->pr_iter = it;
    record_iteration(loc, it, inc, it - it0);
    if (std::max(inc[0], std::max(inc[1], inc[2])) <= tol) break;
  }
  return FSI_OK;
}

// The predictor sweep, then per iteration the fine solves of every slice not
// yet exact (batched) followed by the corrected coarse sweep.
int parareal_serial(fsi_ctx* c, double* U, int max_iter, double tol, fsi_parareal_stats& loc, cudaStream_t st) {
  c->pr_iter = -1;
  TRY(parareal_predictor(c, U, loc, st));
  c->pr_iter = 0;
  return parareal_iterations(c, U, 1, max_iter, tol, loc, st);
}

// Pipelined Parareal (the paper's implementation of Sec. 3 starts a slice's
// fine solve as soon as its coarse value exists; here on one GPU): a host
// thread runs the sequential sweeps (the predictor, then each corrected sweep)
// in a single-slice context on its own high-priority stream, while the calling
// thread runs the fine solves in batches of pipeline_chunk slices on the
// caller's stream, each batch as soon as its inputs exist. The fine inputs of
// iteration it are kept in Uin[it % 2], so the corrected sweep may overwrite U
// while later batches of the same iteration still run. Every slice sees the
// arithmetic of parareal_serial, so the results agree bit for bit.
int parareal_pipelined(fsi_ctx* c, double* U, int max_iter, double tol, fsi_parareal_stats& loc,
                       cudaStream_t st) {
  const int N = c->prm.n_slices;
  const size_t n = c->n;
  const double dt = c->prm.T / N;
  const int B = std::max(1, c->prm.pipeline_chunk);
  const int K = std::min(max_iter, N);
  if (!c->sweep) {
    fsi_params p1 = c->prm;
    p1.max_batch = 1;
    p1.pipeline_chunk = 0;
    fsi_ctx* sw = nullptr;
    TRY(fsi_setup(&c->mesh_desc, &p1, &sw));
    c->sweep = sw;
    int lo = 0, hi = 0;
    CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    CK(cudaStreamCreateWithPriority(&c->sweep_stream, cudaStreamNonBlocking, hi));
  }
  if (!c->Uin) TRY(dalloc(c->owned, &c->Uin, (size_t)2 * N * n));
  fsi_ctx* sw = c->sweep;
  sw->P = c->P;   // materials changed through fsi_set_material
  cudaStream_t ss = c->sweep_stream;
  std::vector<double> t(N);
  for (int i = 0; i < N; ++i) t[i] = i * dt;
  auto Uin = [&](int it, int i) { return c->Uin + ((size_t)(it % 2) * N + i) * n; };

  // progress shared by the two threads, guarded by mu
  std::mutex mu;
  std::condition_variable cv;
  int ready_it = 1, ready = 1;     // the fine inputs of iteration ready_it exist for slices < ready
  int fine_it = 0, fine_done = 0;  // the fine results of iteration fine_it exist for slices < fine_done
  int go_it = 1;                   // fine solves of iterations <= go_it may start
  bool stop = false, abort = false;
  int err = FSI_OK;
  std::string err_msg;
  auto fail_shared = [&](int rc) {
    std::lock_guard<std::mutex> lk(mu);
    if (err == FSI_OK) err = rc, err_msg = fsi_last_error();
    abort = true;
    cv.notify_all();
  };
  fsi_stats coarse_stats{};
  long long coarse_steps = 0;

  // the sweeps start after the caller's queued work (U[0])
  cudaEvent_t start;
  CK(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
  CK(cudaEventRecord(start, st));
  CK(cudaStreamWaitEvent(ss, start, 0));
  CK(cudaEventDestroy(start));
  int dev = 0;
  CK(cudaGetDevice(&dev));

  std::thread sweeper;
  auto sweep_main = [&] {
    cudaSetDevice(dev);
    auto body = [&]() -> int {
      // predictor sweep U[i+1] = C(U[i]), which also gives the fine inputs of iteration 1
      CK(cudaMemcpyAsync(Uin(1, 0), U, n * sizeof(double), cudaMemcpyDeviceToDevice, ss));
      for (int i = 0; i < N; ++i) {
        TRY(propagate_chunked(sw, 1, U + (size_t)i * n, &t[i], c->Cold + (size_t)i * n, false, &coarse_stats, ss));
        CK(cudaMemcpyAsync(U + (size_t)(i + 1) * n, c->Cold + (size_t)i * n, n * sizeof(double),
                           cudaMemcpyDeviceToDevice, ss));
        if (i + 1 < N)
          CK(cudaMemcpyAsync(Uin(1, i + 1), c->Cold + (size_t)i * n, n * sizeof(double), cudaMemcpyDeviceToDevice,
                             ss));
        CK(cudaStreamSynchronize(ss));
        coarse_steps += c->prm.m_coarse;
        std::lock_guard<std::mutex> lk(mu);
        if (abort) return FSI_OK;
        ready = i + 2;
        cv.notify_all();
      }
      for (int it = 1; it <= K; ++it) {
        const int first = it - 1;
        double inc[3] = {0, 0, 0};
        for (int i = first; i < N; ++i) {
          const double* Cn = c->Cold + (size_t)i * n;
          if (i != first) {   // C of the corrected U[i], while later fine batches may still run
            TRY(propagate_chunked(sw, 1, U + (size_t)i * n, &t[i], c->Cnew, false, &coarse_stats, ss));
            coarse_steps += c->prm.m_coarse;
            Cn = c->Cnew;
          }
          {
            std::unique_lock<std::mutex> lk(mu);
            cv.wait(lk, [&] { return abort || (fine_it == it && fine_done > i); });
            if (abort) return FSI_OK;
          }
          TRY(correct_slice(c, i, Cn, U, inc, ss));
          if (i != first)
            CK(cudaMemcpyAsync(c->Cold + (size_t)i * n, c->Cnew, n * sizeof(double), cudaMemcpyDeviceToDevice, ss));
          if (it < K && i + 1 < N)
            CK(cudaMemcpyAsync(Uin(it + 1, i + 1), U + (size_t)(i + 1) * n, n * sizeof(double),
                               cudaMemcpyDeviceToDevice, ss));
          CK(cudaStreamSynchronize(ss));
        }
        record_iteration(loc, it, inc, it - 1);
        std::lock_guard<std::mutex> lk(mu);
        if (std::max(inc[0], std::max(inc[1], inc[2])) <= tol || it == K) {
          stop = true;
        } else {   // every input of iteration it + 1 (slices it .. N-1) exists
          ready_it = it + 1;
          ready = N;
          go_it = it + 1;
        }
        cv.notify_all();
        if (stop) break;
      }
      return FSI_OK;
    };
    const int rc = body();
    if (rc != FSI_OK) fail_shared(rc);
  };
  try {
    sweeper = std::thread(sweep_main);
  } catch (const std::system_error&) {   // no thread to be had: the same iteration, unpipelined
    return parareal_serial(c, U, max_iter, tol, loc, st);
  }

  // the fine solves, on the calling thread in batches of B slices
  for (int it = 1; it <= K; ++it) {
    {
      std::unique_lock<std::mutex> lk(mu);
      cv.wait(lk, [&] { return abort || stop || go_it >= it; });
      if (abort || go_it < it) break;
      fine_it = it;
      fine_done = it - 1;
    }
    bool failed = false;
    for (int s0 = it - 1; s0 < N; s0 += B) {
      const int s1 = std::min(N, s0 + B);
      {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] { return abort || (ready_it == it && ready >= s1); });
        if (abort) {
          failed = true;
          break;
        }
      }
      const int rc = propagate_chunked(c, s1 - s0, Uin(it, s0), &t[s0], c->Fv + (size_t)s0 * n, true, &loc.fine, st);
      if (rc != FSI_OK) {
        fail_shared(rc);
        failed = true;
        break;
      }
      loc.fine_steps += (long long)(s1 - s0) * c->prm.m_fine;
      std::lock_guard<std::mutex> lk(mu);
      fine_done = s1;
      cv.notify_all();
    }
    if (failed) break;
  }
  sweeper.join();
  loc.coarse = coarse_stats;
  loc.coarse_steps = coarse_steps;
  if (err != FSI_OK) return fail(err, err_msg);
  return FSI_OK;
}

}  // namespace

int fsi_record_error(int code, const std::string& msg) { return fail(code, msg); }

extern "C" {

int fsi_dense_invert(int S, int n, const double* A, double* inv, int method, void* stream) {
  if (S < 1 || n < 1 || !A || !inv || method < 0 || method > 1) return fail(FSI_EINVAL, "bad dense inverse arguments");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<void*> own;
  double* D = nullptr;
  int *perm = nullptr, *status = nullptr;
  uint8_t* act = nullptr;
  auto release = [&](int rc) {
    cudaStreamSynchronize(st);
    for (void* q : own) cudaFree(q);
    return rc;
  };
  if (dalloc(own, &D, (size_t)S * n * n) || dalloc(own, &perm, (size_t)S * n) || dalloc(own, &status, S) ||
      dalloc(own, &act, S))
    return release(FSI_ENOMEM);
  std::vector<uint8_t> ones(S, 1);
  std::vector<int> zeros(S, 0), st_h(S);
  int rc = FSI_OK;
  if (cudaMemcpyAsync(D, A, (size_t)S * n * n * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(act, ones.data(), S, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(status, zeros.data(), S * sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return release(fail(FSI_ECUDA, "dense inverse copies failed"));
  rc = dense_invert<double>(S, n, D, perm, act, inv, status, st, method);
  if (rc != FSI_OK) return release(rc);
  if (cudaMemcpyAsync(st_h.data(), status, S * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return release(fail(FSI_ECUDA, "dense inverse failed"));
  for (int s = 0; s < S; ++s)
    if (st_h[s] != 0) return release(fail(FSI_EJAC, "singular matrix in the dense inverse"));
  return release(FSI_OK);
}

int fsi3d_mesh_size(const fsi_mesh3d* mesh, int* n_nodes, int* n_dofs, int* nnzb) {
  if (!mesh || !n_nodes || !n_dofs || !nnzb) return fail(FSI_EINVAL, "null argument");
  const int ns[3] = {mesh->n_xseg, mesh->n_yseg, mesh->n_zseg};
  const double* br[3] = {mesh->x_breaks, mesh->y_breaks, mesh->z_breaks};
  const int* seg[3] = {mesh->nx_seg, mesh->ny_seg, mesh->nz_seg};
  for (int a = 0; a < 3; ++a) {
    if (ns[a] < 1 || !br[a] || !seg[a]) return fail(FSI_EINVAL, "empty 3D mesh axis");
    for (int i = 0; i < ns[a]; ++i)
      if (seg[a][i] < 1 || !(br[a][i + 1] > br[a][i])) return fail(FSI_EINVAL, "bad 3D mesh segments");
  }
  fsi3::HostMesh3 m;
  fsi3::build_mesh3(m, fsi3::axis_vertices3(br[0], seg[0], ns[0]), fsi3::axis_vertices3(br[1], seg[1], ns[1]),
                    fsi3::axis_vertices3(br[2], seg[2], ns[2]), mesh->has_solid ? mesh->solid_box : nullptr);
  *n_nodes = m.n_nodes;
  *n_dofs = 7 * m.n_nodes;
  *nnzb = m.nnzb;
  return FSI_OK;
}

int fsi_mesh_size(const fsi_mesh* mesh, int* n_nodes, int* n_dofs, int* nnzb) {
  if (!n_nodes || !n_dofs || !nnzb) return fail(FSI_EINVAL, "null output");
  TRY(validate_mesh(mesh));
  HostMesh h;
  finest_mesh(mesh, h);
  *n_nodes = h.n_nodes;
  *n_dofs = 5 * h.n_nodes;
  *nnzb = h.nnzb;
  return FSI_OK;
}

const char* fsi_last_error(void) { return g_err.c_str(); }

void fsi_destroy(fsi_ctx* c) {
  if (!c) return;
  if (c->sweep) fsi_destroy(c->sweep);
  if (c->sweep_stream) cudaStreamDestroy(c->sweep_stream);
  for (auto& kv : c->graphs)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  for (double* p : {c->adj_ck, c->adj_sb, c->adj_vec, c->adj_B, c->adj_Bt})
    if (p) cudaFree(p);
  for (auto& L : c->lev)
    for (void* p : L.owned) cudaFree(p);
  for (void* p : c->owned) cudaFree(p);
  delete c;
}

int fsi_setup(const fsi_mesh* mesh, const fsi_params* p, fsi_ctx** out) {
  if (!out) return fail(FSI_EINVAL, "null output pointer");
  *out = nullptr;
  TRY(validate(mesh, p));
  fsi_ctx* c = new fsi_ctx();
  auto cleanup = [&](int rc) {
    fsi_destroy(c);
    return rc;
  };
  c->prm = *p;
  c->mesh_xb.assign(mesh->x_breaks, mesh->x_breaks + mesh->n_xseg + 1);
  c->mesh_yb.assign(mesh->y_breaks, mesh->y_breaks + mesh->n_yseg + 1);
  c->mesh_nx.assign(mesh->nx_seg, mesh->nx_seg + mesh->n_xseg);
  c->mesh_ny.assign(mesh->ny_seg, mesh->ny_seg + mesh->n_yseg);
  c->mesh_desc = *mesh;
  c->mesh_desc.x_breaks = c->mesh_xb.data();
  c->mesh_desc.y_breaks = c->mesh_yb.data();
  c->mesh_desc.nx_seg = c->mesh_nx.data();
  c->mesh_desc.ny_seg = c->mesh_ny.data();
  c->S = p->max_batch;
  c->m = p->gmres_restart;
  c->P = Phys{p->rho_f, p->nu_f, p->rho_s, p->mu_s, p->lambda_s, p->vbar, p->ramp_t,
              mesh->y_breaks[mesh->n_yseg] - mesh->y_breaks[0], mesh->y_breaks[0], p->alpha0};
  const double box[4] = {mesh->solid_x0, mesh->solid_x1, mesh->solid_y0, mesh->solid_y1};
  // level hierarchy
  HostMesh h0;
  finest_mesh(mesh, h0);
  std::vector<HostMesh> hs{h0};
  while ((size_t)hs.back().n_nodes * 5 > (size_t)p->mg_coarsest_max_dofs) {
    const HostMesh& f = hs.back();
    HostMesh hc;
    coarsen_axis(f.xv, f.xseg, hc.xv, hc.xseg);
    coarsen_axis(f.yv, f.yseg, hc.yv, hc.yseg);
    if (hc.xv.size() == f.xv.size() && hc.yv.size() == f.yv.size()) break;
    build_mesh(hc, mesh->has_solid != 0, box);
    hs.push_back(hc);
  }
  if ((size_t)hs.back().n_nodes * 5 > 4096) return cleanup(fail(FSI_EINVAL, "coarsest level too large"));
  c->lev.resize(hs.size());
  int rc = upload_tables();
  if (rc) return cleanup(rc);
  for (size_t l = 0; l < hs.size(); ++l) {
    c->lev[l].h = hs[l];
    const bool ff = p->ff_operator && (p->precision == 0 || (p->precision == 2 && l == 0));
    rc = setup_level(c->lev[l], c->S, l + 1 == hs.size(), l > 0, ff);
    if (rc) return cleanup(rc);
    if (l > 0 && (rc = setup_transfer(c->lev[l], c->lev[l - 1]))) return cleanup(rc);
  }
  c->n = c->lev[0].n;
  if (mesh->has_solid) {
    const HostMesh& h = c->lev[0].h;
    const double xt = 0.5 * (mesh->solid_x0 + mesh->solid_x1), yt = mesh->solid_y1;
    for (int j = 0; j < h.nny; ++j)
      for (int i = 0; i < h.nnx; ++i)
        if (std::fabs(h.xn[i] - xt) < 1e-12 && std::fabs(h.yn[j] - yt) < 1e-12) c->tip = j * h.nnx + i;
  }
  const size_t S = c->S, n = c->n, m = c->m;
  auto A = [&](auto** ptr, size_t cnt) { return dalloc(c->owned, ptr, cnt); };
  if ((rc = A(&c->Uit, S * n)) || (rc = A(&c->Uold, S * n)) || (rc = A(&c->R, S * n)) || (rc = A(&c->dU, S * n)) ||
      (rc = A(&c->w, S * n)) || (rc = A(&c->V, S * (m + 1) * n)) || (rc = A(&c->Z, S * m * n)) ||
      (rc = A(&c->H, S * (m + 1) * m)) || (rc = A(&c->cs, S * m)) || (rc = A(&c->sn, S * m)) ||
      (rc = A(&c->g, S * (m + 1))) || (rc = A(&c->y, S * m)) || (rc = A(&c->hcol, S * (m + 1))) ||
      (rc = A(&c->hcol2, S * (m + 1))) || (rc = A(&c->scal, S)) || (rc = A(&c->resid, S)) ||
      (rc = A(&c->partial, S * nblk(n, RED_CHUNK) * 64)) || (rc = A(&c->nv, S)) || (rc = A(&c->status, S)) ||
      (rc = A(&c->active, S)) || (rc = A(&c->active2, S)) || (rc = A(&c->t_dev, S)) ||
      (rc = A(&c->p_in, S * n)) || (rc = A(&c->p_out, S * n)) || (rc = A(&c->tc_status, 1)))
    return cleanup(rc);
  if (cudaMemset(c->tc_status, 0, sizeof(int)) != cudaSuccess) return cleanup(fail(FSI_ECUDA, "set-up failed"));
  for (auto& L : c->lev) L.async_status = c->tc_status;
  // the tables were copied with synchronous copies on the legacy stream; wait
  // for their DMA without waiting on other contexts' non-blocking streams
  if (cudaStreamSynchronize(cudaStreamLegacy) != cudaSuccess) return cleanup(fail(FSI_ECUDA, "set-up failed"));
  *out = c;
  return FSI_OK;
}

int fsi_n_nodes(const fsi_ctx* c) { return c ? c->lev[0].h.n_nodes : FSI_EINVAL; }
int fsi_n_dofs(const fsi_ctx* c) { return c ? (int)c->n : FSI_EINVAL; }
int fsi_n_levels(const fsi_ctx* c) { return c ? (int)c->lev.size() : FSI_EINVAL; }
int fsi_nnzb(const fsi_ctx* c) { return c ? c->lev[0].h.nnzb : FSI_EINVAL; }

int fsi_bsr_pattern(const fsi_ctx* c, int* rowptr, int* colidx) {
  if (!c || !rowptr || !colidx) return fail(FSI_EINVAL, "null argument");
  const HostMesh& h = c->lev[0].h;
  std::memcpy(rowptr, h.rowptr.data(), h.rowptr.size() * sizeof(int));
  std::memcpy(colidx, h.colidx.data(), h.colidx.size() * sizeof(int));
  return FSI_OK;
}

int fsi_residual(fsi_ctx* c, int S, const double* U, const double* U_old, const double* t_new, double k,
                 double theta, double* R, void* stream) {
  if (!c || !U || !U_old || !t_new || !R) return fail(FSI_EINVAL, "null argument");
  if (S < 1 || S > c->S) return fail(FSI_EINVAL, "batch size outside 1..max_batch");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<uint8_t> act(S, 1);
  CK(cudaMemcpyAsync(c->t_dev, t_new, S * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(c->active, act.data(), S, cudaMemcpyHostToDevice, st));
  c->n_act = g_nact = count_active(act);
  TRY(residual(c, c->lev[0], S, U, U_old, k, theta, c->active, R, st));
  CK(cudaStreamSynchronize(st));
  return FSI_OK;
}

int fsi_jacobian(fsi_ctx* c, int S, const double* U, const double* U_old, double k, double theta, double* vals,
                 void* stream) {
  if (!c || !U || !U_old || !vals) return fail(FSI_EINVAL, "null argument");
  if (S < 1 || S > c->S) return fail(FSI_EINVAL, "batch size outside 1..max_batch");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<uint8_t> act(S, 1);
  CK(cudaMemcpyAsync(c->active, act.data(), S, cudaMemcpyHostToDevice, st));
  c->n_act = g_nact = count_active(act);
  TRY(jacobian<double>(c, c->lev[0], S, U, U_old, k, theta, c->active, vals, st));
  CK(cudaStreamSynchronize(st));
  return FSI_OK;
}

int fsi_jacobian_f32(fsi_ctx* c, int S, const double* U, const double* U_old, double k, double theta, float* vals,
                     void* stream) {
  if (!c || !U || !U_old || !vals) return fail(FSI_EINVAL, "null argument");
  if (S < 1 || S > c->S) return fail(FSI_EINVAL, "batch size outside 1..max_batch");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<uint8_t> act(S, 1);
  CK(cudaMemcpyAsync(c->active, act.data(), S, cudaMemcpyHostToDevice, st));
  c->n_act = g_nact = count_active(act);
  TRY(jacobian<float>(c, c->lev[0], S, U, U_old, k, theta, c->active, vals, st));
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, c->tc_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (flag) return fail(FSI_ECUDA, "tensor-core element Jacobian: an MMA completion was not seen within the poll limit");
  return FSI_OK;
}

int fsi_bsr_spmv(fsi_ctx* c, int S, const double* vals, const double* x, double* y, void* stream) {
  if (!c || !vals || !x || !y) return fail(FSI_EINVAL, "null argument");
  if (S < 1 || S > c->S) return fail(FSI_EINVAL, "batch size outside 1..max_batch");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<uint8_t> act(S, 1);
  CK(cudaMemcpyAsync(c->active, act.data(), S, cudaMemcpyHostToDevice, st));
  c->n_act = g_nact = count_active(act);
  TRY((spmv<double, false>(c->lev[0], S, vals, x, nullptr, c->active, y, st)));
  return FSI_OK;
}

int fsi_bsr_spmv_f32(fsi_ctx* c, int S, const float* vals, const float* x, float* y, void* stream) {
  if (!c || !vals || !x || !y) return fail(FSI_EINVAL, "null argument");
  if (S < 1 || S > c->S) return fail(FSI_EINVAL, "batch size outside 1..max_batch");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<uint8_t> act(S, 1);
  CK(cudaMemcpyAsync(c->active, act.data(), S, cudaMemcpyHostToDevice, st));
  c->n_act = g_nact = count_active(act);
  TRY((spmv<float, false>(c->lev[0], S, vals, x, nullptr, c->active, y, st)));
  return FSI_OK;
}

int fsi_bsr_spmv_ff(fsi_ctx* c, int S, const double* vals, const double* x, double* y, void* stream) {
  if (!c || !vals || !x || !y) return fail(FSI_EINVAL, "null argument");
  if (S < 1 || S > c->S) return fail(FSI_EINVAL, "batch size outside 1..max_batch");
  Level& L = c->lev[0];
  if (!L.Aff) return fail(FSI_EINVAL, "the context was set up without ff_operator");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<uint8_t> act(S, 1);
  CK(cudaMemcpyAsync(c->active, act.data(), S, cudaMemcpyHostToDevice, st));
  c->n_act = g_nact = count_active(act);
  // the operator's float pairs, as a Jacobian assembly leaves them (they then belong to vals)
  const size_t cnt = (size_t)L.h.nnzb * 25;
  LAUNCH_WB(3.0 * cnt * c->n_act, 16.0 * cnt * c->n_act, KI_TO_FF, k_to_ff, (dim3(nblk(cnt, 256), S)), 256, 0, st, cnt, vals, cnt, c->active, L.Aff, cnt);
  TRY(launch_check());
  L.aff_of = vals;
  const int rc = spmv<double, false>(L, S, vals, x, nullptr, c->active, y, st);
  L.aff_of = nullptr;   // the pairs are not the context's operator
  return rc;
}

int fsi_bsr_spmv_variant(fsi_ctx* c, int S, int value_type, int tile_rows, const void* vals, const void* x, void* y,
                         void* stream) {
  if (!c || !vals || !x || !y) return fail(FSI_EINVAL, "null argument");
  if (S < 1 || S > c->S) return fail(FSI_EINVAL, "batch size outside 1..max_batch");
  if (value_type < 0 || value_type > 2) return fail(FSI_EINVAL, "value_type must be 0, 1 or 2");
  Level& L = c->lev[0];
  int t = -1;
  if (tile_rows == 0) t = 0;
  for (int i = 0; i < 4; ++i)
    if (tile_rows == kSptRows[i]) t = i + 1;
  if (t < 0) return fail(FSI_EINVAL, "tile_rows must be 0, 8, 16, 32 or 64");
  const size_t vsz = value_type == 1 ? 4 : 8;
  if (t > 0 && (size_t)L.spt_blocks[t - 1] * 25 * vsz + 16 > kSptMaxSmem)
    return fail(FSI_EINVAL, "the tile's blocks do not fit in shared memory");
  if (value_type == 2 && !L.Aff) return fail(FSI_EINVAL, "the context was set up without ff_operator");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<uint8_t> act(S, 1);
  CK(cudaMemcpyAsync(c->active, act.data(), S, cudaMemcpyHostToDevice, st));
  c->n_act = g_nact = count_active(act);
  const double blocks = (double)L.h.nnzb;
  const double work = 50.0 * blocks * S;
  const double bytes = (double)S * vsz * (25.0 * blocks + 2.0 * (double)L.n) + 4.0 * (blocks + 2.0 * L.h.n_nodes + 1.0);
  if (value_type == 0) {
    spt_run<double, double, false>(L, S, (const double*)vals, (const double*)x, nullptr, c->active, (double*)y, st,
                                   work, bytes, KI_BSR_SPMV, t);
  } else if (value_type == 1) {
    spt_run<float, float, false>(L, S, (const float*)vals, (const float*)x, nullptr, c->active, (float*)y, st, work,
                                 bytes, KI_BSR_SPMV, t);
  } else {
    const size_t cnt = (size_t)L.h.nnzb * 25;
    LAUNCH_WB(3.0 * cnt * S, 16.0 * cnt * S, KI_TO_FF, k_to_ff, (dim3(nblk(cnt, 256), S)), 256, 0, st, cnt, (const double*)vals, cnt, c->active, L.Aff, cnt);
    LAUNCH_WB(3.0 * L.n * S, 16.0 * L.n * S, KI_TO_FF, k_to_ff, (dim3(nblk(L.n, 256), S)), 256, 0, st, L.n, (const double*)x, L.n, c->active, L.xff, L.n);
    L.aff_of = nullptr;   // the pairs are not the context's operator
    spt_run<float2, double, false>(L, S, L.Aff, L.xff, nullptr, c->active, (double*)y, st, work, bytes,
                                   KI_BSR_SPMV_FF, t);
  }
  TRY(launch_check());
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, L.async_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (flag) return fail(FSI_ECUDA, "a bulk copy or MMA completion was not seen within the poll limit");
  return FSI_OK;
}

// Resets the statistics of a call, keeping the caller's per-slice array
// (cleared for the call's S slices).
static void reset_stats(fsi_ctx* c, fsi_stats* stats, int S) {
  c->slice_offset = 0;
  if (!stats) return;
  int* ss = stats->slice_status;
  const int len = stats->slice_status_len;
  *stats = fsi_stats{};
  stats->slice_status = ss;
  stats->slice_status_len = len;
  if (ss)
    for (int s = 0; s < std::min(S, len); ++s) ss[s] = FSI_OK;
}

int fsi_theta_step(fsi_ctx* c, int S, const double* U_old, const double* t_old, double k, double theta,
                   double* U_new, fsi_stats* stats, void* stream) {
  if (!c || !U_old || !t_old || !U_new) return fail(FSI_EINVAL, "null argument");
  reset_stats(c, stats, S);
  // a single step may be large: keep at most the coarsest inverse across Newton iterations
  int rc = theta_step(c, S, U_old, t_old, k, theta, U_new, stats, (cudaStream_t)stream, std::min(c->prm.mg_reuse, 1),
                      false);
  if (stats) stats->status = rc;
  return rc;
}

int fsi_fine(fsi_ctx* c, int S, const double* U0, const double* t0, double* U1, fsi_stats* stats, void* stream) {
  if (!c || !U0 || !t0 || !U1) return fail(FSI_EINVAL, "null argument");
  if (S < 1) return fail(FSI_EINVAL, "empty batch");
  reset_stats(c, stats, S);
  int rc = propagate_chunked(c, S, U0, t0, U1, true, stats, (cudaStream_t)stream);
  if (stats) stats->status = rc;
  return rc;
}

int fsi_coarse(fsi_ctx* c, int S, const double* U0, const double* t0, double* U1, fsi_stats* stats, void* stream) {
  if (!c || !U0 || !t0 || !U1) return fail(FSI_EINVAL, "null argument");
  if (S < 1) return fail(FSI_EINVAL, "empty batch");
  reset_stats(c, stats, S);
  int rc = propagate_chunked(c, S, U0, t0, U1, false, stats, (cudaStream_t)stream);
  if (stats) stats->status = rc;
  return rc;
}

int parareal_iterate(fsi_ctx* c, double* U, int max_iter, double tol, fsi_parareal_stats* stats, void* stream) {
  if (!c || !U) return fail(FSI_EINVAL, "null argument");
  if (max_iter < 0) return fail(FSI_EINVAL, "negative iteration count");
  cudaStream_t st = (cudaStream_t)stream;
  const int N = c->prm.n_slices;
  fsi_parareal_stats loc{};
  if (stats) {
    loc.history = stats->history;
    loc.history_len = stats->history_len;
  }
  TRY(parareal_workspace(c));
  int rc;
  c->pr_iter = -1;
  if (c->prm.pipeline_chunk > 0 && max_iter > 0 && N > 1) {
    rc = parareal_pipelined(c, U, max_iter, tol, loc, st);
    if (rc == FSI_OK) c->pr_iter = loc.iterations;
  } else {
    rc = parareal_serial(c, U, max_iter, tol, loc, st);
  }
  if (rc != FSI_OK) {
    c->pr_iter = -1;
    return rc;
  }
  if (stats) *stats = loc;
  return FSI_OK;
}

int parareal_continue(fsi_ctx* c, double* U, int n_iter, double tol, fsi_parareal_stats* stats, void* stream) {
  if (!c || !U) return fail(FSI_EINVAL, "null argument");
  if (n_iter < 0) return fail(FSI_EINVAL, "negative iteration count");
  if (c->pr_iter < 0 || !c->Cold)
    return fail(FSI_EINVAL, "parareal_continue: no completed Parareal run to continue on this context");
  cudaStream_t st = (cudaStream_t)stream;
  fsi_parareal_stats loc{};
  if (stats) {
    loc.history = stats->history;
    loc.history_len = stats->history_len;
  }
  loc.iterations = c->pr_iter;
  const int it0 = c->pr_iter + 1;
  const int rc = parareal_iterations(c, U, it0, c->pr_iter + n_iter, tol, loc, st);
  if (rc != FSI_OK) {
    c->pr_iter = -1;
    return rc;
  }
  if (stats) *stats = loc;
  return FSI_OK;
}

int fsi_profile_enable(unsigned long long kernel_mask) {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  g_prof.mask = kernel_mask;
  g_prof.used = 0;
  g_prof.rec_id.clear();
  g_prof.rec_ev.clear();
  g_prof.rec_work.clear();
  g_prof.rec_bytes.clear();
  for (int i = 0; i < KI_COUNT; ++i) g_prof.gms[i] = g_prof.gwork[i] = g_prof.gbytes[i] = 0.0, g_prof.gcnt[i] = 0;
  ++g_prof.epoch;
  return FSI_OK;
}

int fsi_profile_read(int kernel_id, double* total_ms, long long* timed_launches, double* total_flops) {
  if (kernel_id < 0 || kernel_id >= KI_COUNT || !total_ms || !timed_launches || !total_flops)
    return fail(FSI_EINVAL, "bad kernel id or null output");
  double ms = 0.0, work = 0.0;
  long long cnt = 0;
  std::lock_guard<std::mutex> lk(g_prof.mu);
  for (size_t r = 0; r < g_prof.rec_id.size(); ++r) {
    if (g_prof.rec_id[r] != kernel_id) continue;
    const size_t ev = g_prof.rec_ev[r];
    CK(cudaEventSynchronize(g_prof.pool[ev + 1]));
    float e = 0.f;
    CK(cudaEventElapsedTime(&e, g_prof.pool[ev], g_prof.pool[ev + 1]));
    ms += e;
    work += g_prof.rec_work[r];
    ++cnt;
  }
  *total_ms = ms + g_prof.gms[kernel_id];
  *timed_launches = cnt + g_prof.gcnt[kernel_id];
  *total_flops = work + g_prof.gwork[kernel_id];
  return FSI_OK;
}

int fsi_profile_read_bytes(int kernel_id, double* total_bytes) {
  if (kernel_id < 0 || kernel_id >= KI_COUNT || !total_bytes) return fail(FSI_EINVAL, "bad kernel id or null output");
  double b = 0.0;
  std::lock_guard<std::mutex> lk(g_prof.mu);
  for (size_t r = 0; r < g_prof.rec_id.size(); ++r)
    if (g_prof.rec_id[r] == kernel_id) b += g_prof.rec_bytes[r];
  *total_bytes = b + g_prof.gbytes[kernel_id];
  return FSI_OK;
}

namespace {
__device__ int g_tc_status;
}

int fsi_tc_tile_product(int nsplit, const float* A, const float* B, float* D, void* stream) {
  if (!A || !B || !D) return fail(FSI_EINVAL, "null argument");
  if (nsplit < 1 || nsplit > 3) return fail(FSI_EINVAL, "fsi_tc_tile_product: nsplit outside 1..3");
  cudaStream_t st = (cudaStream_t)stream;
  int* status = nullptr;
  CK(cudaGetSymbolAddress((void**)&status, g_tc_status));
  CK(cudaMemsetAsync(status, 0, sizeof(int), st));
  if (nsplit == 1) k_tc_tile_product<1><<<1, 128, 0, st>>>(A, B, D, status);
  else if (nsplit == 2) k_tc_tile_product<2><<<1, 128, 0, st>>>(A, B, D, status);
  else k_tc_tile_product<3><<<1, 128, 0, st>>>(A, B, D, status);
  TRY(launch_check());
  int h = 0;
  CK(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (h) return fail(FSI_ECUDA, "fsi_tc_tile_product: MMA completion not seen within the poll limit");
  return FSI_OK;
}

int fsi_fp64_probe(int blocks, int iters, double seed, double* sink, void* stream) {
  if (blocks < 1 || iters < 1 || !sink) return fail(FSI_EINVAL, "fsi_fp64_probe: bad size or null sink");
  k_fma_probe<<<blocks, FMA_PROBE_THREADS, 0, (cudaStream_t)stream>>>(iters, seed, sink);
  return launch_check();
}

long long fsi_launch_count(int kernel_id) {
  if (kernel_id < 0) return g_prof.total.load();
  return kernel_id < KI_COUNT ? g_prof.launches[kernel_id].load() : -1LL;
}

int fsi_kernel_count(void) { return KI_COUNT; }

const char* fsi_kernel_name(int kernel_id) {
  return (kernel_id >= 0 && kernel_id < KI_COUNT) ? kKernelNames[kernel_id] : "";
}

int fsi_jacobian_old(fsi_ctx* c, int S, const double* U, const double* U_old, double k, double theta,
                     double* vals, void* stream) {
  if (!c || !U || !U_old || !vals) return fail(FSI_EINVAL, "null argument");
  if (S < 1 || S > c->S) return fail(FSI_EINVAL, "batch size outside 1..max_batch");
  cudaStream_t st = (cudaStream_t)stream;
  Level& L = c->lev[0];
  std::vector<uint8_t> act(S, 1);
  CK(cudaMemcpyAsync(c->active, act.data(), S, cudaMemcpyHostToDevice, st));
  c->n_act = g_nact = S;
  LAUNCH(KI_CELL_JACOBIAN_OLD, k_cell_jacobian<true>, (dim3(L.h.n_cells, S)), JAC_THREADS, 0, st, L.dm, c->P, U, U_old, L.n, k, theta, 1.0, c->active, L.Ke);
  LAUNCH(KI_ASSEMBLE_BSR, k_assemble_bsr<double>, (dim3(nblk((size_t)L.h.nnzb * 5, 128), S)), 128, 0, st, L.dm, L.Ke, c->active, vals, 0.0);
  TRY(launch_check());
  CK(cudaStreamSynchronize(st));
  return FSI_OK;
}

int fsi_set_material(fsi_ctx* c, double mu_s, double lambda_s, double vbar) {
  if (!c || !(mu_s > 0) || !(lambda_s > 0) || !(vbar >= 0)) return fail(FSI_EINVAL, "bad material");
  c->prm.mu_s = c->P.mu_s = mu_s;
  c->prm.lambda_s = c->P.lambda_s = lambda_s;
  c->prm.vbar = c->P.vbar = vbar;
  return FSI_OK;
}

int fsi_adjoint(fsi_ctx* c, const double* U0, double t0, int n_steps, double* J_out, double* grad, fsi_stats* stats,
                void* stream) {
  if (!c || !U0 || !J_out || !grad) return fail(FSI_EINVAL, "null argument");
  if (stats) *stats = fsi_stats{};
  int rc = adjoint_impl(c, U0, t0, n_steps, J_out, grad, stats, (cudaStream_t)stream);
  if (stats) stats->status = rc;
  return rc;
}

int fsi_residual_noalloc(fsi_ctx* c, int S, const double* U, const double* U_old, const double* t_new, double k,
                         double theta, double* R, void* stream) {
  if (!c || !U || !U_old || !t_new || !R) return fail(FSI_EINVAL, "null argument");
  if (S < 1 || S > kNaMaxSlices) return fail(FSI_EINVAL, "fsi_residual_noalloc: S outside 1..256");
  Level& L = c->lev[0];
  if ((size_t)S * L.h.n_cells * 45 > kNaDoubles - kNaCellOffset)
    return fail(FSI_EINVAL, "fsi_residual_noalloc: S * cells * 45 exceeds the 16 MiB static scratch "
                            "(2,096,864 doubles)");
  double* scratch = nullptr;
  TRY(na_scratch(&scratch));
  cudaStream_t st = (cudaStream_t)stream;
  uint8_t* act = reinterpret_cast<uint8_t*>(scratch);
  double* t_dev = scratch + 32;
  double* cellbuf = scratch + kNaCellOffset;
  CK(cudaMemsetAsync(act, 1, S, st));   // every slice active
  CK(cudaMemcpyAsync(t_dev, t_new, S * sizeof(double), cudaMemcpyHostToDevice, st));
  g_nact = S;
  LAUNCH(KI_CELL_RESIDUAL, k_cell_residual, (dim3(nblk(L.h.n_cells, 128), S)), 128, 0, st, L.dm, c->P, U, U_old, L.n,
         k, theta, act, cellbuf);
  LAUNCH(KI_GATHER_RESIDUAL, k_gather_residual, (dim3(nblk(L.h.n_nodes, 128), S)), 128, 0, st, L.dm, c->P, cellbuf,
         U, L.n, t_dev, act, R);
  TRY(launch_check());
  CK(cudaStreamSynchronize(st));
  return FSI_OK;
}

}  // extern "C"
