// 3D path of the library: hexahedral Q2 elements with 7 unknowns per node
// (v, u, p). The theta step of Sec. 2.3 is solved by Newton's method, with
// FGMRES preconditioned by a geometric multigrid V-cycle (block Vanka smoother,
// additive or over eight cell colours; Q2 transfers; a dense inverse or
// smoother sweeps on the coarsest level), for S slices per launch (grid.y =
// slice). On top sit the propagators F and C of Sec. 3 and the Parareal
// iteration. Every per-entry step is a __host__ __device__ function of the 3D
// headers, which are also run on the host against the oracle. This file holds
// the device tables, the kernels that run those functions, and the solver loops.
//
// Layout in HBM: states [S][n_nodes][7] FP64; Jacobian blocks [S][nnzb][7][7]
// (FP64 for the Krylov operator, T = FP64 or FP32 for the multigrid levels);
// element matrices [S][cells][189][189] FP64 (scratch of the assembly); Vanka
// factors [S][cells][189^2] in T; Krylov bases [S][m+1][n] FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/fsi.h"
#include "fsi_element3d.cuh"
#include "fsi_internal.h"
#include "fsi_mesh3d.h"
#include "fsi_mg3d.h"
#include "fsi_vanka3.h"

namespace {

int fail3(int code, const std::string& msg) { return fsi_record_error(code, msg); }

#define CK3(call)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) return fail3(FSI_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define TRY3(call)                  \
  do {                              \
    int rc_ = (call);               \
    if (rc_ != FSI_OK) return rc_;  \
  } while (0)

inline unsigned nb3(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

int launched3() {
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FSI_OK : fail3(FSI_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
}

// Launch accounting of the 3D kernels: every launch is counted; with profiling
// on, each launch is bracketed by two CUDA events on its stream, read later
// (no synchronisation on the launch path).
enum Ki3 {
  KI3_CELL_JACOBIAN,
  KI3_CELL_RESIDUAL,
  KI3_GATHER_RESIDUAL,
  KI3_ASSEMBLE,
  KI3_INTERP_STATE,
  KI3_AXPBY,
  KI3_DENSE_FROM_BSR,
  KI3_IDENTITY_INACTIVE,
  KI3_CONVERT,
  KI3_VANKA_SETUP,
  KI3_RESID_ROWS,
  KI3_VANKA_APPLY,
  KI3_VANKA_SCATTER,
  KI3_SPMV,
  KI3_VANKA_GATHER,
  KI3_FILL,
  KI3_DENSE_APPLY,
  KI3_RESTRICT,
  KI3_PROLONG_ADD,
  KI3_DOTS_PARTIAL,
  KI3_DOTS_FINISH,
  KI3_SCALE,
  KI3_SUB_BASIS,
  KI3_ADD_BASIS,
  KI3_APPLY_DIRICHLET,
  KI3_PARAREAL_CORRECT,
  KI3_COUNT
};
const char* const kKernelNames3[KI3_COUNT] = {
    "k3_cell_jacobian",
    "k3_cell_residual",
    "k3_gather_residual",
    "k3_assemble",
    "k3_interp_state",
    "k3_axpby",
    "k3_dense_from_bsr",
    "k3_identity_inactive",
    "k3_convert",
    "k3_vanka_setup",
    "k3_resid_rows",
    "k3_vanka_apply",
    "k3_vanka_scatter",
    "k3_spmv",
    "k3_vanka_gather",
    "k3_fill",
    "k3_dense_apply",
    "k3_restrict",
    "k3_prolong_add",
    "k3_dots_partial",
    "k3_dots_finish",
    "k3_scale",
    "k3_sub_basis",
    "k3_add_basis",
    "k3_apply_dirichlet",
    "k3_parareal_correct",
};

struct Prof3 {
  std::mutex mu;
  std::atomic<bool> on{false};
  std::atomic<long long> launches[KI3_COUNT] = {};
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[KI3_COUNT];
};
Prof3 g_prof3;

inline void prof3_pre(int id, cudaStream_t st, cudaEvent_t* a) {
  g_prof3.launches[id].fetch_add(1, std::memory_order_relaxed);
  *a = nullptr;
  if (!g_prof3.on.load(std::memory_order_relaxed)) return;
  if (cudaEventCreate(a) != cudaSuccess || cudaEventRecord(*a, st) != cudaSuccess) *a = nullptr;
}

inline void prof3_post(int id, cudaEvent_t a, cudaStream_t st) {
  if (!a) return;
  cudaEvent_t b = nullptr;
  if (cudaEventCreate(&b) != cudaSuccess || cudaEventRecord(b, st) != cudaSuccess) {
    cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    return;
  }
  std::lock_guard<std::mutex> lock(g_prof3.mu);
  g_prof3.ev[id].push_back({a, b});
}

#define P3(id, kern, grid, block, smem, st, ...)   \
  do {                                              \
    cudaEvent_t ev_;                                \
    prof3_pre(id, st, &ev_);                        \
    kern<<<grid, block, smem, st>>>(__VA_ARGS__);   \
    prof3_post(id, ev_, st);                        \
  } while (0)

__constant__ fsi3::Tables3 c_tab3;

// Device tables of one level.
struct Dev3 {
  fsi3::Mesh3View v;          // device pointers
  const int* cell_nodes;      // [cells][27]
  const double* cell_h;       // [cells][3]
  const int* rowptr;          // [n_nodes + 1]
  int nnzb, nx, ny, nz;
};

struct Phys3D {
  double rho_f, nu_f, rho_s, mu_s, lambda_s, vbar, ramp_t, alpha0;
};

// ---------------------------------------------------------------------------
// Kernels (blockIdx.y = slice; inactive slices return at once)
// ---------------------------------------------------------------------------
__global__ void k3_apply_dirichlet(Dev3 d, Phys3D P, double* __restrict__ U, size_t stride,
                                   const double* __restrict__ t, const uint8_t* __restrict__ active) {
  const int s = blockIdx.y;
  const int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || node >= d.v.n_nodes) return;
  const uint8_t nf = d.v.node_flags[node];
  double* x = U + s * stride + (size_t)node * 7;
  for (int c = 0; c < 6; ++c)
    if (fsi3::identity_row3(nf, c)) x[c] = fsi3::dirichlet3(d.v, node, c, t[s], P.vbar, P.ramp_t);
}

// Per cell: stabilisation weight from the old state, then the cell residual
// Re[s][cell][189]; one CTA per (cell, slice) running the cooperative routine.
constexpr int CR3_THREADS = 192;

__global__ void __launch_bounds__(CR3_THREADS, 1) k3_cell_residual(Dev3 d, Phys3D P, const double* __restrict__ U,
                                                               const double* __restrict__ Uo, size_t stride, double k,
                                                               double theta, const uint8_t* __restrict__ active,
                                                               double* __restrict__ Re) {
  const int s = blockIdx.y;
  const int cell = blockIdx.x;
  if (!active[s] || cell >= d.v.n_cells) return;
  __shared__ double shr[fsi3::CR3_TOTAL];
  __shared__ double alpha_s;
  const int* cn = d.cell_nodes + (size_t)cell * 27;
  for (int e = threadIdx.x; e < 189; e += blockDim.x) {
    const size_t g = s * stride + (size_t)cn[e / 7] * 7 + e % 7;
    shr[fsi3::CR3_UE + e] = U[g];
    shr[fsi3::CR3_UE + 189 + e] = Uo[g];
  }
  __syncthreads();
  const double* h = d.cell_h + (size_t)cell * 3;
  if (threadIdx.x == 0) alpha_s = fsi3::stab_weight3(c_tab3, shr + fsi3::CR3_UE + 189, h, P.alpha0, P.rho_f, P.nu_f);
  __syncthreads();
  const uint8_t cf = d.v.cell_flags[cell];
  const fsi3::Phys3 ph{P.rho_f, P.nu_f, P.rho_s, P.mu_s, P.lambda_s};
  fsi3::cell_residual3_cta(fsi3::DevCta{(int)threadIdx.x, (int)blockDim.x}, ph, c_tab3, h, cf & fsi3::C3_SOLID,
                           cf & fsi3::C3_OUTFLOW, k, theta, alpha_s, shr,
                           Re + ((size_t)s * d.v.n_cells + cell) * 189);
}

__global__ void k3_gather_residual(Dev3 d, Phys3D P, const double* __restrict__ Re, const double* __restrict__ U,
                                   size_t stride, const double* __restrict__ t, const uint8_t* __restrict__ active,
                                   double* __restrict__ R) {
  const int s = blockIdx.y;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || e >= d.v.n_nodes * 7) return;
  R[s * stride + e] = fsi3::gather3(d.v, Re + (size_t)s * d.v.n_cells * 189, U + s * stride, e / 7, e % 7, t[s],
                                    P.vbar, P.ramp_t);
}

// Per cell: the element matrix Ke[s][cell][189][189], one CTA per (cell, slice)
// running the cooperative routine; lps_scale multiplies the stabilisation
// weight (coarse multigrid levels). Dynamic shared memory CJ3_TOTAL doubles.
constexpr int CJ3_THREADS = 256;
static_assert(CJ3_THREADS >= 7 * 32, "the cell Jacobian's field flags take one warp per test field");

__global__ void __launch_bounds__(CJ3_THREADS) k3_cell_jacobian(Dev3 d, Phys3D P, const double* __restrict__ U,
                                                               const double* __restrict__ Uo, size_t stride, double k,
                                                               double theta, double lps_scale,
                                                               const uint8_t* __restrict__ active,
                                                               double* __restrict__ Ke) {
  const int s = blockIdx.y;
  const int cell = blockIdx.x;
  if (!active[s] || cell >= d.v.n_cells) return;
  extern __shared__ __align__(16) double shj[];
  const int* cn = d.cell_nodes + (size_t)cell * 27;
  for (int e = threadIdx.x; e < 189; e += blockDim.x) {
    const size_t g = s * stride + (size_t)cn[e / 7] * 7 + e % 7;
    shj[fsi3::CJ3_UE + e] = U[g];
    shj[fsi3::CJ3_UE + 189 + e] = Uo[g];
  }
  __syncthreads();
  const double* h = d.cell_h + (size_t)cell * 3;
  double* alpha_slot = shj + fsi3::CJ3_FLAG + 7;   // the eighth flag slot is free
  if (threadIdx.x == 0)
    *alpha_slot = lps_scale * fsi3::stab_weight3(c_tab3, shj + fsi3::CJ3_UE + 189, h, P.alpha0, P.rho_f, P.nu_f);
  __syncthreads();
  const double alpha = *alpha_slot;
  const uint8_t cf = d.v.cell_flags[cell];
  const fsi3::Phys3 ph{P.rho_f, P.nu_f, P.rho_s, P.mu_s, P.lambda_s};
  fsi3::cell_jacobian3_cta(fsi3::DevCta{(int)threadIdx.x, (int)blockDim.x}, ph, c_tab3, h, cf & fsi3::C3_SOLID,
                           cf & fsi3::C3_OUTFLOW, k, theta, alpha, shj,
                           Ke + ((size_t)s * d.v.n_cells + cell) * 189 * 189);
}

int launch_cell_jacobian(const Dev3& d, int n_cells, int S, const Phys3D& P, const double* U, const double* Uo,
                         size_t stride, double k, double theta, double lps, const uint8_t* act, double* Ke,
                         cudaStream_t st) {
  const int smem = fsi3::CJ3_TOTAL * (int)sizeof(double);
  CK3(cudaFuncSetAttribute(k3_cell_jacobian, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  P3(KI3_CELL_JACOBIAN, (k3_cell_jacobian), (dim3(n_cells, S)), CJ3_THREADS, smem, st, d, P, U, Uo, stride, k, theta, lps, act, Ke);
  return launched3();
}

// A[s][b][r][c] = the fixed-order gather of the element matrices (identity rows: unit diagonal).
template <typename TO>
__global__ void k3_assemble(Dev3 d, const double* __restrict__ Ke, const uint8_t* __restrict__ active,
                            TO* __restrict__ A) {
  const int s = blockIdx.y;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || e >= (size_t)d.nnzb * 49) return;
  const int b = (int)(e / 49), rc = (int)(e % 49);
  A[(size_t)s * d.nnzb * 49 + e] =
      (TO)fsi3::assemble3(d.v, Ke + (size_t)s * d.v.n_cells * 189 * 189, b, rc / 7, rc % 7);
}

// y = b - A x (RESID) or y = A x, one thread per row; x has slice stride xstride,
// b and y slice stride ystride.
template <typename T, bool RESID>
__global__ void k3_spmv(Dev3 d, const T* __restrict__ A, const T* __restrict__ x, size_t xstride,
                        const T* __restrict__ bvec, size_t ystride, const uint8_t* __restrict__ active,
                        T* __restrict__ y) {
  const int s = blockIdx.y;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || e >= d.v.n_nodes * 7) return;
  const int node = e / 7, r = e % 7;
  const T* As = A + (size_t)s * d.nnzb * 49;
  const T* xs = x + s * xstride;
  T acc = 0;
  for (int b = d.rowptr[node]; b < d.rowptr[node + 1]; ++b) {
    const T* blk = As + (size_t)b * 49 + r * 7;
    const T* xj = xs + (size_t)d.v.colidx[b] * 7;
    for (int c = 0; c < 7; ++c) acc += blk[c] * xj[c];
  }
  y[s * ystride + e] = RESID ? bvec[s * ystride + e] - acc : acc;
}

// r = b - A x on the listed rows only (the nodes of one colour's cells; other rows untouched).
template <typename T>
__global__ void k3_resid_rows(Dev3 d, const T* __restrict__ A, const T* __restrict__ x, const T* __restrict__ bvec,
                              size_t stride, const int* __restrict__ nodes, int nnodes,
                              const uint8_t* __restrict__ active, T* __restrict__ y) {
  const int s = blockIdx.y;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || e >= nnodes * 7) return;
  const int node = nodes[e / 7], r = e % 7;
  const T* As = A + (size_t)s * d.nnzb * 49;
  const T* xs = x + s * stride;
  T acc = 0;
  for (int b = d.rowptr[node]; b < d.rowptr[node + 1]; ++b) {
    const T* blk = As + (size_t)b * 49 + r * 7;
    const T* xj = xs + (size_t)d.v.colidx[b] * 7;
    for (int c = 0; c < 7; ++c) acc += blk[c] * xj[c];
  }
  const size_t o = s * stride + (size_t)node * 7 + r;
  y[o] = bvec[o] - acc;
}

// y = a x + b y (types may differ: precision conversions of the preconditioner)
template <typename TI, typename TO>
__global__ void k3_axpby(int n, double a, const TI* __restrict__ x, size_t xs, double b,
                         const uint8_t* __restrict__ active, TO* __restrict__ y, size_t ys) {
  const int s = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || r >= n) return;
  const double yv = b == 0.0 ? 0.0 : b * (double)y[s * ys + r];
  y[s * ys + r] = (TO)(a * (double)x[s * xs + r] + yv);
}

template <typename T>
__global__ void k3_fill(int n, T v, const uint8_t* __restrict__ active, T* __restrict__ y, size_t ys) {
  const int s = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || r >= n) return;
  y[s * ys + r] = v;
}

// Block Vanka setup: one CTA per (cell, slice); dynamic shared memory vk3_setup_smem_bytes<T>().
template <typename T>
__global__ void __launch_bounds__(256) k3_vanka_setup(Dev3 d, const T* __restrict__ A,
                                                     const uint8_t* __restrict__ active, T* __restrict__ inv,
                                                     int* __restrict__ status) {
  const int s = blockIdx.y;
  const int cell = blockIdx.x;
  if (!active[s] || cell >= d.v.n_cells) return;
  extern __shared__ __align__(16) unsigned char smem3[];
  T* sh = reinterpret_cast<T*>(smem3);
  int* ish = reinterpret_cast<int*>(sh + fsi3::VK3_SH_T);
  const fsi3::DevCta cta{(int)threadIdx.x, (int)blockDim.x};
  const bool ok = fsi3::vk3_setup_cell(cta, d.v, A + (size_t)s * d.nnzb * 49, cell, sh, ish,
                                       inv + ((size_t)s * d.v.n_cells + cell) * fsi3::VK3_SIZE);
  if (!ok && threadIdx.x == 0) status[s] = -6;
}

// Local corrections cz[s][cell][189] of the listed cells (all cells when cells == nullptr).
template <typename T>
__global__ void __launch_bounds__(128) k3_vanka_apply(Dev3 d, const T* __restrict__ inv, const T* __restrict__ r,
                                                     size_t stride, const uint8_t* __restrict__ active,
                                                     const int* __restrict__ cells, int ncells, T* __restrict__ cz) {
  const int s = blockIdx.y;
  if (!active[s] || (int)blockIdx.x >= ncells) return;
  const int cell = cells ? cells[blockIdx.x] : (int)blockIdx.x;
  __shared__ T rl[189];
  __shared__ T ap[fsi3::VK3_AP_T];
  const int* cn = d.cell_nodes + (size_t)cell * 27;
  for (int e = threadIdx.x; e < 189; e += blockDim.x) rl[e] = r[s * stride + (size_t)cn[e / 7] * 7 + e % 7];
  __syncthreads();
  const fsi3::DevCta cta{(int)threadIdx.x, (int)blockDim.x};
  fsi3::vk3_apply_cell(cta, (d.v.cell_flags[cell] & fsi3::C3_U_DECOUPLED) != 0,
                       inv + ((size_t)s * d.v.n_cells + cell) * fsi3::VK3_SIZE, rl, ap,
                       cz + ((size_t)s * d.v.n_cells + cell) * 189);
}

// Additive smoothing: x += omega / cnt * (sum of the node's cell corrections).
template <typename T>
__global__ void k3_vanka_gather(Dev3 d, const T* __restrict__ cz, double omega, size_t stride,
                                const uint8_t* __restrict__ active, T* __restrict__ x) {
  const int s = blockIdx.y;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || e >= d.v.n_nodes * 7) return;
  x[s * stride + e] += fsi3::vk3_gather(d.v, cz + (size_t)s * d.v.n_cells * 189, omega, e / 7, e % 7);
}

// Multiplicative smoothing, one colour: its cells share no node, so every dof of
// those cells takes its one cell's correction: x += omega z.
template <typename T>
__global__ void k3_vanka_scatter(Dev3 d, const int* __restrict__ cells, int ncells, const T* __restrict__ cz,
                                 double omega, size_t stride, const uint8_t* __restrict__ active,
                                 T* __restrict__ x) {
  const int s = blockIdx.y;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || e >= ncells * 189) return;
  const int cell = cells[e / 189], ld = e % 189;
  const int node = d.cell_nodes[(size_t)cell * 27 + ld / 7];
  x[s * stride + (size_t)node * 7 + ld % 7] += (T)omega * cz[((size_t)s * d.v.n_cells + cell) * 189 + ld];
}

template <typename T>
__global__ void k3_restrict(fsi3::Transfer3View tv, const uint8_t* __restrict__ nf_f, const uint8_t* __restrict__ nf_c,
                            const T* __restrict__ rf, size_t sf, size_t sc, int n_c, const uint8_t* __restrict__ active,
                            T* __restrict__ rc) {
  const int s = blockIdx.y;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || e >= n_c * 7) return;
  rc[s * sc + e] = fsi3::restrict3(tv, nf_f, nf_c, rf + s * sf, e / 7, e % 7);
}

template <typename T>
__global__ void k3_prolong_add(fsi3::Transfer3View tv, const uint8_t* __restrict__ nf_f, const T* __restrict__ xc,
                               size_t sf, size_t sc, int n_f, const uint8_t* __restrict__ active,
                               T* __restrict__ xf) {
  const int s = blockIdx.y;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || e >= n_f * 7) return;
  xf[s * sf + e] += fsi3::prolong3(tv, nf_f, xc + s * sc, e / 7, e % 7);
}

__global__ void k3_interp_state(fsi3::Transfer3View tv, const double* __restrict__ Uf, size_t sf, size_t sc, int n_c,
                                const uint8_t* __restrict__ active, double* __restrict__ Uc) {
  const int s = blockIdx.y;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || e >= n_c * 7) return;
  Uc[s * sc + e] = fsi3::interp_state3(tv, Uf + s * sf, e / 7, e % 7);
}

// Dense copy D[s][n][n] (row-major, zero-filled before) of the coarsest level's blocks.
template <typename T>
__global__ void k3_dense_from_bsr(Dev3 d, const T* __restrict__ A, const uint8_t* __restrict__ active,
                                  double* __restrict__ D) {
  const int s = blockIdx.y;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || e >= (size_t)d.nnzb * 49) return;
  const int b = (int)(e / 49), rc = (int)(e % 49);
  const size_t n = (size_t)d.v.n_nodes * 7;
  const size_t row = (size_t)d.v.blk_row[b] * 7 + rc / 7, col = (size_t)d.v.colidx[b] * 7 + rc % 7;
  D[(size_t)s * n * n + row * n + col] = (double)A[(size_t)s * d.nnzb * 49 + e];
}

// Inactive slices get the identity as their coarsest matrix (so the batched inverse stays regular).
__global__ void k3_identity_inactive(int n, const uint8_t* __restrict__ active, double* __restrict__ D) {
  const int s = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (active[s] || i >= n) return;
  D[(size_t)s * n * n + (size_t)i * n + i] = 1.0;
}

// x = Dinv b on the coarsest level: one warp per row.
template <typename T>
__global__ void k3_dense_apply(int n, const T* __restrict__ Dinv, const T* __restrict__ b, size_t stride,
                               const uint8_t* __restrict__ active, T* __restrict__ x) {
  const int s = blockIdx.y;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) / 32, lane = threadIdx.x % 32;
  if (!active[s] || warp >= n) return;
  const T* row = Dinv + ((size_t)s * n + warp) * n;
  const T* bs = b + s * stride;
  T acc = 0;
  for (int j = lane; j < n; j += 32) acc += row[j] * bs[j];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) x[s * stride + warp] = acc;
}

// Convert FP64 -> T (dense inverses of the preconditioner)
template <typename T>
__global__ void k3_convert(size_t n, const double* __restrict__ in, T* __restrict__ out) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) out[e] = (T)in[e];
}

constexpr int R3_THREADS = 256;
constexpr int R3_CHUNK = 2048;   // rows per block: the partition (and the sums) depend on n only

// partial[s][blk][i] = sum over the block's rows of V[s][i][row] * w[s][row], i < nv (<= 64).
__global__ void __launch_bounds__(R3_THREADS) k3_dots_partial(int n, int nv, const double* __restrict__ V,
                                                             size_t vstride, size_t vslice,
                                                             const double* __restrict__ w, size_t wstride,
                                                             const uint8_t* __restrict__ active,
                                                             double* __restrict__ partial) {
  const int s = blockIdx.y;
  if (!active[s]) return;
  __shared__ double red[R3_THREADS / 32][64];
  const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
  const int r0 = blockIdx.x * R3_CHUNK, r1 = min(n, r0 + R3_CHUNK);
  const double* ws = w + s * wstride;
  for (int i = 0; i < nv; ++i) {
    const double* vi = V + s * vslice + i * vstride;
    double acc = 0.0;
    for (int r = r0 + tid; r < r1; r += R3_THREADS) acc += vi[r] * ws[r];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) red[warp][i] = acc;
  }
  __syncthreads();
  for (int i = tid; i < nv; i += R3_THREADS) {
    double acc = 0.0;
    for (int wv = 0; wv < R3_THREADS / 32; ++wv) acc += red[wv][i];
    partial[((size_t)s * gridDim.x + blockIdx.x) * 64 + i] = acc;
  }
}

// out[s][i] = sum over blocks (fixed order) of partial[s][blk][i].
__global__ void k3_dots_finish(int nblk, int nv, const double* __restrict__ partial,
                               const uint8_t* __restrict__ active, double* __restrict__ out) {
  const int s = blockIdx.x, i = threadIdx.x;
  if (!active[s] || i >= nv) return;
  double acc = 0.0;
  for (int b = 0; b < nblk; ++b) acc += partial[((size_t)s * nblk + b) * 64 + i];
  out[s * 64 + i] = acc;
}

// w[s] -= sum_{i < nv} h[s][i] V[s][i]
__global__ void k3_sub_basis(int n, int nv, const double* __restrict__ V, size_t vstride, size_t vslice,
                             const double* __restrict__ h, const uint8_t* __restrict__ active,
                             double* __restrict__ w, size_t wstride) {
  const int s = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || r >= n) return;
  double acc = w[s * wstride + r];
  for (int i = 0; i < nv; ++i) acc -= h[s * 64 + i] * V[s * vslice + i * vstride + r];
  w[s * wstride + r] = acc;
}

// x[s] += sum_{i < cnt[s]} y[s][i] Z[s][i]
__global__ void k3_add_basis(int n, const double* __restrict__ Z, size_t zstride, size_t zslice,
                             const double* __restrict__ y, const int* __restrict__ cnt,
                             const uint8_t* __restrict__ active, double* __restrict__ x, size_t xstride) {
  const int s = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || r >= n) return;
  double acc = x[s * xstride + r];
  for (int i = 0; i < cnt[s]; ++i) acc += y[s * 64 + i] * Z[s * zslice + i * zstride + r];
  x[s * xstride + r] = acc;
}

// v[s] = w[s] * scale[s]
__global__ void k3_scale(int n, const double* __restrict__ w, size_t ws, const double* __restrict__ scale,
                         const uint8_t* __restrict__ active, double* __restrict__ v, size_t vs) {
  const int s = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (!active[s] || r >= n) return;
  v[s * vs + r] = w[s * ws + r] * scale[s];
}

// Parareal correction U_next = F + (C_new - C_old), with per-field partial sums
// of the squared increment and of the new state (fields: v = 0..2, u = 3..5, p = 6).
__global__ void __launch_bounds__(R3_THREADS) k3_parareal_correct(int n, const double* __restrict__ Fv,
                                                                 const double* __restrict__ Cnew,
                                                                 const double* __restrict__ Cold,
                                                                 double* __restrict__ Unext,
                                                                 double* __restrict__ partial) {
  __shared__ double red[R3_THREADS / 32][6];
  const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
  double a[6] = {0, 0, 0, 0, 0, 0};
  for (int r = blockIdx.x * blockDim.x + tid; r < n; r += gridDim.x * blockDim.x) {
    const double un = Fv[r] + (Cnew[r] - Cold[r]);
    const double dd = un - Unext[r];
    const int c = r % 7;
    const int f = c < 3 ? 0 : (c < 6 ? 1 : 2);
    a[f] += dd * dd;
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
    for (int w = 0; w < R3_THREADS / 32; ++w) v += red[w][tid];
    partial[blockIdx.x * 6 + tid] = v;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
struct fsi3_level {
  fsi3::HostMesh3 h;
  std::vector<double> xv[3];
  std::vector<int> seg[3];
  fsi3::Transfer3 T;                 // from the next finer level (level >= 1), host tables
  fsi3::Transfer3View tv{};          // the same, device pointers
  Dev3 d{};
  std::vector<void*> owned;
  size_t n = 0;
  bool coarsest = false;
  bool dense = false;                // coarsest level solved with its dense inverse
  std::vector<int> colour_cells[8];  // cells per colour (multiplicative smoother)
  std::vector<int> colour_nodes[8];  // the nodes of those cells, ascending
  const int* colour_dev[8] = {};
  const int* colour_nodes_dev[8] = {};
  // workspace (T = the multigrid precision; double when FP64)
  void *A = nullptr, *inv = nullptr, *r = nullptr, *b = nullptr, *x = nullptr, *cz = nullptr, *Dinv = nullptr;
  double *U = nullptr, *Uo = nullptr, *D = nullptr, *Dinv64 = nullptr;
};

struct fsi3_ctx {
  fsi_params prm{};
  Phys3D P{};
  int S = 0, m = 0;
  size_t n = 0;
  std::vector<fsi3_level> lev;
  std::vector<void*> owned;
  double *Uit = nullptr, *Uold = nullptr, *R = nullptr, *A64 = nullptr, *Ke = nullptr, *Re = nullptr;
  double *V = nullptr, *Z = nullptr, *w = nullptr, *xk = nullptr, *bk = nullptr;
  double *partial = nullptr, *dots = nullptr, *dots_b = nullptr, *dots_n = nullptr, *scal = nullptr, *ycoef = nullptr,
         *t_dev = nullptr;
  int *cnt = nullptr, *status = nullptr;
  uint8_t *active = nullptr;
  double *Cold = nullptr, *Fv = nullptr, *Cnew = nullptr, *ppart = nullptr;
  int red_blocks = 0;
  bool mg32 = false;                 // multigrid in FP32 (precision 2)
  bool hierarchy_built = false;
  double* sub[2] = {nullptr, nullptr};   // states of the half-step fallback, one buffer per depth
};

namespace {

template <typename T>
int dal3(std::vector<void*>& own, T** p, size_t count) {
  void* q = nullptr;
  if (count == 0) count = 1;
  const cudaError_t e = cudaMalloc(&q, count * sizeof(T));
  if (e != cudaSuccess) return fail3(FSI_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  own.push_back(q);
  *p = (T*)q;
  return FSI_OK;
}

template <typename T>
int up3(std::vector<void*>& own, const T** p, const std::vector<T>& v) {
  T* q;
  TRY3(dal3(own, &q, v.size()));
  if (!v.empty()) CK3(cudaMemcpy(q, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  *p = q;
  return FSI_OK;
}

void free_all(std::vector<void*>& own) {
  for (void* p : own) cudaFree(p);
  own.clear();
}

// The reference tables are the same for every context: one upload per device,
// serialised across host threads.
constexpr int kMaxDevices3 = 64;
std::mutex g_tab3_mutex;
bool g_tab3_done[kMaxDevices3] = {};

int setup_tables3() {
  int dev = 0;
  CK3(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices3) return fail3(FSI_EINVAL, "device index beyond the supported range");
  std::lock_guard<std::mutex> lock(g_tab3_mutex);
  if (g_tab3_done[dev]) return FSI_OK;
  std::vector<fsi3::Tables3> T(1);
  fsi3::build_tables3(T[0]);
  const cudaError_t e = cudaMemcpyToSymbol(c_tab3, T.data(), sizeof(fsi3::Tables3));
  if (e != cudaSuccess) return fail3(FSI_ECUDA, std::string("tables: ") + cudaGetErrorString(e));
  g_tab3_done[dev] = true;
  return FSI_OK;
}

int setup_level3(fsi3_level& L, int S, bool mg32, bool need_state) {
  fsi3::HostMesh3& h = L.h;
  Dev3& d = L.d;
  const double *yn, *zn, *ch;
  const uint8_t *cf, *nf;
  const int *nc, *br, *ci, *bs, *cb, *cn, *rp;
  TRY3(up3(L.owned, &yn, h.yn));
  TRY3(up3(L.owned, &zn, h.zn));
  TRY3(up3(L.owned, &cf, h.cell_flags));
  TRY3(up3(L.owned, &nf, h.node_flags));
  TRY3(up3(L.owned, &nc, h.node_cells));
  TRY3(up3(L.owned, &br, h.blk_row));
  TRY3(up3(L.owned, &ci, h.colidx));
  TRY3(up3(L.owned, &bs, h.blk_src));
  TRY3(up3(L.owned, &cb, h.cell_blk));
  TRY3(up3(L.owned, &cn, h.cell_nodes));
  TRY3(up3(L.owned, &ch, h.cell_h));
  TRY3(up3(L.owned, &rp, h.rowptr));
  d.v = fsi3::Mesh3View{h.nnx, h.nny, h.nnz, h.n_nodes, h.n_cells, yn, zn, cf, nf, nc, h.y0, h.y1, h.z0, h.z1,
                        br, ci, bs, cb};
  d.cell_nodes = cn;
  d.cell_h = ch;
  d.rowptr = rp;
  d.nnzb = h.nnzb;
  d.nx = h.nx;
  d.ny = h.ny;
  d.nz = h.nz;
  L.n = (size_t)h.n_nodes * 7;
  for (int c = 0; c < h.n_cells; ++c) {
    const int cx = c % h.nx, cy = (c / h.nx) % h.ny, cz = c / (h.nx * h.ny);
    L.colour_cells[(cx & 1) + 2 * (cy & 1) + 4 * (cz & 1)].push_back(c);
  }
  for (int k = 0; k < 8; ++k) {
    std::vector<char> seen(h.n_nodes, 0);
    for (int c : L.colour_cells[k])
      for (int l = 0; l < 27; ++l) seen[h.cell_nodes[(size_t)c * 27 + l]] = 1;
    for (int nd = 0; nd < h.n_nodes; ++nd)
      if (seen[nd]) L.colour_nodes[k].push_back(nd);
    TRY3(up3(L.owned, &L.colour_dev[k], L.colour_cells[k]));
    TRY3(up3(L.owned, &L.colour_nodes_dev[k], L.colour_nodes[k]));
  }
  const size_t ts = mg32 ? sizeof(float) : sizeof(double);
  auto A = [&](void** p, size_t bytes) -> int {
    unsigned char* q;
    TRY3(dal3(L.owned, &q, bytes));
    *p = q;
    return FSI_OK;
  };
  TRY3(A(&L.A, (size_t)S * h.nnzb * 49 * ts));
  TRY3(A(&L.r, (size_t)S * L.n * ts));
  TRY3(A(&L.b, (size_t)S * L.n * ts));
  TRY3(A(&L.x, (size_t)S * L.n * ts));
  if (L.dense) {
    const size_t nn = L.n * L.n;
    TRY3(dal3(L.owned, &L.D, (size_t)S * nn));
    TRY3(dal3(L.owned, &L.Dinv64, (size_t)S * nn));
    if (mg32) TRY3(A(&L.Dinv, (size_t)S * nn * ts));
    else L.Dinv = L.Dinv64;
  } else {
    TRY3(A(&L.inv, (size_t)S * h.n_cells * fsi3::VK3_SIZE * ts));
    TRY3(A(&L.cz, (size_t)S * h.n_cells * 189 * ts));
  }
  if (need_state) {
    TRY3(dal3(L.owned, &L.U, (size_t)S * L.n));
    TRY3(dal3(L.owned, &L.Uo, (size_t)S * L.n));
  }
  return FSI_OK;
}

int setup_transfer3(fsi3_level& C, const fsi3_level& F) {
  const std::vector<double> xf[3] = {F.h.xn, F.h.yn, F.h.zn}, xc[3] = {C.h.xn, C.h.yn, C.h.zn};
  fsi3::build_transfer3(C.T, C.xv, xc, F.xv, xf);
  fsi3::Transfer3View& v = C.tv;
  for (int a = 0; a < 3; ++a) {
    v.nn_f[a] = C.T.nn_f[a];
    v.nn_c[a] = C.T.nn_c[a];
    TRY3(up3(C.owned, &v.pidx[a], C.T.pidx[a]));
    TRY3(up3(C.owned, &v.ridx[a], C.T.ridx[a]));
    TRY3(up3(C.owned, &v.iidx[a], C.T.iidx[a]));
    TRY3(up3(C.owned, &v.pw[a], C.T.pw[a]));
    TRY3(up3(C.owned, &v.rw[a], C.T.rw[a]));
    TRY3(up3(C.owned, &v.iw[a], C.T.iw[a]));
  }
  return FSI_OK;
}

int validate_mesh3(const fsi_mesh3d* m) {
  if (!m) return fail3(FSI_EINVAL, "null mesh");
  const int ns[3] = {m->n_xseg, m->n_yseg, m->n_zseg};
  const double* br[3] = {m->x_breaks, m->y_breaks, m->z_breaks};
  const int* sg[3] = {m->nx_seg, m->ny_seg, m->nz_seg};
  for (int a = 0; a < 3; ++a) {
    if (ns[a] < 1 || !br[a] || !sg[a]) return fail3(FSI_EINVAL, "mesh axis without segments");
    for (int i = 0; i < ns[a]; ++i)
      if (sg[a][i] < 1 || !(br[a][i + 1] > br[a][i])) return fail3(FSI_EINVAL, "bad mesh segment");
  }
  return FSI_OK;
}

// ---------------------------------------------------------------------------
// Residual, Jacobian, hierarchy
// ---------------------------------------------------------------------------
int residual3(fsi3_ctx* c, int S, const double* U, const double* Uo, double k, double theta, const uint8_t* act,
              double* R, cudaStream_t st) {
  const fsi3_level& L = c->lev[0];
  P3(KI3_CELL_RESIDUAL, (k3_cell_residual), (dim3(L.h.n_cells, S)), CR3_THREADS, 0, st, L.d, c->P, U, Uo, L.n, k, theta,
     act, c->Re);
  TRY3(launched3());
  P3(KI3_GATHER_RESIDUAL, (k3_gather_residual), (dim3(nb3(L.n, 256), S)), 256, 0, st, L.d, c->P, c->Re, U, L.n, c->t_dev, act, R);
  return launched3();
}

// FP64 blocks of level L for the state (U, Uo) into A64 (or the level's own FP64 buffer).
int jacobian3(fsi3_ctx* c, fsi3_level& L, int S, const double* U, const double* Uo, double k, double theta,
              double lps, const uint8_t* act, double* A, cudaStream_t st) {
  TRY3(launch_cell_jacobian(L.d, L.h.n_cells, S, c->P, U, Uo, L.n, k, theta, lps, act, c->Ke, st));
  P3(KI3_ASSEMBLE, (k3_assemble<double>), (dim3(nb3((size_t)L.h.nnzb * 49, 256), S)), 256, 0, st, L.d, c->Ke, act, A);
  return launched3();
}

template <typename T>
int mg_setup3(fsi3_ctx* c, int S, const double* U, const double* Uo, double k, double theta, const uint8_t* act,
              cudaStream_t st) {
  double lps = 1.0;
  for (size_t l = 0; l < c->lev.size(); ++l) {
    fsi3_level& L = c->lev[l];
    const double *Ul = U, *Uol = Uo;
    if (l > 0) {
      const fsi3_level& F = c->lev[l - 1];
      const double* Uf = l == 1 ? U : F.U;
      const double* Uof = l == 1 ? Uo : F.Uo;
      P3(KI3_INTERP_STATE, (k3_interp_state), (dim3(nb3(L.n, 256), S)), 256, 0, st, L.tv, Uf, F.n, L.n, L.h.n_nodes, act, L.U);
      P3(KI3_INTERP_STATE, (k3_interp_state), (dim3(nb3(L.n, 256), S)), 256, 0, st, L.tv, Uof, F.n, L.n, L.h.n_nodes, act, L.Uo);
      TRY3(launched3());
      Ul = L.U;
      Uol = L.Uo;
      lps *= c->prm.mg_coarse_lps;
    }
    T* A = reinterpret_cast<T*>(L.A);
    if (l == 0) {   // the Krylov operator, and its copy in T for the preconditioner
      TRY3(jacobian3(c, L, S, Ul, Uol, k, theta, 1.0, act, c->A64, st));
      P3(KI3_AXPBY, (k3_axpby<double, T>), (dim3(nb3((size_t)L.h.nnzb * 49, 256), S)), 256, 0, st, 
          L.h.nnzb * 49, 1.0, c->A64, (size_t)L.h.nnzb * 49, 0.0, act, A, (size_t)L.h.nnzb * 49);
      TRY3(launched3());
    } else {
      TRY3(launch_cell_jacobian(L.d, L.h.n_cells, S, c->P, Ul, Uol, L.n, k, theta, lps, act, c->Ke, st));
      P3(KI3_ASSEMBLE, (k3_assemble<T>), (dim3(nb3((size_t)L.h.nnzb * 49, 256), S)), 256, 0, st, L.d, c->Ke, act, A);
      TRY3(launched3());
    }
    if (L.dense) {
      const size_t nn = L.n * L.n;
      CK3(cudaMemsetAsync(L.D, 0, (size_t)S * nn * sizeof(double), st));
      P3(KI3_DENSE_FROM_BSR, (k3_dense_from_bsr<T>), (dim3(nb3((size_t)L.h.nnzb * 49, 256), S)), 256, 0, st, L.d, A, act, L.D);
      P3(KI3_IDENTITY_INACTIVE, (k3_identity_inactive), (dim3(nb3(L.n, 256), S)), 256, 0, st, (int)L.n, act, L.D);
      TRY3(launched3());
      const int rc = fsi_dense_invert(S, (int)L.n, L.D, L.Dinv64, 0, st);
      if (rc != FSI_OK) return rc;
      if (c->mg32) {
        P3(KI3_CONVERT, (k3_convert<T>), (nb3((size_t)S * nn, 256)), 256, 0, st, (size_t)S * nn, L.Dinv64, reinterpret_cast<T*>(L.Dinv));
        TRY3(launched3());
      }
    } else {
      const int smem = fsi3::vk3_setup_smem_bytes<T>();
      CK3(cudaFuncSetAttribute(k3_vanka_setup<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
      P3(KI3_VANKA_SETUP, (k3_vanka_setup<T>), (dim3(L.h.n_cells, S)), 256, smem, st, L.d, A, act, reinterpret_cast<T*>(L.inv),
                                                                   c->status);
      TRY3(launched3());
    }
  }
  c->hierarchy_built = true;
  return FSI_OK;
}

// ---------------------------------------------------------------------------
// V-cycle (in T), FGMRES (FP64)
// ---------------------------------------------------------------------------
template <typename T>
int smooth3(fsi3_ctx* c, fsi3_level& L, int S, const T* b, bool first, const uint8_t* act, cudaStream_t st) {
  T* x = reinterpret_cast<T*>(L.x);
  T* r = reinterpret_cast<T*>(L.r);
  T* cz = reinterpret_cast<T*>(L.cz);
  const T* A = reinterpret_cast<const T*>(L.A);
  const T* inv = reinterpret_cast<const T*>(L.inv);
  const double om = c->prm.mg_omega;
  if (c->prm.mg_smoother == 1) {
    for (int k = 0; k < 8; ++k) {
      const int nc = (int)L.colour_cells[k].size();
      if (nc == 0) continue;
      const int nn = (int)L.colour_nodes[k].size();
      P3(KI3_RESID_ROWS, (k3_resid_rows<T>), (dim3(nb3((size_t)nn * 7, 256), S)), 256, 0, st, L.d, A, x, b, L.n, L.colour_nodes_dev[k],
                                                                          nn, act, r);
      P3(KI3_VANKA_APPLY, (k3_vanka_apply<T>), (dim3(nc, S)), 128, 0, st, L.d, inv, r, L.n, act, L.colour_dev[k], nc, cz);
      P3(KI3_VANKA_SCATTER, (k3_vanka_scatter<T>), (dim3(nb3((size_t)nc * 189, 256), S)), 256, 0, st, L.d, L.colour_dev[k], nc, cz, om, L.n,
                                                                                 act, x);
      TRY3(launched3());
    }
    return FSI_OK;
  }
  const T* rr = b;
  if (!first) {
    P3(KI3_SPMV, (k3_spmv<T, true>), (dim3(nb3(L.n, 256), S)), 256, 0, st, L.d, A, x, L.n, b, L.n, act, r);
    rr = r;
  }
  P3(KI3_VANKA_APPLY, (k3_vanka_apply<T>), (dim3(L.h.n_cells, S)), 128, 0, st, L.d, inv, rr, L.n, act, nullptr, L.h.n_cells, cz);
  P3(KI3_VANKA_GATHER, (k3_vanka_gather<T>), (dim3(nb3(L.n, 256), S)), 256, 0, st, L.d, cz, om, L.n, act, x);
  return launched3();
}

// L.x = one V-cycle applied to b.
template <typename T>
int vcycle3(fsi3_ctx* c, size_t l, int S, const T* b, const uint8_t* act, cudaStream_t st) {
  fsi3_level& L = c->lev[l];
  T* x = reinterpret_cast<T*>(L.x);
  if (L.coarsest && !L.dense) {   // smoother sweeps in place of the coarsest solve
    P3(KI3_FILL, (k3_fill<T>), (dim3(nb3(L.n, 256), S)), 256, 0, st, (int)L.n, T(0), act, x, L.n);
    TRY3(launched3());
    for (int i = 0; i < c->prm.mg_coarse_sweeps; ++i) TRY3(smooth3<T>(c, L, S, b, i == 0, act, st));
    return FSI_OK;
  }
  if (L.coarsest) {
    P3(KI3_DENSE_APPLY, (k3_dense_apply<T>), (dim3(nb3(L.n * 32, 256), S)), 256, 0, st, (int)L.n, reinterpret_cast<const T*>(L.Dinv), b,
                                                                    L.n, act, x);
    return launched3();
  }
  P3(KI3_FILL, (k3_fill<T>), (dim3(nb3(L.n, 256), S)), 256, 0, st, (int)L.n, T(0), act, x, L.n);
  TRY3(launched3());
  for (int i = 0; i < c->prm.mg_smooth; ++i) TRY3(smooth3<T>(c, L, S, b, i == 0, act, st));
  fsi3_level& C = c->lev[l + 1];
  T* r = reinterpret_cast<T*>(L.r);
  P3(KI3_SPMV, (k3_spmv<T, true>), (dim3(nb3(L.n, 256), S)), 256, 0, st, L.d, reinterpret_cast<const T*>(L.A), x, L.n, b, L.n,
                                                            act, r);
  P3(KI3_RESTRICT, (k3_restrict<T>), (dim3(nb3(C.n, 128), S)), 128, 0, st, C.tv, L.d.v.node_flags, C.d.v.node_flags, r, L.n, C.n,
                                                          C.h.n_nodes, act, reinterpret_cast<T*>(C.b));
  TRY3(launched3());
  TRY3(vcycle3<T>(c, l + 1, S, reinterpret_cast<const T*>(C.b), act, st));
  P3(KI3_PROLONG_ADD, (k3_prolong_add<T>), (dim3(nb3(L.n, 128), S)), 128, 0, st, C.tv, L.d.v.node_flags, reinterpret_cast<const T*>(C.x),
                                                             L.n, C.n, L.h.n_nodes, act, x);
  TRY3(launched3());
  for (int i = 0; i < c->prm.mg_smooth; ++i) TRY3(smooth3<T>(c, L, S, b, false, act, st));
  return FSI_OK;
}

// Batched dots on the device: out[s * 64 + i] = <V[s][i], w[s]>, i < nv (fixed reduction order).
int dots3_dev(fsi3_ctx* c, int S, int nv, const double* V, size_t vstride, size_t vslice, const double* w,
              const uint8_t* act, double* out, cudaStream_t st) {
  const int n = (int)c->n;
  const unsigned nblk = nb3(n, R3_CHUNK);
  P3(KI3_DOTS_PARTIAL, (k3_dots_partial), (dim3(nblk, S)), R3_THREADS, 0, st, n, nv, V, vstride, vslice, w, c->n, act,
     c->partial);
  P3(KI3_DOTS_FINISH, (k3_dots_finish), (S), 64, 0, st, (int)nblk, nv, c->partial, act, out);
  return launched3();
}

// Batched dots: out[s][i] = <V[s][i], w[s]>, i < nv, to the host array h[S][64].
int dots3(fsi3_ctx* c, int S, int nv, const double* V, size_t vstride, size_t vslice, const double* w,
          const uint8_t* act, std::vector<double>& h, cudaStream_t st) {
  const int n = (int)c->n;
  const unsigned nblk = nb3(n, R3_CHUNK);
  P3(KI3_DOTS_PARTIAL, (k3_dots_partial), (dim3(nblk, S)), R3_THREADS, 0, st, n, nv, V, vstride, vslice, w, c->n, act, c->partial);
  P3(KI3_DOTS_FINISH, (k3_dots_finish), (S), 64, 0, st, (int)nblk, nv, c->partial, act, c->dots);
  TRY3(launched3());
  h.assign((size_t)S * 64, 0.0);
  CK3(cudaMemcpyAsync(h.data(), c->dots, (size_t)S * 64 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK3(cudaStreamSynchronize(st));
  return FSI_OK;
}

// FGMRES(m) on the FP64 Jacobian A64, right-preconditioned by the V-cycle in T:
// x = A^{-1} b per active slice to ||b - A x|| <= max(rtol ||b||, target[s]).
// Hessenberg matrices and Givens rotations on the host (one synchronisation per iteration).
template <typename T>
int fgmres3(fsi3_ctx* c, int S, const double* b, double* x, std::vector<uint8_t> act, double rtol,
            const std::vector<double>& target, fsi_stats* stats, cudaStream_t st, std::vector<int>* codes = nullptr) {
  // codes (optional, [S]): FSI_EGMRES or FSI_ENAN for the slices that stopped that way
  auto mark = [&](int s, int code) {
    if (codes) (*codes)[s] = code;
  };
  fsi3_level& L = c->lev[0];
  const size_t n = c->n;
  const int m = c->m;
  const size_t vsl = (size_t)(m + 1) * n, zsl = (size_t)m * n;
  const unsigned g = nb3(n, 256);
  CK3(cudaMemcpyAsync(c->active, act.data(), S, cudaMemcpyHostToDevice, st));
  P3(KI3_FILL, (k3_fill<double>), (dim3(g, S)), 256, 0, st, (int)n, 0.0, c->active, x, n);
  TRY3(launched3());
  std::vector<double> hb;
  TRY3(dots3(c, S, 1, b, 0, n, b, c->active, hb, st));
  std::vector<double> tgt(S, 0.0);
  int status = FSI_OK;
  for (int s = 0; s < S; ++s) {
    if (!act[s]) continue;
    const double bn = std::sqrt(hb[(size_t)s * 64]);
    if (!std::isfinite(bn)) {
      status = FSI_ENAN;
      mark(s, FSI_ENAN);
      act[s] = 0;
      continue;
    }
    if (!(bn > 0.0)) act[s] = 0;
    tgt[s] = std::max(rtol * bn, target.empty() ? 0.0 : target[s]);
  }
  std::vector<double> H((size_t)S * (m + 1) * m), cs((size_t)S * m), sn((size_t)S * m), gv((size_t)S * (m + 1));
  std::vector<int> its(S, 0), jn(S, 0);
  auto any = [](const std::vector<uint8_t>& a) { return std::any_of(a.begin(), a.end(), [](uint8_t v) { return v != 0; }); };
  std::vector<double> h1, h2, scal(S, 0.0), y((size_t)S * 64, 0.0);
  while (any(act)) {
    CK3(cudaMemcpyAsync(c->active, act.data(), S, cudaMemcpyHostToDevice, st));
    // r = b - A x into V[0]; beta
    P3(KI3_SPMV, (k3_spmv<double, true>), (dim3(g, S)), 256, 0, st, L.d, c->A64, x, n, b, n, c->active, c->w);
    TRY3(launched3());
    TRY3(dots3(c, S, 1, c->w, 0, n, c->w, c->active, h1, st));
    std::vector<uint8_t> cyc = act;   // slices iterating in this cycle
    for (int s = 0; s < S; ++s) {
      if (!act[s]) continue;
      const double beta = std::sqrt(h1[(size_t)s * 64]);
      if (!std::isfinite(beta)) {
        status = FSI_ENAN;
        mark(s, FSI_ENAN);
        act[s] = cyc[s] = 0;
        continue;
      }
      if (beta <= tgt[s]) {
        act[s] = cyc[s] = 0;
        continue;
      }
      if (its[s] >= c->prm.gmres_maxit) {
        status = FSI_EGMRES;
        mark(s, FSI_EGMRES);
        act[s] = cyc[s] = 0;
        continue;
      }
      scal[s] = 1.0 / beta;
      std::fill(&gv[(size_t)s * (m + 1)], &gv[(size_t)s * (m + 1)] + m + 1, 0.0);
      gv[(size_t)s * (m + 1)] = beta;
      jn[s] = 0;
    }
    if (!any(cyc)) break;
    CK3(cudaMemcpyAsync(c->active, cyc.data(), S, cudaMemcpyHostToDevice, st));
    CK3(cudaMemcpyAsync(c->scal, scal.data(), S * sizeof(double), cudaMemcpyHostToDevice, st));
    P3(KI3_SCALE, (k3_scale), (dim3(g, S)), 256, 0, st, (int)n, c->w, n, c->scal, c->active, c->V, vsl);
    TRY3(launched3());
    std::vector<uint8_t> run = cyc;   // slices still adding basis vectors in this cycle
    for (int j = 0; j < m && any(run); ++j) {
      CK3(cudaMemcpyAsync(c->active, run.data(), S, cudaMemcpyHostToDevice, st));
      // z_j = M^{-1} v_j (in T), w = A z_j
      T* xin = reinterpret_cast<T*>(L.b);
      P3(KI3_AXPBY, (k3_axpby<double, T>), (dim3(g, S)), 256, 0, st, (int)n, 1.0, c->V + (size_t)j * n, vsl, 0.0, c->active, xin, n);
      TRY3(launched3());
      TRY3(vcycle3<T>(c, 0, S, xin, c->active, st));
      P3(KI3_AXPBY, (k3_axpby<T, double>), (dim3(g, S)), 256, 0, st, (int)n, 1.0, reinterpret_cast<const T*>(L.x), n, 0.0, c->active,
                                                      c->Z + (size_t)j * n, zsl);
      P3(KI3_SPMV, (k3_spmv<double, false>), (dim3(g, S)), 256, 0, st, L.d, c->A64, c->Z + (size_t)j * n, zsl, nullptr, n,
                                                        c->active, c->w);
      TRY3(launched3());
      // classical Gram-Schmidt, twice: the coefficients stay on the device for the subtractions, and the
      // host reads both passes and the new norm after one synchronisation
      TRY3(dots3_dev(c, S, j + 1, c->V, n, vsl, c->w, c->active, c->dots, st));
      P3(KI3_SUB_BASIS, (k3_sub_basis), (dim3(g, S)), 256, 0, st, (int)n, j + 1, c->V, n, vsl, c->dots, c->active, c->w, n);
      TRY3(launched3());
      TRY3(dots3_dev(c, S, j + 1, c->V, n, vsl, c->w, c->active, c->dots_b, st));
      P3(KI3_SUB_BASIS, (k3_sub_basis), (dim3(g, S)), 256, 0, st, (int)n, j + 1, c->V, n, vsl, c->dots_b, c->active, c->w,
         n);
      TRY3(launched3());
      TRY3(dots3_dev(c, S, 1, c->w, 0, n, c->w, c->active, c->dots_n, st));
      std::vector<double> hn((size_t)S * 64);
      h1.assign((size_t)S * 64, 0.0);
      h2.assign((size_t)S * 64, 0.0);
      CK3(cudaMemcpyAsync(h1.data(), c->dots, (size_t)S * 64 * sizeof(double), cudaMemcpyDeviceToHost, st));
      CK3(cudaMemcpyAsync(h2.data(), c->dots_b, (size_t)S * 64 * sizeof(double), cudaMemcpyDeviceToHost, st));
      CK3(cudaMemcpyAsync(hn.data(), c->dots_n, (size_t)S * 64 * sizeof(double), cudaMemcpyDeviceToHost, st));
      CK3(cudaStreamSynchronize(st));
      for (int s = 0; s < S; ++s) {
        if (!run[s]) continue;
        double hcol[65];
        for (int i = 0; i <= j; ++i) hcol[i] = h1[(size_t)s * 64 + i] + h2[(size_t)s * 64 + i];
        hcol[j + 1] = std::sqrt(hn[(size_t)s * 64]);
        scal[s] = hcol[j + 1] > 0.0 ? 1.0 / hcol[j + 1] : 0.0;
        double* csv = &cs[(size_t)s * m];
        double* snv = &sn[(size_t)s * m];
        for (int i = 0; i < j; ++i) {
          const double a = hcol[i], bb = hcol[i + 1];
          hcol[i] = csv[i] * a + snv[i] * bb;
          hcol[i + 1] = -snv[i] * a + csv[i] * bb;
        }
        const double den = std::hypot(hcol[j], hcol[j + 1]);
        csv[j] = den > 0.0 ? hcol[j] / den : 1.0;
        snv[j] = den > 0.0 ? hcol[j + 1] / den : 0.0;
        hcol[j] = den;
        double* gs = &gv[(size_t)s * (m + 1)];
        gs[j + 1] = -snv[j] * gs[j];
        gs[j] = csv[j] * gs[j];
        for (int i = 0; i <= j; ++i) H[((size_t)s * (m + 1) + i) * m + j] = hcol[i];
        jn[s] = j + 1;
        ++its[s];
        if (!std::isfinite(gs[j + 1])) {
          status = FSI_ENAN;
          mark(s, FSI_ENAN);
          run[s] = 0;
          act[s] = 0;
        } else if (std::fabs(gs[j + 1]) <= tgt[s] || its[s] >= c->prm.gmres_maxit || !(den > 0.0)) {
          run[s] = 0;
        }
      }
      CK3(cudaMemcpyAsync(c->scal, scal.data(), S * sizeof(double), cudaMemcpyHostToDevice, st));
      P3(KI3_SCALE, (k3_scale), (dim3(g, S)), 256, 0, st, (int)n, c->w, n, c->scal, c->active, c->V + (size_t)(j + 1) * n, vsl);
      TRY3(launched3());
    }
    // x += Z y per slice (back substitution on the host)
    std::vector<int> cnt(S, 0);
    std::fill(y.begin(), y.end(), 0.0);
    for (int s = 0; s < S; ++s) {
      if (!cyc[s]) continue;
      const int jj = jn[s];
      cnt[s] = jj;
      for (int i = jj - 1; i >= 0; --i) {
        double acc = gv[(size_t)s * (m + 1) + i];
        for (int q = i + 1; q < jj; ++q) acc -= H[((size_t)s * (m + 1) + i) * m + q] * y[(size_t)s * 64 + q];
        y[(size_t)s * 64 + i] = acc / H[((size_t)s * (m + 1) + i) * m + i];
      }
    }
    CK3(cudaMemcpyAsync(c->active, cyc.data(), S, cudaMemcpyHostToDevice, st));
    CK3(cudaMemcpyAsync(c->ycoef, y.data(), y.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    CK3(cudaMemcpyAsync(c->cnt, cnt.data(), S * sizeof(int), cudaMemcpyHostToDevice, st));
    P3(KI3_ADD_BASIS, (k3_add_basis), (dim3(g, S)), 256, 0, st, (int)n, c->Z, n, zsl, c->ycoef, c->cnt, c->active, x, n);
    TRY3(launched3());
  }
  if (stats)
    for (int s = 0; s < S; ++s) {
      stats->gmres_iters += its[s];
      stats->max_gmres = std::max(stats->max_gmres, its[s]);
    }
  return status;
}

// ---------------------------------------------------------------------------
// Theta step, propagators, Parareal
// ---------------------------------------------------------------------------
int theta_step3(fsi3_ctx* c, int S, const double* U_old, const double* t_old, double k, double theta, double* U_new,
                fsi_stats* stats, cudaStream_t st, int reuse, bool hierarchy_valid,
                std::vector<int>* why_out = nullptr) {
  if (S < 1 || S > c->S) return fail3(FSI_EINVAL, "batch size outside 1..max_batch");
  const size_t n = c->n;
  std::vector<double> tn(S);
  for (int s = 0; s < S; ++s) tn[s] = t_old[s] + k;
  CK3(cudaMemcpyAsync(c->t_dev, tn.data(), S * sizeof(double), cudaMemcpyHostToDevice, st));
  CK3(cudaMemcpyAsync(c->Uold, U_old, S * n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CK3(cudaMemcpyAsync(c->Uit, U_old, S * n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  std::vector<uint8_t> act(S, 1);
  std::vector<int> st_h(S, 0);
  CK3(cudaMemcpyAsync(c->active, act.data(), S, cudaMemcpyHostToDevice, st));
  CK3(cudaMemcpyAsync(c->status, st_h.data(), S * sizeof(int), cudaMemcpyHostToDevice, st));
  const fsi3_level& L = c->lev[0];
  P3(KI3_APPLY_DIRICHLET, (k3_apply_dirichlet), (dim3(nb3(L.h.n_nodes, 128), S)), 128, 0, st, L.d, c->P, c->Uit, n, c->t_dev, c->active);
  TRY3(launched3());
  std::vector<double> r0(S, 0.0), nr(S), hr;
  std::vector<int> nit(S, 0), why(S, 0);
  // gmiss: an FGMRES solve of the slice stopped at its iteration limit; its correction is
  // still applied (inexact Newton), and the slice fails only if Newton then fails (FSI_EGMRES)
  std::vector<uint8_t> gmiss(S, 0);
  const bool trace = std::getenv("FSI_TRACE_NEWTON") != nullptr;
  std::vector<std::vector<double>> hist(trace ? S : 0);
  int status = FSI_OK;
  for (int it = 0;; ++it) {
    CK3(cudaMemcpyAsync(c->active, act.data(), S, cudaMemcpyHostToDevice, st));
    TRY3(residual3(c, S, c->Uit, c->Uold, k, theta, c->active, c->R, st));
    TRY3(dots3(c, S, 1, c->R, 0, n, c->R, c->active, hr, st));
    bool any = false;
    for (int s = 0; s < S; ++s) {
      if (!act[s]) continue;
      nr[s] = std::sqrt(hr[(size_t)s * 64]);
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
        if (trace) {
          std::fprintf(stderr, "[fsi trace] 3D slice %d t=%.6g k=%.6g status %d, Newton residuals:", s,
                       t_old[s] + k, k, why[s]);
          for (double x : hist[s]) std::fprintf(stderr, " %.3e", x);
          std::fprintf(stderr, "\n");
        }
        act[s] = 0;
        continue;
      }
      nit[s] = it + 1;
      any = true;
    }
    if (!any) break;
    CK3(cudaMemcpyAsync(c->active, act.data(), S, cudaMemcpyHostToDevice, st));
    // inexact Newton forcing terms (as in the 2D solver)
    std::vector<double> target(S, 0.0);
    double rtol = c->prm.gmres_rtol;
    if (c->prm.newton_eta > 0.0) {
      rtol = it == 0 ? std::max(c->prm.gmres_rtol, c->prm.gmres_rtol_first) : c->prm.gmres_rtol;
      if (it > 0)
        for (int s = 0; s < S; ++s)
          target[s] = std::min(1e-2 * nr[s], c->prm.newton_eta * c->prm.newton_tol * std::max(r0[s], 1.0));
    }
    const bool keep_all = (it == 0) ? hierarchy_valid && c->hierarchy_built : reuse >= 2;
    if (keep_all) {
      TRY3(jacobian3(c, c->lev[0], S, c->Uit, c->Uold, k, theta, 1.0, c->active, c->A64, st));
    } else if (c->mg32) {
      TRY3(mg_setup3<float>(c, S, c->Uit, c->Uold, k, theta, c->active, st));
    } else {
      TRY3(mg_setup3<double>(c, S, c->Uit, c->Uold, k, theta, c->active, st));
    }
    P3(KI3_AXPBY, (k3_axpby<double, double>), (dim3(nb3(n, 256), S)), 256, 0, st, (int)n, -1.0, c->R, n, 0.0, c->active, c->bk, n);
    TRY3(launched3());
    std::vector<int> codes(S, 0);
    int rc = c->mg32 ? fgmres3<float>(c, S, c->bk, c->xk, act, rtol, target, stats, st, &codes)
                     : fgmres3<double>(c, S, c->bk, c->xk, act, rtol, target, stats, st, &codes);
    CK3(cudaMemcpyAsync(st_h.data(), c->status, S * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK3(cudaStreamSynchronize(st));
    for (int s = 0; s < S; ++s)
      if (act[s] && st_h[s] != 0) {
        status = why[s] = FSI_EJAC;
        act[s] = 0;
      }
    if (rc != FSI_OK && rc != FSI_EGMRES && rc != FSI_ENAN) return rc;
    for (int s = 0; s < S; ++s) {
      if (!act[s]) continue;
      if (codes[s] == FSI_EGMRES) {
        gmiss[s] = 1;
        if (trace) std::fprintf(stderr, "[fsi trace] 3D slice %d t=%.6g Newton it %d: FGMRES at its limit\n", s,
                                t_old[s] + k, it);
      } else if (codes[s] == FSI_ENAN) {
        if (!why[s]) why[s] = FSI_ENAN;
        status = FSI_ENAN;
      }
    }
    CK3(cudaMemcpyAsync(c->active, act.data(), S, cudaMemcpyHostToDevice, st));
    P3(KI3_AXPBY, (k3_axpby<double, double>), (dim3(nb3(n, 256), S)), 256, 0, st, (int)n, 1.0, c->xk, n, 1.0, c->active, c->Uit, n);
    TRY3(launched3());
  }
  CK3(cudaMemcpyAsync(U_new, c->Uit, S * n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (why_out) *why_out = why;
  if (stats) {
    for (int s = 0; s < S; ++s) {
      stats->newton_iters += nit[s];
      stats->max_newton = std::max(stats->max_newton, nit[s]);
      if (stats->slice_status && s < stats->slice_status_len && !stats->slice_status[s]) stats->slice_status[s] = why[s];
    }
    stats->status = status;
  }
  if (status != FSI_OK) {
    char buf[96];
    std::snprintf(buf, sizeof buf, "3D theta step failed with status %d", status);
    return fail3(status, buf);
  }
  return FSI_OK;
}

// Fallback of the propagators. The slices of a batch whose step failed in Newton's method
// or in FGMRES (not by a NaN or a singular element) take it again from the same state as
// two steps of half the length (fine: shifted Crank-Nicolson with theta = 1/2 + theta0 k/2;
// coarse: implicit Euler), each with the same fallback, halving at most kSubstepDepth times.
// Steps that converge are unchanged; a slice's fallback depends on its own state only. The
// step after a fallback rebuilds the multigrid hierarchy of the whole batch.
constexpr int kSubstepDepth = 2;

int step3_with_fallback(fsi3_ctx* c, int S, const double* src, const double* t, double k, bool fine, double* dst,
                        fsi_stats* stats, cudaStream_t st, int reuse, bool hierarchy_valid, int depth = 0) {
  const size_t n = c->n;
  const double theta = fine ? 0.5 + c->prm.theta0 * k : 1.0;
  std::vector<int> saved;   // the caller's per-slice statuses before the step
  if (stats && stats->slice_status)
    saved.assign(stats->slice_status, stats->slice_status + std::min(S, stats->slice_status_len));
  std::vector<int> why;
  const int rc = theta_step3(c, S, src, t, k, theta, dst, stats, st, reuse, hierarchy_valid, &why);
  if (rc == FSI_OK || depth >= kSubstepDepth || (int)why.size() != S) return rc;
  std::vector<int> redo;
  for (int s = 0; s < S; ++s) {
    if (why[s] == FSI_ENEWTON || why[s] == FSI_EGMRES) redo.push_back(s);
    else if (why[s] != FSI_OK) return rc;   // a NaN or a singular element stands
  }
  if (redo.empty()) return rc;
  if (!c->sub[depth]) TRY3(dal3(c->owned, &c->sub[depth], (size_t)c->S * n));
  double* buf = c->sub[depth];
  const int R = (int)redo.size();
  std::vector<double> tr(R);
  for (int i = 0; i < R; ++i) {   // the step's input is still in Uold (src may alias dst)
    CK3(cudaMemcpyAsync(buf + (size_t)i * n, c->Uold + (size_t)redo[i] * n, n * sizeof(double),
                        cudaMemcpyDeviceToDevice, st));
    tr[i] = t[redo[i]];
  }
  if (std::getenv("FSI_TRACE_NEWTON"))
    std::fprintf(stderr, "[fsi trace] 3D: %d slice(s) of the batch retry t=%.6g as two steps of k=%.6g\n", R,
                 t[redo[0]] + k, 0.5 * k);
  fsi_stats sub{};
  if (stats) {
    sub = *stats;
    sub.slice_status = nullptr;
    sub.slice_status_len = 0;
  }
  for (int h = 0; h < 2; ++h) {
    const int rc2 = step3_with_fallback(c, R, buf, tr.data(), 0.5 * k, fine, buf, stats ? &sub : nullptr, st, reuse,
                                        false, depth + 1);
    if (stats) {
      stats->newton_iters = sub.newton_iters;
      stats->gmres_iters = sub.gmres_iters;
      stats->max_newton = std::max(stats->max_newton, sub.max_newton);
      stats->max_gmres = std::max(stats->max_gmres, sub.max_gmres);
    }
    c->hierarchy_built = false;   // the hierarchy now belongs to the sub-batch
    if (rc2 != FSI_OK) return rc;  // the first failure stands
    for (double& x : tr) x += 0.5 * k;
  }
  for (int i = 0; i < R; ++i)
    CK3(cudaMemcpyAsync(dst + (size_t)redo[i] * n, buf + (size_t)i * n, n * sizeof(double),
                        cudaMemcpyDeviceToDevice, st));
  if (stats) {
    stats->status = FSI_OK;
    for (size_t s = 0; s < saved.size(); ++s) stats->slice_status[s] = saved[s];
  }
  return FSI_OK;
}

int propagate3(fsi3_ctx* c, int S, const double* U0, const double* t0, double* U1, bool fine, fsi_stats* stats,
               cudaStream_t st) {
  const int m = fine ? c->prm.m_fine : c->prm.m_coarse;
  const double k = c->prm.T / c->prm.n_slices / m;
  const int every = std::max(1, c->prm.mg_rebuild_every);
  for (int s0 = 0; s0 < S; s0 += c->S) {
    const int b = std::min(c->S, S - s0);
    std::vector<double> t(t0 + s0, t0 + s0 + b);
    const double* src = U0 + (size_t)s0 * c->n;
    double* dst = U1 + (size_t)s0 * c->n;
    for (int j = 0; j < m; ++j) {
      const int reuse = fine ? c->prm.mg_reuse : std::min(c->prm.mg_reuse, 1);
      TRY3(step3_with_fallback(c, b, src, t.data(), k, fine, dst, stats, st, reuse, fine && j % every != 0));
      for (double& x : t) x += k;
      src = dst;
    }
    if (m == 0 && dst != src) CK3(cudaMemcpyAsync(dst, src, (size_t)b * c->n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  return FSI_OK;
}

int correct3(fsi3_ctx* c, int i, const double* Cn, double* U, double inc[3], cudaStream_t st) {
  const size_t n = c->n;
  const int nrb = c->red_blocks;
  P3(KI3_PARAREAL_CORRECT, (k3_parareal_correct), (nrb), R3_THREADS, 0, st, (int)n, c->Fv + (size_t)i * n, Cn, c->Cold + (size_t)i * n,
                                                  U + (size_t)(i + 1) * n, c->ppart);
  TRY3(launched3());
  std::vector<double> part((size_t)nrb * 6);
  CK3(cudaMemcpyAsync(part.data(), c->ppart, part.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK3(cudaStreamSynchronize(st));
  double a[6] = {0, 0, 0, 0, 0, 0};
  for (int b = 0; b < nrb; ++b)
    for (int f = 0; f < 6; ++f) a[f] += part[(size_t)b * 6 + f];
  for (int f = 0; f < 3; ++f) {
    const double rel = a[3 + f] > 0 ? std::sqrt(a[f] / a[3 + f]) : std::sqrt(a[f]);
    if (!std::isfinite(rel)) return fail3(FSI_EDIVERGE, "Parareal increment is not finite");
    inc[f] = std::max(inc[f], rel);
  }
  return FSI_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI (3D)
// ---------------------------------------------------------------------------
extern "C" {

int fsi3_kernel_count(void) { return KI3_COUNT; }

const char* fsi3_kernel_name(int id) { return (id >= 0 && id < KI3_COUNT) ? kKernelNames3[id] : nullptr; }

long long fsi3_launch_count(int id) {
  if (id >= KI3_COUNT) return -1;
  if (id >= 0) return g_prof3.launches[id].load();
  long long t = 0;
  for (int k = 0; k < KI3_COUNT; ++k) t += g_prof3.launches[k].load();
  return t;
}

int fsi3_profile_enable(int on) {
  std::lock_guard<std::mutex> lock(g_prof3.mu);
  for (auto& v : g_prof3.ev) {
    for (auto& pr : v) {
      cudaEventSynchronize(pr.second);
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
    v.clear();
  }
  g_prof3.on.store(on != 0);
  return FSI_OK;
}

int fsi3_profile_read(int id, double* total_ms, long long* timed_launches) {
  if (id < 0 || id >= KI3_COUNT || !total_ms || !timed_launches) return fail3(FSI_EINVAL, "bad profile query");
  std::lock_guard<std::mutex> lock(g_prof3.mu);
  double t = 0.0;
  for (auto& pr : g_prof3.ev[id]) {
    float ms = 0.0f;
    CK3(cudaEventSynchronize(pr.second));
    CK3(cudaEventElapsedTime(&ms, pr.first, pr.second));
    t += ms;
  }
  *total_ms = t;
  *timed_launches = (long long)g_prof3.ev[id].size();
  return FSI_OK;
}

void fsi3_destroy(fsi3_ctx* c) {
  if (!c) return;
  for (auto& L : c->lev) free_all(L.owned);
  free_all(c->owned);
  delete c;
}

int fsi3_setup(const fsi_mesh3d* mesh, const fsi_params* p, fsi3_ctx** out) {
  if (!out || !p) return fail3(FSI_EINVAL, "null argument");
  *out = nullptr;
  TRY3(validate_mesh3(mesh));
  if (p->max_batch < 1 || p->gmres_restart < 1 || p->gmres_restart > 63 || p->n_slices < 1 || p->m_fine < 1 ||
      p->m_coarse < 0 || !(p->T > 0.0) || p->mg_smooth < 0 || p->mg_coarsest_max_dofs < 7 ||
      !(p->mg_coarse_lps > 0.0) || p->newton_maxit < 0 || p->gmres_maxit < 1 || !(p->newton_tol > 0.0) ||
      !(p->gmres_rtol > 0.0) || !(p->newton_eta >= 0.0) || !(p->gmres_rtol_first >= 0.0))
    return fail3(FSI_EINVAL, "invalid solver parameters (3D: gmres_restart <= 63)");
  if (p->precision == 1) return fail3(FSI_EINVAL, "the 3D path supports precision 0 and 2");
  if (p->mg_smoother != 0 && p->mg_smoother != 1) return fail3(FSI_EINVAL, "mg_smoother must be 0 or 1");
  if (p->mg_coarse_sweeps < 0 || p->mg_coarse_sweeps > 1000) return fail3(FSI_EINVAL, "mg_coarse_sweeps outside 0..1000");
  fsi3_ctx* c = new fsi3_ctx;
  auto cleanup = [&](int rc) {
    fsi3_destroy(c);
    return rc;
  };
  c->prm = *p;
  c->S = p->max_batch;
  c->m = p->gmres_restart;
  c->mg32 = p->precision == 2;
  c->P = Phys3D{p->rho_f, p->nu_f, p->rho_s, p->mu_s, p->lambda_s, p->vbar, p->ramp_t, p->alpha0};
  // hierarchy: pair cells per segment until the dofs fit, or no axis coarsens
  const double* br[3] = {mesh->x_breaks, mesh->y_breaks, mesh->z_breaks};
  const int* sg[3] = {mesh->nx_seg, mesh->ny_seg, mesh->nz_seg};
  const int ns[3] = {mesh->n_xseg, mesh->n_yseg, mesh->n_zseg};
  const double* box = mesh->has_solid ? mesh->solid_box : nullptr;
  c->lev.emplace_back();
  for (int a = 0; a < 3; ++a) {
    c->lev[0].xv[a] = fsi3::axis_vertices3(br[a], sg[a], ns[a]);
    c->lev[0].seg[a].assign(sg[a], sg[a] + ns[a]);
  }
  fsi3::build_mesh3(c->lev[0].h, c->lev[0].xv[0], c->lev[0].xv[1], c->lev[0].xv[2], box);
  while ((size_t)c->lev.back().h.n_nodes * 7 > (size_t)p->mg_coarsest_max_dofs) {
    fsi3_level C;
    bool changed = false;
    for (int a = 0; a < 3; ++a) {
      fsi3::coarsen_axis3(c->lev.back().xv[a], c->lev.back().seg[a], C.xv[a], C.seg[a]);
      changed |= C.xv[a].size() != c->lev.back().xv[a].size();
    }
    if (!changed) break;
    fsi3::build_mesh3(C.h, C.xv[0], C.xv[1], C.xv[2], box);
    c->lev.push_back(std::move(C));
  }
  if (c->lev.size() < 2) return cleanup(fail3(FSI_EINVAL, "the mesh needs at least one coarser level"));
  c->lev.back().coarsest = true;
  c->lev.back().dense = p->mg_coarse_sweeps == 0;
  if (c->lev.back().dense && (size_t)c->lev.back().h.n_nodes * 7 > 4096)
    return cleanup(fail3(FSI_EINVAL, "coarsest level above 4096 dofs"));
  int rc = setup_tables3();
  if (rc) return cleanup(rc);
  for (size_t l = 0; l < c->lev.size(); ++l) {
    rc = setup_level3(c->lev[l], c->S, c->mg32, l > 0);
    if (rc) return cleanup(rc);
    if (l > 0 && (rc = setup_transfer3(c->lev[l], c->lev[l - 1]))) return cleanup(rc);
  }
  c->n = c->lev[0].n;
  const size_t S = c->S, n = c->n, m = c->m;
  const fsi3_level& L0 = c->lev[0];
  size_t cells_max = 0;
  for (const auto& L : c->lev) cells_max = std::max(cells_max, (size_t)L.h.n_cells);
  auto A = [&](auto** ptr, size_t cnt) { return dal3(c->owned, ptr, cnt); };
  if ((rc = A(&c->Uit, S * n)) || (rc = A(&c->Uold, S * n)) || (rc = A(&c->R, S * n)) || (rc = A(&c->xk, S * n)) ||
      (rc = A(&c->bk, S * n)) || (rc = A(&c->w, S * n)) || (rc = A(&c->V, S * (m + 1) * n)) ||
      (rc = A(&c->Z, S * m * n)) || (rc = A(&c->A64, S * (size_t)L0.h.nnzb * 49)) ||
      (rc = A(&c->Ke, S * cells_max * 189 * 189)) || (rc = A(&c->Re, S * (size_t)L0.h.n_cells * 189)) ||
      (rc = A(&c->partial, S * (size_t)nb3(n, R3_CHUNK) * 64)) || (rc = A(&c->dots, S * 64)) ||
      (rc = A(&c->dots_b, S * 64)) || (rc = A(&c->dots_n, S * 64)) ||
      (rc = A(&c->scal, S)) || (rc = A(&c->ycoef, S * 64)) || (rc = A(&c->t_dev, S)) || (rc = A(&c->cnt, S)) ||
      (rc = A(&c->status, S)) || (rc = A(&c->active, S)))
    return cleanup(rc);
  const size_t N = p->n_slices;
  c->red_blocks = (int)std::min<size_t>(nb3(n, R3_THREADS), 304);
  if ((rc = A(&c->Cold, N * n)) || (rc = A(&c->Fv, N * n)) || (rc = A(&c->Cnew, n)) ||
      (rc = A(&c->ppart, (size_t)c->red_blocks * 6)))
    return cleanup(rc);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cleanup(fail3(FSI_ECUDA, std::string("setup: ") + cudaGetErrorString(e)));
  *out = c;
  return FSI_OK;
}

int fsi3_n_nodes(const fsi3_ctx* c) { return c ? c->lev[0].h.n_nodes : -1; }
int fsi3_n_dofs(const fsi3_ctx* c) { return c ? (int)c->n : -1; }
int fsi3_n_levels(const fsi3_ctx* c) { return c ? (int)c->lev.size() : -1; }
int fsi3_nnzb(const fsi3_ctx* c) { return c ? c->lev[0].h.nnzb : -1; }

int fsi3_bsr_pattern(const fsi3_ctx* c, int* rowptr, int* colidx) {
  if (!c || !rowptr || !colidx) return fail3(FSI_EINVAL, "null argument");
  std::copy(c->lev[0].h.rowptr.begin(), c->lev[0].h.rowptr.end(), rowptr);
  std::copy(c->lev[0].h.colidx.begin(), c->lev[0].h.colidx.end(), colidx);
  return FSI_OK;
}

int fsi3_residual(fsi3_ctx* c, int S, const double* U, const double* U_old, const double* t_new, double k,
                  double theta, double* R, void* stream) {
  if (!c || !U || !U_old || !t_new || !R) return fail3(FSI_EINVAL, "null argument");
  if (S < 1 || S > c->S) return fail3(FSI_EINVAL, "batch size outside 1..max_batch");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<uint8_t> act(S, 1);
  CK3(cudaMemcpyAsync(c->active, act.data(), S, cudaMemcpyHostToDevice, st));
  CK3(cudaMemcpyAsync(c->t_dev, t_new, S * sizeof(double), cudaMemcpyHostToDevice, st));
  TRY3(residual3(c, S, U, U_old, k, theta, c->active, R, st));
  CK3(cudaStreamSynchronize(st));
  return FSI_OK;
}

int fsi3_jacobian(fsi3_ctx* c, int S, const double* U, const double* U_old, double k, double theta, double* vals,
                  void* stream) {
  if (!c || !U || !U_old || !vals) return fail3(FSI_EINVAL, "null argument");
  if (S < 1 || S > c->S) return fail3(FSI_EINVAL, "batch size outside 1..max_batch");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<uint8_t> act(S, 1);
  CK3(cudaMemcpyAsync(c->active, act.data(), S, cudaMemcpyHostToDevice, st));
  TRY3(jacobian3(c, c->lev[0], S, U, U_old, k, theta, 1.0, c->active, vals, st));
  CK3(cudaStreamSynchronize(st));
  return FSI_OK;
}

int fsi3_theta_step(fsi3_ctx* c, int S, const double* U_old, const double* t_old, double k, double theta,
                    double* U_new, fsi_stats* stats, void* stream) {
  if (!c || !U_old || !t_old || !U_new) return fail3(FSI_EINVAL, "null argument");
  if (stats) {
    int* ss = stats->slice_status;
    const int sl = stats->slice_status_len;
    std::memset(stats, 0, sizeof(*stats));
    stats->slice_status = ss;
    stats->slice_status_len = sl;
    if (ss)
      for (int s = 0; s < std::min(S, sl); ++s) ss[s] = 0;
  }
  cudaStream_t st = (cudaStream_t)stream;
  TRY3(theta_step3(c, S, U_old, t_old, k, theta, U_new, stats, st, std::min(c->prm.mg_reuse, 1), false));
  CK3(cudaStreamSynchronize(st));
  return FSI_OK;
}

static int fsi3_propagate(fsi3_ctx* c, int S, const double* U0, const double* t0, double* U1, bool fine,
                          fsi_stats* stats, void* stream) {
  if (!c || !U0 || !t0 || !U1) return fail3(FSI_EINVAL, "null argument");
  if (S < 1) return fail3(FSI_EINVAL, "S < 1");
  if (stats) {
    int* ss = stats->slice_status;
    const int sl = stats->slice_status_len;
    std::memset(stats, 0, sizeof(*stats));
    stats->slice_status = ss;
    stats->slice_status_len = sl;
  }
  cudaStream_t st = (cudaStream_t)stream;
  TRY3(propagate3(c, S, U0, t0, U1, fine, stats, st));
  CK3(cudaStreamSynchronize(st));
  return FSI_OK;
}

int fsi3_fine(fsi3_ctx* c, int S, const double* U0, const double* t0, double* U1, fsi_stats* stats, void* stream) {
  return fsi3_propagate(c, S, U0, t0, U1, true, stats, stream);
}

int fsi3_coarse(fsi3_ctx* c, int S, const double* U0, const double* t0, double* U1, fsi_stats* stats, void* stream) {
  return fsi3_propagate(c, S, U0, t0, U1, false, stats, stream);
}

int fsi3_parareal(fsi3_ctx* c, double* U, int max_iter, double tol, fsi_parareal_stats* stats, void* stream) {
  if (!c || !U) return fail3(FSI_EINVAL, "null argument");
  if (max_iter < 0 || !(tol >= 0.0)) return fail3(FSI_EINVAL, "max_iter < 0 or tol < 0");
  cudaStream_t st = (cudaStream_t)stream;
  fsi_parareal_stats loc{};
  if (stats) {
    loc.history = stats->history;
    loc.history_len = stats->history_len;
  }
  const int N = c->prm.n_slices;
  const size_t n = c->n;
  const double dt = c->prm.T / N;
  std::vector<double> t(N);
  for (int i = 0; i < N; ++i) t[i] = i * dt;
  for (int i = 0; i < N; ++i) {   // predictor sweep
    TRY3(propagate3(c, 1, U + (size_t)i * n, &t[i], c->Cold + (size_t)i * n, false, &loc.coarse, st));
    CK3(cudaMemcpyAsync(U + (size_t)(i + 1) * n, c->Cold + (size_t)i * n, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    loc.coarse_steps += c->prm.m_coarse;
  }
  for (int it = 1; it <= max_iter && it <= N; ++it) {
    const int first = it - 1, S = N - first;
    TRY3(propagate3(c, S, U + (size_t)first * n, &t[first], c->Fv + (size_t)first * n, true, &loc.fine, st));
    loc.fine_steps += (long long)S * c->prm.m_fine;
    double inc[3] = {0, 0, 0};
    for (int i = first; i < N; ++i) {
      const double* Cn;
      if (i == first) {
        Cn = c->Cold + (size_t)i * n;   // unchanged input: the coarse difference is zero exactly
      } else {
        TRY3(propagate3(c, 1, U + (size_t)i * n, &t[i], c->Cnew, false, &loc.coarse, st));
        loc.coarse_steps += c->prm.m_coarse;
        Cn = c->Cnew;
      }
      TRY3(correct3(c, i, Cn, U, inc, st));
      if (i != first)
        CK3(cudaMemcpyAsync(c->Cold + (size_t)i * n, c->Cnew, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    loc.increment_v = inc[0];
    loc.increment_u = inc[1];
    loc.increment_p = inc[2];
    if (loc.history && it - 1 < loc.history_len)
      for (int f = 0; f < 3; ++f) loc.history[(it - 1) * 3 + f] = inc[f];
    loc.iterations = it;
    if (std::max(inc[0], std::max(inc[1], inc[2])) <= tol) break;
  }
  CK3(cudaStreamSynchronize(st));
  if (stats) *stats = loc;
  return FSI_OK;
}

}  // extern "C"
