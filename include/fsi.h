/*
 * fsi.h -- C ABI of the GB300 library for Parareal time stepping of monolithic
 * ALE fluid-structure interaction (Margenberg & Richter, "Parallel
 * time-stepping for fluid-structure interactions").
 *
 * The library advances the fully discrete ALE-FSI system of Sec. 2
 * (equal-order Q2 elements, shifted Crank-Nicolson step of Sec. 2.3 with the
 * forms of Eq. (semiforms)) for many time slices at once on one GPU, and runs
 * the Parareal iteration of Sec. 3, Eq. (parareal:iteration).
 *
 * Conventions shared by every entry point
 *   - State layout: one state is n_dofs = 5 * n_nodes doubles, node-major,
 *     components (v_x, v_y, u_x, u_y, p). Node (i, j) of the Q2 node grid
 *     (2nx+1) x (2ny+1) has id j * (2nx+1) + i (x fastest). A batch of S
 *     states is S contiguous states.
 *   - Pointers documented "device" are CUDA device pointers owned by the
 *     caller; "host" pointers are ordinary host memory owned by the caller.
 *     The library never frees caller memory and never keeps a caller pointer
 *     after a call returns.
 *   - stream: a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Every kernel of a call runs on that stream. Calls that report
 *     iteration statistics synchronise the stream before they return.
 *   - Return value: FSI_OK (0) on success, a negative FSI_E* code otherwise;
 *     fsi_last_error() then returns a message (thread-local). No entry point
 *     aborts, exits, traps on the device or leaves a kernel waiting without
 *     an iteration limit.
 *   - The context owns all workspace (allocated in fsi_setup for batches of
 *     up to params->max_batch slices). A context must not be used by two
 *     host threads at the same time; different contexts may be used from
 *     different threads concurrently, each on its own stream.
 */
#ifndef FSI_H
#define FSI_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
  FSI_OK = 0,
  FSI_EINVAL = -1,    /* invalid argument or size */
  FSI_ENOMEM = -2,    /* device allocation failed */
  FSI_ECUDA = -3,     /* CUDA runtime error */
  FSI_ENEWTON = -4,   /* Newton did not reach its tolerance within newton_maxit */
  FSI_EGMRES = -5,    /* as FSI_ENEWTON, after at least one of the slice's FGMRES solves
                         stopped at gmres_maxit (such a solve's correction is still
                         applied; a slice whose Newton iteration converges anyway
                         succeeds) */
  FSI_EJAC = -6,      /* singular local block (Vanka or coarsest solve) or J <= 0 */
  FSI_ENAN = -7,      /* non-finite residual */
  FSI_EDIVERGE = -8   /* Parareal increment is not finite */
};

/* Interface-fitted tensor-product mesh of the reference domain (Sec. 2.2:
 * the interface is resolved by cell faces). Break points split each axis into
 * segments with nx_seg[i] (ny_seg[j]) uniform cells. Cells whose centre lies
 * in the solid box are solid. Host pointers, read during fsi_setup only. */
typedef struct fsi_mesh {
  int n_xseg;
  const double* x_breaks; /* [n_xseg + 1], increasing */
  const int* nx_seg;      /* [n_xseg], each >= 1 */
  int n_yseg;
  const double* y_breaks; /* [n_yseg + 1], increasing */
  const int* ny_seg;      /* [n_yseg], each >= 1 */
  int has_solid;
  double solid_x0, solid_x1, solid_y0, solid_y1;
} fsi_mesh;

/* Material, time and solver parameters. Materials: Eq. (stress) (Newtonian
 * fluid, St. Venant-Kirchhoff solid). theta = 1/2 + theta0 * k for the fine
 * step (Sec. 2.3); the coarse step uses theta = 1. alpha0 scales the local
 * projection stabilisation (Sec. 2.2 requires one; its form is a reading).
 * The Parareal interval [0, T] is cut into n_slices slices of m_fine fine and
 * m_coarse coarse steps (Sec. 3, T/L = m k = M K). */
typedef struct fsi_params {
  double rho_f, nu_f, rho_s, mu_s, lambda_s;
  double vbar, ramp_t;     /* mean inflow velocity, inflow ramp duration */
  double theta0, alpha0;
  double T;
  int n_slices, m_fine, m_coarse;
  double newton_tol;       /* stop when ||R||_2 <= newton_tol * max(||R_0||_2, 1) */
  int newton_maxit;
  int gmres_restart;       /* FGMRES restart length m */
  int gmres_maxit;         /* total FGMRES iterations per linear solve */
  double gmres_rtol;       /* relative residual reduction per linear solve */
  double gmres_rtol_first; /* with newton_eta > 0: reduction of the first Newton
                              correction of a step */
  double newton_eta;       /* > 0: later Newton corrections stop once the linear
                              residual is newton_eta x the Newton target (inexact
                              Newton, per slice); 0: every solve to gmres_rtol */
  int mg_coarsest_max_dofs;/* coarsen the multigrid hierarchy until <= this */
  int mg_smooth;           /* Vanka sweeps before and after the coarse correction */
  double mg_omega;         /* Vanka damping */
  int mg_smoother;         /* 0: additive Vanka (all cells at once, corrections
                              averaged over the cells of a node); 1: multiplicative,
                              four colours of cells that share no node, one after
                              the other with the residual updated in between */
  double mg_coarse_lps;    /* preconditioner only: the stabilisation weight on
                              multigrid level l is multiplied by mg_coarse_lps^l
                              (rediscretised coarse levels otherwise carry far more
                              pressure stabilisation than the fine operator) */
  int mg_reuse;            /* what the preconditioner keeps from the first Newton
                              iteration of a step (the Krylov operator is always the
                              current exact Jacobian): 0 nothing, 1 the coarsest-level
                              inverse, 2 the whole multigrid hierarchy. Coarse steps
                              and fsi_theta_step use at most 1 (a stale hierarchy
                              fails on large steps); the fine propagator uses it as is */
  int mg_rebuild_every;    /* fine propagator: rebuild the hierarchy at the first
                              Newton iteration of every mg_rebuild_every-th step and
                              keep it in between (>= 1; 1 = every step) */
  int graph_max_batch;     /* batches of at most this many slices run each FGMRES
                              iteration as one CUDA graph (captured once per batch
                              size and Krylov index); 0 disables graphs */
  int precision;           /* 0: FP64 throughout. 1: the whole linear solver (FGMRES,
                              multigrid, Vanka, block-sparse operator) in FP32 inside
                              the FP64 Newton loop (inner tolerance >= 1e-6); the
                              Newton refinement only contracts while cond(J) times the
                              FP32 unit roundoff stays below one (large steps of stiff
                              problems can violate it). 2: FP64 FGMRES on the FP64 Jacobian,
                              preconditioned by the multigrid V-cycle in FP32 (Vanka
                              inverses, transfers, level operators): GMRES-based
                              refinement, as accurate as 0. In every mode the Newton
                              residual, J = det F and the Parareal correction are FP64 */
  int pipeline_chunk;      /* parareal_iterate: 0 runs the sweeps and the batched fine
                              solves one after the other; > 0 pipelines them (a host
                              thread runs the sequential coarse sweeps in a second,
                              single-slice context on a high-priority stream while
                              the fine solves run in batches of pipeline_chunk slices
                              as soon as their inputs exist). Results are identical */
  int max_batch;           /* most slices advanced in one call */
  int mg_coarse_sweeps;    /* 3D path only: 0 solves the coarsest level with its dense
                              inverse; > 0 applies that many smoother sweeps there
                              instead (no inverse to build for each coarse step) */
  int tc_contraction;      /* 2D path, FP32 element matrices (precision 1, and the FP32
                              multigrid levels of precision 2): 1 computes the tangent D
                              in FP32 and runs the element contraction B^T D B on the
                              tensor cores (tcgen05.mma, each FP32 operand as three BF16
                              terms, FP32 accumulation in tensor memory); 0 computes D
                              in FP64 and contracts on the CUDA cores in FP32. These
                              matrices only feed the FP32 solver; the Newton residual
                              stays FP64 either way */
  int ff_operator;         /* 2D path, FP64 operators (precision 0, and the Krylov
                              operator of precision 2): 1 applies the block-sparse
                              product in the Krylov solver and in the multigrid
                              residuals with the blocks and the input vector as float
                              pairs hi + lo and a compensated FP32 accumulation (about
                              2^-48 relative to the sum of |a x|, on the FP32 pipe); 0
                              with FP64 FMAs. The Newton residual, the Jacobian and
                              every state stay FP64 either way */
} fsi_params;

/* Iteration statistics of one call (filled when the pointer is non-NULL). */
typedef struct fsi_stats {
  long long newton_iters;  /* Newton iterations summed over slices and steps */
  long long gmres_iters;   /* FGMRES iterations summed over slices and solves */
  int max_newton;          /* most Newton iterations of one slice in one step */
  int max_gmres;           /* most FGMRES iterations of one slice in one solve */
  int status;              /* same code as the return value */
  int* slice_status;       /* optional host array [slice_status_len] (NULL to skip):
                              fsi_theta_step, fsi_fine and fsi_coarse set entry s of
                              the call's S slices to FSI_OK, or to the first failure
                              of slice s (FSI_ENAN, FSI_ENEWTON, FSI_EJAC, FSI_EGMRES);
                              other entry points leave it alone */
  int slice_status_len;
} fsi_stats;

typedef struct fsi_parareal_stats {
  int iterations;          /* Parareal iterations done (the predictor sweep is 0) */
  double increment_v, increment_u, increment_p; /* last relative increments */
  long long fine_steps;    /* fine theta steps run (slices x steps) */
  long long coarse_steps;  /* coarse theta steps run */
  fsi_stats fine, coarse;  /* summed solver statistics */
  double* history;         /* optional host array [history_len][3]: the relative
                              increments (v, u, p) of every iteration; NULL to skip */
  int history_len;
} fsi_parareal_stats;

typedef struct fsi_ctx fsi_ctx;

/* Build the mesh hierarchy, the dof tables and all device workspace.
 * Errors: FSI_EINVAL (bad mesh/params), FSI_ENOMEM, FSI_ECUDA. */
int fsi_setup(const fsi_mesh* mesh, const fsi_params* params, fsi_ctx** out);
void fsi_destroy(fsi_ctx* ctx);
const char* fsi_last_error(void);
int fsi_n_nodes(const fsi_ctx* ctx);
int fsi_n_dofs(const fsi_ctx* ctx);
int fsi_n_levels(const fsi_ctx* ctx);   /* multigrid levels of the linear solver */

/* Residual of one theta step t_{n-1} -> t_n = t_new (Sec. 2.3, the step
 * equation with the forms of Eq. (semiforms)) for S slices at once.
 * U, U_old, R: device [S][n_dofs]; t_new: host [S]. Rows with Dirichlet data
 * carry U - g(t_new); pressure rows of nodes that touch no fluid cell carry p.
 * Errors: FSI_EINVAL (S outside 1..max_batch). */
int fsi_residual(fsi_ctx* ctx, int S, const double* U, const double* U_old,
                 const double* t_new, double k, double theta, double* R, void* stream);

/* Allocation-free variant of fsi_residual, for callers that must not allocate
 * device memory when they evaluate residuals: code running inside a framework
 * that owns the whole device memory pool, or a loop with a fixed memory budget.
 * The paper has no counterpart; it computes exactly what fsi_residual computes.
 * The entry point calls no cudaMalloc/cudaFree and no allocating library
 * routine: its scratch (slice flags, times and the per-cell contributions) is
 * one file-scope static __device__ array of 16 MiB, which every GPU that loads
 * the library holds until the process exits. The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress, with that device
 * current) and caches it; make that first call before any stream capture.
 * The context is only read (its tables were built by fsi_setup), so S is not
 * bounded by max_batch. Limits: 1 <= S <= 256 and S * cells * 45 <= 2,096,864
 * doubles (e.g. 11 slices of the 128 x 32 mesh); larger sizes return
 * FSI_EINVAL with a message. Every call on a device shares the one array and
 * overwrites it completely (nothing needs to start at zero), so calls that
 * overlap on the GPU (other streams, other host threads) race: serialise them.
 * Arguments, layout and errors as fsi_residual; the call synchronises the stream. */
int fsi_residual_noalloc(fsi_ctx* ctx, int S, const double* U, const double* U_old,
                         const double* t_new, double k, double theta, double* R, void* stream);

/* Jacobian dR/dU of the same residual, assembled as a block-sparse matrix with
 * 5x5 node blocks: vals device [S][nnzb][5][5] (row-major blocks), pattern
 * from fsi_bsr_pattern. Errors: FSI_EINVAL. */
int fsi_jacobian(fsi_ctx* ctx, int S, const double* U, const double* U_old,
                 double k, double theta, double* vals, void* stream);

/* The same Jacobian with FP32 element matrices and FP32 blocks, as the FP32
 * linear solver builds it (precision 1): vals device float [S][nnzb][5][5].
 * Tangent and element contraction as params->tc_contraction says (FP32 tangent
 * and tensor cores, or FP64 tangent and CUDA cores). Errors: FSI_EINVAL,
 * FSI_ECUDA (also when a tensor-core MMA completion was not seen). */
int fsi_jacobian_f32(fsi_ctx* ctx, int S, const double* U, const double* U_old,
                     double k, double theta, float* vals, void* stream);
int fsi_nnzb(const fsi_ctx* ctx);
/* Host copy of the block pattern: rowptr [n_nodes + 1], colidx [nnzb]. */
int fsi_bsr_pattern(const fsi_ctx* ctx, int* rowptr, int* colidx);

/* y = A x for S slices sharing the pattern: vals device [S][nnzb][25],
 * x, y device [S][n_dofs]. Errors: FSI_EINVAL. */
int fsi_bsr_spmv(fsi_ctx* ctx, int S, const double* vals, const double* x,
                 double* y, void* stream);
/* The same product with FP32 values and vectors (the FP32 linear solver's
 * operator), one warp per node row: vals device [S][nnzb][25], x, y device
 * [S][n_dofs], all float. Errors: FSI_EINVAL. */
int fsi_bsr_spmv_f32(fsi_ctx* ctx, int S, const float* vals, const float* x,
                     float* y, void* stream);
/* The FP64 product as the float-float option computes it: vals and x split
 * into float pairs hi + lo (a context scratch buffer), every row summed with
 * compensated FP32 arithmetic, y in FP64 (about 2^-48 of sum |a x| per row).
 * Shapes as fsi_bsr_spmv. Errors: FSI_EINVAL, also when the context was set
 * up without ff_operator. */
int fsi_bsr_spmv_ff(fsi_ctx* ctx, int S, const double* vals, const double* x,
                    double* y, void* stream);

/* The product y = A x over all node rows in one chosen kernel variant, for
 * tests and tuning: value_type 0 FP64 (vals, x, y double), 1 FP32 (all float),
 * 2 FP64 values and vector carried as float pairs (vals, x, y double; needs
 * ff_operator); tile_rows 0 the row-list kernel (one thread per row component),
 * or 8, 16, 32, 64: the row-tile kernel, whose CTA stages the contiguous blocks
 * of that many consecutive rows in shared memory by a bulk asynchronous copy.
 * Every variant sums each row component over its blocks in the same order, so
 * all give the same bits (the library's own products pick the fastest per
 * level, value type and batch size on first use). Shapes as fsi_bsr_spmv;
 * synchronises the stream. Errors: FSI_EINVAL (also a tile whose blocks exceed
 * 200 KiB of shared memory), FSI_ECUDA when a bulk copy did not complete within
 * its poll limit (the outputs of its tile are NaN). */
int fsi_bsr_spmv_variant(fsi_ctx* ctx, int S, int value_type, int tile_rows,
                         const void* vals, const void* x, void* y, void* stream);

/* One theta step for S slices: Newton's method (exact Jacobian, no damping;
 * Sec. 1 and 4 solve each step's nonlinear system by Newton) with FGMRES
 * preconditioned by a geometric multigrid V-cycle with Vanka smoothing.
 * U_old, U_new: device [S][n_dofs] (may alias); t_old: host [S].
 * Errors: FSI_ENEWTON, FSI_EGMRES, FSI_EJAC, FSI_ENAN, FSI_EINVAL. */
int fsi_theta_step(fsi_ctx* ctx, int S, const double* U_old, const double* t_old,
                   double k, double theta, double* U_new, fsi_stats* stats, void* stream);

/* Fine propagator F of Sec. 3 for S slices at once: m_fine shifted
 * Crank-Nicolson steps of k = T / n_slices / m_fine from t0[s].
 * U0, U1: device [S][n_dofs] (may alias); t0: host [S]. */
int fsi_fine(fsi_ctx* ctx, int S, const double* U0, const double* t0, double* U1,
             fsi_stats* stats, void* stream);

/* Coarse propagator C of Sec. 3: m_coarse theta = 1 steps of
 * K = T / n_slices / m_coarse. Same arguments as fsi_fine. */
int fsi_coarse(fsi_ctx* ctx, int S, const double* U0, const double* t0, double* U1,
               fsi_stats* stats, void* stream);

/* Parareal, Eq. (parareal:iteration): predictor sweep with C, then iterations
 * U_{n+1}^{i+1} = F(U_n^i) + (C(U_n^{i+1}) - C(U_n^i)); fine solves of all
 * slices not yet exact run batched. U: device [n_slices + 1][n_dofs]; on entry
 * U[0] is the initial state, on return U holds the last iterate at all slice
 * boundaries. Stops when the largest relative boundary increment of v, u and
 * p is <= tol, or after max_iter iterations (max_iter >= n_slices gives the
 * serial fine solution). Errors: as fsi_theta_step, FSI_EDIVERGE. */
int parareal_iterate(fsi_ctx* ctx, double* U, int max_iter, double tol,
                     fsi_parareal_stats* stats, void* stream);

/* Continue the context's Parareal run (Sec. 3, Eq. (parareal:iteration)) by up
 * to n_iter further iterations, numbered on from the run's last completed one:
 * parareal_iterate(U, a) followed by parareal_continue(U, b) computes the same
 * bits as parareal_iterate(U, a + b) (the same tol stops either early).
 * parareal_iterate with max_iter = 0 runs only the predictor sweep, so
 * successive parareal_continue(U, 1) calls step a run one iteration at a time.
 * U: device [n_slices + 1][n_dofs], the U the previous call of the run returned
 * (it may have been copied to the host and back in between, but not changed);
 * the context keeps the coarse values of the last sweep. Iterations always use
 * the serial schedule (results are identical to the pipelined one). No
 * iteration runs past n_slices (the iterate is then the serial fine solution).
 * stats->iterations is the run's iteration count after the call; the other
 * counts and history rows cover this call's iterations. Errors: FSI_EINVAL when
 * the context has no completed run (none yet, or its last Parareal call
 * failed), and as parareal_iterate; a failed call ends the run. */
int parareal_continue(fsi_ctx* ctx, double* U, int n_iter, double tol,
                      fsi_parareal_stats* stats, void* stream);

/* Jacobian of the same step residual with respect to the old state U_{n-1}
 * (Sec. 2.3: U_{n-1} enters the ALE mass term, the (1 - theta) terms, the
 * kinematic and harmonic rows and, through the cell-mean velocity, the
 * stabilisation weight; the old pressure does not enter). Same layout as
 * fsi_jacobian; rows with Dirichlet data or p = 0 are zero. The stabilisation
 * weight is not differentiable where a cell mean velocity is exactly zero;
 * there its derivative is taken as zero. Errors: FSI_EINVAL. */
int fsi_jacobian_old(fsi_ctx* ctx, int S, const double* U, const double* U_old,
                     double k, double theta, double* vals, void* stream);

/* Change the solid Lame parameters and the mean inflow velocity of a context
 * (Eq. (stress) material, Sec. 4 inflow profile). Errors: FSI_EINVAL. */
int fsi_set_material(fsi_ctx* ctx, double mu_s, double lambda_s, double vbar);

/* Discrete adjoint of the fine trajectory (the paper gives no adjoint; this is
 * the exact derivative of its discrete scheme, the theta step of Sec. 2.3).
 * One slice: n_steps fine steps (k = T / n_slices / m_fine, theta = 1/2 +
 * theta0 k) from the device state U0 [n_dofs] at time t0. Functional
 *   J = sum_{n=0}^{n_steps} w_n |u(x_tip, t_n)|^2, trapezoid weights w_n (k/2 at the ends),
 * x_tip the node at the top centre of the solid box. Output (host): J_out and
 * grad[3] = (dJ/dmu_s, dJ/dlambda_s, dJ/dvbar), all partial derivatives.
 * Backward sweep: (dR_n/dU_n)^T lam_n = -w_n dg/dU_n - (dR_{n+1}/dU_n)^T lam_{n+1},
 * dJ/dp = sum_n lam_n^T dR_n/dp; transposed solves by FGMRES with the multigrid
 * hierarchy of the transposed operators. States are checkpointed at slice
 * boundaries (every m_fine steps) and recomputed slice by slice. Needs
 * precision 0. The first call allocates the adjoint workspace of the context.
 * Errors: FSI_EINVAL (no tip node, n_steps < 1), solver errors as fsi_theta_step. */
int fsi_adjoint(fsi_ctx* ctx, const double* U0, double t0, int n_steps, double* J_out,
                double* grad, fsi_stats* stats, void* stream);

/* Dense inverse of S independent n x n matrices, the solver of the coarsest
 * multigrid level (Gauss-Jordan with partial pivoting, in place). A, inv:
 * device [S][n][n] row-major; A is not modified; inv receives A^{-1}.
 * method 0: on a thread-block cluster of 8 CTAs per matrix when its rows fit
 * in the cluster's shared memory, else one CTA per matrix; method 1: always
 * one CTA per matrix. Both choose the same pivots and give the same inverse.
 * Allocates its own scratch; synchronises the stream.
 * Errors: FSI_EINVAL, FSI_ENOMEM, FSI_EJAC (a singular matrix), FSI_ECUDA. */
int fsi_dense_invert(int S, int n, const double* A, double* inv, int method, void* stream);

/* Sizes of the finest level of a mesh, on the host only (no GPU, no context):
 * nodes, dofs (5 per node) and 5x5 blocks of the Jacobian's block pattern, as
 * fsi_n_nodes / fsi_n_dofs / fsi_nnzb of a context built on the same mesh.
 * Outputs: host ints. Errors: FSI_EINVAL (bad mesh, null output). */
int fsi_mesh_size(const fsi_mesh* mesh, int* n_nodes, int* n_dofs, int* nnzb);

/* 3D interface-fitted hexahedral mesh (the 3D channel of the uneven and 3D
 * workloads): break points and cells per segment on the three axes, and an
 * optional solid box. Host pointers, read during the call only. */
typedef struct fsi_mesh3d {
  int n_xseg;
  const double* x_breaks; /* [n_xseg + 1], increasing */
  const int* nx_seg;      /* [n_xseg], each >= 1 */
  int n_yseg;
  const double* y_breaks;
  const int* ny_seg;
  int n_zseg;
  const double* z_breaks;
  const int* nz_seg;
  int has_solid;
  double solid_box[6];    /* x0, x1, y0, y1, z0, z1 */
} fsi_mesh3d;

/* Sizes of a 3D mesh on the host only (no GPU): nodes of the Q2 hexahedra
 * (2nx+1)(2ny+1)(2nz+1), dofs (7 per node: v, u, p) and 7 x 7 blocks of the
 * Jacobian's node pattern. Errors: FSI_EINVAL (bad mesh, null output). */
int fsi3d_mesh_size(const fsi_mesh3d* mesh, int* n_nodes, int* n_dofs, int* nnzb);

/* ---- 3D path: the same method on hexahedral Q2 elements ------------------
 * The theta step of Sec. 2.3 in three dimensions: 27-node hexahedra, 7
 * unknowns per node (v_x, v_y, v_z, u_x, u_y, u_z, p), 3 x 3 x 3 Gauss points.
 * Fluid: no-slip on the four lateral walls; inflow 36 vbar s(t) (y - y0)(y1 - y)
 * (z - z0)(z1 - z) / ((y1 - y0)^2 (z1 - z0)^2) with the ramp s(t) of the 2D
 * path; free outflow. Displacement: zero on the outer boundary. Solved by Newton with FGMRES (classical
 * Gram-Schmidt twice; the Hessenberg matrices live on the host) and a V-cycle
 * over interface-fitted coarsenings. The V-cycle uses block Vanka local solves:
 * velocity-pressure block and displacement Schur complement, in FP64 or
 * (precision 2) FP32, and a dense inverse on the coarsest level (at most 4096
 * dofs) or, with mg_coarse_sweeps > 0, that many smoother sweeps there. Parameters as fsi_params, with these limits: precision 0 or 2;
 * gmres_restart <= 63; the mesh must coarsen at least once; mg_smoother 1
 * sweeps eight cell colours; graph_max_batch and pipeline_chunk are ignored.
 * Device arrays are [S][n_dofs] (node-major, 7 per node); Jacobian blocks are
 * [S][nnzb][7][7] row-major. Calls on one context are serialised by the caller.
 * Every call synchronises its stream before it returns. */
typedef struct fsi3_ctx fsi3_ctx;

/* Build the level hierarchy and all device workspace. Errors: FSI_EINVAL (bad
 * mesh or parameters), FSI_ENOMEM, FSI_ECUDA. */
int fsi3_setup(const fsi_mesh3d* mesh, const fsi_params* params, fsi3_ctx** out);
void fsi3_destroy(fsi3_ctx* ctx);
int fsi3_n_nodes(const fsi3_ctx* ctx);
int fsi3_n_dofs(const fsi3_ctx* ctx);
int fsi3_n_levels(const fsi3_ctx* ctx);
int fsi3_nnzb(const fsi3_ctx* ctx);
/* Host copy of the block pattern: rowptr [n_nodes + 1], colidx [nnzb]. */
int fsi3_bsr_pattern(const fsi3_ctx* ctx, int* rowptr, int* colidx);

/* Residual of one theta step for S slices (as fsi_residual): U, U_old, R
 * device [S][n_dofs], t_new host [S]. Errors: FSI_EINVAL. */
int fsi3_residual(fsi3_ctx* ctx, int S, const double* U, const double* U_old,
                  const double* t_new, double k, double theta, double* R, void* stream);

/* Jacobian dR/dU in 7 x 7 blocks: vals device [S][nnzb][49]. Errors: FSI_EINVAL. */
int fsi3_jacobian(fsi3_ctx* ctx, int S, const double* U, const double* U_old,
                  double k, double theta, double* vals, void* stream);

/* One theta step for S slices (as fsi_theta_step). Errors: FSI_ENEWTON,
 * FSI_EGMRES, FSI_EJAC, FSI_ENAN, FSI_EINVAL. */
int fsi3_theta_step(fsi3_ctx* ctx, int S, const double* U_old, const double* t_old,
                    double k, double theta, double* U_new, fsi_stats* stats, void* stream);

/* Fine and coarse propagators of Sec. 3 (as fsi_fine, fsi_coarse); S may exceed
 * max_batch (batches of max_batch). */
int fsi3_fine(fsi3_ctx* ctx, int S, const double* U0, const double* t0, double* U1,
              fsi_stats* stats, void* stream);
int fsi3_coarse(fsi3_ctx* ctx, int S, const double* U0, const double* t0, double* U1,
                fsi_stats* stats, void* stream);

/* Parareal iteration of Sec. 3 (as parareal_iterate, serial sweeps): U device
 * [n_slices + 1][n_dofs]. Errors: as fsi3_theta_step, FSI_EDIVERGE. */
int fsi3_parareal(fsi3_ctx* ctx, double* U, int max_iter, double tol,
                  fsi_parareal_stats* stats, void* stream);

/* Launch accounting of the 3D kernels (process-wide, all threads): every launch
 * is counted; fsi3_profile_enable(1) clears the recorded times and brackets each
 * later launch with two CUDA events on its stream (0 stops recording).
 * fsi3_profile_read waits for the recorded events of kernel id and returns their
 * summed device time and count. fsi3_launch_count(-1) sums over all kernels.
 * Errors: FSI_EINVAL (bad id or null output), FSI_ECUDA. */
int fsi3_kernel_count(void);
const char* fsi3_kernel_name(int kernel_id);
long long fsi3_launch_count(int kernel_id);
int fsi3_profile_enable(int on);
int fsi3_profile_read(int kernel_id, double* total_ms, long long* timed_launches);

/* ---- Batches of independent problems (beyond the paper, which solves one
 * problem at a time) ----------------------------------------------------
 * Many independent FSI problems of uneven meshes, materials and slice counts,
 * each advanced by the Parareal iteration of Sec. 3 (parareal_iterate).
 * Worker host threads, each with its own non-blocking CUDA stream, take the
 * problems longest first (estimated cost: dofs x fine steps still iterated,
 * plus the single-slice coarse steps weighted 8x) and run each in its own
 * context, created and released around it; kernels of different workers run
 * concurrently on the GPU. A problem's result is bit-identical to running it
 * alone with parareal_iterate. A problem whose set-up runs out of device memory
 * next to the others is run again after all workers finish, alone. */
typedef struct fsi_instance {
  fsi_mesh mesh;               /* host pointers, read during the call */
  fsi_params params;           /* max_batch is ignored: taken as n_slices */
  double* U;                   /* device [n_slices + 1][n_dofs], caller-owned;
                                  in/out exactly as in parareal_iterate */
  int max_iter;                /* Parareal iterations, as parareal_iterate */
  double tol;                  /* increment tolerance, as parareal_iterate */
  fsi_parareal_stats stats;    /* out; set history/history_len before the
                                  call to record increments (host memory) */
  int status;                  /* out: FSI_OK or this problem's error code */
  int worker;                  /* out: worker thread that ran it */
  double seconds;              /* out: host wall time of set-up, Parareal
                                  and release of this problem */
} fsi_instance;

/* The schedule the batch runner follows, on the host only: order[n] = the
 * problems longest first (ties by index), cost[n] = estimated cost,
 * worker[n] = the worker each problem gets when every worker runs exactly the
 * estimate (greedy: next problem to the least loaded worker, ties by index),
 * makespan (may be NULL) = the largest worker load of that schedule.
 * Errors: FSI_EINVAL (n < 0, workers < 1, null outputs, a bad mesh). */
int fsi_batch_plan(const fsi_instance* inst, int n, int workers, int* order, int* worker,
                   double* cost, double* makespan);

/* Run the batch with `workers` concurrent workers (at most n are started).
 * The workers start after the work already queued on `stream`, and `stream`
 * continues after all of theirs. Returns FSI_OK when every problem succeeded,
 * otherwise the first failing problem's code (its message names the problem);
 * every problem's own status is in inst[i].status either way.
 * Errors: FSI_EINVAL (bad arguments: nothing runs), FSI_ECUDA, the problems' codes. */
int fsi_batch_parareal(fsi_instance* inst, int n, int workers, void* stream);

/* Autotuner for the worker count: one untimed run with candidates[0] (module
 * loading, CUDA graph capture), then one timed run per candidate (host wall
 * time between stream synchronisations). seconds[n_candidates] receives the
 * times, *best the fastest worker count. Every run recomputes the same results
 * from U[0] of each problem, so inst holds the results on return.
 * Errors: FSI_EINVAL, and those of fsi_batch_parareal. */
int fsi_batch_autotune(fsi_instance* inst, int n, const int* candidates, int n_candidates,
                       double* seconds, int* best, void* stream);

/* Measurement hooks (the paper has no counterpart; they serve benchmarking).
 * Process-wide; counts and timings include every host thread's launches
 * (profile_enable and profile_read themselves must not run while another
 * thread is inside the library). Every kernel launch of the library is
 * counted per kernel id (0 .. fsi_kernel_count()-1, names from
 * fsi_kernel_name). fsi_profile_enable(mask) clears the timing records and
 * brackets each later launch of the kernels whose id bit is set with two CUDA
 * events on the launching stream; fsi_profile_read synchronises on those
 * events and returns the summed duration, the number of timed launches and the
 * algorithmic floating-point operations the library attributes to them.
 * fsi_launch_count(-1) is the total over all kernels. */
int fsi_profile_enable(unsigned long long kernel_mask);
int fsi_profile_read(int kernel_id, double* total_ms, long long* timed_launches,
                     double* total_flops);   /* algorithmic FP64 flops of the timed launches (0 if not counted) */
/* Algorithmic DRAM bytes the library attributes to the timed launches of a
 * kernel since fsi_profile_enable (the data each launch must move at least
 * once: for the block-sparse product the blocks, the input and output vectors
 * of every active slice and, once per launch, the index arrays); 0 for
 * kernels without a byte count. Errors: FSI_EINVAL. */
int fsi_profile_read_bytes(int kernel_id, double* total_bytes);

/* FP64 FMA throughput probe (the paper has no counterpart; it measures the
 * FP64 peak that the FP64 kernels' rooflines divide by): launches `blocks`
 * CTAs of 256 threads on `stream`, each thread running eight independent FMA
 * chains of `iters` steps, i.e. blocks * 256 * iters * 16 flops. sink: device
 * pointer to one double (written only in a case no input reaches). The caller
 * times the launch with events on the same stream. Errors: FSI_EINVAL, FSI_ECUDA. */
int fsi_fp64_probe(int blocks, int iters, double seed, double* sink, void* stream);

/* Tensor-core tile product (the paper has no counterpart; it is the primitive of
 * the tensor-core element contraction, exposed so that it can be tested alone):
 * D = A B^T with A device [128][32], B device [16][32] and D device [128][16],
 * all FP32 row-major. Each FP32 operand enters the BF16 tcgen05 MMA as nsplit
 * BF16 terms (1: plain BF16 rounding; 2 or 3: the rounding residuals as
 * further terms, 3 giving FP32-level accuracy); products accumulate in FP32
 * in tensor memory. Synchronises the stream. Errors: FSI_EINVAL, FSI_ECUDA
 * (also when the MMA completion is not seen within the kernel's poll limit). */
int fsi_tc_tile_product(int nsplit, const float* A, const float* B, float* D, void* stream);

long long fsi_launch_count(int kernel_id);
int fsi_kernel_count(void);
const char* fsi_kernel_name(int kernel_id);

#ifdef __cplusplus
}
#endif
#endif /* FSI_H */
