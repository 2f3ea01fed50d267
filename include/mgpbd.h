/*
 * mgpbd.h -- C ABI of the GB300 (sm_103a) global XPBD solver of MGPBD
 * (Li et al., "MGPBD: A Multigrid Accelerated Global XPBD Solver",
 * SIGGRAPH 2025).
 *
 * One handle holds one simulation instance resident in device memory.  Every
 * call is asynchronous on the CUDA stream given at create time unless its
 * comment says that it synchronises.  All device pointers are plain CUDA
 * global-memory addresses; host pointers are ordinary (pageable or pinned)
 * memory.  No call retains a caller pointer after it returns.
 *
 * Errors: every call returns an mgpbd_status; a negative value is an error,
 * a positive value a warning.  mgpbd_last_error() gives a thread-local text
 * for the most recent error of the calling thread.  No call throws.
 */
#ifndef MGPBD_H
#define MGPBD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque instance handle, owned by the library. */
typedef struct mgpbd_handle mgpbd_handle_t;

typedef int mgpbd_status;
enum {
  MGPBD_OK = 0,
  MGPBD_W_NOT_CONVERGED = 1,  /* PCG stopped at pcg_maxiter above pcg_rtol */
  MGPBD_E_INVALID = -1,       /* bad argument or mesh */
  MGPBD_E_OOM = -2,           /* device allocation failed */
  MGPBD_E_BREAKDOWN = -3,     /* PCG: p^T A p <= 0, r^T z <= 0, or NaN */
  MGPBD_E_SINGULAR = -4,      /* coarsest Cholesky pivot <= 0 */
  MGPBD_E_DEVICE_TIMEOUT = -5,/* a bounded device wait ran out */
  MGPBD_E_CUDA = -6,          /* a CUDA runtime call failed */
  MGPBD_E_BUDGET = -7,        /* device-memory budget exceeded */
  MGPBD_E_SETUP = -8          /* AMG setup could not coarsen to a solvable size */
};

enum { MGPBD_MEM_HOST = 0, MGPBD_MEM_DEVICE = 1 };
enum { MGPBD_SMOOTH_JACOBI = 0, MGPBD_SMOOTH_MCGS = 1, MGPBD_SMOOTH_CHEBYSHEV = 2 };
enum { MGPBD_FP64 = 0, MGPBD_MIXED = 1 };

/* Problem definition (eq. 1-3 of the paper).  Host pointers, copied at
 * create.  Rows of the constraint system are all distance rows (in the order
 * of `dist`) followed by one row per tetrahedron (in the order of `tet`).
 *   rest_pos  [n_verts*3]  rest shape (AoS xyz), defines L0, V0 and Dm
 *   inv_mass  [n_verts]    M^-1 per vertex; 0 pins the vertex
 *   dist      [n_dist*2]   distance pairs, C = |x_a - x_b| - L0
 *   tet       [n_tet*4]    tetrahedra; their rows are, by tet_kind,
 *                          0: volume, C = V(x) - V0 with V = det[x1-x0,x2-x0,x3-x0]/6
 *                          1: ARAP (Sec. 5.3), C = |F - R|_F^2 with F = Ds Dm^-1 the
 *                             deformation gradient and R its polar rotation
 *   alpha     [n_dist+n_tet] compliance per row; alpha~ = alpha/dt^2 (eq. 2)
 *                          (Sec. 5.3 uses alpha = 1/(mu V_tet) for ARAP rows)
 * A zero-initialised descriptor has tet_kind 0. */
typedef struct {
  int n_verts;
  const double *rest_pos;
  const double *inv_mass;
  int n_dist;
  const int32_t *dist;
  int n_tet;
  const int32_t *tet;
  const double *alpha;
  int tet_kind;
} mgpbd_mesh_desc;

/* Solver parameters.  mgpbd_default_params() fills the paper's defaults:
 * theta_s = 0.1 (Sec. 4.1), 2 smoothing sweeps (Sec. 4.5), lambda_min
 * estimate 0.1 (Sec. 4.5), coarsest below 400 rows (Sec. 4.1, setup-pipeline figure), omega_x 0.25. */
typedef struct {
  double dt;            /* time step */
  double gravity[3];    /* f_ext / m */
  double omega_x;       /* position relaxation of Alg. 1 */
  int max_iter;         /* global iterations per frame (Alg. 1) */
  double eps_b;         /* stop the frame when |b| < eps_b (0 disables) */
  double pcg_rtol;      /* PCG stop: |r|/|b| <= pcg_rtol */
  int pcg_maxiter;      /* PCG iteration cap (a safeguard; default 20000) */
  int setup_interval;   /* lazy setup every k global iterations (Sec. 4.2) */
  int nk_sweeps;        /* near-kernel Jacobi sweeps on A x = 0 (Sec. 4.3) */
  double nk_omega;      /* their weight */
  double theta_s;       /* strength threshold (Sec. 4.1) */
  int smoother;         /* MGPBD_SMOOTH_JACOBI (weighted Jacobi, default),
                           MGPBD_SMOOTH_MCGS (multicolour Gauss-Seidel: forward colours
                           before, reverse colours after the coarse correction) or
                           MGPBD_SMOOTH_CHEBYSHEV (Chebyshev polynomial of degree
                           smooth_sweeps on [lambda_min_est, safety*lambda_max]) */
  int smooth_sweeps;    /* pre- and post-smoothing sweeps (Sec. 4.5) */
  double lambda_min_est;/* lambda_min estimate in omega_opt (Sec. 4.5) */
  int power_iters;      /* power-method iterations for lambda_max */
  double power_safety;  /* factor on the lambda_max estimate */
  int coarse_max;       /* stop coarsening below this many rows (Sec. 4.1, setup-pipeline figure) */
  int max_levels;       /* hard cap on the number of levels */
  int precision;        /* MGPBD_FP64 or MGPBD_MIXED */
  int backtrack;        /* 0: x += omega_x dx; k > 0: start at omega_x and halve omega
                           while the dual residual |b| does not decrease, at most k
                           times (the paper's backtracking option, Sec. 4) */
  int autotune;         /* 0: lanes per matrix row by a fixed rule (reproducible
                           bit for bit); 1: time the row kernels of every level at
                           each setup and keep the fastest shape (rounding of the
                           row sums then depends on the choice) */
  int level0_op;        /* 0: level-0 products (A.p, V-cycle sweeps and residual) with
                           the assembled CSR matrix; 1: matrix-free, y = J (W (J^T x))
                           + alpha~ x through the constraint gradients (the paper's
                           future-work direction, Sec. 6).  Setup and Galerkin
                           products always use the assembled matrix. */
  int use_graphs;       /* 1: capture chunks of 8 PCG iterations into a CUDA graph and
                           replay it (one launch instead of ~40 per iteration; the
                           graph is re-captured after each setup); 0: plain launches.
                           Needs a stream of the caller's own: on the legacy default
                           stream (NULL) launches stay plain. */
  int linear_solver;    /* 0: MGPCG (Sec. 4.4); 1: XPBD's local step dl_j = b_j / A_jj
                           (eq. 4, the Jacobi form the paper compares against) */
  int nk_vectors;       /* k near-kernel vectors (Sec. 4.3; the paper uses six), 1..8: P
                           has k columns per aggregate from a QR of each aggregate's
                           block of B, coarse levels have k unknowns per aggregate */
  int ap_split;         /* 0: the PCG recurrence's A.p in FP64 (default); 1 (needs
                           precision MGPBD_MIXED and level0_op 1): A.p matrix-free
                           from float-float pairs (every FP64 operand stored as FP32
                           high and low parts, products and sums by error-free
                           transformations on the FP32 pipe, ~2^-46 relative per
                           product), with the recursive residual replaced by an FP64
                           b - A x whenever |r| has fallen tenfold since the solve's
                           start or its last replacement.  x, r, p and the scalars
                           stay FP64.  Instances with it set step outside a cohort. */
  uint64_t seed_nk, seed_agg, seed_col, seed_pow;
} mgpbd_params;

typedef struct {
  int pcg_iters;
  int status;           /* MGPBD_OK, MGPBD_W_NOT_CONVERGED or an error */
  double bnorm;         /* |b|_2 of the solved system */
  double rel_res;       /* recursive |r|/|b| at exit */
  double true_rel_res;  /* |b - A dlambda| / |b| recomputed in FP64 */
  double omega;         /* relaxation used for x (after backtracking) */
  double bnorm_after;   /* |b| at the updated state (backtracking only, else -1) */
  int replacements;     /* residual replacements of the solve (params.ap_split) */
} mgpbd_solve_info;

typedef struct {
  int levels;           /* number of AMG levels (1 = direct solve) */
  int n_setups;         /* setups run so far */
  int64_t global_iters; /* global iterations run so far */
  double op_complexity; /* sum nnz_l / nnz_0 (Table 1 column C) */
  size_t device_bytes;  /* device memory held by the handle */
  double ms_setup, ms_galerkin, ms_solve, ms_other; /* accumulated phase times */
  size_t peak_device_bytes; /* high-water mark of device_bytes since create */
} mgpbd_stats_t;

typedef struct {
  int n;                /* rows */
  int64_t nnz;
  int n_agg;            /* aggregates (0 on the coarsest level) */
  int n_colors;         /* colours of the multicolour ordering (0 if none) */
  double lmax, omega;   /* power-method lambda_max(D^-1 A) and Jacobi weight */
  int lanes_fp32, lanes_fp64; /* lanes per row picked by the autotuner (0 = rule) */
} mgpbd_level_info;

/* Fills p with the defaults listed above.  Never fails for p != NULL. */
mgpbd_status mgpbd_default_params(mgpbd_params *p);

/* Creates an instance (Alg. 1 problem set-up; fixed CSR pattern, Sec. 4.2).
 * Uploads the mesh, computes rest lengths/volumes, builds the vertex
 * incidence, the diagonal-last CSR pattern of A and its assembly map on the
 * device.  `stream` is a cudaStream_t (NULL = legacy default stream).
 * Positions start at rest_pos, velocities at 0.  Synchronises the stream.
 * Errors: MGPBD_E_INVALID (index out of range, nnz >= 2^31, bad params),
 * MGPBD_E_OOM, MGPBD_E_CUDA.  *out is NULL on error. */
mgpbd_status mgpbd_create(const mgpbd_mesh_desc *mesh, const mgpbd_params *p, void *stream,
                          mgpbd_handle_t **out);

/* mgpbd_create with every device array of the instance placed in a buffer
 * the caller owns (for example a torch uint8 tensor), so that the caller
 * decides where, and within what budget, the instance lives.
 *   d_workspace  device memory, 256-byte aligned; the library carves its
 *                arrays out of it (first fit, freed ranges reused) and never
 *                frees it; it must outlive mgpbd_destroy of the handle
 *   bytes        its size; mgpbd_workspace_size bounds what create and the
 *                first setup hold (nk_vectors = 1); a later setup whose
 *                coarse levels outgrow their capacity re-allocates them with
 *                25% headroom and may need more
 * Pinned host scalars, events and CUDA graphs are still allocated by the
 * runtime.  Results are bitwise those of mgpbd_create: no kernel depends on
 * where its arrays lie.  Errors: as mgpbd_create; MGPBD_E_INVALID for a NULL,
 * misaligned or non-device workspace; MGPBD_E_BUDGET when an allocation does
 * not fit, at create or later (a setup whose hierarchy needs more), with the
 * handle left valid in the latter case. */
mgpbd_status mgpbd_create_in_workspace(const mgpbd_mesh_desc *mesh, const mgpbd_params *p,
                                       void *d_workspace, size_t bytes, void *stream,
                                       mgpbd_handle_t **out);

/* Frees everything the handle holds.  Synchronises its stream. NULL is a no-op. */
void mgpbd_destroy(mgpbd_handle_t *h);

/* Positions and velocities, AoS [n_verts*3] doubles, host or device memory
 * per `mem`.  Either pointer may be NULL to leave that array unchanged.
 * Host-memory transfers synchronise the stream. */
mgpbd_status mgpbd_set_state(mgpbd_handle_t *h, const double *x, const double *v, int mem);
mgpbd_status mgpbd_get_state(mgpbd_handle_t *h, double *x, double *v, int mem);

/* Alg. 1 for n_frames frames: per frame semi-implicit Euler and lambda = 0,
 * max_iter global iterations (C and grad C, assembly, b, lazy setup or
 * Galerkin re-form, coarsest Cholesky, MGPCG, dx, lambda and x update,
 * |b| < eps_b test), then the velocity update.  Synchronises at lazy-setup
 * points and at PCG convergence polls.  Returns the worst PCG status seen
 * (MGPBD_W_NOT_CONVERGED when any solve hit pcg_maxiter) or an error. */
mgpbd_status mgpbd_step(mgpbd_handle_t *h, int n_frames);

/* The pieces of mgpbd_step: the frame prologue (semi-Euler, lambda = 0),
 * one global iteration (info may be NULL) and the frame epilogue (velocity). */
mgpbd_status mgpbd_begin_frame(mgpbd_handle_t *h);
mgpbd_status mgpbd_iterate(mgpbd_handle_t *h, mgpbd_solve_info *info);
mgpbd_status mgpbd_end_frame(mgpbd_handle_t *h);

/* Evaluates C, grad C, b = -C - alpha~ lambda and the values of A at the
 * current positions (Alg. 1, eq. 3), without solving. */
mgpbd_status mgpbd_eval_assemble(mgpbd_handle_t *h);

/* Runs the full AMG setup (Sec. 4.1-4.3, setup-pipeline figure) on the current A. */
mgpbd_status mgpbd_setup(mgpbd_handle_t *h);

/* Readies the current A for solving: setup if none exists, else the
 * Galerkin re-form of every coarse operator (Sec. 4.4); then the coarsest
 * Cholesky.  Synchronises. */
mgpbd_status mgpbd_prepare_solve(mgpbd_handle_t *h);

/* MGPCG (Sec. 4.4) on the current hierarchy: solves A dl = b from dl = 0.
 * d_b, d_dl: device arrays of n_rows doubles (d_b is not modified).
 * Synchronises; fills info if not NULL. */
mgpbd_status mgpbd_solve(mgpbd_handle_t *h, const double *d_b, double *d_dl,
                         mgpbd_solve_info *info);

/* One V-cycle z = V(r) of the current hierarchy (the preconditioner of
 * Sec. 4.4); device arrays of n_rows doubles. */
mgpbd_status mgpbd_vcycle(mgpbd_handle_t *h, const double *d_r, double *d_z);

/* y = A x with the level-0 matrix of eq. 3 (A = grad C M^-1 grad C^T +
 * alpha~) at the last mgpbd_eval_assemble, in one of the forms the PCG
 * recurrence's A.p takes (Sec. 4.4): form 0 the assembled CSR matrix in FP64;
 * 1 matrix-free in FP64 (needs params.level0_op 1); 2 matrix-free from
 * float-float pairs (needs params.ap_split).  d_x, d_y: device arrays of
 * n_rows doubles, not overlapping.  MGPBD_E_INVALID when the form is not
 * prepared on the instance (before the first mgpbd_eval_assemble, or its
 * parameters off).  Synchronises. */
mgpbd_status mgpbd_apply(mgpbd_handle_t *h, const double *d_x, double *d_y, int form);

/* Counters and phase times.  Synchronises. */
mgpbd_status mgpbd_stats(mgpbd_handle_t *h, mgpbd_stats_t *s);

/* ---- inspection (host or device destinations per `mem`; synchronise) ---- */
mgpbd_status mgpbd_sizes(mgpbd_handle_t *h, int *n_verts, int *n_rows, int64_t *nnz);
mgpbd_status mgpbd_level_info_get(mgpbd_handle_t *h, int level, mgpbd_level_info *info);
/* Shapes of the row kernels (not in the paper: they decide only how the
 * GPU splits a row sum or a vertex sum among threads, which changes the
 * rounding order of that sum).  mgpbd_set_lanes forces, for every level,
 *   csr32, csr64    lanes per CSR row of the FP32 and FP64 row kernels
 *                   (sweeps, residuals, A.p): 4, 8, 16 or 32
 *   vert32, vert64  lanes per vertex of the matrix-free vertex pass
 *                   u = W J^T x in FP32 and FP64: 4, 8 or 16
 * with 0 meaning "the autotuner's pick, else the fixed rule".  Forced shapes
 * take precedence over params.autotune and stay in force across setups.  No
 * device work.  MGPBD_E_INVALID for another value.  mgpbd_get_lanes returns
 * the shapes in effect on level `level` (the vertex shapes are level 0's). */
mgpbd_status mgpbd_set_lanes(mgpbd_handle_t *h, int csr32, int csr64, int vert32, int vert64);
mgpbd_status mgpbd_get_lanes(mgpbd_handle_t *h, int level, int *csr32, int *csr64, int *vert32,
                             int *vert64);
/* The V-cycle below level 0 (Sec. 4.4: smoothing, residual and restriction
 * down to the coarsest level, its dense solve, prolongation and smoothing back
 * up to level 1).  By default each step is its own launch.
 * mgpbd_set_coarse_tail(h, 1) runs them, where it applies (weighted-Jacobi
 * smoother, one near-kernel vector, a level between level 0 and the coarsest)
 * from the first level of at most 16,384 rows, as one cooperative kernel over
 * two blocks per SM with a grid barrier between dependent steps; the results
 * are the same bits either way (no step of it sums across rows).  A
 * cooperative launch needs every SM at once, so it waits for other streams'
 * kernels; on these workloads it is no faster than the separate launches
 * inside a CUDA graph.  0 restores the default.  No device work;
 * MGPBD_E_INVALID for another value.
 * mgpbd_set_wait_limit bounds how many times a block of the cooperative kernel
 * polls a grid barrier (default 2^24, one to two seconds); when a wait runs
 * out the solve stops and returns MGPBD_E_DEVICE_TIMEOUT, and the next solve
 * starts from a reset barrier.  0 makes every waiting block give up at once
 * (to test that path).  MGPBD_E_INVALID for polls < 0. */
mgpbd_status mgpbd_set_coarse_tail(mgpbd_handle_t *h, int enable);
mgpbd_status mgpbd_set_wait_limit(mgpbd_handle_t *h, long long polls);
/* CSR of level `level`: ptr [n+1] int64, col [nnz] int32, val [nnz] double
 * (diagonal last in each row); any pointer may be NULL. */
mgpbd_status mgpbd_get_matrix(mgpbd_handle_t *h, int level, int64_t *ptr, int32_t *col,
                              double *val, int mem);
/* assembly map of level 0: per nnz, bits 0-1 the number of shared vertices,
 * pair p at bits 2+4p (slot in row i) and 4+4p (slot in row j) */
mgpbd_status mgpbd_get_map(mgpbd_handle_t *h, uint16_t *map, int mem);
/* vertex -> incident rows, ascending: vptr [n_verts+1], vrow [2*n_dist+4*n_tet] */
mgpbd_status mgpbd_get_incidence(mgpbd_handle_t *h, int64_t *vptr, int32_t *vrow, int mem);
/* aggregates, MIS-2 roots, P values and near-kernel B of level `level`:
 * agg, root [n]; P, B [n * nk_vectors], row-major (row i of P holds the
 * values of columns agg[i]*k .. agg[i]*k + k-1) */
mgpbd_status mgpbd_get_aggregates(mgpbd_handle_t *h, int level, int32_t *agg, uint8_t *root,
                                  double *P, double *B, int mem);
/* multicolour ordering of each level (Jones-Plassmann, used by the Gauss-Seidel
 * smoother); computed at setup when the smoother needs it or when
 * mgpbd_set_colouring(h, 1) was called before the setup */
mgpbd_status mgpbd_get_colors(mgpbd_handle_t *h, int level, int32_t *color, int mem);
mgpbd_status mgpbd_set_colouring(mgpbd_handle_t *h, int enable);
/* C [m], b [m], distance gradients n [n_dist*3], tet gradients [n_tet*12] */
mgpbd_status mgpbd_get_constraints(mgpbd_handle_t *h, double *C, double *b, double *gd,
                                   double *gt, int mem);
mgpbd_status mgpbd_get_lambda(mgpbd_handle_t *h, double *lambda, double *dlambda, int mem);

/* ---- measurement ----
 * mgpbd_profile(h, enable) with enable a mask: bit 0 (1) records a CUDA event
 * pair around every level-0 smoother sweep (one CSR launch, or the vertex and
 * row passes of the matrix-free sweep) (the dominant kernel of the V-cycle,
 * Sec. 5.2 of the paper: the V-cycle takes most of an iteration and the
 * smoother most of the V-cycle); bit 1 (2) around every A.p of the PCG
 * recurrence (read with mgpbd_profile_read_ap); 0 stops.  Each event pair
 * costs a few microseconds of the iteration, so record only what is read.
 * Other values are MGPBD_E_INVALID.  Every call resets the totals and
 * synchronises.  mgpbd_profile_read returns the summed kernel time, the number
 * of timed launches (launches skipped after PCG convergence are excluded)
 * and the algorithmic bytes of one launch (CSR values and columns once, row
 * pointers, and four row vectors).  mgpbd_launch_count is the number of
 * kernels this library has launched in the process so far. */
mgpbd_status mgpbd_profile(mgpbd_handle_t *h, int enable);
mgpbd_status mgpbd_profile_read(mgpbd_handle_t *h, double *total_ms, int64_t *launches,
                                double *bytes_per_launch);
/* The same for the A.p of the PCG recurrence (Sec. 4.4): one timed launch is
 * the product of one iteration (matrix-free: its vertex and row passes, in
 * FP64 or from float-float pairs per params.ap_split; assembled: the FP64 CSR
 * product), its algorithmic bytes counted once per array (every value 8
 * bytes in both matrix-free forms). */
mgpbd_status mgpbd_profile_read_ap(mgpbd_handle_t *h, double *total_ms, int64_t *launches,
                                   double *bytes_per_launch);
unsigned long long mgpbd_launch_count(void);

/* ---- serving: continuous batching of many instances ----
 * Not in the paper, which steps one instance at a time.  A batch holds many
 * instances (meshes with their parameters and state) and serves step
 * requests: one request = `frames` frames of Alg. 1 on one instance.  It is
 * a request loop: mgpbd_batch_admit submits a request at any time, from any
 * thread, also while other requests run; mgpbd_batch_tick returns the
 * requests that have finished since the previous tick.  A request starts as
 * soon as its instance is idle, one of max_active worker threads is free and
 * the instance fits the device-memory budget (idle resident instances are
 * evicted least recently used first; their state moves to host memory and
 * back on their next admission).  Running requests step on their instances'
 * own CUDA streams, so their kernels overlap on the GPU.  Requests of one
 * instance run in submission order.  Times are seconds on the batch's clock,
 * which starts at mgpbd_batch_create.  A request whose instance can never fit
 * the budget finishes at once with MGPBD_E_BUDGET.  Instances may be added
 * at any time; their indices are 0, 1, 2, ... in order of addition. */
typedef struct mgpbd_batch mgpbd_batch_t;
typedef struct {
  size_t hbm_budget;  /* bytes of device memory the resident instances may hold */
  int max_active;     /* requests stepping at the same time, 1..256 (1..64 with cohort) */
  int cohort;         /* 0: each running request on its own stream and worker thread;
                         1: one stepping thread runs every running request together:
                         the PCG iterations of all of them run as ONE launch per step
                         (A.p passes, x/r update, level-0 sweeps and residual,
                         restriction, the V-cycle below level 0 as one cooperative
                         kernel, prolongation, final sweep, p update), each instance
                         keeping the grid and reduction order of its own solve, so
                         its results are bit for bit those of running alone.  Covers
                         mixed precision, matrix-free level 0, two weighted-Jacobi
                         sweeps, one near-kernel vector and at least two levels;
                         other instances solve alone on the same thread. */
} mgpbd_batch_config;
typedef struct {
  int id;             /* caller's request id, copied to the result (mgpbd_batch_run) */
  int instance;       /* instance index returned by mgpbd_batch_add_instance */
  int frames;         /* frames of Alg. 1 to run (each max_iter global iterations) */
  double arrival_s;   /* arrival time, seconds after mgpbd_batch_run starts */
} mgpbd_step_request;
typedef struct {
  int id;             /* ticket of mgpbd_batch_admit (the request's id under mgpbd_batch_run) */
  int instance, status;
  double arrival_s, start_s, finish_s;  /* latency = finish_s - arrival_s */
  int64_t global_iters, pcg_iters;
} mgpbd_step_result;
/* Upper estimate of the device bytes an instance of this mesh holds after
 * create and its first setup (the figure the service admits instances by,
 * and a buffer size that mgpbd_create_in_workspace accepts for them),
 * computed on the host from the mesh alone: per nonzero of A (bounded by the
 * sum over rows of their vertices' degrees) column, FP64 and FP32 values,
 * assembly map and strength mask; per row, vertex and incidence entry the
 * vectors, gradients and matrix-free arrays; the dense coarsest factor and
 * inverse for a coarsest level below p->coarse_max rows.  For nk_vectors = 1.
 * No device work.  MGPBD_E_INVALID for a malformed descriptor. */
mgpbd_status mgpbd_workspace_size(const mgpbd_mesh_desc *mesh, const mgpbd_params *p,
                                  size_t *bytes);
mgpbd_status mgpbd_batch_create(const mgpbd_batch_config *cfg, mgpbd_batch_t **out);
/* copies the mesh (host pointers) and the initial state (x0/v0 may be NULL:
 * rest positions, zero velocity); the instance is not resident until needed */
mgpbd_status mgpbd_batch_add_instance(mgpbd_batch_t *b, const mgpbd_mesh_desc *mesh,
                                      const mgpbd_params *p, const double *x0, const double *v0,
                                      int *instance);
/* Submits one request now (its arrival time is the call's time on the
 * batch's clock) and returns at once with its ticket (0, 1, 2, ... per
 * batch), which its result carries as `id`.  Thread-safe.  MGPBD_E_INVALID
 * for an unknown instance or frames < 1. */
mgpbd_status mgpbd_batch_admit(mgpbd_batch_t *b, int instance, int frames, int *ticket);
/* Copies up to `max` results of requests that finished since the previous
 * tick into res[0 .. *n), in finishing order, waiting up to wait_s seconds for
 * the first one when none is ready (0: poll).  A result is returned once. */
mgpbd_status mgpbd_batch_tick(mgpbd_batch_t *b, double wait_s, mgpbd_step_result *res, int max,
                              int *n);
/* Requests queued (not started), running, finished but not yet returned by a
 * tick, and the batch's clock now (seconds); any pointer may be NULL. */
mgpbd_status mgpbd_batch_counts(mgpbd_batch_t *b, int *queued, int *running, int *unreported,
                                double *clock);
/* Text of the error of the most recently failed request of the batch ("" if
 * none), valid until the calling thread's next call of this function.  The
 * failure itself is the request's status. */
const char *mgpbd_batch_error(mgpbd_batch_t *b);
/* Cohort mode only (zeros otherwise): rounds of the stepping thread, batched
 * PCG iterations launched (eight per round that has a solving instance), and
 * the wall time in seconds spent in the batched chunks (launch, completion,
 * scalar read-back) and in everything else of the rounds (the instances' own
 * work between solves: frame steps, C and A, setup or re-form, coarsest
 * factorisation, the start and end of each solve).  Any pointer may be NULL. */
mgpbd_status mgpbd_batch_cohort_stats(mgpbd_batch_t *b, int64_t *rounds, int64_t *batched_iters,
                                      double *chunk_s, double *other_s);
/* Replays a list of timed requests through the request loop: admits each
 * when its arrival time (seconds after the call) has passed and returns
 * when all have finished, res[i] holding request i's result (its caller id,
 * times in seconds after the call; arrival_s is the time it was admitted).
 * Results of requests admitted by other calls stay for mgpbd_batch_tick.
 * Returns the first error of a request, else MGPBD_OK. */
mgpbd_status mgpbd_batch_run(mgpbd_batch_t *b, const mgpbd_step_request *req, int n_req,
                             mgpbd_step_result *res);
/* host copy of an instance's positions/velocities (waits while a request steps
 * the instance; synchronises if it is resident) */
mgpbd_status mgpbd_batch_get_state(mgpbd_batch_t *b, int instance, double *x, double *v);
/* resident instances and bytes held now */
mgpbd_status mgpbd_batch_resident(mgpbd_batch_t *b, int *n_resident, size_t *bytes);
/* Waits for the requests that have started, drops the queued ones, frees
 * every instance. */
void mgpbd_batch_destroy(mgpbd_batch_t *b);

/* ---- precision conversions of the mixed-precision path ----
 * The paper has no counterpart of this call: it exposes the conversions the
 * MGPBD_MIXED solve uses between its FP64 Krylov vectors and its FP32
 * V-cycle, integer implementations of IEEE 754-2008 binary64 -> binary32
 * with roundTiesToEven (section 4.3.1) and of the exact binary32 ->
 * binary64 widening.  d_in64 (n doubles) is narrowed into d_out32 (n floats)
 * and d_in32 (n floats) is widened into d_out64 (n doubles); either pair may
 * be NULL/NULL to skip it.  All four are device pointers owned by the caller.
 * Asynchronous on `stream` (a cudaStream_t; NULL = legacy default stream).
 * MGPBD_E_INVALID for n < 0 or a pair given by half. */
mgpbd_status mgpbd_convert(const double *d_in64, float *d_out32, const float *d_in32,
                           double *d_out64, int64_t n, void *stream);

/* ---- allocation-free entry point ----
 * The paper has no counterpart of this call; it exists for callers that
 * cannot allocate device memory while they run: a thread capturing a CUDA
 * stream into a graph (cudaMalloc is not allowed during global-mode
 * capture), a real-time loop that must not wait on the allocator, or an
 * application whose device memory belongs to another pool.
 * It computes the FP64 true relative residual |b - A x|_2 / |b|_2 of the
 * instance's level-0 matrix (the check mgpbd_solve reports as true_rel_res)
 * into d_out[0] (device memory; 0 when b = 0), asynchronously on the
 * instance's stream.  d_b and d_x are device arrays of n_rows doubles owned
 * by the caller.  It calls no cudaMalloc, cudaFree or allocating library
 * routine: its per-block partial sums live in one static device array of
 * about 1 MiB that every GPU loading the library holds until the process
 * exits.  All calls share that array and it keeps the last call's contents
 * (the block counter is cleared before each launch), so calls that overlap
 * on the GPU race and must be serialised by the caller.  The first call on a
 * device looks up the array's address (once per device); make it before any
 * stream capture starts.  The instance's device (current at its create) must
 * be the current device, else MGPBD_E_INVALID.  Instances with more than 4,194,304 constraint rows
 * are rejected with MGPBD_E_INVALID (the array holds 65,536 blocks of 64 rows). */
mgpbd_status mgpbd_true_residual_noalloc(mgpbd_handle_t *h, const double *d_b, const double *d_x,
                                         double *d_out);

/* Thread-local text of the calling thread's last error ("" if none). */
const char *mgpbd_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
