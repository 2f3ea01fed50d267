/*
 * mgpbd_oracle.c -- plain, slow, single-threaded FP64 CPU oracle of the MGPBD
 * global XPBD solve (Li et al., "MGPBD: A Multigrid Accelerated Global XPBD
 * Solver", SIGGRAPH 2025).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark call this file.  The CUDA library shares no
 * code, header, table or helper with it.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -shared -fPIC (no FMA
 * contraction: every fused multiply-add below is an explicit fma() call).
 *
 * What it computes, step by step in the order of Algorithm 1:
 *   semi-implicit Euler predict and lambda reset        (Alg. 1, Sec. 3 eq. 1)
 *   constraint values C and gradients: distance, volume
 *     and ARAP rows                                      (Alg. 1, eq. 3, Sec. 5.3)
 *   A = grad C  M^-1  grad C^T + alpha~ on a fixed CSR
 *     pattern, off-diagonals first, diagonal last        (eq. 3, Sec. 4.2)
 *   b = -C - alpha~ lambda                               (eq. 3)
 *   lazy UA-AMG setup: near-kernel sweeps (k vectors),
 *     strength filter, aggregation, injection (QR per
 *     aggregate for k > 1), next-level near-kernel,
 *     Galerkin, recursion below 400 rows                 (Sec. 4.1-4.3, setup-pipeline figure)
 *   Galerkin coarse operators P^T A P                    (Sec. 4.4, eq. 6)
 *   coarsest dense Cholesky                              (reading: Sec. 4.1 size rule)
 *   PCG with one V-cycle per iteration                   (Sec. 4.4)
 *   weighted-Jacobi / multicolour GS / Chebyshev
 *     smoothing, omega from the power method and the
 *     lambda_min estimate                                (Sec. 4.5)
 *   or XPBD's local step dlambda_j = b_j / A_jj          (eq. 4)
 *   dx = M^-1 grad C^T dlambda, lambda and x update,
 *     optionally with backtracking of omega_x            (eq. 5, Alg. 1, Sec. 4)
 *   velocity update                                      (Alg. 1)
 *
 * Readings where the paper is silent (the constraint forms, the
 * deterministic MIS-2 aggregation, the number of near-kernel vectors,
 * summation orders, the coarsest solve) are listed in the design notes and
 * restated at each function below.
 *
 * How it is pinned (tests/test_oracle_pins.py, test_oracle_arap.py,
 * test_oracle_nearkernel.py): against published generator outputs, finite
 * differences, closed forms, dense J M^-1 J^T + alpha~ built in numpy,
 * brute-force patterns, aggregations and colourings, scipy's P^T A P, dense
 * Cholesky solves, the textbook XPBD update and a compliant two-particle
 * solution, V-cycle symmetry and the Chebyshev polynomial.
 * tests/test_oracle_mutants.py plants 58 plausible mistakes in a copy of
 * this file, one at a time, and each is caught by a named pin.
 * Parity unpinned: whole-frame trajectories of the stiff meshes beyond those
 * invariants (the paper prints no trajectory).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXL 16

/* Loops over independent rows carry ORC_ROWS.  The plain build ignores it;
   the -fopenmp build (liborc_omp.so, used to time the oracle on all host
   cores and to run it at test sizes where one core is too slow) splits the
   rows among threads.  Each row's arithmetic is the same in both, so both
   builds give the same bits.  Sums across rows (dot products, norms) stay
   sequential. */
#define ORC_ROWS _Pragma("omp parallel for schedule(static)")

enum {
  ORC_OK = 0,
  ORC_W_NOT_CONVERGED = 1,
  ORC_E_INVALID = -1,
  ORC_E_OOM = -2,
  ORC_E_BREAKDOWN = -3,
  ORC_E_SINGULAR = -4,
  ORC_E_SETUP = -8
};

typedef struct {
  double dt;
  double gravity[3];
  double omega_x;
  int max_iter;
  double eps_b;
  double pcg_rtol;
  int pcg_maxiter;
  int setup_interval;
  int nk_sweeps;
  double nk_omega;
  double theta_s;
  int smoother; /* 0 weighted Jacobi, 1 multicolour Gauss-Seidel, 2 Chebyshev */
  int smooth_sweeps;
  double lambda_min_est;
  int power_iters;
  double power_safety;
  int coarse_max;
  int max_levels;
  int backtrack;  /* 0: fixed omega_x; k > 0: halve omega up to k times (Sec. 4) */
  int linear_solver; /* 0: MGPCG (Sec. 4.4); 1: XPBD diagonal step dl_j = b_j / A_jj (eq. 4) */
  int nk_vectors;    /* k near-kernel vectors, k columns of P per aggregate (Sec. 4.3) */
  uint64_t seed_nk, seed_agg, seed_col, seed_pow;
} orc_params;

typedef struct {
  int n;
  int64_t nnz;
  int64_t *ptr;
  int32_t *col;
  double *val;
} orc_csr;

typedef struct {
  orc_csr A;
  /* prolongator to the next level (absent on the coarsest) */
  int n_agg;
  int32_t *agg;     /* aggregate of each row */
  uint8_t *root;    /* 1 for the MIS-2 roots */
  double *B;        /* near-kernel at this level, n x k row-major */
  double *P;        /* row i of P: k values in columns agg_i*k .. agg_i*k+k-1 */
  uint8_t *pdead;   /* n_agg*k: 1 where a column of P is zero (rank-deficient B_a) */
  int64_t *mptr;    /* members of each aggregate, ascending */
  int32_t *mrow;
  double lmax, omega;
  int n_colors;
  int32_t *color;
  double *x, *b, *r, *t; /* V-cycle work vectors */
} orc_level;

typedef struct {
  int pcg_iters;
  int status;
  double bnorm;
  double rel_res;      /* recursive residual at exit */
  double true_rel_res; /* ||b - A dl|| / ||b|| in FP64 */
  double omega;        /* position relaxation used by the update */
  double bnorm_after;  /* |b| at the updated x and lambda (backtracking only) */
} orc_solve_info;

typedef struct {
  int N, E, T, m;
  double *rest, *w, *alpha, *alpha_t, *L0, *V0;
  int tet_kind;  /* 0: volume rows; 1: ARAP rows (Sec. 5.3) */
  double *Dminv; /* ARAP: inverse rest edge matrix per tet, row-major [T][9] */
  int32_t *edge, *tet;
  orc_params p;
  double *x, *v, *xold, *lambda;
  double *C, *b, *gd, *gt, *dl, *dx, *xbak;
  orc_csr A;
  uint16_t *map;
  int64_t *vptr;
  int32_t *vrow;
  int L; /* number of levels */
  int have_setup;
  orc_level lev[ORC_MAXL];
  double *chol;
  int chol_n;
  long it_global;
  /* PCG vectors */
  double *pr, *pz, *pp, *pq;
  orc_solve_info last;
  int n_setups;
} orc;

/* ------------------------------------------------------------------------- */
/* counter-based generator: SplitMix64 output function (Steele, Lea, Flood,   */
/* "Fast splittable pseudorandom number generators", OOPSLA 2014; the         */
/* constants are those of its public reference implementation).              */
/* ------------------------------------------------------------------------- */
static uint64_t h64(uint64_t k) {
  uint64_t z = k + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
/* key of row i at level l for a given seed: seed<<40 | l<<32 | i */
static uint64_t hkey(uint64_t seed, int l, int i) {
  return (seed << 40) | ((uint64_t)(uint32_t)l << 32) | (uint64_t)(uint32_t)i;
}
/* uniform in (0,1): ((h >> 11) + 0.5) * 2^-53 */
static double u01(uint64_t h) { return ((double)(h >> 11) + 0.5) * 0x1p-53; }

uint64_t orc_h64(uint64_t k) { return h64(k); }

#ifdef _OPENMP
#include <omp.h>
#endif
/* threads the row loops use (1 in the plain build); n > 0 sets them */
int orc_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

static void *xcalloc(size_t n, size_t s) { return calloc(n ? n : 1, s ? s : 1); }

static void csr_free(orc_csr *a) {
  free(a->ptr); free(a->col); free(a->val);
  memset(a, 0, sizeof(*a));
}

static void level_free(orc_level *L) {
  csr_free(&L->A);
  free(L->agg); free(L->root); free(L->B); free(L->P); free(L->pdead); free(L->mptr); free(L->mrow);
  free(L->color); free(L->x); free(L->b); free(L->r); free(L->t);
  memset(L, 0, sizeof(*L));
}

/* vertices of row j; returns the count (2 for distance, 4 for volume rows) */
static int row_verts(const orc *o, int j, int32_t *v) {
  if (j < o->E) { v[0] = o->edge[2 * j]; v[1] = o->edge[2 * j + 1]; return 2; }
  const int32_t *t = o->tet + 4 * (int64_t)(j - o->E);
  v[0] = t[0]; v[1] = t[1]; v[2] = t[2]; v[3] = t[3];
  return 4;
}

/* gradient of row j with respect to its vertex in slot s */
static void row_grad(const orc *o, int j, int s, double g[3]) {
  if (j < o->E) {
    const double *n = o->gd + 3 * (int64_t)j;
    if (s == 0) { g[0] = n[0]; g[1] = n[1]; g[2] = n[2]; }
    else { g[0] = -n[0]; g[1] = -n[1]; g[2] = -n[2]; }
    return;
  }
  const double *t = o->gt + 12 * (int64_t)(j - o->E) + 3 * s;
  g[0] = t[0]; g[1] = t[1]; g[2] = t[2];
}

/* ------------------------------------------------------------------------- */
/* Constraint functions (reading: the paper uses distance constraints,       */
/* Sec. 4.2 and the cloth scene, without printing them; volume constraints   */
/* are this build's reading for tetrahedral meshes).                         */
/* ------------------------------------------------------------------------- */

/* distance: C = |xa - xb| - L0, grad_a = n = (xa - xb)/|xa - xb|, grad_b = -n;
   |d| = sqrt(fma(dz,dz, fma(dy,dy, dx*dx))); n = 0 when |d| = 0. */
static double dist_eval(const double *xa, const double *xb, double L0, double n[3]) {
  double d0 = xa[0] - xb[0], d1 = xa[1] - xb[1], d2 = xa[2] - xb[2];
  double len = sqrt(fma(d2, d2, fma(d1, d1, d0 * d0)));
  if (len > 0.0) { n[0] = d0 / len; n[1] = d1 / len; n[2] = d2 / len; }
  else { n[0] = n[1] = n[2] = 0.0; }
  return len - L0;
}

static void cross(const double *a, const double *b, double *c) {
  double t1, t2;
  t1 = a[1] * b[2]; t2 = a[2] * b[1]; c[0] = t1 - t2;
  t1 = a[2] * b[0]; t2 = a[0] * b[2]; c[1] = t1 - t2;
  t1 = a[0] * b[1]; t2 = a[1] * b[0]; c[2] = t1 - t2;
}

/* volume: e_k = x_k - x_0; V = e1.(e2 x e3)/6; C = V - V0;
   g1 = (e2 x e3)/6, g2 = (e3 x e1)/6, g3 = (e1 x e2)/6, g0 = -((g1+g2)+g3). */
static double tet_eval(const double *x0, const double *x1, const double *x2,
                       const double *x3, double V0, double g[12]) {
  double e1[3], e2[3], e3[3], c23[3], c31[3], c12[3];
  for (int k = 0; k < 3; ++k) { e1[k] = x1[k] - x0[k]; e2[k] = x2[k] - x0[k]; e3[k] = x3[k] - x0[k]; }
  cross(e2, e3, c23); cross(e3, e1, c31); cross(e1, e2, c12);
  for (int k = 0; k < 3; ++k) {
    g[3 + k] = c23[k] / 6.0;
    g[6 + k] = c31[k] / 6.0;
    g[9 + k] = c12[k] / 6.0;
    g[k] = -((g[3 + k] + g[6 + k]) + g[9 + k]);
  }
  double V = fma(e1[2], c23[2], fma(e1[1], c23[1], e1[0] * c23[0])) / 6.0;
  return V - V0;
}

/* ARAP constraint (Sec. 5.3): C = |F - R|_F^2 with F = Ds Dm^-1 the
   deformation gradient (Ds, Dm: edge matrices [x1-x0, x2-x0, x3-x0] now and
   at rest) and R the rotation of F's polar decomposition F = R S.
   R: Newton's iteration for the orthogonal polar factor, R <- (R + R^-T)/2
   from R = F, a fixed ARAP_POLAR_ITERS times (quadratic convergence; the
   singular values map to (s + 1/s)/2).  R^-T = [c1 x c2, c2 x c0, c0 x c1] /
   det R for the columns c_k of R.  A singular F (det F = 0) has no unique
   polar factor: the row gets C = 0 and zero gradient.
   Gradient: dC = 2 (F - R) : dF (the term (F - R) : dR vanishes because
   R^T (F - R) = S - I is symmetric and R^T dR is skew), so with B = Dm^-1
   dC/dx_k = 2 (F - R) B^T e_k for k = 1..3 and dC/dx_0 = -((g1 + g2) + g3).
   Inverse rest edge matrix: the rows of Dm^-1 are (e2 x e3, e3 x e1,
   e1 x e2) / det Dm. */
#define ARAP_POLAR_ITERS 20

static void arap_rest(const double *x0, const double *x1, const double *x2, const double *x3,
                      double B[9]) {
  double e1[3], e2[3], e3[3], c[3][3];
  for (int k = 0; k < 3; ++k) { e1[k] = x1[k] - x0[k]; e2[k] = x2[k] - x0[k]; e3[k] = x3[k] - x0[k]; }
  cross(e2, e3, c[0]); cross(e3, e1, c[1]); cross(e1, e2, c[2]);
  double det = fma(e1[2], c[0][2], fma(e1[1], c[0][1], e1[0] * c[0][0]));
  for (int r = 0; r < 3; ++r)
    for (int k = 0; k < 3; ++k) B[3 * r + k] = det != 0.0 ? c[r][k] / det : 0.0;
}

static double arap_eval(const double *x0, const double *x1, const double *x2, const double *x3,
                        const double B[9], double g[12]) {
  double d[3][3]; /* d[k] = x_{k+1} - x_0 (column k of Ds) */
  for (int a = 0; a < 3; ++a) { d[0][a] = x1[a] - x0[a]; d[1][a] = x2[a] - x0[a]; d[2][a] = x3[a] - x0[a]; }
  double F[3][3], R[3][3];
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c)
      F[a][c] = fma(d[2][a], B[6 + c], fma(d[1][a], B[3 + c], d[0][a] * B[c]));
  /* det F = c0 . (c1 x c2) over the columns of F */
  double col[3][3], x12[3];
  for (int k = 0; k < 3; ++k) for (int a = 0; a < 3; ++a) col[k][a] = F[a][k];
  cross(col[1], col[2], x12);
  double detF = fma(col[0][2], x12[2], fma(col[0][1], x12[1], col[0][0] * x12[0]));
  if (detF == 0.0) {
    for (int k = 0; k < 12; ++k) g[k] = 0.0;
    return 0.0;
  }
  memcpy(R, F, sizeof(R));
  for (int it = 0; it < ARAP_POLAR_ITERS; ++it) {
    double cc[3][3], dual[3][3];
    for (int k = 0; k < 3; ++k) for (int a = 0; a < 3; ++a) cc[k][a] = R[a][k];
    cross(cc[1], cc[2], dual[0]); cross(cc[2], cc[0], dual[1]); cross(cc[0], cc[1], dual[2]);
    double det = fma(cc[0][2], dual[0][2], fma(cc[0][1], dual[0][1], cc[0][0] * dual[0][0]));
    for (int a = 0; a < 3; ++a)
      for (int k = 0; k < 3; ++k) R[a][k] = 0.5 * (R[a][k] + dual[k][a] / det);
  }
  double C = 0.0, D[3][3];
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) {
      D[a][c] = F[a][c] - R[a][c];
      C = fma(D[a][c], D[a][c], C);
    }
  for (int k = 0; k < 3; ++k)
    for (int a = 0; a < 3; ++a) {
      double t = fma(D[a][2], B[3 * k + 2], fma(D[a][1], B[3 * k + 1], D[a][0] * B[3 * k]));
      g[3 * (k + 1) + a] = 2.0 * t;
    }
  for (int a = 0; a < 3; ++a) g[a] = -((g[3 + a] + g[6 + a]) + g[9 + a]);
  return C;
}

/* Alg. 1 (calculate C and grad C), eq. 3 (b = -C - alpha~ lambda) */
static void eval_constraints(orc *o) {
  ORC_ROWS
  for (int j = 0; j < o->E; ++j) {
    const double *xa = o->x + 3 * (int64_t)o->edge[2 * j];
    const double *xb = o->x + 3 * (int64_t)o->edge[2 * j + 1];
    o->C[j] = dist_eval(xa, xb, o->L0[j], o->gd + 3 * (int64_t)j);
  }
  ORC_ROWS
  for (int t = 0; t < o->T; ++t) {
    const int32_t *tv = o->tet + 4 * (int64_t)t;
    const double *p0 = o->x + 3 * (int64_t)tv[0], *p1 = o->x + 3 * (int64_t)tv[1];
    const double *p2 = o->x + 3 * (int64_t)tv[2], *p3 = o->x + 3 * (int64_t)tv[3];
    o->C[o->E + t] = o->tet_kind == 1
                         ? arap_eval(p0, p1, p2, p3, o->Dminv + 9 * (int64_t)t, o->gt + 12 * (int64_t)t)
                         : tet_eval(p0, p1, p2, p3, o->V0[t], o->gt + 12 * (int64_t)t);
  }
  ORC_ROWS
  for (int j = 0; j < o->m; ++j) {
    double t = o->alpha_t[j] * o->lambda[j];
    o->b[j] = (-o->C[j]) - t;
  }
}

/* ------------------------------------------------------------------------- */
/* Fixed CSR pattern of A (Sec. 4.2: three fixed-length arrays, off-diagonal */
/* terms first, diagonal last).  Row i's off-diagonals are all rows j != i   */
/* sharing at least one vertex with i (pinned or not), ascending j.  The     */
/* assembly map of each off-diagonal lists the shared vertices in ascending  */
/* vertex id as (slot in i, slot in j) pairs:                                */
/*   bits 0-1 count, pair p at bits 2+4p (slot in i) and 4+4p (slot in j).   */
/* ------------------------------------------------------------------------- */
static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

static int build_pattern(orc *o) {
  int N = o->N, m = o->m;
  /* vertex -> incident rows, ascending row id */
  o->vptr = (int64_t *)xcalloc((size_t)N + 1, sizeof(int64_t));
  int32_t vv[4];
  for (int j = 0; j < m; ++j) {
    int c = row_verts(o, j, vv);
    for (int k = 0; k < c; ++k) o->vptr[vv[k] + 1]++;
  }
  for (int v = 0; v < N; ++v) o->vptr[v + 1] += o->vptr[v];
  o->vrow = (int32_t *)xcalloc((size_t)o->vptr[N], sizeof(int32_t));
  int64_t *fill = (int64_t *)xcalloc((size_t)N, sizeof(int64_t));
  for (int j = 0; j < m; ++j) {
    int c = row_verts(o, j, vv);
    for (int k = 0; k < c; ++k) o->vrow[o->vptr[vv[k]] + fill[vv[k]]++] = j;
  }
  free(fill);

  /* count pass */
  int32_t *mark = (int32_t *)xcalloc((size_t)m, sizeof(int32_t));
  for (int j = 0; j < m; ++j) mark[j] = -1;
  int64_t *ptr = (int64_t *)xcalloc((size_t)m + 1, sizeof(int64_t));
  int maxdeg = 0;
  for (int i = 0; i < m; ++i) {
    int c = row_verts(o, i, vv), cnt = 0;
    for (int k = 0; k < c; ++k)
      for (int64_t q = o->vptr[vv[k]]; q < o->vptr[vv[k] + 1]; ++q) {
        int j = o->vrow[q];
        if (j != i && mark[j] != i) { mark[j] = i; ++cnt; }
      }
    ptr[i + 1] = ptr[i] + cnt + 1;
    if (cnt > maxdeg) maxdeg = cnt;
  }
  int64_t nnz = ptr[m];
  int32_t *col = (int32_t *)xcalloc((size_t)nnz, sizeof(int32_t));
  uint16_t *map = (uint16_t *)xcalloc((size_t)nnz, sizeof(uint16_t));
  double *val = (double *)xcalloc((size_t)nnz, sizeof(double));
  if (!col || !map || !val) { free(mark); free(ptr); free(col); free(map); free(val); return ORC_E_OOM; }
  int32_t *tmp = (int32_t *)xcalloc((size_t)maxdeg + 1, sizeof(int32_t));
  for (int j = 0; j < m; ++j) mark[j] = -1;
  for (int i = 0; i < m; ++i) {
    int c = row_verts(o, i, vv), cnt = 0;
    for (int k = 0; k < c; ++k)
      for (int64_t q = o->vptr[vv[k]]; q < o->vptr[vv[k] + 1]; ++q) {
        int j = o->vrow[q];
        if (j != i && mark[j] != i) { mark[j] = i; tmp[cnt++] = j; }
      }
    qsort(tmp, (size_t)cnt, sizeof(int32_t), cmp_i32);
    int64_t base = ptr[i];
    for (int q = 0; q < cnt; ++q) {
      int j = tmp[q];
      int32_t wv[4];
      int cj = row_verts(o, j, wv);
      /* shared vertices, ascending vertex id */
      int32_t sv[4]; int si[4], sj[4], ns = 0;
      for (int a = 0; a < c; ++a)
        for (int bb = 0; bb < cj; ++bb)
          if (vv[a] == wv[bb]) { sv[ns] = vv[a]; si[ns] = a; sj[ns] = bb; ++ns; }
      for (int a = 1; a < ns; ++a)  /* insertion sort by vertex id */
        for (int bb = a; bb > 0 && sv[bb - 1] > sv[bb]; --bb) {
          int32_t t0 = sv[bb]; sv[bb] = sv[bb - 1]; sv[bb - 1] = t0;
          int t1 = si[bb]; si[bb] = si[bb - 1]; si[bb - 1] = t1;
          int t2 = sj[bb]; sj[bb] = sj[bb - 1]; sj[bb - 1] = t2;
        }
      if (ns > 3) ns = 3; /* two distinct rows share at most 3 vertices */
      uint16_t code = (uint16_t)ns;
      for (int pp = 0; pp < ns; ++pp)
        code |= (uint16_t)((si[pp] << (2 + 4 * pp)) | (sj[pp] << (4 + 4 * pp)));
      col[base + q] = j;
      map[base + q] = code;
    }
    col[base + cnt] = i; /* diagonal last */
    map[base + cnt] = 0;
  }
  free(tmp); free(mark);
  o->A.n = m; o->A.nnz = nnz; o->A.ptr = ptr; o->A.col = col; o->A.val = val;
  o->map = map;
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Assembly of A's values (Alg. 1; Sec. 4.2 formulas for A_ii and A_ij).     */
/*   A_ij = sum over shared v (ascending id) of acc = fma(w_v, g_i.g_j, acc)  */
/*   g_i.g_j = fma(gz_i, gz_j, fma(gy_i, gy_j, gx_i*gx_j))                    */
/*   A_ii = same over the row's own slots in slot order, then + alpha~_i     */
/* ------------------------------------------------------------------------- */
static double gdot(const double *a, const double *b) {
  return fma(a[2], b[2], fma(a[1], b[1], a[0] * b[0]));
}

static void assemble(orc *o) {
  ORC_ROWS
  for (int i = 0; i < o->m; ++i) {
    int32_t vv[4];
    int c = row_verts(o, i, vv);
    double gi[4][3];
    for (int s = 0; s < c; ++s) row_grad(o, i, s, gi[s]);
    int64_t e = o->A.ptr[i + 1] - 1;
    for (int64_t k = o->A.ptr[i]; k < e; ++k) {
      int j = o->A.col[k];
      uint16_t code = o->map[k];
      int ns = code & 3;
      double acc = 0.0;
      for (int pp = 0; pp < ns; ++pp) {
        int si = (code >> (2 + 4 * pp)) & 3, sj = (code >> (4 + 4 * pp)) & 3;
        double gj[3];
        row_grad(o, j, sj, gj);
        acc = fma(o->w[vv[si]], gdot(gi[si], gj), acc);
      }
      o->A.val[k] = acc;
    }
    double acc = 0.0;
    for (int s = 0; s < c; ++s) acc = fma(o->w[vv[s]], gdot(gi[s], gi[s]), acc);
    o->A.val[e] = acc + o->alpha_t[i];
  }
}

/* ------------------------------------------------------------------------- */
/* Sparse helpers (plain definitions)                                        */
/* ------------------------------------------------------------------------- */
static double diag_of(const orc_csr *A, int i) { return A->val[A->ptr[i + 1] - 1]; }

/* y_i = sum over row i in storage order of fma(A_ij, x_j, s) */
static void spmv(const orc_csr *A, const double *x, double *y) {
  ORC_ROWS
  for (int i = 0; i < A->n; ++i) {
    double s = 0.0;
    for (int64_t k = A->ptr[i]; k < A->ptr[i + 1]; ++k) s = fma(A->val[k], x[A->col[k]], s);
    y[i] = s;
  }
}

/* ascending-index dot with fma accumulation */
static double dot(int n, const double *x, const double *y) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s = fma(x[i], y[i], s);
  return s;
}

/* ------------------------------------------------------------------------- */
/* Setup phase (Sec. 4.1 and its setup-pipeline figure): filter, aggregate, inject.                */
/* ------------------------------------------------------------------------- */

/* Strength filter (Sec. 4.1): off-diagonal A_ij is strong unless
   |A_ij| < theta_s * sqrt(|A_ii| |A_jj|); evaluated as mul, sqrt, mul. */
static uint8_t *strength(const orc_csr *A, double theta) {
  uint8_t *S = (uint8_t *)xcalloc((size_t)A->nnz, 1);
  for (int i = 0; i < A->n; ++i) {
    double aii = fabs(diag_of(A, i));
    for (int64_t k = A->ptr[i]; k < A->ptr[i + 1] - 1; ++k) {
      int j = A->col[k];
      double prod = aii * fabs(diag_of(A, j));
      double thr = theta * sqrt(prod);
      S[k] = fabs(A->val[k]) >= thr;
    }
  }
  return S;
}

/* Aggregation (Sec. 4.1, reading: deterministic MIS-2 aggregation).
   Rows without any strong off-diagonal are "left alone": they get no
   aggregate (agg = -1, a zero row of P) and are handled by the smoother only.
   Roots: greedy distance-2 independent set of the strength graph over the
   other rows, visiting them by decreasing priority h64(key(seed_agg, l, i)).
   Aggregate ids are the roots in ascending row order.  Pass 1: strong
   neighbours of a root join it.  Pass 2: every other row with a strong
   neighbour joins the aggregate of the pass-1 member among its strong
   neighbours with the largest |A_ij| (ties: smaller aggregate id, then
   smaller neighbour index): a leftover row goes to the aggregate it is
   most strongly coupled to. */
typedef struct { uint64_t pri; int32_t i; } orc_pri;
static int cmp_pri_desc(const void *a, const void *b) {
  const orc_pri *x = (const orc_pri *)a, *y = (const orc_pri *)b;
  if (x->pri != y->pri) return x->pri < y->pri ? 1 : -1;
  return (x->i < y->i) ? 1 : (x->i > y->i ? -1 : 0);
}

static int aggregate(const orc_csr *A, const uint8_t *S, uint64_t seed, int l,
                     int32_t *agg, uint8_t *root) {
  int n = A->n;
  if (n <= 0) return 0;
  orc_pri *ord = (orc_pri *)xcalloc((size_t)n, sizeof(orc_pri));
  for (int i = 0; i < n; ++i) { ord[i].pri = h64(hkey(seed, l, i)); ord[i].i = i; }
  qsort(ord, (size_t)n, sizeof(orc_pri), cmp_pri_desc);
  uint8_t *blocked = (uint8_t *)xcalloc((size_t)n, 1);
  uint8_t *isolated = (uint8_t *)xcalloc((size_t)n, 1);
  memset(root, 0, (size_t)n);
  for (int i = 0; i < n; ++i) {
    int any = 0;
    for (int64_t k = A->ptr[i]; k < A->ptr[i + 1] - 1; ++k) any |= S[k];
    isolated[i] = !any;
    blocked[i] = isolated[i];
  }
  for (int q = 0; q < n; ++q) {
    int u = ord[q].i;
    if (blocked[u]) continue;
    root[u] = 1;
    blocked[u] = 1;
    for (int64_t k = A->ptr[u]; k < A->ptr[u + 1] - 1; ++k) {
      if (!S[k]) continue;
      int w = A->col[k];
      blocked[w] = 1;
      for (int64_t k2 = A->ptr[w]; k2 < A->ptr[w + 1] - 1; ++k2)
        if (S[k2]) blocked[A->col[k2]] = 1;
    }
  }
  free(blocked); free(ord);
  int na = 0;
  for (int i = 0; i < n; ++i) agg[i] = root[i] ? na++ : -1;
  /* pass 1 */
  int32_t *p1 = (int32_t *)xcalloc((size_t)n, sizeof(int32_t));
  for (int i = 0; i < n; ++i) p1[i] = agg[i];
  for (int i = 0; i < n; ++i) {
    if (!root[i]) continue;
    for (int64_t k = A->ptr[i]; k < A->ptr[i + 1] - 1; ++k)
      if (S[k]) p1[A->col[k]] = agg[i];
  }
  /* pass 2 (reads pass-1 state only) */
  for (int i = 0; i < n; ++i) {
    if (p1[i] >= 0) { agg[i] = p1[i]; continue; }
    if (isolated[i]) { agg[i] = -1; continue; }
    double best = -1.0; int ba = -1, bw = -1;
    for (int64_t k = A->ptr[i]; k < A->ptr[i + 1] - 1; ++k) {
      if (!S[k]) continue;
      int w = A->col[k];
      if (p1[w] < 0) continue;
      double s = fabs(A->val[k]);
      int a = p1[w];
      if (s > best || (s == best && (a < ba || (a == ba && w < bw)))) { best = s; ba = a; bw = w; }
    }
    agg[i] = ba; /* >= 0 by maximality of the distance-2 independent set */
  }
  free(p1);
  for (int i = 0; i < n; ++i)
    if (agg[i] < 0 && !isolated[i]) { free(isolated); return -1; }
  free(isolated);
  return na;
}

/* Near-kernel (Sec. 4.3): sweeps of weighted Jacobi on A x = 0 from
   x0_i = u_i * max|A_ij| (u_i in (0,1) from the counter generator).
   Sweep: s_i = sum over storage order fma(A_ij, x_j, s);
          x_i <- fma(-omega_nk, s_i / A_ii, x_i). */
static void near_kernel_one(const orc_csr *A, const orc_params *p, uint64_t seed, double *B) {
  int n = A->n;
  double amax = 0.0;
  for (int64_t k = 0; k < A->nnz; ++k) if (fabs(A->val[k]) > amax) amax = fabs(A->val[k]);
  for (int i = 0; i < n; ++i) B[i] = u01(h64(hkey(seed, 0, i))) * amax;
  double *s = (double *)xcalloc((size_t)n, sizeof(double));
  for (int sw = 0; sw < p->nk_sweeps; ++sw) {
    spmv(A, B, s);
    ORC_ROWS
    for (int i = 0; i < n; ++i) B[i] = fma(-p->nk_omega, s[i] / diag_of(A, i), B[i]);
  }
  free(s);
}

/* k vectors (Sec. 4.3 repeats the sweeps for each B): vector c starts from
   the generator stream seed_nk + c; B is n x k row-major. */
static void near_kernel(const orc_csr *A, const orc_params *p, double *B) {
  int n = A->n, k = p->nk_vectors;
  if (k == 1) { near_kernel_one(A, p, p->seed_nk, B); return; }
  double *v = (double *)xcalloc((size_t)n, sizeof(double));
  for (int c = 0; c < k; ++c) {
    near_kernel_one(A, p, p->seed_nk + (uint64_t)c, v);
    for (int i = 0; i < n; ++i) B[(size_t)i * k + c] = v[i];
  }
  free(v);
}

/* Injection with k = 1 (Sec. 4.1 setup-pipeline figure): per aggregate a (members
   ascending) nrm_a = sqrt(sum fma(B_i, B_i, .)); P_i = B_i / nrm_a;
   the next level's near-kernel is the R factor, B_{l+1}[a] = nrm_a.
   If nrm_a == 0: P_i = 1/sqrt(|a|). */
#define ORC_QR_DROP 1e-6

static void inject_k(orc_level *L, orc_level *Lc, int k);

static void inject(orc_level *L, orc_level *Lc, int k) {
  if (k > 1) { inject_k(L, Lc, k); return; }
  int n = L->A.n, na = L->n_agg;
  L->mptr = (int64_t *)xcalloc((size_t)na + 1, sizeof(int64_t));
  L->mrow = (int32_t *)xcalloc((size_t)n, sizeof(int32_t));
  for (int i = 0; i < n; ++i) if (L->agg[i] >= 0) L->mptr[L->agg[i] + 1]++;
  for (int a = 0; a < na; ++a) L->mptr[a + 1] += L->mptr[a];
  int64_t *f = (int64_t *)xcalloc((size_t)na, sizeof(int64_t));
  for (int i = 0; i < n; ++i) if (L->agg[i] >= 0) L->mrow[L->mptr[L->agg[i]] + f[L->agg[i]]++] = i;
  free(f);
  L->P = (double *)xcalloc((size_t)n, sizeof(double)); /* 0 on left-alone rows */
  Lc->B = (double *)xcalloc((size_t)na, sizeof(double));
  for (int a = 0; a < na; ++a) {
    double acc = 0.0;
    for (int64_t q = L->mptr[a]; q < L->mptr[a + 1]; ++q) {
      double bi = L->B[L->mrow[q]];
      acc = fma(bi, bi, acc);
    }
    double nrm = sqrt(acc);
    int64_t sz = L->mptr[a + 1] - L->mptr[a];
    for (int64_t q = L->mptr[a]; q < L->mptr[a + 1]; ++q) {
      int i = L->mrow[q];
      L->P[i] = nrm > 0.0 ? L->B[i] / nrm : 1.0 / sqrt((double)sz);
    }
    Lc->B[a] = nrm;
  }
}

static void member_lists(orc_level *L) {
  int n = L->A.n, na = L->n_agg;
  L->mptr = (int64_t *)xcalloc((size_t)na + 1, sizeof(int64_t));
  L->mrow = (int32_t *)xcalloc((size_t)n, sizeof(int32_t));
  for (int i = 0; i < n; ++i) if (L->agg[i] >= 0) L->mptr[L->agg[i] + 1]++;
  for (int a = 0; a < na; ++a) L->mptr[a + 1] += L->mptr[a];
  int64_t *f = (int64_t *)xcalloc((size_t)na, sizeof(int64_t));
  for (int i = 0; i < n; ++i) if (L->agg[i] >= 0) L->mrow[L->mptr[L->agg[i]] + f[L->agg[i]]++] = i;
  free(f);
}

/* Injection with k > 1 (Sec. 4.3, six vectors in the paper; the tentative prolongator of
   smoothed-aggregation AMG): per aggregate a the member rows of B (|a| x k)
   are factored B_a = Q R by modified Gram-Schmidt with one re-orthogonal-
   isation pass (the smoothed near-kernel columns are close to dependent on
   small aggregates), column by column, each sum over the members in
   ascending order with fma:
     v = B_a[:,c]; twice: for d < c: r = q_d . v, R[d][c] += r,
                                     v = v - r q_d  (fma(-r, q_d, v))
     r_cc = |v|; q_c = v / r_cc, or q_c = 0 (a dead column) when
     r_cc <= ORC_QR_DROP * |B_a[:,c]| (B_a numerically rank-deficient).
   P rows of a take Q; the next level's near-kernel rows (a, d) take R[d][:].
   Rows left alone keep zero rows of P. */
static void inject_k(orc_level *L, orc_level *Lc, int k) {
  int n = L->A.n, na = L->n_agg;
  member_lists(L);
  L->P = (double *)xcalloc((size_t)n * k, sizeof(double));
  L->pdead = (uint8_t *)xcalloc((size_t)na * k, 1);
  Lc->B = (double *)xcalloc((size_t)na * k * k, sizeof(double));
  double *v = (double *)xcalloc((size_t)n, sizeof(double)); /* by member position */
  for (int a = 0; a < na; ++a) {
    int64_t q0 = L->mptr[a], q1 = L->mptr[a + 1];
    double *R = Lc->B + (size_t)a * k * k; /* rows (a, d), column c: R[d * k + c] */
    for (int c = 0; c < k; ++c) {
      for (int64_t q = q0; q < q1; ++q) v[q - q0] = L->B[(size_t)L->mrow[q] * k + c];
      for (int pass = 0; pass < 2; ++pass)
        for (int d = 0; d < c; ++d) {
          double r = 0.0;
          for (int64_t q = q0; q < q1; ++q) r = fma(L->P[(size_t)L->mrow[q] * k + d], v[q - q0], r);
          R[d * k + c] = pass ? R[d * k + c] + r : r;
          for (int64_t q = q0; q < q1; ++q)
            v[q - q0] = fma(-r, L->P[(size_t)L->mrow[q] * k + d], v[q - q0]);
        }
      double nb = 0.0, nv = 0.0;
      for (int64_t q = q0; q < q1; ++q) {
        double bq = L->B[(size_t)L->mrow[q] * k + c];
        nb = fma(bq, bq, nb);
        nv = fma(v[q - q0], v[q - q0], nv);
      }
      double nrm = sqrt(nv);
      int live = nv > 0.0 && nrm > ORC_QR_DROP * sqrt(nb);
      for (int64_t q = q0; q < q1; ++q)
        L->P[(size_t)L->mrow[q] * k + c] = live ? v[q - q0] / nrm : 0.0;
      R[c * k + c] = live ? nrm : 0.0;
      L->pdead[(size_t)a * k + c] = (uint8_t)!live;
    }
  }
  free(v);
}

/* Coarse pattern of P^T A P (eq. 6): row a holds every aggregate b reached
   from a member row of a (left-alone columns have P_j = 0 and add nothing);
   off-diagonals ascending, diagonal last. */
static int cmp_i32c(const void *a, const void *b) { return cmp_i32(a, b); }

static void galerkin_pattern(const orc_level *L, orc_csr *Ac) {
  int na = L->n_agg;
  Ac->n = na;
  Ac->ptr = (int64_t *)xcalloc((size_t)na + 1, sizeof(int64_t));
  int32_t *mark = (int32_t *)xcalloc((size_t)na, sizeof(int32_t));
  for (int a = 0; a < na; ++a) mark[a] = -1;
  for (int a = 0; a < na; ++a) {
    int cnt = 0;
    for (int64_t q = L->mptr[a]; q < L->mptr[a + 1]; ++q) {
      int i = L->mrow[q];
      for (int64_t k = L->A.ptr[i]; k < L->A.ptr[i + 1]; ++k) {
        int b = L->agg[L->A.col[k]];
        if (b >= 0 && mark[b] != a) { mark[b] = a; ++cnt; }
      }
    }
    Ac->ptr[a + 1] = Ac->ptr[a] + cnt;
  }
  Ac->nnz = Ac->ptr[na];
  Ac->col = (int32_t *)xcalloc((size_t)Ac->nnz, sizeof(int32_t));
  Ac->val = (double *)xcalloc((size_t)Ac->nnz, sizeof(double));
  for (int a = 0; a < na; ++a) mark[a] = -1;
  for (int a = 0; a < na; ++a) {
    int64_t base = Ac->ptr[a];
    int cnt = 0;
    for (int64_t q = L->mptr[a]; q < L->mptr[a + 1]; ++q) {
      int i = L->mrow[q];
      for (int64_t k = L->A.ptr[i]; k < L->A.ptr[i + 1]; ++k) {
        int b = L->agg[L->A.col[k]];
        if (b >= 0 && b != a && mark[b] != a) { mark[b] = a; Ac->col[base + cnt++] = b; }
      }
    }
    qsort(Ac->col + base, (size_t)cnt, sizeof(int32_t), cmp_i32c);
    Ac->col[base + cnt] = a;
  }
  free(mark);
}

static int64_t find_col(const orc_csr *A, int a, int b) {
  int64_t lo = A->ptr[a], hi = A->ptr[a + 1] - 1; /* off-diagonals [lo, hi) */
  if (b == a) return hi;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (A->col[mid] < b) lo = mid + 1; else hi = mid;
  }
  return (lo < A->ptr[a + 1] - 1 && A->col[lo] == b) ? lo : -1;
}

/* Galerkin values A_{l+1} = P^T A_l P (eq. 6), canonical order:
   entry (a, b) with b >= a sums, over member rows i of a ascending and row
   i's storage order, acc = fma(P_i * A_ij, P_j, acc) for agg[j] == b (rows
   left alone have no aggregate and are skipped); entries with b < a are
   copied from (b, a), so A_{l+1} is exactly symmetric. */
static void galerkin_values(const orc_level *L, orc_csr *Ac) {
  int na = L->n_agg;
  double *acc = (double *)xcalloc((size_t)na, sizeof(double));
  for (int a = 0; a < na; ++a) {
    for (int64_t k = Ac->ptr[a]; k < Ac->ptr[a + 1]; ++k) acc[Ac->col[k]] = 0.0;
    for (int64_t q = L->mptr[a]; q < L->mptr[a + 1]; ++q) {
      int i = L->mrow[q];
      double pi = L->P[i];
      for (int64_t k = L->A.ptr[i]; k < L->A.ptr[i + 1]; ++k) {
        int j = L->A.col[k];
        int b = L->agg[j];
        if (b < a) continue;
        double t = pi * L->A.val[k];
        acc[b] = fma(t, L->P[j], acc[b]);
      }
    }
    for (int64_t k = Ac->ptr[a]; k < Ac->ptr[a + 1]; ++k)
      if (Ac->col[k] >= a) Ac->val[k] = acc[Ac->col[k]];
  }
  for (int a = 0; a < na; ++a)
    for (int64_t k = Ac->ptr[a]; k < Ac->ptr[a + 1] - 1; ++k) {
      int b = Ac->col[k];
      if (b < a) Ac->val[k] = Ac->val[find_col(Ac, b, a)];
    }
  free(acc);
}

/* Coarse pattern with k unknowns per aggregate (Sec. 4.3): aggregate a's
   block list is every aggregate reached from a member row of a, a included,
   ascending; coarse row (a, p) = a*k+p holds the columns b*k+q of those
   blocks in ascending order with its own diagonal moved last. */
static void galerkin_pattern_k(const orc_level *L, orc_csr *Ac, int k) {
  int na = L->n_agg, nc = na * k;
  int32_t *mark = (int32_t *)xcalloc((size_t)na, sizeof(int32_t));
  int32_t *blk = (int32_t *)xcalloc((size_t)na + 1, sizeof(int32_t));
  for (int a = 0; a < na; ++a) mark[a] = -1;
  Ac->n = nc;
  Ac->ptr = (int64_t *)xcalloc((size_t)nc + 1, sizeof(int64_t));
  for (int a = 0; a < na; ++a) {
    int cnt = 0;
    for (int64_t q = L->mptr[a]; q < L->mptr[a + 1]; ++q) {
      int i = L->mrow[q];
      for (int64_t e = L->A.ptr[i]; e < L->A.ptr[i + 1]; ++e) {
        int b = L->agg[L->A.col[e]];
        if (b >= 0 && mark[b] != a) { mark[b] = a; ++cnt; }
      }
    }
    for (int p = 0; p < k; ++p) Ac->ptr[(int64_t)a * k + p + 1] = (int64_t)cnt * k;
  }
  for (int r = 0; r < nc; ++r) Ac->ptr[r + 1] += Ac->ptr[r];
  Ac->nnz = Ac->ptr[nc];
  Ac->col = (int32_t *)xcalloc((size_t)Ac->nnz, sizeof(int32_t));
  Ac->val = (double *)xcalloc((size_t)Ac->nnz, sizeof(double));
  for (int a = 0; a < na; ++a) mark[a] = -1;
  for (int a = 0; a < na; ++a) {
    int cnt = 0;
    for (int64_t q = L->mptr[a]; q < L->mptr[a + 1]; ++q) {
      int i = L->mrow[q];
      for (int64_t e = L->A.ptr[i]; e < L->A.ptr[i + 1]; ++e) {
        int b = L->agg[L->A.col[e]];
        if (b >= 0 && mark[b] != a) { mark[b] = a; blk[cnt++] = b; }
      }
    }
    qsort(blk, (size_t)cnt, sizeof(int32_t), cmp_i32c);
    for (int p = 0; p < k; ++p) {
      int r = a * k + p;
      int64_t w = Ac->ptr[r];
      for (int t = 0; t < cnt; ++t)
        for (int q = 0; q < k; ++q) {
          int c = blk[t] * k + q;
          if (c != r) Ac->col[w++] = c;
        }
      Ac->col[w] = r;
    }
  }
  free(mark); free(blk);
}

/* Galerkin values with k unknowns per aggregate (eq. 6), the canonical
   order of the k = 1 case per entry: entry (r, c) = ((a,p), (b,q)) with
   c >= r sums, over member rows i of a ascending and row i's storage order,
   acc = fma(P_ip * A_ij, P_jq, acc) for agg[j] == b; entries with c < r are
   copied from (c, r).  A dead column (a, p) of P leaves a zero row and
   column; its diagonal is set to 1 so that the coarse matrix stays SPD. */
static void galerkin_values_k(const orc_level *L, orc_csr *Ac, int k) {
  int na = L->n_agg, nc = na * k;
  int32_t *slot = (int32_t *)xcalloc((size_t)na, sizeof(int32_t));
  for (int a = 0; a < na; ++a) slot[a] = -1;
  int maxblk = 0;
  for (int a = 0; a < na; ++a) {
    int len = (int)(Ac->ptr[a * k + 1] - Ac->ptr[a * k]) / k;
    if (len > maxblk) maxblk = len;
  }
  double *acc = (double *)xcalloc((size_t)k * maxblk * k, sizeof(double));
  int32_t *blk = (int32_t *)xcalloc((size_t)maxblk, sizeof(int32_t));
  for (int a = 0; a < na; ++a) {
    /* block list of a from row (a, 0): its columns in blocks of k, with
       (a, 0) moved last */
    int r0 = a * k, nb = 0;
    for (int64_t e = Ac->ptr[r0]; e < Ac->ptr[r0 + 1]; ++e) {
      int b = Ac->col[e] / k;
      if (slot[b] != -2 - a) { slot[b] = -2 - a; blk[nb++] = b; }
    }
    qsort(blk, (size_t)nb, sizeof(int32_t), cmp_i32c);
    for (int t = 0; t < nb; ++t) slot[blk[t]] = t;
    memset(acc, 0, sizeof(double) * (size_t)k * nb * k);
    for (int64_t q = L->mptr[a]; q < L->mptr[a + 1]; ++q) {
      int i = L->mrow[q];
      for (int64_t e = L->A.ptr[i]; e < L->A.ptr[i + 1]; ++e) {
        int j = L->A.col[e];
        int b = L->agg[j];
        if (b < a) continue;
        int sb = slot[b];
        for (int p = 0; p < k; ++p) {
          double t = L->P[(size_t)i * k + p] * L->A.val[e];
          for (int qq = (b == a ? p : 0); qq < k; ++qq) {
            double *cell = acc + (size_t)p * nb * k + (size_t)sb * k + qq;
            *cell = fma(t, L->P[(size_t)j * k + qq], *cell);
          }
        }
      }
    }
    for (int p = 0; p < k; ++p) {
      int r = a * k + p;
      for (int64_t e = Ac->ptr[r]; e < Ac->ptr[r + 1]; ++e) {
        int c = Ac->col[e];
        if (c >= r) Ac->val[e] = acc[(size_t)p * nb * k + (size_t)slot[c / k] * k + c % k];
      }
    }
    for (int t = 0; t < nb; ++t) slot[blk[t]] = -1;
  }
  for (int r = 0; r < nc; ++r)
    for (int64_t e = Ac->ptr[r]; e < Ac->ptr[r + 1] - 1; ++e) {
      int c = Ac->col[e];
      if (c < r) Ac->val[e] = Ac->val[find_col(Ac, c, r)];
    }
  for (int r = 0; r < nc; ++r)
    if (L->pdead[r]) Ac->val[Ac->ptr[r + 1] - 1] = 1.0;
  free(acc); free(blk); free(slot);
}

/* Multicolour ordering (Sec. 4.5, "parallel GS"): greedy colouring in
   decreasing priority h64(key(seed_col, l, i)); each row takes the smallest
   colour absent among its already-coloured (higher-priority) neighbours.  This
   is what Jones-Plassmann rounds produce. */
static int colour(const orc_csr *A, uint64_t seed, int l, int32_t *color) {
  int n = A->n, nc = 0;
  orc_pri *ord = (orc_pri *)xcalloc((size_t)n, sizeof(orc_pri));
  for (int i = 0; i < n; ++i) { ord[i].pri = h64(hkey(seed, l, i)); ord[i].i = i; color[i] = -1; }
  qsort(ord, (size_t)n, sizeof(orc_pri), cmp_pri_desc);
  int cap = 64;
  uint8_t *used = (uint8_t *)xcalloc((size_t)cap, 1);
  for (int q = 0; q < n; ++q) {
    int u = ord[q].i;
    int deg = (int)(A->ptr[u + 1] - A->ptr[u]);
    if (deg + 1 > cap) { free(used); cap = 2 * (deg + 1); used = (uint8_t *)xcalloc((size_t)cap, 1); }
    memset(used, 0, (size_t)cap);
    for (int64_t k = A->ptr[u]; k < A->ptr[u + 1] - 1; ++k) {
      int c = color[A->col[k]];
      if (c >= 0 && c < cap) used[c] = 1;
    }
    int c = 0;
    while (used[c]) ++c;
    color[u] = c;
    if (c + 1 > nc) nc = c + 1;
  }
  free(used); free(ord);
  return nc;
}

/* Power method for lambda_max(D^-1 A) (Sec. 4.5): y0_i = u(seed_pow, l, i);
   repeat: z = D^-1 A y, lambda = |z|/|y|, y = z/|z|.  omega is
   2 / (safety * lambda + lambda_min_est). */
static double power_lmax(const orc_csr *A, const orc_params *p, int l) {
  int n = A->n;
  double *y = (double *)xcalloc((size_t)n, sizeof(double));
  double *z = (double *)xcalloc((size_t)n, sizeof(double));
  for (int i = 0; i < n; ++i) y[i] = u01(h64(hkey(p->seed_pow, l, i)));
  double lam = 0.0;
  for (int it = 0; it < p->power_iters; ++it) {
    spmv(A, y, z);
    ORC_ROWS
    for (int i = 0; i < n; ++i) z[i] = z[i] / diag_of(A, i);
    double nz = sqrt(dot(n, z, z)), ny = sqrt(dot(n, y, y));
    lam = nz / ny;
    if (!(nz > 0.0)) break;
    ORC_ROWS
    for (int i = 0; i < n; ++i) y[i] = z[i] / nz;
  }
  free(y); free(z);
  return lam;
}

/* Coarsest solve (reading: the paper only fixes its size): dense Cholesky
   A = L L^T, column by column; fails if a pivot is not positive. */
static int cholesky(orc *o) {
  const orc_csr *A = &o->lev[o->L - 1].A;
  int n = A->n;
  if (o->chol_n != n) { free(o->chol); o->chol = (double *)xcalloc((size_t)n * n, sizeof(double)); o->chol_n = n; }
  double *Lm = o->chol;
  memset(Lm, 0, sizeof(double) * (size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int64_t k = A->ptr[i]; k < A->ptr[i + 1]; ++k) Lm[(size_t)i * n + A->col[k]] = A->val[k];
  for (int j = 0; j < n; ++j) {
    double d = Lm[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) d = fma(-Lm[(size_t)j * n + k], Lm[(size_t)j * n + k], d);
    if (!(d > 0.0)) return ORC_E_SINGULAR;
    double ljj = sqrt(d);
    Lm[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double s = Lm[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) s = fma(-Lm[(size_t)i * n + k], Lm[(size_t)j * n + k], s);
      Lm[(size_t)i * n + j] = s / ljj;
    }
    for (int i = 0; i < j; ++i) Lm[(size_t)i * n + j] = 0.0;
  }
  return ORC_OK;
}

static void chol_solve(const orc *o, const double *b, double *x) {
  int n = o->chol_n;
  const double *Lm = o->chol;
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s = fma(-Lm[(size_t)i * n + k], x[k], s);
    x[i] = s / Lm[(size_t)i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = x[i];
    for (int k = i + 1; k < n; ++k) s = fma(-Lm[(size_t)k * n + i], x[k], s);
    x[i] = s / Lm[(size_t)i * n + i];
  }
}

static void level_alloc_work(orc_level *L) {
  int n = L->A.n;
  L->x = (double *)xcalloc((size_t)n, sizeof(double));
  L->b = (double *)xcalloc((size_t)n, sizeof(double));
  L->r = (double *)xcalloc((size_t)n, sizeof(double));
  L->t = (double *)xcalloc((size_t)n, sizeof(double));
}

/* Node matrix of a coarse level with k unknowns per node (k > 1): node a
   holds rows a*k .. a*k+k-1; its row lists the nodes its rows reach (off-
   diagonals ascending, itself last) with the Frobenius norm of each k x k
   block, |A_ab|_F = sqrt(sum over rows p ascending and their storage order
   of fma(v, v, .)).  Aggregating nodes keeps a node's k unknowns together
   (smoothed-aggregation practice for several near-kernel vectors). */
static void node_matrix(const orc_csr *A, int k, orc_csr *N) {
  int nn = A->n / k;
  N->n = nn;
  N->ptr = (int64_t *)xcalloc((size_t)nn + 1, sizeof(int64_t));
  int32_t *mark = (int32_t *)xcalloc((size_t)nn, sizeof(int32_t));
  int32_t *slot = (int32_t *)xcalloc((size_t)nn, sizeof(int32_t));
  for (int a = 0; a < nn; ++a) mark[a] = -1;
  for (int a = 0; a < nn; ++a) {
    int cnt = 0;
    for (int p = 0; p < k; ++p)
      for (int64_t e = A->ptr[a * k + p]; e < A->ptr[a * k + p + 1]; ++e) {
        int b = A->col[e] / k;
        if (mark[b] != a) { mark[b] = a; ++cnt; }
      }
    N->ptr[a + 1] = N->ptr[a] + cnt;
  }
  N->nnz = N->ptr[nn];
  N->col = (int32_t *)xcalloc((size_t)N->nnz, sizeof(int32_t));
  N->val = (double *)xcalloc((size_t)N->nnz, sizeof(double));
  for (int a = 0; a < nn; ++a) mark[a] = -1;
  for (int a = 0; a < nn; ++a) {
    int64_t base = N->ptr[a];
    int cnt = 0;
    for (int p = 0; p < k; ++p)
      for (int64_t e = A->ptr[a * k + p]; e < A->ptr[a * k + p + 1]; ++e) {
        int b = A->col[e] / k;
        if (b != a && mark[b] != a) { mark[b] = a; N->col[base + cnt++] = b; }
      }
    qsort(N->col + base, (size_t)cnt, sizeof(int32_t), cmp_i32c);
    N->col[base + cnt] = a;
    for (int t = 0; t <= cnt; ++t) slot[N->col[base + t]] = t;
    for (int p = 0; p < k; ++p)
      for (int64_t e = A->ptr[a * k + p]; e < A->ptr[a * k + p + 1]; ++e) {
        double v = A->val[e];
        double *c = N->val + base + slot[A->col[e] / k];
        *c = fma(v, v, *c);
      }
    for (int t = 0; t <= cnt; ++t) N->val[base + t] = sqrt(N->val[base + t]);
  }
  free(mark); free(slot);
}

/* Full setup from the current level-0 matrix (Sec. 4.1, setup-pipeline figure): level 0 takes the
   near-kernel sweeps; each level filters, aggregates, injects and forms the
   next Galerkin operator, until the size is below coarse_max or max_levels is
   reached.  Smoother weights (and colourings) are set lazily here too. */
static int setup(orc *o) {
  for (int l = 1; l < ORC_MAXL; ++l) level_free(&o->lev[l]);
  orc_level *L0 = &o->lev[0];
  free(L0->agg); free(L0->root); free(L0->B); free(L0->P); free(L0->pdead); free(L0->mptr); free(L0->mrow);
  free(L0->color);
  L0->agg = NULL; L0->root = NULL; L0->B = NULL; L0->P = NULL; L0->pdead = NULL; L0->mptr = NULL;
  L0->mrow = NULL; L0->color = NULL;
  L0->B = (double *)xcalloc((size_t)o->m * o->p.nk_vectors, sizeof(double));
  near_kernel(&L0->A, &o->p, L0->B);
  int l = 0;
  for (;;) {
    orc_level *L = &o->lev[l];
    int n = L->A.n;
    if (!L->x) level_alloc_work(L);
    if (n < o->p.coarse_max || l == o->p.max_levels - 1 || l == ORC_MAXL - 1) break;
    L->agg = (int32_t *)xcalloc((size_t)n, sizeof(int32_t));
    L->root = (uint8_t *)xcalloc((size_t)n, 1);
    const int k = o->p.nk_vectors;
    int na, units = n;
    if (k > 1 && l > 0) {
      /* coarse levels with k unknowns per node aggregate whole nodes */
      orc_csr N;
      memset(&N, 0, sizeof(N));
      node_matrix(&L->A, k, &N);
      units = N.n;
      uint8_t *S = strength(&N, o->p.theta_s);
      int32_t *nagg = (int32_t *)xcalloc((size_t)N.n, sizeof(int32_t));
      uint8_t *nroot = (uint8_t *)xcalloc((size_t)N.n, 1);
      na = aggregate(&N, S, o->p.seed_agg, l, nagg, nroot);
      for (int i = 0; i < n; ++i) { L->agg[i] = nagg[i / k]; L->root[i] = nroot[i / k]; }
      free(S); free(nagg); free(nroot); csr_free(&N);
    } else {
      uint8_t *S = strength(&L->A, o->p.theta_s);
      na = aggregate(&L->A, S, o->p.seed_agg, l, L->agg, L->root);
      free(S);
    }
    if (na < 0) return ORC_E_SETUP;
    if (na == 0 || na == units) { /* nothing to coarsen: stop here */
      free(L->agg); free(L->root); L->agg = NULL; L->root = NULL;
      break;
    }
    L->n_agg = na;
    orc_level *Lc = &o->lev[l + 1];
    inject(L, Lc, o->p.nk_vectors);
    if (o->p.nk_vectors > 1) {
      galerkin_pattern_k(L, &Lc->A, o->p.nk_vectors);
      galerkin_values_k(L, &Lc->A, o->p.nk_vectors);
    } else {
      galerkin_pattern(L, &Lc->A);
      galerkin_values(L, &Lc->A);
    }
    ++l;
  }
  o->L = l + 1;
  if (o->lev[o->L - 1].A.n > 4096) return ORC_E_SETUP;
  for (int q = 0; q + 1 < o->L; ++q) {
    orc_level *L = &o->lev[q];
    L->lmax = power_lmax(&L->A, &o->p, q);
    L->omega = 2.0 / (o->p.power_safety * L->lmax + o->p.lambda_min_est);
    free(L->color);
    L->color = (int32_t *)xcalloc((size_t)L->A.n, sizeof(int32_t));
    L->n_colors = colour(&L->A, o->p.seed_col, q, L->color);
  }
  o->have_setup = 1;
  o->n_setups++;
  return ORC_OK;
}

/* Galerkin re-form on reuse (Sec. 4.4): P kept, values recomputed. */
static void reform(orc *o) {
  for (int l = 0; l + 1 < o->L; ++l) {
    if (o->p.nk_vectors > 1) galerkin_values_k(&o->lev[l], &o->lev[l + 1].A, o->p.nk_vectors);
    else galerkin_values(&o->lev[l], &o->lev[l + 1].A);
  }
}

/* ------------------------------------------------------------------------- */
/* Smoothers and V-cycle (Sec. 4.4-4.5)                                      */
/* ------------------------------------------------------------------------- */

/* weighted Jacobi: x_i <- fma(omega, (b_i - s_i)/A_ii, x_i), s = A x */
static void jacobi(const orc_level *L, double *x, const double *b, double *t) {
  spmv(&L->A, x, t);
  ORC_ROWS
  for (int i = 0; i < L->A.n; ++i) x[i] = fma(L->omega, (b[i] - t[i]) / diag_of(&L->A, i), x[i]);
}

/* Gauss-Seidel over one colour class, in place */
static void gs_colour(const orc_level *L, double *x, const double *b, int c) {
  const orc_csr *A = &L->A;
  for (int i = 0; i < A->n; ++i) {
    if (L->color[i] != c) continue;
    double s = 0.0;
    for (int64_t k = A->ptr[i]; k < A->ptr[i + 1]; ++k) s = fma(A->val[k], x[A->col[k]], s);
    x[i] = x[i] + (b[i] - s) / diag_of(A, i);
  }
}

/* Chebyshev smoother (Sec. 4.5): the Chebyshev iteration on D^-1 A x = D^-1 b
   over the eigenvalue interval [lo, hi] = [lambda_min_est, safety * lambda_max]
   (the interval of the omega-Jacobi formula, whose weight 2/(lo+hi) is the
   degree-1 case), with smooth_sweeps products:
     theta = (hi+lo)/2, delta = (hi-lo)/2, sigma = theta/delta, rho = 1/sigma
     r = D^-1 (b - A x), d = r/theta
     repeat: x += d; r -= D^-1 A d; rho' = 1/(2 sigma - rho);
             d = rho' rho d + (2 rho'/delta) r; rho = rho'
   A polynomial in D^-1 A, so identical pre and post smoothing keeps the
   V-cycle symmetric. */
static void chebyshev(const orc *o, const orc_level *L, double *x, const double *b, double *t) {
  int n = L->A.n;
  double lo = o->p.lambda_min_est, hi = o->p.power_safety * L->lmax;
  double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo);
  double sigma = theta / delta, rho = 1.0 / sigma;
  double *r = (double *)xcalloc((size_t)n, sizeof(double));
  double *d = (double *)xcalloc((size_t)n, sizeof(double));
  spmv(&L->A, x, t);
  ORC_ROWS
  for (int i = 0; i < n; ++i) {
    r[i] = (b[i] - t[i]) / diag_of(&L->A, i);
    d[i] = r[i] / theta;
  }
  for (int k = 0; k < o->p.smooth_sweeps; ++k) {
    ORC_ROWS
    for (int i = 0; i < n; ++i) x[i] = x[i] + d[i];
    if (k + 1 == o->p.smooth_sweeps) break;
    spmv(&L->A, d, t);
    ORC_ROWS
    for (int i = 0; i < n; ++i) r[i] = r[i] - t[i] / diag_of(&L->A, i);
    double rho2 = 1.0 / (2.0 * sigma - rho);
    double c1 = rho2 * rho, c2 = 2.0 * rho2 / delta;
    ORC_ROWS
    for (int i = 0; i < n; ++i) d[i] = fma(c1, d[i], c2 * r[i]);
    rho = rho2;
  }
  free(r);
  free(d);
}

static void smooth(const orc *o, const orc_level *L, double *x, const double *b, double *t, int post) {
  if (o->p.smoother == 2) {
    chebyshev(o, L, x, b, t);
    return;
  }
  for (int s = 0; s < o->p.smooth_sweeps; ++s) {
    if (o->p.smoother == 1) {
      if (!post) for (int c = 0; c < L->n_colors; ++c) gs_colour(L, x, b, c);
      else for (int c = L->n_colors - 1; c >= 0; --c) gs_colour(L, x, b, c);
    } else {
      jacobi(L, x, b, t);
    }
  }
}

/* One V-cycle z = V(r) from a zero start: pre-smooth, residual, restrict
   b_{l+1,a} = sum_{i in a} fma(P_i, r_i, .), recurse, prolong
   x_i = fma(P_i, x_{l+1}[agg_i], x_i), post-smooth; Cholesky on the coarsest. */
static void vcycle_level(orc *o, int l) {
  orc_level *L = &o->lev[l];
  int n = L->A.n;
  if (l == o->L - 1) { chol_solve(o, L->b, L->x); return; }
  memset(L->x, 0, sizeof(double) * (size_t)n);
  smooth(o, L, L->x, L->b, L->t, 0);
  spmv(&L->A, L->x, L->t);
  ORC_ROWS
  for (int i = 0; i < n; ++i) L->r[i] = L->b[i] - L->t[i];
  orc_level *Lc = &o->lev[l + 1];
  const int k = o->p.nk_vectors;
  ORC_ROWS
  for (int a = 0; a < L->n_agg; ++a)
    for (int c = 0; c < k; ++c) {
      double acc = 0.0;
      for (int64_t q = L->mptr[a]; q < L->mptr[a + 1]; ++q) {
        int i = L->mrow[q];
        acc = fma(L->P[(size_t)i * k + c], L->r[i], acc);
      }
      Lc->b[a * k + c] = acc;
    }
  vcycle_level(o, l + 1);
  ORC_ROWS
  for (int i = 0; i < n; ++i)
    if (L->agg[i] >= 0)
      for (int c = 0; c < k; ++c)
        L->x[i] = fma(L->P[(size_t)i * k + c], Lc->x[L->agg[i] * k + c], L->x[i]);
  smooth(o, L, L->x, L->b, L->t, 1);
}

static void vcycle(orc *o, const double *r, double *z) {
  memcpy(o->lev[0].b, r, sizeof(double) * (size_t)o->m);
  vcycle_level(o, 0);
  memcpy(z, o->lev[0].x, sizeof(double) * (size_t)o->m);
}

/* MGPCG (Sec. 4.4): PCG from a zero start, one V-cycle per iteration, stop
   when |r|_2 <= rtol |b|_2 (recursive residual); then one FP64 true residual. */
static int pcg(orc *o, const double *b, double *x, orc_solve_info *info) {
  int n = o->m;
  const orc_csr *A = &o->lev[0].A;
  double *r = o->pr, *z = o->pz, *p = o->pp, *q = o->pq;
  memset(info, 0, sizeof(*info));
  memset(x, 0, sizeof(double) * (size_t)n);
  double bnorm = sqrt(dot(n, b, b));
  info->bnorm = bnorm;
  if (bnorm == 0.0) { info->status = ORC_OK; return ORC_OK; }
  memcpy(r, b, sizeof(double) * (size_t)n);
  vcycle(o, r, z);
  memcpy(p, z, sizeof(double) * (size_t)n);
  double rz = dot(n, r, z);
  int status = ORC_W_NOT_CONVERGED, k;
  double rr = bnorm * bnorm;
  for (k = 1; k <= o->p.pcg_maxiter; ++k) {
    spmv(A, p, q);
    double pq = dot(n, p, q);
    if (!(pq > 0.0) || !(rz > 0.0)) { status = ORC_E_BREAKDOWN; break; }
    double al = rz / pq;
    ORC_ROWS
    for (int i = 0; i < n; ++i) { x[i] = fma(al, p[i], x[i]); r[i] = fma(-al, q[i], r[i]); }
    rr = dot(n, r, r);
    if (sqrt(rr) <= o->p.pcg_rtol * bnorm) { status = ORC_OK; break; }
    vcycle(o, r, z);
    double rz2 = dot(n, r, z);
    double be = rz2 / rz;
    rz = rz2;
    ORC_ROWS
    for (int i = 0; i < n; ++i) p[i] = fma(be, p[i], z[i]);
  }
  info->pcg_iters = k > o->p.pcg_maxiter ? o->p.pcg_maxiter : k;
  info->rel_res = sqrt(rr) / bnorm;
  spmv(A, x, q);
  ORC_ROWS
  for (int i = 0; i < n; ++i) q[i] = b[i] - q[i];
  info->true_rel_res = sqrt(dot(n, q, q)) / bnorm;
  info->status = status;
  return status;
}

/* ------------------------------------------------------------------------- */
/* Integrator (Alg. 1)                                                       */
/* ------------------------------------------------------------------------- */

/* semi-implicit Euler (Alg. 1 first line): free vertices v += dt g,
   x_old = x, x += dt v; pinned vertices (w = 0) keep v = 0 and x.
   Then lambda = 0. */
void orc_begin_frame(orc *o) {
  for (int v = 0; v < o->N; ++v) {
    double *x = o->x + 3 * (int64_t)v, *vel = o->v + 3 * (int64_t)v, *xo = o->xold + 3 * (int64_t)v;
    for (int k = 0; k < 3; ++k) xo[k] = x[k];
    if (o->w[v] == 0.0) { vel[0] = vel[1] = vel[2] = 0.0; continue; }
    for (int k = 0; k < 3; ++k) {
      double t = o->p.dt * o->p.gravity[k];
      vel[k] = vel[k] + t;
      double t2 = o->p.dt * vel[k];
      x[k] = x[k] + t2;
    }
  }
  memset(o->lambda, 0, sizeof(double) * (size_t)o->m);
}

/* v = (x - x_old) / dt (Alg. 1 last line) */
void orc_end_frame(orc *o) {
  for (int64_t q = 0; q < 3 * (int64_t)o->N; ++q) o->v[q] = (o->x[q] - o->xold[q]) / o->p.dt;
}

/* eq. 5: dx_v = w_v * sum_{j incident to v, ascending} fma(g_{j,v}, dl_j, .) */
static void position_correction(orc *o) {
  int32_t vv[4];
  for (int v = 0; v < o->N; ++v) {
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t q = o->vptr[v]; q < o->vptr[v + 1]; ++q) {
      int j = o->vrow[q];
      int c = row_verts(o, j, vv), s = 0;
      while (s < c && vv[s] != v) ++s;
      double g[3];
      row_grad(o, j, s, g);
      for (int k = 0; k < 3; ++k) acc[k] = fma(g[k], o->dl[j], acc[k]);
    }
    for (int k = 0; k < 3; ++k) o->dx[3 * (int64_t)v + k] = o->w[v] * acc[k];
  }
}

/* Alg. 1 update: lambda += dl; x = fma(omega, dx, x).  With backtracking
   (Sec. 4: omega "halves when the residual increases") the step starts at
   omega_x and halves while the dual residual |b| = |-C - alpha~ lambda| at
   the new x and lambda is not below the current one, at most `backtrack`
   times; the last trial is kept. */
static void update_positions(orc *o, orc_solve_info *info) {
  position_correction(o);
  for (int j = 0; j < o->m; ++j) o->lambda[j] = o->lambda[j] + o->dl[j];
  int64_t n3 = 3 * (int64_t)o->N;
  double om = o->p.omega_x;
  if (o->p.backtrack <= 0) {
    for (int64_t q = 0; q < n3; ++q) o->x[q] = fma(om, o->dx[q], o->x[q]);
    info->omega = om;
    info->bnorm_after = -1.0;
    return;
  }
  memcpy(o->xbak, o->x, sizeof(double) * (size_t)n3);
  double nb = 0.0;
  for (int t = 0; t <= o->p.backtrack; ++t) {
    for (int64_t q = 0; q < n3; ++q) o->x[q] = fma(om, o->dx[q], o->xbak[q]);
    eval_constraints(o);
    nb = sqrt(dot(o->m, o->b, o->b));
    if (nb < info->bnorm || t == o->p.backtrack) break;
    om = om * 0.5;
  }
  info->omega = om;
  info->bnorm_after = nb;
}

/* C, gradients, A and b at the current positions */
void orc_eval_assemble(orc *o) {
  eval_constraints(o);
  assemble(o);
}

int orc_setup(orc *o) { return setup(o); }

/* Galerkin re-form plus coarsest factorisation for the current A */
int orc_prepare_solve(orc *o) {
  if (!o->have_setup) { int s = setup(o); if (s) return s; }
  else reform(o);
  return cholesky(o);
}

/* One global iteration (Alg. 1 loop body).  Returns 1 if the loop should
   stop (|b| < eps_b), 0 to go on, < 0 on error. */
/* XPBD's local solve (eq. 4): every constraint takes dl_j = b_j / A_jj from
   the same state (the Jacobi form the paper compares against). */
static int xpbd_step(orc *o, orc_solve_info *info) {
  memset(info, 0, sizeof(*info));
  info->bnorm = sqrt(dot(o->m, o->b, o->b));
  for (int j = 0; j < o->m; ++j) o->dl[j] = o->b[j] / diag_of(&o->A, j);
  info->pcg_iters = 1;
  info->status = ORC_OK;
  return ORC_OK;
}

int orc_iterate(orc *o, orc_solve_info *info) {
  eval_constraints(o);
  assemble(o);
  int st;
  if (o->p.linear_solver == 1) {
    xpbd_step(o, info);
    o->it_global++;
    update_positions(o, info);
    o->last = *info;
    return info->bnorm < o->p.eps_b ? 1 : 0;
  }
  int fresh = 0;
  if (!o->have_setup || (o->p.setup_interval > 0 && o->it_global % o->p.setup_interval == 0)) {
    st = setup(o);
    if (st) return st;
    fresh = 1;
  } else {
    reform(o);
  }
  st = cholesky(o);
  if (st) return st;
  st = pcg(o, o->b, o->dl, info);
  /* Reading of the lazy setup (Sec. 4.2, 4.5): P and omega are reused while
     they still fit A.  A breakdown on a reused hierarchy (omega or P built for
     an A that has since changed, e.g. ARAP rows leaving the rest state) sets
     up afresh for the current A and solves once more. */
  if (st == ORC_E_BREAKDOWN && !fresh) {
    st = setup(o);
    if (st) return st;
    st = cholesky(o);
    if (st) return st;
    st = pcg(o, o->b, o->dl, info);
  }
  o->it_global++;
  if (st < 0) { o->last = *info; return st; }
  update_positions(o, info);
  o->last = *info;
  double bn = info->bnorm;
  return bn < o->p.eps_b ? 1 : 0;
}

int orc_step(orc *o, int n_frames, orc_solve_info *hist /* n_frames*max_iter or NULL */) {
  for (int f = 0; f < n_frames; ++f) {
    orc_begin_frame(o);
    for (int it = 0; it < o->p.max_iter; ++it) {
      orc_solve_info inf;
      int st = orc_iterate(o, &inf);
      if (hist) hist[(int64_t)f * o->p.max_iter + it] = inf;
      if (st < 0) return st;
      if (st == 1) break;
    }
    orc_end_frame(o);
  }
  return ORC_OK;
}

/* PCG on the current hierarchy for a caller-given right-hand side */
int orc_solve(orc *o, const double *b, double *x, orc_solve_info *info) {
  return pcg(o, b, x, info);
}

void orc_vcycle(orc *o, const double *r, double *z) { vcycle(o, r, z); }

/* ------------------------------------------------------------------------- */
/* create / destroy / state / getters                                        */
/* ------------------------------------------------------------------------- */
void orc_destroy(orc *o) {
  if (!o) return;
  free(o->rest); free(o->w); free(o->alpha); free(o->alpha_t); free(o->L0); free(o->V0); free(o->Dminv);
  free(o->edge); free(o->tet); free(o->x); free(o->v); free(o->xold); free(o->lambda);
  free(o->C); free(o->b); free(o->gd); free(o->gt); free(o->dl); free(o->dx); free(o->xbak);
  csr_free(&o->A);
  o->lev[0].A.ptr = NULL; o->lev[0].A.col = NULL; o->lev[0].A.val = NULL;
  for (int l = 0; l < ORC_MAXL; ++l) level_free(&o->lev[l]);
  free(o->map); free(o->vptr); free(o->vrow); free(o->chol);
  free(o->pr); free(o->pz); free(o->pp); free(o->pq);
  free(o);
}

orc *orc_create(int N, const double *rest, const double *inv_mass, int E, const int32_t *edge,
                int T, const int32_t *tet, int tet_kind, const double *alpha, const orc_params *p,
                int *status) {
  *status = ORC_E_INVALID;
  if (N <= 0 || E < 0 || T < 0 || !p || p->dt <= 0.0 || tet_kind < 0 || tet_kind > 1 ||
      p->nk_vectors < 1 || p->nk_vectors > 8) return NULL;
  for (int j = 0; j < 2 * E; ++j) if (edge[j] < 0 || edge[j] >= N) return NULL;
  for (int64_t j = 0; j < 4 * (int64_t)T; ++j) if (tet[j] < 0 || tet[j] >= N) return NULL;
  orc *o = (orc *)xcalloc(1, sizeof(orc));
  o->N = N; o->E = E; o->T = T; o->m = E + T; o->p = *p; o->tet_kind = tet_kind;
  int m = o->m;
  o->rest = (double *)xcalloc(3 * (size_t)N, sizeof(double));
  o->w = (double *)xcalloc((size_t)N, sizeof(double));
  o->edge = (int32_t *)xcalloc(2 * (size_t)E, sizeof(int32_t));
  o->tet = (int32_t *)xcalloc(4 * (size_t)T, sizeof(int32_t));
  o->alpha = (double *)xcalloc((size_t)m, sizeof(double));
  o->alpha_t = (double *)xcalloc((size_t)m, sizeof(double));
  o->L0 = (double *)xcalloc((size_t)E, sizeof(double));
  o->V0 = (double *)xcalloc((size_t)T, sizeof(double));
  o->Dminv = (double *)xcalloc(9 * (size_t)T + 1, sizeof(double));
  o->x = (double *)xcalloc(3 * (size_t)N, sizeof(double));
  o->v = (double *)xcalloc(3 * (size_t)N, sizeof(double));
  o->xold = (double *)xcalloc(3 * (size_t)N, sizeof(double));
  o->lambda = (double *)xcalloc((size_t)m, sizeof(double));
  o->C = (double *)xcalloc((size_t)m, sizeof(double));
  o->b = (double *)xcalloc((size_t)m, sizeof(double));
  o->dl = (double *)xcalloc((size_t)m, sizeof(double));
  o->dx = (double *)xcalloc(3 * (size_t)N, sizeof(double));
  o->xbak = (double *)xcalloc(3 * (size_t)N, sizeof(double));
  o->gd = (double *)xcalloc(3 * (size_t)E, sizeof(double));
  o->gt = (double *)xcalloc(12 * (size_t)T, sizeof(double));
  o->pr = (double *)xcalloc((size_t)m, sizeof(double));
  o->pz = (double *)xcalloc((size_t)m, sizeof(double));
  o->pp = (double *)xcalloc((size_t)m, sizeof(double));
  o->pq = (double *)xcalloc((size_t)m, sizeof(double));
  memcpy(o->rest, rest, sizeof(double) * 3 * (size_t)N);
  memcpy(o->x, rest, sizeof(double) * 3 * (size_t)N);
  memcpy(o->w, inv_mass, sizeof(double) * (size_t)N);
  if (E) memcpy(o->edge, edge, sizeof(int32_t) * 2 * (size_t)E);
  if (T) memcpy(o->tet, tet, sizeof(int32_t) * 4 * (size_t)T);
  memcpy(o->alpha, alpha, sizeof(double) * (size_t)m);
  /* alpha~ = alpha / dt^2 (eq. 2) */
  double dt2 = p->dt * p->dt;
  for (int j = 0; j < m; ++j) o->alpha_t[j] = alpha[j] / dt2;
  /* rest lengths and rest volumes from the rest shape */
  double n3[3], g12[12];
  for (int j = 0; j < E; ++j)
    o->L0[j] = dist_eval(rest + 3 * (int64_t)edge[2 * j], rest + 3 * (int64_t)edge[2 * j + 1], 0.0, n3);
  for (int t = 0; t < T; ++t) {
    const int32_t *tv = tet + 4 * (int64_t)t;
    o->V0[t] = tet_eval(rest + 3 * (int64_t)tv[0], rest + 3 * (int64_t)tv[1], rest + 3 * (int64_t)tv[2],
                        rest + 3 * (int64_t)tv[3], 0.0, g12);
    arap_rest(rest + 3 * (int64_t)tv[0], rest + 3 * (int64_t)tv[1], rest + 3 * (int64_t)tv[2],
              rest + 3 * (int64_t)tv[3], o->Dminv + 9 * (int64_t)t);
  }
  int st = build_pattern(o);
  if (st) { orc_destroy(o); *status = st; return NULL; }
  o->lev[0].A = o->A; /* level 0 aliases the assembled matrix */
  level_alloc_work(&o->lev[0]);
  *status = ORC_OK;
  return o;
}

void orc_set_state(orc *o, const double *x, const double *v) {
  if (x) memcpy(o->x, x, sizeof(double) * 3 * (size_t)o->N);
  if (v) memcpy(o->v, v, sizeof(double) * 3 * (size_t)o->N);
}
void orc_get_state(const orc *o, double *x, double *v) {
  if (x) memcpy(x, o->x, sizeof(double) * 3 * (size_t)o->N);
  if (v) memcpy(v, o->v, sizeof(double) * 3 * (size_t)o->N);
}
int64_t orc_nnz(const orc *o, int l) { return (l < o->L || l == 0) ? o->lev[l].A.nnz : -1; }
int orc_rows(const orc *o, int l) { return (l < o->L || l == 0) ? o->lev[l].A.n : -1; }
int orc_levels(const orc *o) { return o->L; }
int orc_n_setups(const orc *o) { return o->n_setups; }
void orc_matrix(const orc *o, int l, int64_t *ptr, int32_t *col, double *val) {
  const orc_csr *A = &o->lev[l].A;
  if (ptr) memcpy(ptr, A->ptr, sizeof(int64_t) * ((size_t)A->n + 1));
  if (col) memcpy(col, A->col, sizeof(int32_t) * (size_t)A->nnz);
  if (val) memcpy(val, A->val, sizeof(double) * (size_t)A->nnz);
}
void orc_map(const orc *o, uint16_t *map) { memcpy(map, o->map, sizeof(uint16_t) * (size_t)o->A.nnz); }
void orc_incidence(const orc *o, int64_t *vptr, int32_t *vrow) {
  memcpy(vptr, o->vptr, sizeof(int64_t) * ((size_t)o->N + 1));
  memcpy(vrow, o->vrow, sizeof(int32_t) * (size_t)o->vptr[o->N]);
}
/* aggregates, roots, P and B of level l (l < levels-1) */
int orc_level_agg(const orc *o, int l, int32_t *agg, uint8_t *root, double *P, double *B) {
  const orc_level *L = &o->lev[l];
  const size_t nk = (size_t)L->A.n * o->p.nk_vectors;
  if (l + 1 >= o->L) { if (B && L->B) memcpy(B, L->B, sizeof(double) * nk); return 0; }
  if (agg) memcpy(agg, L->agg, sizeof(int32_t) * (size_t)L->A.n);
  if (root) memcpy(root, L->root, (size_t)L->A.n);
  if (P) memcpy(P, L->P, sizeof(double) * nk);
  if (B) memcpy(B, L->B, sizeof(double) * nk);
  return L->n_agg;
}
int orc_level_color(const orc *o, int l, int32_t *color) {
  const orc_level *L = &o->lev[l];
  if (!L->color) return 0;
  memcpy(color, L->color, sizeof(int32_t) * (size_t)L->A.n);
  return L->n_colors;
}
void orc_level_omega(const orc *o, int l, double *lmax, double *omega) {
  *lmax = o->lev[l].lmax; *omega = o->lev[l].omega;
}
void orc_constraints(const orc *o, double *C, double *b, double *gd, double *gt) {
  if (C) memcpy(C, o->C, sizeof(double) * (size_t)o->m);
  if (b) memcpy(b, o->b, sizeof(double) * (size_t)o->m);
  if (gd) memcpy(gd, o->gd, sizeof(double) * 3 * (size_t)o->E);
  if (gt) memcpy(gt, o->gt, sizeof(double) * 12 * (size_t)o->T);
}
void orc_rest(const orc *o, double *L0, double *V0) {
  if (L0) memcpy(L0, o->L0, sizeof(double) * (size_t)o->E);
  if (V0) memcpy(V0, o->V0, sizeof(double) * (size_t)o->T);
}
void orc_lambda(const orc *o, double *lam, double *dl) {
  if (lam) memcpy(lam, o->lambda, sizeof(double) * (size_t)o->m);
  if (dl) memcpy(dl, o->dl, sizeof(double) * (size_t)o->m);
}
void orc_set_lambda(orc *o, const double *lam) { memcpy(o->lambda, lam, sizeof(double) * (size_t)o->m); }
int orc_sizeof_info(void) { return (int)sizeof(orc_solve_info); }
int orc_sizeof_params(void) { return (int)sizeof(orc_params); }

/* ------------------------------------------------------------------------- */
/* Test-only entry points on a caller-given CSR matrix (diagonal last)       */
/* ------------------------------------------------------------------------- */
int orc_aggregate_csr(int n, const int64_t *ptr, const int32_t *col, const double *val,
                      double theta, uint64_t seed, int l, int32_t *agg, uint8_t *root,
                      uint8_t *S_out) {
  if (n <= 0) return 0;
  orc_csr A = {n, ptr[n], (int64_t *)ptr, (int32_t *)col, (double *)val};
  uint8_t *S = strength(&A, theta);
  if (S_out) memcpy(S_out, S, (size_t)A.nnz);
  int na = aggregate(&A, S, seed, l, agg, root);
  free(S);
  return na;
}

int orc_colour_csr(int n, const int64_t *ptr, const int32_t *col, uint64_t seed, int l,
                   int32_t *color) {
  if (n <= 0) return 0;
  orc_csr A = {n, ptr[n], (int64_t *)ptr, (int32_t *)col, NULL};
  return colour(&A, seed, l, color);
}

/* test-only: one pre-smoothing of level l from x = 0 */
void orc_smooth_test(orc *o, int l, const double *b, double *x) {
  orc_level *L = &o->lev[l];
  memset(x, 0, sizeof(double) * (size_t)L->A.n);
  smooth(o, L, x, b, L->t, 0);
}
