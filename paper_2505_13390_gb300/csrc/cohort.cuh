// Batched PCG of several instances ("a cohort"): the records a batched
// launch reads its per-instance arguments from (internal, not part of the ABI).
//
// Each step of a PCG iteration (the vertex and row passes of A.p, the x/r
// update, the level-0 sweeps and residual, restriction, the V-cycle below
// level 0, prolongation, the final sweep and the p update) runs as ONE launch
// for every instance of the cohort.  Each instance keeps the grid its own
// launch would have: a block reads its instance, its index among that
// instance's blocks and their number from a per-block table and runs the
// standalone kernel's body with them.  Every reduction is therefore partitioned, and every sum
// rounded, exactly as in the instance's standalone solve.
#pragma once

#include "reduce.cuh"

namespace mg {

// one CSR level of the V-cycle below level 0
template <class T>
struct TailLevel {
  int n, G, n_agg;
  T omega;
  const int64_t *ptr;
  const int32_t *col;
  const T *val, *dinv;
  T *x, *x2, *b, *r;
  const int32_t *agg;
  const T *P;
  const int64_t *mptr;
  const int32_t *mrow;
};

template <class T>
struct TailDesc {
  int first, coarsest, sweeps;  // levels first .. coarsest-1 smooth; coarsest solves
  const double *cinv;
  TailLevel<T> lev[kMaxLevels];
};

// the steps of a batched PCG iteration that have a per-instance grid
enum CohortStep {
  CS_VERT64 = 0,  // vertex pass of A.p (FP64)
  CS_ROW_PQ,      // row pass of A.p with p.Ap
  CS_XR,          // x, r update with r.r and the next V-cycle's start
  CS_VERT32,      // vertex pass of a level-0 sweep or residual (FP32)
  CS_ROW,         // row pass of a level-0 sweep or the residual
  CS_RESTRICT,    // level 0 to level 1
  CS_PROLONG,     // level 1 to level 0
  CS_ROW_FINAL,   // last post-sweep: z in FP64 and r.z
  CS_PUPD,        // p = z + beta p
  CS_STEPS
};

// One instance of a cohort: mixed precision, matrix-free level 0,
// weighted-Jacobi smoothing (two sweeps), one column of P per aggregate and
// at least one level below level 0.
struct CohortMember {
  int m, N, E;
  int gv64, gv32;  // lanes per vertex of the FP64 and FP32 vertex passes
  const int32_t *edge, *tet, *vorder;
  const int64_t *vptr;
  const int32_t *vrow;
  const double *ginc64, *w, *gd, *gt, *at;
  const float4 *ginc4;
  const float *w32, *gd32, *gt32, *at32;
  double *u64;
  float *u32;
  // Krylov vectors, scalars and the reductions of p.q, r.r and r.z
  double *x, *r, *z, *p, *q;
  PcgScalars *sc;
  DotCtx c_pq, c_rr, c_rz;
  // level 0 of the V-cycle (FP32): right-hand side, iterate pair, residual
  float *b0, *x0, *x20, *r0;
  const float *dinv0;
  float om0;
  int n_agg0;
  const int64_t *mptr0;
  const int32_t *mrow0;
  const float *P0;
  const int32_t *agg0;
  const float *xc1;  // where level 1 leaves its result for the prolongation
  TailDesc<float> tail;  // levels 1 .. coarsest
  int grid[CS_STEPS];    // blocks of each step in the instance's standalone solve
};

// one block of a batched launch: its instance, its index among that
// instance's blocks and their number, and the instance's PCG scalars (read
// first: a finished instance's blocks leave after one load)
struct __align__(16) CohortBlock {
  int k, vb, vn, pad;
  const PcgScalars *sc;
  const void *pad2;
};

// ---- host side (solve.cu and mfree.cu) ----
constexpr int kCohortMax = 64;

// A set of instances (same stream, each cohort_eligible) whose PCG
// iterations run together.  A member between solves (its scalars say done)
// costs its blocks one flag read per launch.
struct Cohort {
  cudaStream_t stream = nullptr;
  std::vector<Handle *> hs;                 // members, in table order
  std::vector<unsigned long long> gens;     // each member's arrays at the build
  int K = 0, cap = 0, maxc = 1;
  int gv32 = 0;                             // the members' common lanes per FP32 vertex (0: mixed)
  int blocks[CS_STEPS] = {};                // blocks of each batched step
  CohortMember *d_mem = nullptr;
  CohortBlock *d_blk = nullptr;             // the blocks of every step, step after step
  int blk_off[CS_STEPS] = {};               // first block record of each step
  size_t blk_cap = 0;
  PcgScalars *d_sc = nullptr, *h_sc = nullptr;  // members' scalars after a chunk
  unsigned int *bar = nullptr;              // grid barrier of the batched tail
  long long wait_limit = 1ll << 24;
  cudaGraphExec_t graph = nullptr;
  int graph_iters = 0;
  unsigned long long graph_kernels = 0;
  ~Cohort();
};
bool cohort_eligible(const Handle *h);
mgpbd_status cohort_build(Cohort *c);
bool cohort_stale(const Cohort *c);
mgpbd_status cohort_chunk(Cohort *c, int iters);
// the standalone grids of the matrix-free steps of h's solve
void mf_cohort_grids(const Handle *h, int grid[CS_STEPS]);
// one batched matrix-free step for every member: which = CS_VERT64,
// CS_ROW_PQ, CS_VERT32 (sel 0: from x0, 1: from x20), CS_ROW (sel 0: sweep
// x0 -> x20, 1: residual x20 -> r0, 2: sweep x20 -> x0) or CS_ROW_FINAL;
// gv32 is the members' common lanes per FP32 vertex, 0 when they differ
mgpbd_status mf_cohort_step(int which, int sel, const CohortMember *d_mem,
                            const CohortBlock *d_blk, int blocks, int gv32, cudaStream_t st);

}  // namespace mg
