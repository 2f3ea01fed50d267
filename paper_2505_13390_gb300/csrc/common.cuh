// Internal declarations of the GB300 MGPBD library (not part of the ABI).
//
// Compiled with --fmad=false: a*b+c is never contracted, and every fused
// multiply-add is an explicit fma()/fmaf().  Constraint evaluation, assembly,
// near-kernel sweeps, strength, aggregation, injection and the canonical
// Galerkin product therefore reproduce a plain IEEE-754 FP64 program exactly.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/mgpbd.h"

namespace mg {

constexpr int kMaxLevels = 16;
constexpr int kWarp = 32;

// ---------------------------------------------------------------------------
// error plumbing
// ---------------------------------------------------------------------------
void set_error(const std::string &msg);
mgpbd_status cuda_fail(cudaError_t e, const char *what, const char *file, int line);

#define MG_CUDA(call)                                                     \
  do {                                                                    \
    cudaError_t e_ = (call);                                              \
    if (e_ != cudaSuccess) return mg::cuda_fail(e_, #call, __FILE__, __LINE__); \
  } while (0)
// every kernel launch is followed by MG_LAUNCH, which also counts it
extern unsigned long long g_launches;  // updated atomically
#define MG_LAUNCH(what)                                                   \
  do {                                                                    \
    __atomic_fetch_add(&mg::g_launches, 1ull, __ATOMIC_RELAXED);          \
    cudaError_t e_ = cudaGetLastError();                                  \
    if (e_ != cudaSuccess) return mg::cuda_fail(e_, what, __FILE__, __LINE__); \
  } while (0)
#define MG_TRY(expr)                                                      \
  do {                                                                    \
    mgpbd_status s_ = (expr);                                             \
    if (s_ < 0) return s_;                                                \
  } while (0)

// ---------------------------------------------------------------------------
// device memory owned by a handle
// ---------------------------------------------------------------------------
// Stream-ordered allocations on the owning handle's stream (cudaMallocAsync /
// cudaFreeAsync): freeing never synchronises the whole device, so instances
// that run side by side on their own streams do not stall each other.
//
// With a caller workspace (base != nullptr) the arena instead carves every
// array out of the caller's buffer [base, base + cap): first fit over a list
// of free ranges, freed ranges merged with their neighbours.  A range freed
// here is reused only by arrays the same handle allocates later, and all of
// the handle's work is ordered on its one stream, so a reused range is never
// written while an earlier kernel still reads it (the ordering
// cudaFreeAsync gives the pooled mode).  Exhausting the buffer is
// MGPBD_E_BUDGET.
struct Arena {
  size_t bytes = 0;  // live bytes
  size_t peak = 0;   // high-water mark of `bytes`
  cudaStream_t stream = nullptr;
  std::vector<std::pair<void *, size_t>> live;
  char *base = nullptr;             // caller workspace, or nullptr (pooled)
  size_t cap = 0;                   // usable bytes of the workspace
  std::map<size_t, size_t> holes;   // offset -> length of each free range
  void use_workspace(void *p, size_t n);
  mgpbd_status alloc(void **p, size_t n);
  void release(void *p);
  void release_all();
};

template <class T>
inline mgpbd_status alloc_n(Arena &a, T **p, size_t n) {
  return a.alloc(reinterpret_cast<void **>(p), n * sizeof(T));
}

// ---------------------------------------------------------------------------
// PCG scalars that live on the device (no host round trip per iteration)
// ---------------------------------------------------------------------------
struct PcgScalars {
  double bnorm2;   // |b|^2
  double rz;       // r.z of the current iteration
  double rz_new;
  double pq;       // p.q
  double rr;       // r.r
  double alpha, beta;
  double tr2;      // |b - A x|^2 (true residual)
  int done;        // 1 once converged or failed
  int iters;       // PCG iterations taken
  int status;      // MGPBD_OK / MGPBD_W_NOT_CONVERGED / MGPBD_E_BREAKDOWN
  int pad;
};

// ---------------------------------------------------------------------------
// one AMG level
// ---------------------------------------------------------------------------
struct Level {
  int n = 0;
  int64_t nnz = 0;
  int64_t *ptr = nullptr;
  int32_t *col = nullptr;
  double *val = nullptr;   // FP64 values (canonical)
  float *val32 = nullptr;  // FP32 mirror (mixed precision)
  double *dinv = nullptr;  // 1/A_ii
  float *dinv32 = nullptr;
  // capacity of the coarse-level buffers (levels >= 1)
  int cap_n = 0;
  int64_t cap_nnz = 0;
  // prolongation to level+1 (absent on the coarsest)
  int n_agg = 0;
  int32_t *agg = nullptr;
  uint8_t *root = nullptr;
  double *P = nullptr;
  float *P32 = nullptr;
  double *B = nullptr;       // near-kernel of this level
  int64_t *mptr = nullptr;   // members of each aggregate (ascending rows)
  int32_t *mrow = nullptr;
  // level 0 with the matrix-free operator and one column of P: each row's
  // position in the member list (-1: in no aggregate) and P in member order
  // (the V-cycle's precision), so that the residual is written and the
  // restriction reads it in member order
  int32_t *mpos = nullptr;
  void *Pm = nullptr;
  int max_members = 0;
  int max_coarse_row = 0;    // longest row of level+1 (Galerkin smem size), in aggregates
  // k > 1 near-kernel vectors: dead columns of P and the aggregate-level
  // pattern of level+1 (kept for the Galerkin re-form)
  uint8_t *pdead = nullptr;
  int64_t *gbptr = nullptr;
  int32_t *gbcol = nullptr;
  int64_t cap_gb = 0;
  int G32 = 0, G64 = 0;      // lanes per row of the FP32 / FP64 row kernels (0 = rule)
  int32_t *color = nullptr;
  int n_colors = 0;
  int32_t *crow = nullptr;          // rows grouped by colour (multicolour GS)
  std::vector<int64_t> hcptr;       // host offsets of each colour in crow
  double lmax = 0.0, omega = 0.0;
  // V-cycle vectors in the working precision (double or float)
  void *x = nullptr, *x2 = nullptr, *b = nullptr, *r = nullptr, *t = nullptr;
};

enum ProfChannel { PROF_SWEEP = 0, PROF_AP = 1, PROF_CH = 2 };

struct Handle {
  cudaStream_t stream = nullptr;
  int device = 0;            // CUDA device that was current at create
  mgpbd_params p{};
  int N = 0, E = 0, T = 0, m = 0;
  Arena arena;
  // mesh (device)
  double *rest = nullptr, *w = nullptr, *alpha_t = nullptr, *L0 = nullptr, *V0 = nullptr;
  int32_t *edge = nullptr, *tet = nullptr;
  int tet_kind = 0;          // tet rows: 0 volume, 1 ARAP (Sec. 5.3)
  double *Dminv = nullptr;   // ARAP: inverse rest edge matrix per tet, row-major [T][9]
  // incidence
  int64_t *vptr = nullptr;
  int32_t *vrow = nullptr;
  // state
  double *x = nullptr, *v = nullptr, *xold = nullptr, *lambda = nullptr;
  // per-iteration
  double *C = nullptr, *b = nullptr, *gd = nullptr, *gt = nullptr, *dl = nullptr;
  double *dx = nullptr, *xbak = nullptr;  // position correction and backtracking base
  // matrix-free level-0 operator: gradients in incidence order, FP32 copies
  uint8_t *vslot = nullptr;
  double *ginc64 = nullptr, *u64 = nullptr;
  float4 *ginc4 = nullptr;  // FP32 gradient and row id (bits in .w) per incidence
  float *gd32 = nullptr, *gt32 = nullptr, *at32 = nullptr, *w32 = nullptr, *u32 = nullptr;
  // float-float A.p (params.ap_split): low parts beside the FP32 high parts
  // above (gradients in incidence and row order, alpha~, w), u as high and
  // low parts (four slots per vertex), and p as (high, low) pairs written by
  // the p update
  float *ginc_lo = nullptr, *gd_lo = nullptr, *gt_lo = nullptr, *at_lo = nullptr,
        *w_lo = nullptr, *u_hi = nullptr, *u_lo = nullptr;
  float2 *p_df = nullptr;
  int n_replace = 0;           // residual replacements of the current solve
  int mf_g32 = 8, mf_g64 = 4;  // lanes per vertex of the vertex pass (autotuned)
  // lanes forced by mgpbd_set_lanes (0 = autotuned or rule): CSR rows in FP32
  // and FP64, matrix-free vertices in FP32 and FP64
  int force_csr32 = 0, force_csr64 = 0, force_vert32 = 0, force_vert64 = 0;
  int32_t *vorder = nullptr;   // vertex-pass order: by incidence count within windows
  uint16_t *map = nullptr;
  uint8_t *S = nullptr;  // strength mask, reused per level (grown when a level has more nnz)
  int64_t cap_S = 0;
  // hierarchy
  int L = 0;
  bool have_setup = false;
  Level lev[kMaxLevels];
  // coarsest dense factor and inverse (FP64)
  int nc = 0, cap_nc = 0;
  double *cdense = nullptr;  // n_c x n_c: A, then L (lower)
  double *cinv = nullptr;    // n_c x n_c: A^-1
  int *cstat = nullptr;      // Cholesky status (device)
  // PCG
  double *pr = nullptr, *pz = nullptr, *pp = nullptr, *pq = nullptr;
  PcgScalars *sc = nullptr;
  PcgScalars *sc_host = nullptr;  // pinned mirror for polls
  // the V-cycle below level 0 as one cooperative kernel (solve.cu)
  bool tail = false;                 // use it where it applies (mgpbd_set_coarse_tail)
  unsigned int *gbar = nullptr;      // its grid barrier word
  long long wait_limit = 1ll << 24;  // polls a block waits at the barrier
  double *partials = nullptr;     // dot-product block partials
  unsigned int *counter = nullptr;
  // scratch for setup
  void *tmp = nullptr;
  size_t tmp_bytes = 0;
  int *flag = nullptr;       // device int scratch (round counters)
  int *flag_host = nullptr;  // pinned
  // counters
  int64_t it_global = 0;
  int n_setups = 0;
  double ms_setup = 0, ms_galerkin = 0, ms_solve = 0, ms_other = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  int last_pcg_iters = 0;
  bool want_colors = false;  // colour every level at setup even for Jacobi
  mgpbd_solve_info last{};
  // optional event timing, per channel (PROF_SWEEP: the level-0 smoother
  // sweeps, the dominant kernel; PROF_AP: the PCG recurrence's A.p)
  bool prof = false;
  int prof_mask = 0;  // channels recorded: bit PROF_SWEEP, bit PROF_AP
  std::vector<cudaEvent_t> pev[PROF_CH];  // pairs
  std::vector<int> pev_iter[PROF_CH];     // PCG iteration of each pair (-1 = initial V-cycle)
  int pev_used[PROF_CH] = {};
  int pcg_k = -1;                         // PCG iteration being launched
  double prof_ms[PROF_CH] = {};
  long long prof_n[PROF_CH] = {};
  // the same timing inside a captured PCG chunk: event-record nodes of the
  // graph, read back after every replay
  bool capturing = false;
  std::vector<cudaEvent_t> gev[PROF_CH];  // pairs
  std::vector<int> gev_iter[PROF_CH];     // iteration within the chunk of each pair
  int gev_used[PROF_CH] = {};
  bool graph_prof = false;       // the captured graph records gev
  // CUDA graph of a chunk of PCG iterations, valid while `graph_gen` matches
  unsigned long long gen = 1;      // bumped whenever device pointers or setup change
  unsigned long long graph_gen = 0;
  const double *graph_x = nullptr;
  int graph_chunk = 0;
  unsigned long long graph_kernels = 0;  // kernels in one replay of the graph
  cudaGraphExec_t pcg_graph = nullptr;
};

// event pair around one launch of the profiled kernel (no-op when disabled)
mgpbd_status prof_reserve_graph(Handle *h, int pairs);
mgpbd_status prof_harvest_graph(Handle *h, int first_iter);
mgpbd_status prof_begin(Handle *h, int ch = PROF_SWEEP);
mgpbd_status prof_end(Handle *h, int ch = PROF_SWEEP);
// sums the pairs recorded during the last solve that belong to iterations that ran
mgpbd_status prof_harvest(Handle *h, int iters);

// grid sizing
int num_sms();
// blocks of `kernel` (with `threads` per block) that fit on the GPU at once:
// kernels that end in a last-block reduction run as one such wave, so that
// each block's serialised tail (fence, counter atomic) is paid once
int wave_blocks(const void *kernel, int threads);
inline int blocks_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  return (int)(b < 1 ? 1 : (b > 1048576 ? 1048576 : b));
}

// device scratch of at least `bytes`
mgpbd_status ensure_tmp(Handle *h, size_t bytes);

// ---------------------------------------------------------------------------
// building blocks (definitions in the .cu files)
// ---------------------------------------------------------------------------
// exclusive scan of n int64 counts in place into out[0..n] (out[n] = total)
mgpbd_status scan_counts(Handle *h, const int64_t *counts, int64_t *out, int64_t n);
// read one int64 from device memory (synchronises)
mgpbd_status read_i64(Handle *h, const int64_t *d, int64_t *out);

// pattern.cu
mgpbd_status build_incidence(Handle *h);
mgpbd_status build_pattern(Handle *h);

// physics.cu
mgpbd_status rest_shape(Handle *h);
mgpbd_status launch_begin_frame(Handle *h);
mgpbd_status launch_end_frame(Handle *h);
mgpbd_status launch_eval(Handle *h);
mgpbd_status launch_assemble(Handle *h);
mgpbd_status launch_update(Handle *h, mgpbd_solve_info *info);

// api.cu: one global iteration of Alg. 1 around its MGPCG solve
mgpbd_status iterate_prepare(Handle *h, bool *due);
mgpbd_status iterate_complete(Handle *h, mgpbd_status st, mgpbd_solve_info *inf, bool due,
                              mgpbd_solve_info *info);

// setup.cu
mgpbd_status amg_setup(Handle *h);
mgpbd_status galerkin_reform(Handle *h);
mgpbd_status level_precision_copies(Handle *h, int l);

// mfree.cu (matrix-free level-0 operator)
mgpbd_status mf_create(Handle *h);
mgpbd_status mf_prepare(Handle *h);

// solve.cu
int group_for(const Handle *h, const Level &L, bool fp64);  // lanes per row in effect
mgpbd_status autotune_levels(Handle *h);
mgpbd_status coarsest_factor(Handle *h);
mgpbd_status pcg_solve(Handle *h, const double *d_b, double *d_x, mgpbd_solve_info *info);
// the solve's start (x = 0, r = b, z = V(r), p = z) and end (true residual,
// status into info; synchronises), between which chunks of iterations run
mgpbd_status pcg_begin(Handle *h, const double *d_b, double *d_x);
mgpbd_status pcg_finish(Handle *h, const double *d_b, double *d_x, mgpbd_solve_info *info);
mgpbd_status vcycle_apply(Handle *h, const double *d_r, double *d_z);
mgpbd_status apply_level0(Handle *h, int form, const double *x, double *y);
mgpbd_status dot_dd(Handle *h, const double *x, const double *y, int64_t n, double *d_out);
mgpbd_status xpbd_step(Handle *h, mgpbd_solve_info *info);
mgpbd_status power_method(Handle *h, int l);
mgpbd_status evict_l2(Handle *h);  // autotuner: start timings from an evicted L2

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
// SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014)
__host__ __device__ __forceinline__ uint64_t h64(uint64_t k) {
  uint64_t z = k + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t hkey(uint64_t seed, int l, int i) {
  return (seed << 40) | ((uint64_t)(uint32_t)l << 32) | (uint64_t)(uint32_t)i;
}
__host__ __device__ __forceinline__ double u01(uint64_t hv) {
  return ((double)(hv >> 11) + 0.5) * 0x1p-53;
}

// Conversions between IEEE 754 binary64 and binary32 written with integer
// operations.  The hardware conversion instructions between the two formats
// issue on the FP64 pipe, which is narrow on this GPU (a level-0 vector of
// 3.7M entries took ~28 us to convert), while the integer pipes are wide.
//
// binary32 -> binary64 is exact: rebias the exponent (127 -> 1023), widen the
// fraction, normalise subnormals; infinities and NaNs keep sign and payload.
__device__ __forceinline__ double f32_to_f64(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t s = u & 0x80000000u, e = (u >> 23) & 0xffu;
  uint32_t m = u & 0x7fffffu, hi, lo;
  if (e == 0xffu) {
    hi = s | 0x7ff00000u | (m >> 3);
    lo = m << 29;
  } else if (e != 0u) {
    hi = s | ((e + 896u) << 20) | (m >> 3);
    lo = m << 29;
  } else if (m == 0u) {
    hi = s;
    lo = 0u;
  } else {  // subnormal m * 2^-149: shift the leading one to bit 23
    const int n = __clz(m) - 8;
    m = (m << n) & 0x7fffffu;
    hi = s | ((uint32_t)(897 - n) << 20) | (m >> 3);
    lo = m << 29;
  }
  return __hiloint2double((int)hi, (int)lo);
}

// binary64 -> binary32 with roundTiesToEven (IEEE 754-2008, 4.3.1): keep the
// leading 24 significant bits, round on the dropped bits (above half: up;
// exactly half: to the even neighbour), overflow to infinity, results below
// the binary32 normal range rounded in units of 2^-149.
__device__ __forceinline__ float f64_to_f32(double d) {
  const uint32_t hi = (uint32_t)__double2hiint(d), lo = (uint32_t)__double2loint(d);
  const uint32_t s = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu);
  const uint64_t m = ((uint64_t)(hi & 0xfffffu) << 32) | lo;
  if (e == 0x7ff) return __uint_as_float(s | 0x7f800000u | (m ? 0x400000u | (uint32_t)(m >> 29) : 0u));
  const int ef = e - 896;  // binary32 biased exponent
  if (ef >= 0xff) return __uint_as_float(s | 0x7f800000u);
  if (ef >= 1) {
    const uint32_t r = (uint32_t)(m >> 29), rem = (uint32_t)m & 0x1fffffffu;
    uint32_t bits = ((uint32_t)ef << 23) | r;
    if (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) bits += 1u;  // carries into exponent
    return __uint_as_float(s | bits);
  }
  // value = (2^52 + m) * 2^(e - 1075) = sig * 2^(ef - 30) units of 2^-149
  const int sh = 30 - ef;
  if (e == 0 || sh >= 54) return __uint_as_float(s);  // below half the smallest subnormal
  const uint64_t sig = m | (1ull << 52);
  const uint32_t q = (uint32_t)(sig >> sh);
  const uint64_t rem = sig & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
  return __uint_as_float(s | (q + ((rem > half || (rem == half && (q & 1u))) ? 1u : 0u)));
}

template <class T>
__device__ __forceinline__ T narrow(double v);
template <>
__device__ __forceinline__ float narrow<float>(double v) { return f64_to_f32(v); }
template <>
__device__ __forceinline__ double narrow<double>(double v) { return v; }
__device__ __forceinline__ double widen(float v) { return f32_to_f64(v); }
__device__ __forceinline__ double widen(double v) { return v; }

// a binary64 value as a float-float pair (h, l): h = RN32(a), l = RN32(a - h).
// a - h is exact in binary64 (a multiple of a's last place below half of h's,
// at most 30 significant bits), so h + l carries 48 of a's 53 significant
// bits inside the binary32 normal range; one FP64 subtraction.
__device__ __forceinline__ float2 df_split(double a) {
  const float h = f64_to_f32(a);
  return make_float2(h, f64_to_f32(a - f32_to_f64(h)));
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace mg
