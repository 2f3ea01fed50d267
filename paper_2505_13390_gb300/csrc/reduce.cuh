// Deterministic reductions and row-group helpers shared by the solve kernels.
//
// Every dot product is a fixed-grid two-stage reduction: each block folds its
// threads in a fixed order, the last block to finish folds the per-block
// partials in block order and applies the next PCG recurrence step on the
// device (dot_finalize).  Results are therefore identical run to run.
#pragma once

#include "common.cuh"

namespace mg {

constexpr int kDotThreads = 256;

enum DotMode {
  DOT_STORE = 0,  // *out = s
  DOT_BNORM,      // |b|^2; zero right-hand side finishes at once
  DOT_RZ0,        // initial r.z
  DOT_PQ,         // p.q and alpha
  DOT_RR,         // r.r, iteration count and convergence test
  DOT_RZ,         // new r.z and beta
  DOT_TR          // |b - A x|^2
};

struct DotCtx {
  double *partials;
  unsigned int *counter;
  PcgScalars *sc;
  double *out;
  int mode;
  double rtol;
  int maxiter;
};

static __device__ void dot_finalize(const DotCtx &c, double s) {
  PcgScalars *sc = c.sc;
  switch (c.mode) {
    case DOT_STORE:
      *c.out = s;
      break;
    case DOT_BNORM:
      sc->bnorm2 = s;
      sc->iters = 0;
      sc->rr = s;
      if (s == 0.0) {
        sc->done = 1;
        sc->status = MGPBD_OK;
      } else if (!(s == s) || isinf(s)) {
        sc->done = 1;
        sc->status = MGPBD_E_BREAKDOWN;
      }
      break;
    case DOT_RZ0:
      sc->rz = s;
      if (!(s > 0.0)) {
        sc->done = 1;
        sc->status = MGPBD_E_BREAKDOWN;
      }
      break;
    case DOT_PQ:
      sc->pq = s;
      if (!(s > 0.0)) {
        sc->done = 1;
        sc->status = MGPBD_E_BREAKDOWN;
      } else {
        sc->alpha = sc->rz / s;
      }
      break;
    case DOT_RR:
      sc->rr = s;
      sc->iters += 1;
      if (!(s == s)) {
        sc->done = 1;
        sc->status = MGPBD_E_BREAKDOWN;
      } else if (sqrt(s) <= c.rtol * sqrt(sc->bnorm2)) {
        sc->done = 1;
        sc->status = MGPBD_OK;
      } else if (sc->iters >= c.maxiter) {
        sc->done = 1;
        sc->status = MGPBD_W_NOT_CONVERGED;
      }
      break;
    case DOT_RZ:
      if (!(s > 0.0)) {
        sc->done = 1;
        sc->status = MGPBD_E_BREAKDOWN;
      } else {
        sc->beta = s / sc->rz;
        sc->rz = s;
      }
      break;
    case DOT_TR:
      sc->tr2 = s;
      break;
  }
}

// block reduce of one value per thread in a fixed order, then the last block
// folds the partials (fixed order) and finalizes.  vb and vn are the block's
// index and the number of blocks of its reduction: the launch's own, or one
// instance's share of a launch that serves several instances (the partition
// into blocks, and so every rounding, is the instance's own either way).
static __device__ void block_dot_finish_vg(double v, const DotCtx &c, int vb, int vn) {
  __shared__ double ws[32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) ws[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += ws[w];
    c.partials[vb] = s;
    __threadfence();
    unsigned t = atomicAdd(c.counter, 1u);
    last = (t == (unsigned)vn - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s = 0.0;
  for (int b = threadIdx.x; b < vn; b += blockDim.x)
    s += ((volatile double *)c.partials)[b];
  s = warp_sum(s);
  if (lane == 0) ws[wid] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    dot_finalize(c, t);
    *c.counter = 0;
  }
}

static __device__ __forceinline__ void block_dot_finish(double v, const DotCtx &c) {
  block_dot_finish_vg(v, c, blockIdx.x, gridDim.x);
}

static __device__ __forceinline__ bool is_done(const PcgScalars *sc) {
  return ((volatile const PcgScalars *)sc)->done != 0;
}


template <int G, class T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of three values over the G lanes of a group (G >= 4) by
// reduce-scatter with a zero fourth slot: two exchange steps leave each lane
// one component summed over four lanes, butterflies finish it.  Lane g ends
// with component 2 * [g & G/2] + [g & G/4]; log2(G) + 1 adds per lane instead
// of 3 log2(G) for three butterflies (the FP64 vertex pass is bound by them).
template <int G, class T>
__device__ __forceinline__ T group_sum3(T a0, T a1, T a2, int g) {
  static_assert(G >= 4 && G <= 32, "group of 4..32 lanes");
  constexpr int o1 = G / 2, o2 = G / 4;
  const bool h1 = (g & o1) != 0, h2 = (g & o2) != 0;
  T k0 = h1 ? a2 : a0, k1 = h1 ? (T)0 : a1;  // kept: components (0,1) or (2,3)
  T s0 = h1 ? a0 : a2, s1 = h1 ? a1 : (T)0;  // sent to the partner
  k0 += __shfl_xor_sync(0xffffffffu, s0, o1);
  k1 += __shfl_xor_sync(0xffffffffu, s1, o1);
  T k = h2 ? k1 : k0, s = h2 ? k0 : k1;
  k += __shfl_xor_sync(0xffffffffu, s, o2);
#pragma unroll
  for (int o = o2 / 2; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
  return k;
}

template <int G>
__device__ __forceinline__ int group_sum3_component(int g) {
  return 2 * ((g & (G / 2)) != 0) + ((g & (G / 4)) != 0);
}

// partial row dot of lane g of a G-lane group (no shuffles: callers reduce).
// Four entries per trip are loaded before any is used, so a lane has four
// gathers in flight; the sum order is the plain lane-strided order.
template <int G, class VT, class AT, class XT>
__device__ __forceinline__ AT row_dot(const int64_t *ptr, const int32_t *col, const VT *val,
                                      const XT *x, int i, int g) {
  AT acc = 0;
  int64_t k = ptr[i] + g;
  const int64_t e = ptr[i + 1];
  for (; k + 3 * G < e; k += 4 * G) {
    const int32_t c0 = col[k], c1 = col[k + G], c2 = col[k + 2 * G], c3 = col[k + 3 * G];
    const VT v0 = val[k], v1 = val[k + G], v2 = val[k + 2 * G], v3 = val[k + 3 * G];
    const XT x0 = x[c0], x1 = x[c1], x2 = x[c2], x3 = x[c3];
    acc = fma((AT)v0, (AT)x0, acc);
    acc = fma((AT)v1, (AT)x1, acc);
    acc = fma((AT)v2, (AT)x2, acc);
    acc = fma((AT)v3, (AT)x3, acc);
  }
  for (; k < e; k += G) acc = fma((AT)val[k], (AT)x[col[k]], acc);
  return acc;
}

// Rows handled by G-lane groups, 32/G rows per warp per trip, over warps
// w0, w0 + nw, ...  The loop bound is uniform across the warp, so full-mask
// shuffles inside are safe; `valid` marks groups past the last row.  Which
// warp takes a row never changes that row's arithmetic.
#define GROUP_ROWS_OVER(G, n, w0, nw)                                             \
  const int lane_ = threadIdx.x & 31;                                             \
  const int g = lane_ & ((G) - 1);                                                \
  const int sub_ = lane_ / (G);                                                   \
  const int64_t warp_ = (w0);                                                     \
  const int64_t nwarp_ = (nw);                                                    \
  for (int64_t base_ = warp_ * (32 / (G)), i = base_ + sub_; base_ < (n);         \
       base_ += nwarp_ * (32 / (G)), i = base_ + sub_)                            \
    if (const bool valid = i < (n); true)

// the same over every warp of the launch
#define GROUP_ROWS(G, n)                                                          \
  GROUP_ROWS_OVER(G, n, (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5,    \
                  ((int64_t)gridDim.x * blockDim.x) >> 5)

// the launch's own warps as (first warp, number of warps)
#define HW_WARPS                                                                  \
  (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5,                          \
      ((int64_t)gridDim.x * blockDim.x) >> 5

// the warps of virtual block vb of a grid of vn blocks
#define VG_WARPS(vb, vn)                                                          \
  ((int64_t)(vb) * blockDim.x + threadIdx.x) >> 5, ((int64_t)(vn) * blockDim.x) >> 5

// matrix-free level-0 products (mfree.cu)
mgpbd_status mf_apply_pq(Handle *h, const double *p, double *q, const DotCtx &c);
mgpbd_status mf_apply_pq_form(Handle *h, bool pairs, const double *p, double *q,
                              const DotCtx &c);
mgpbd_status mf_residual64(Handle *h, const double *x, const double *b, double *r);
mgpbd_status mf_split(Handle *h, const double *a, float2 *out, int64_t n);
template <class T>
mgpbd_status mf_level0(Handle *h, int mode, const T *x, const T *b, const T *dinv, T omega,
                       T *out);
constexpr int kMfSweep = 0, kMfResid = 1, kMfApply = 3, kMfResidMember = 6;
mgpbd_status mf_autotune(Handle *h);

// The last level-0 sweep of a top V-cycle can write the preconditioned
// residual z = x_new straight in FP64 and fold r.z into the PCG scalars.
struct TopOut {
  const double *r;  // FP64 residual the V-cycle was applied to
  double *z;        // FP64 output
  DotCtx c;         // r.z reduction (when dot is set)
  bool dot;
};
template <class T>
mgpbd_status mf_level0_final(Handle *h, const T *x, const T *b, const T *dinv, T omega,
                             const TopOut &o);

}  // namespace mg
