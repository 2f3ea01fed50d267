// Solve phase (Sec. 4.4-4.5): MGPCG with one V-cycle per iteration, the
// weighted-Jacobi smoother, restriction/prolongation through the aggregates,
// the coarsest dense Cholesky, and the power method for lambda_max(D^-1 A).
//
// Scalars of the PCG recurrence (r.z, p.q, alpha, beta, |r|) stay on the
// device: every dot product is a fixed-grid two-stage reduction whose last
// block folds the per-block partials in a fixed order and applies the next
// recurrence step, so results are deterministic run to run and no host round
// trip is needed inside an iteration.  Kernels of an iteration return at once
// when the device flag `done` is set, so the host launches iterations in
// chunks and polls the flag between chunks.
//
// Precision: MGPBD_FP64 runs everything in FP64.  MGPBD_MIXED runs the
// V-cycle bulk (smoothing, residuals, restriction, prolongation) with FP32
// values, vectors and accumulation; A.p, the dot products, alpha/beta, the
// Krylov vectors, the true residual and the coarsest factorisation stay FP64.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "cohort.cuh"
#include "reduce.cuh"

namespace mg {

// blocks of a dot-product kernel over n entries: about 4 entries per thread,
// at least two blocks per SM, at most the 4096 partials the handle holds
static int dot_grid(int64_t n) {
  return (int)std::min<int64_t>(4096, std::max<int64_t>(2 * num_sms(), (n + 1023) / 1024));
}

static DotCtx make_ctx(Handle *h, int mode, double *out = nullptr) {
  DotCtx c;
  c.partials = h->partials;
  c.counter = h->counter;
  c.sc = h->sc;
  c.out = out;
  c.mode = mode;
  c.rtol = h->p.pcg_rtol;
  c.maxiter = h->p.pcg_maxiter;
  return c;
}

// ---------------------------------------------------------------------------
// plain vector kernels
// ---------------------------------------------------------------------------
__global__ void k_dot(int64_t n, const double *x, const double *y, DotCtx c, int check_done) {
  if (check_done && is_done(c.sc)) return;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    acc = fma(x[i], y[i], acc);
  block_dot_finish(acc, c);
}

// x += alpha p; r -= alpha q; then r.r (convergence test).  The start of the
// next V-cycle is folded in: bl = r in the V-cycle's precision (MGPBD_MIXED)
// and, with the Jacobi smoother, its first sweep from zero x0 = omega D^-1 r.
// In mixed precision each thread sums the squares of its FP32 copies of r in
// FP32 (the stopping test needs a few digits, and every FP64 operation is
// scarce); the sum over threads stays FP64.  Each thread takes two adjacent
// entries per trip with 16-byte loads (the vectors are 256-byte aligned).
template <class T>
struct Pair;
template <>
struct Pair<float> {
  using V = float2;
};
template <>
struct Pair<double> {
  using V = double2;
};

template <class T>
__device__ __forceinline__ T xr_entry(double al, double &xi, double &ri, double pi, double qi,
                                      T di, T om, T *bi_out, T *x0i) {
  xi = fma(al, pi, xi);
  ri = fma(-al, qi, ri);
  const T bi = narrow<T>(ri);
  *bi_out = bi;
  *x0i = om * (bi * di);
  return bi;
}

template <class T>
__device__ __forceinline__ void xr_update_body(int vb, int vn, int64_t n, double *x, double *r,
                                               const double *p, const double *q, const DotCtx &c,
                                               T *bl, const T *dinv, T om, T *x0) {
  using V = typename Pair<T>::V;
  const double al = c.sc->alpha;
  T acc = 0;
  const int64_t n2 = n / 2;
  for (int64_t k = vb * (int64_t)blockDim.x + threadIdx.x; k < n2;
       k += (int64_t)vn * blockDim.x) {
    double2 xv = reinterpret_cast<const double2 *>(x)[k];
    double2 rv = reinterpret_cast<const double2 *>(r)[k];
    const double2 pv = reinterpret_cast<const double2 *>(p)[k];
    const double2 qv = reinterpret_cast<const double2 *>(q)[k];
    V dv = {};
    if (x0) dv = reinterpret_cast<const V *>(dinv)[k];
    V bv, xv0;
    const T b0 = xr_entry<T>(al, xv.x, rv.x, pv.x, qv.x, dv.x, om, &bv.x, &xv0.x);
    const T b1 = xr_entry<T>(al, xv.y, rv.y, pv.y, qv.y, dv.y, om, &bv.y, &xv0.y);
    acc = fma(b0, b0, acc);
    acc = fma(b1, b1, acc);
    reinterpret_cast<double2 *>(x)[k] = xv;
    reinterpret_cast<double2 *>(r)[k] = rv;
    if (bl) reinterpret_cast<V *>(bl)[k] = bv;
    if (x0) reinterpret_cast<V *>(x0)[k] = xv0;
  }
  if ((n & 1) && vb == 0 && threadIdx.x == 0) {
    const int64_t i = n - 1;
    double xi = x[i], ri = r[i];
    T bi, x0i;
    const T b0 = xr_entry<T>(al, xi, ri, p[i], q[i], x0 ? dinv[i] : (T)0, om, &bi, &x0i);
    acc = fma(b0, b0, acc);
    x[i] = xi;
    r[i] = ri;
    if (bl) bl[i] = bi;
    if (x0) x0[i] = x0i;
  }
  block_dot_finish_vg(widen(acc), c, vb, vn);
}

template <class T>
__global__ void k_xr_update(int64_t n, double *x, double *r, const double *p, const double *q,
                            DotCtx c, T *bl, const T *dinv, T om, T *x0) {
  if (is_done(c.sc)) return;
  xr_update_body<T>(blockIdx.x, gridDim.x, n, x, r, p, q, c, bl, dinv, om, x0);
}

// the same start of a V-cycle on its own: bl = r in the V-cycle's precision,
// x0 = omega D^-1 bl (Jacobi)
template <class T>
__global__ void k_top_prep(int64_t n, const double *r, T *bl, const T *dinv, T om, T *x0,
                           const PcgScalars *sc) {
  if (sc && is_done(sc)) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    T bi = narrow<T>(r[i]);
    if (bl) bl[i] = bi;
    if (x0) x0[i] = om * (bi * dinv[i]);
  }
}

// p = z + beta p, two entries per thread (16-byte loads; p and z are
// 256-byte aligned); with pdf, p also as float-float pairs for the pair form
// of A.p (params.ap_split)
__device__ __forceinline__ void p_update_body(int vb, int vn, int64_t n, double *p,
                                              const double *z, const PcgScalars *sc,
                                              float2 *pdf = nullptr) {
  const double be = sc->beta;
  const int64_t n2 = n / 2, h2 = (n2 + 1) / 2;  // pairs k and k + h2 per thread
  double2 *p2 = reinterpret_cast<double2 *>(p);
  const double2 *z2 = reinterpret_cast<const double2 *>(z);
  for (int64_t k = vb * (int64_t)blockDim.x + threadIdx.x; k < h2;
       k += (int64_t)vn * blockDim.x) {
    const int64_t k2 = k + h2;
    const bool two = k2 < n2;
    double2 pa = p2[k], za = z2[k], pb = {0.0, 0.0}, zb = {0.0, 0.0};
    if (two) {
      pb = p2[k2];
      zb = z2[k2];
    }
    pa.x = fma(be, pa.x, za.x);
    pa.y = fma(be, pa.y, za.y);
    p2[k] = pa;
    if (pdf) {
      const float2 s0 = df_split(pa.x), s1 = df_split(pa.y);
      reinterpret_cast<float4 *>(pdf)[k] = make_float4(s0.x, s0.y, s1.x, s1.y);
    }
    if (two) {
      pb.x = fma(be, pb.x, zb.x);
      pb.y = fma(be, pb.y, zb.y);
      p2[k2] = pb;
      if (pdf) {
        const float2 s0 = df_split(pb.x), s1 = df_split(pb.y);
        reinterpret_cast<float4 *>(pdf)[k2] = make_float4(s0.x, s0.y, s1.x, s1.y);
      }
    }
  }
  if ((n & 1) && vb == 0 && threadIdx.x == 0) {
    p[n - 1] = fma(be, p[n - 1], z[n - 1]);
    if (pdf) pdf[n - 1] = df_split(p[n - 1]);
  }
}

__global__ void k_p_update(int64_t n, double *p, const double *z, const PcgScalars *sc,
                           float2 *pdf) {
  if (is_done(sc)) return;
  p_update_body(blockIdx.x, gridDim.x, n, p, z, sc, pdf);
}

__global__ void k_pcg_init(PcgScalars *sc, unsigned int *bar) {
  bar[0] = 0;  // the coarse tail's barrier word starts each solve at zero
  sc->done = 0;
  sc->iters = 0;
  sc->status = MGPBD_W_NOT_CONVERGED;
  sc->rz = sc->pq = sc->rr = sc->alpha = sc->beta = sc->tr2 = 0.0;
}

template <class D>
__device__ __forceinline__ D convert_to(float v);
template <>
__device__ __forceinline__ float convert_to<float>(float v) { return v; }
template <>
__device__ __forceinline__ double convert_to<double>(float v) { return f32_to_f64(v); }
template <class D>
__device__ __forceinline__ D convert_to(double v) { return narrow<D>(v); }

template <class S, class D>
__global__ void k_convert(int64_t n, const S *a, D *b, const PcgScalars *sc) {
  if (sc && is_done(sc)) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = convert_to<D>(a[i]);
}

// ---------------------------------------------------------------------------
// sparse kernels: G lanes per row (G in 4, 8, 16, 32)
// ---------------------------------------------------------------------------
// q = A p (PCG operator) fused with p.q
template <int G, class VT, class AT>
__global__ void k_spmv_pq(int n, const int64_t *ptr, const int32_t *col, const VT *val,
                          const double *p, double *q, DotCtx c) {
  if (is_done(c.sc)) return;
  double acc = 0.0;
  GROUP_ROWS(G, n) {
    AT s = valid ? row_dot<G, VT, AT, double>(ptr, col, val, p, (int)i, g) : (AT)0;
    s = group_sum<G>(s);
    if (valid && g == 0) {
      double qi = (double)s;
      q[i] = qi;
      acc = fma(p[i], qi, acc);
    }
  }
  block_dot_finish(acc, c);
}

// r_t = b - A x in FP64, |r_t|^2
__global__ void k_true_resid(int n, const int64_t *ptr, const int32_t *col, const double *val,
                             const double *x, const double *b, DotCtx c) {
  double acc = 0.0;
  GROUP_ROWS(4, n) {
    double s = valid ? row_dot<4, double, double, double>(ptr, col, val, x, (int)i, g) : 0.0;
    s = group_sum<4>(s);
    if (valid && g == 0) {
      double ri = b[i] - s;
      acc = fma(ri, ri, acc);
    }
  }
  block_dot_finish(acc, c);
}

// weighted Jacobi, first sweep from x = 0: x = omega D^-1 b
template <class T>
__global__ void k_jacobi0(int n, const T *b, const T *dinv, T omega, T *x, const PcgScalars *sc) {
  if (is_done(sc)) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    x[i] = omega * (b[i] * dinv[i]);
}

// Gauss-Seidel over the rows of one colour, in place (rows of one colour are
// not coupled): x_i += (b_i - sum_j A_ij x_j) / A_ii
template <int G, class T>
__global__ void k_gs_colour(int nrows, const int32_t *crow, const int64_t *ptr,
                            const int32_t *col, const T *val, const T *dinv, const T *b, T *x,
                            const PcgScalars *sc) {
  if (is_done(sc)) return;
  GROUP_ROWS(G, nrows) {
    int row = valid ? crow[i] : 0;
    T s = valid ? row_dot<G, T, T, T>(ptr, col, val, x, row, g) : (T)0;
    s = group_sum<G>(s);
    if (valid && g == 0) x[row] = fma(b[row] - s, dinv[row], x[row]);
  }
}

// y = A v (Chebyshev products on CSR levels)
template <int G, class T>
__global__ void k_spmv_plain(int n, const int64_t *ptr, const int32_t *col, const T *val,
                             const T *v, T *y, const PcgScalars *sc) {
  if (is_done(sc)) return;
  GROUP_ROWS(G, n) {
    T s = valid ? row_dot<G, T, T, T>(ptr, col, val, v, (int)i, g) : (T)0;
    s = group_sum<G>(s);
    if (valid && g == 0) y[i] = s;
  }
}

// Chebyshev recurrence: start r = D^-1 (b - A x), d = r / theta, x += d;
// step r -= D^-1 (A d), d = c1 d + c2 r, x += d
template <class T>
__global__ void k_cheb_start(int n, const T *b, const T *Ax, const T *dinv, T inv_theta, T *r,
                             T *d, T *x, const PcgScalars *sc) {
  if (is_done(sc)) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    T ri = (Ax ? b[i] - Ax[i] : b[i]) * dinv[i];  // no Ax: x = 0 on entry
    T di = ri * inv_theta;
    r[i] = ri;
    d[i] = di;
    x[i] = Ax ? x[i] + di : di;
  }
}

template <class T>
__global__ void k_cheb_step(int n, const T *Ad, const T *dinv, T c1, T c2, T *r, T *d, T *x,
                            const PcgScalars *sc) {
  if (is_done(sc)) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    T ri = r[i] - Ad[i] * dinv[i];
    T di = fma(c1, d[i], c2 * ri);
    r[i] = ri;
    d[i] = di;
    x[i] = x[i] + di;
  }
}

// Row bodies of the CSR-level V-cycle steps, over the warps w0, w0 + nw, ...
// (a launch's own warps, or every warp of the cooperative coarse tail).
// weighted Jacobi sweep: xn = x + omega D^-1 (b - A x)
template <int G, class T>
__device__ __forceinline__ void jacobi_rows(int64_t w0, int64_t nw, int n, const int64_t *ptr,
                                            const int32_t *col, const T *val, const T *dinv,
                                            T omega, const T *b, const T *x, T *xn) {
  GROUP_ROWS_OVER(G, n, w0, nw) {
    T s = valid ? row_dot<G, T, T, T>(ptr, col, val, x, (int)i, g) : (T)0;
    s = group_sum<G>(s);
    if (valid && g == 0) xn[i] = fma(omega, (b[i] - s) * dinv[i], x[i]);
  }
}

// r = b - A x
template <int G, class T>
__device__ __forceinline__ void resid_rows(int64_t w0, int64_t nw, int n, const int64_t *ptr,
                                           const int32_t *col, const T *val, const T *b,
                                           const T *x, T *r) {
  GROUP_ROWS_OVER(G, n, w0, nw) {
    T s = valid ? row_dot<G, T, T, T>(ptr, col, val, x, (int)i, g) : (T)0;
    s = group_sum<G>(s);
    if (valid && g == 0) r[i] = b[i] - s;
  }
}

template <int G, class T>
__global__ void k_jacobi(int n, const int64_t *ptr, const int32_t *col, const T *val,
                         const T *dinv, T omega, const T *b, const T *x, T *xn,
                         const PcgScalars *sc) {
  if (is_done(sc)) return;
  jacobi_rows<G, T>(HW_WARPS, n, ptr, col, val, dinv, omega, b, x, xn);
}

template <int G, class T>
__global__ void k_resid(int n, const int64_t *ptr, const int32_t *col, const T *val, const T *b,
                        const T *x, T *r, const PcgScalars *sc) {
  if (sc && is_done(sc)) return;
  resid_rows<G, T>(HW_WARPS, n, ptr, col, val, b, x, r);
}

// b_c[a*k+c] = sum_{i in a} P_ic r_i (warp per aggregate, k columns of P per
// aggregate); with xc given, also the coarse level's first Jacobi sweep from
// zero, xc = omega_c b_c / A_c,diag
template <class T>
__device__ __forceinline__ void restrict_aggs(int64_t w, int64_t nw, int na, int k,
                                              const int64_t *mptr, const int32_t *mrow,
                                              const T *P, const T *r, T *bc, const T *dinv_c,
                                              T om_c, T *xc) {
  const int lane = threadIdx.x & 31;
  for (int64_t a = w; a < na; a += nw) {
    for (int c = 0; c < k; ++c) {
      T acc = 0;
      for (int64_t q = mptr[a] + lane; q < mptr[a + 1]; q += 32) {
        int i = mrow[q];
        acc = fma(P[(int64_t)i * k + c], r[i], acc);
      }
      acc = warp_sum(acc);
      if (lane == 0) {
        const int64_t ac = a * k + c;
        bc[ac] = acc;
        if (xc) xc[ac] = om_c * (acc * dinv_c[ac]);
      }
    }
  }
}

// restrict_aggs with one column of P, on P and r stored in member order
// (level 0, matrix-free): the same products in the same order, streamed
template <class T>
__global__ void k_restrict_member(int na, const int64_t *mptr, const T *Pm, const T *rm, T *bc,
                                  const PcgScalars *sc, const T *dinv_c, T om_c, T *xc) {
  if (is_done(sc)) return;
  const int lane = threadIdx.x & 31;
  for (int64_t a = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; a < na;
       a += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    T acc = 0;
    for (int64_t q = mptr[a] + lane; q < mptr[a + 1]; q += 32) acc = fma(Pm[q], rm[q], acc);
    acc = warp_sum(acc);
    if (lane == 0) {
      bc[a] = acc;
      if (xc) xc[a] = om_c * (acc * dinv_c[a]);
    }
  }
}

template <class T>
__global__ void k_restrict(int na, int k, const int64_t *mptr, const int32_t *mrow, const T *P,
                           const T *r, T *bc, const PcgScalars *sc, const T *dinv_c = nullptr,
                           T om_c = 0, T *xc = nullptr) {
  if (is_done(sc)) return;
  restrict_aggs<T>(HW_WARPS, na, k, mptr, mrow, P, r, bc, dinv_c, om_c, xc);
}

// x_i += P_i x_c[agg_i] (rows left alone have no aggregate); each thread
// takes four rows a block-width apart so that its loads are in flight together
constexpr int kProlongRows = 4;
template <class T>
__device__ __forceinline__ void prolong_rows(int64_t blk, int64_t nblk, int n, const int32_t *agg,
                                             const T *P, const T *xc, T *x) {
  const int64_t tile = (int64_t)blockDim.x * kProlongRows;
  for (int64_t base = blk * tile + threadIdx.x; base < n; base += nblk * tile) {
    int a[kProlongRows];
    T p[kProlongRows], xv[kProlongRows];
#pragma unroll
    for (int k = 0; k < kProlongRows; ++k) {
      const int64_t i = base + k * (int64_t)blockDim.x;
      a[k] = i < n ? agg[i] : -1;
    }
#pragma unroll
    for (int k = 0; k < kProlongRows; ++k) {
      const int64_t i = base + k * (int64_t)blockDim.x;
      if (a[k] >= 0) {  // left-alone rows: P_i = 0
        p[k] = P[i];
        xv[k] = x[i];
      }
    }
#pragma unroll
    for (int k = 0; k < kProlongRows; ++k) {
      const int64_t i = base + k * (int64_t)blockDim.x;
      if (a[k] >= 0) x[i] = fma(p[k], xc[a[k]], xv[k]);
    }
  }
}

template <class T>
__global__ void k_prolong(int n, const int32_t *agg, const T *P, const T *xc, T *x,
                          const PcgScalars *sc) {  // one column of P per aggregate
  if (is_done(sc)) return;
  prolong_rows<T>(blockIdx.x, gridDim.x, n, agg, P, xc, x);
}

// x_i += sum_c P_ic x_c[agg_i*k + c], c ascending (k columns of P per aggregate)
template <class T>
__global__ void k_prolong_k(int n, int k, const int32_t *agg, const T *P, const T *xc, T *x,
                            const PcgScalars *sc) {
  if (is_done(sc)) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int a = agg[i];
    if (a < 0) continue;  // left-alone rows: P_i = 0
    T xi = x[i];
    for (int c = 0; c < k; ++c) xi = fma(P[i * k + c], xc[(int64_t)a * k + c], xi);
    x[i] = xi;
  }
}

// coarsest: x = A_c^-1 b with the explicit FP64 inverse (warp per row)
template <class T>
__device__ __forceinline__ void coarse_rows(int64_t w, int64_t nw, int n, const double *inv,
                                            const T *b, T *x) {
  const int lane = threadIdx.x & 31;
  for (int64_t i = w; i < n; i += nw) {
    double acc = 0.0;
    for (int j = lane; j < n; j += 32) acc = fma(inv[i * (int64_t)n + j], widen(b[j]), acc);
    acc = warp_sum(acc);
    if (lane == 0) x[i] = narrow<T>(acc);
  }
}

template <class T>
__global__ void k_coarse_apply(int n, const double *inv, const T *b, T *x, const PcgScalars *sc) {
  if (sc && is_done(sc)) return;
  coarse_rows<T>(HW_WARPS, n, inv, b, x);
}

// ---------------------------------------------------------------------------
// coarsest dense Cholesky (FP64) and explicit inverse
// ---------------------------------------------------------------------------
__global__ void k_dense_fill(int n, const int64_t *ptr, const int32_t *col, const double *val,
                             double *Ad) {
  for (int i = blockIdx.x; i < n; i += gridDim.x)
    for (int64_t k = ptr[i] + threadIdx.x; k < ptr[i + 1]; k += blockDim.x)
      Ad[(int64_t)i * n + col[k]] = val[k];
}

// Tiled over 16 x 16 tiles, one tile per block of 256 threads (one entry per
// thread).  FP64 throughput per SM is low on this part (about 1.6 fused
// multiply-adds per clock), so the n^3 work is spread over many blocks and
// the dependent chains inside a tile are kept short.  Right-looking, for each
// tile column k (Li holds L^-1; its tiles start at zero):
//   panel launch: every block factors the diagonal tile A_kk in shared memory
//     (redundantly, so no block waits on another), getting L_kk and L_kk^-1;
//     blocks below form L_ik = A_ik L_kk^-T, block 0 stores Li_kk = L_kk^-1,
//     and blocks left of the diagonal finish Li_kj = L_kk^-1 S_kj;
//   trailing launch: A_ij -= L_ik L_jk^T right of column k, and the running
//     sums S_ij -= L_ik Li_kj of L^-1's tiles in the rows below k;
// then A^-1 = L^-T L^-1 in one launch, tile (i, j) summing Li_ki^T Li_kj over
// k >= max(i, j) in ascending k (so A^-1 is bitwise symmetric).  Entries
// outside the n x n matrix read as 0 (1 on the diagonal of the last diagonal
// tile), i.e. the factorisation of diag(A, I), whose leading block is A's;
// they are never stored.  A pivot <= 0 sets *status to MGPBD_E_SINGULAR and
// every later launch returns at once.
constexpr int kCT = 16;
constexpr int kCThreads = kCT * kCT;

__device__ __forceinline__ bool chol_failed(const int *status) {
  return *(volatile const int *)status != MGPBD_OK;
}

__device__ __forceinline__ double tile_get(const double *M, int n, int ti, int tj, int r, int c,
                                           bool ident) {
  const int gr = ti * kCT + r, gc = tj * kCT + c;
  if (gr < n && gc < n) return M[(int64_t)gr * n + gc];
  return (ident && gr == gc) ? 1.0 : 0.0;
}

__device__ __forceinline__ void tile_put(double *M, int n, int ti, int tj, int r, int c,
                                         double v) {
  const int gr = ti * kCT + r, gc = tj * kCT + c;
  if (gr < n && gc < n) M[(int64_t)gr * n + gc] = v;
}

// Cholesky of the tile in D (lower part, in place) and, in the same
// right-looking loop, the inverse X of the lower factor (X starts as the
// identity; step j scales row j of X by 1/L_jj and subtracts L_ij times it
// from the rows below).  False on a pivot <= 0 (the same in every thread).
__device__ bool tile_factor(double (*D)[kCT + 1], double (*X)[kCT + 1], double *rinv, int *bad) {
  const int t = threadIdx.x, r = t / kCT, c = t % kCT;
  X[r][c] = r == c ? 1.0 : 0.0;
  for (int j = 0; j < kCT; ++j) {
    if (t == 0) {
      const double d = D[j][j];
      if (!(d > 0.0)) {
        *bad = 1;
      } else {
        const double l = sqrt(d);
        D[j][j] = l;
        *rinv = 1.0 / l;
      }
    }
    __syncthreads();
    if (*bad) return false;
    const double inv = *rinv;
    if (c == j && r > j) D[r][j] = D[r][j] * inv;
    if (r == j && c <= j) X[j][c] = X[j][c] * inv;
    __syncthreads();
    if (c > j && r >= c) D[r][c] = fma(-D[r][j], D[c][j], D[r][c]);
    if (r > j && c <= j) X[r][c] = fma(-D[r][j], X[j][c], X[r][c]);
    __syncthreads();
  }
  return true;
}

// panel of tile column k: blocks 0 .. T-k-1 handle tile rows k .. T-1 of L
// (block 0 stores L_kk^-1 into Li), blocks T-k .. T-1 finish the tiles
// Li_kj, j = 0 .. k-1, of L^-1's row k.  A_kk is read by every block and
// written by none.
__global__ void __launch_bounds__(kCThreads) k_chol_panel(int n, int T, int k, double *A,
                                                          double *Li, int *status) {
  __shared__ double D[kCT][kCT + 1], X[kCT][kCT + 1];
  __shared__ double rinv;
  __shared__ int bad;
  if (chol_failed(status)) return;
  const int t = threadIdx.x, r = t / kCT, c = t % kCT;
  if (t == 0) bad = 0;
  D[r][c] = tile_get(A, n, k, k, r, c, true);
  __syncthreads();
  if (!tile_factor(D, X, &rinv, &bad)) {
    if (blockIdx.x == 0 && t == 0) *status = MGPBD_E_SINGULAR;
    return;
  }
  const int b = blockIdx.x;
  if (b == 0) {
    tile_put(Li, n, k, k, r, c, X[r][c]);
    return;
  }
  if (b < T - k) {  // L_ik = A_ik L_kk^-T, i = k + b
    const int i = k + b;
    D[r][c] = tile_get(A, n, i, k, r, c, false);  // D is free after the factor
    __syncthreads();
    double s = 0.0;
    for (int q = 0; q <= c; ++q) s = fma(D[r][q], X[c][q], s);
    tile_put(A, n, i, k, r, c, s);
    return;
  }
  const int j = b - (T - k);  // Li_kj = L_kk^-1 S_kj
  D[r][c] = tile_get(Li, n, k, j, r, c, false);
  __syncthreads();
  double s = 0.0;
  for (int q = 0; q <= r; ++q) s = fma(X[r][q], D[q][c], s);
  tile_put(Li, n, k, j, r, c, s);
}

// trailing update after tile column k: block (x, y) is tile column x of tile
// row i = k+1+y: A_ix -= L_ik L_xk^T for k < x <= i (blocks with x > i
// return), S_ix -= L_ik Li_kx for x <= k
__global__ void __launch_bounds__(kCThreads) k_chol_trail(int n, int k, double *A, double *Li,
                                                          const int *status) {
  __shared__ double Lr[kCT][kCT + 1], M[kCT][kCT + 1];
  if (chol_failed(status)) return;
  const int i = k + 1 + blockIdx.y, x = blockIdx.x;
  if (x > i) return;
  const int t = threadIdx.x, r = t / kCT, c = t % kCT;
  Lr[r][c] = tile_get(A, n, i, k, r, c, false);
  if (x > k) {
    M[r][c] = tile_get(A, n, x, k, r, c, false);
    __syncthreads();
    double a = tile_get(A, n, i, x, r, c, false);
    for (int q = 0; q < kCT; ++q) a = fma(-Lr[r][q], M[c][q], a);
    tile_put(A, n, i, x, r, c, a);
  } else {
    M[r][c] = tile_get(Li, n, k, x, r, c, false);
    __syncthreads();
    double a = tile_get(Li, n, i, x, r, c, false);
    for (int q = 0; q < kCT; ++q) a = fma(-Lr[r][q], M[q][c], a);
    tile_put(Li, n, i, x, r, c, a);
  }
}

// A^-1 = L^-T L^-1: block (x, y) is tile (y, x)
__global__ void __launch_bounds__(kCThreads) k_inv_gram(int n, int T, const double *Li,
                                                        double *inv, const int *status) {
  __shared__ double Pt[kCT][kCT + 1], Qt[kCT][kCT + 1];
  if (chol_failed(status)) return;
  const int i = blockIdx.y, j = blockIdx.x;
  const int t = threadIdx.x, r = t / kCT, c = t % kCT;
  double s = 0.0;
  for (int k = max(i, j); k < T; ++k) {
    Pt[r][c] = tile_get(Li, n, k, i, r, c, false);
    Qt[r][c] = tile_get(Li, n, k, j, r, c, false);
    __syncthreads();
    for (int q = 0; q < kCT; ++q) s = fma(Pt[q][r], Qt[q][c], s);
    __syncthreads();
  }
  tile_put(inv, n, i, j, r, c, s);
}

mgpbd_status coarsest_factor(Handle *h) {
  if (!h->have_setup || h->m == 0) return MGPBD_OK;
  Level &L = h->lev[h->L - 1];
  int n = L.n;
  if (n > h->cap_nc) {
    h->arena.release(h->cdense);
    h->arena.release(h->cinv);
    MG_TRY(alloc_n(h->arena, &h->cdense, (size_t)n * n));
    MG_TRY(alloc_n(h->arena, &h->cinv, 2 * (size_t)n * n));
    h->cap_nc = n;
    h->gen++;  // captured PCG graphs refer to the old buffers
  }
  h->nc = n;
  MG_CUDA(cudaMemsetAsync(h->cdense, 0, sizeof(double) * (size_t)n * n, h->stream));
  k_dense_fill<<<std::max(1, std::min(n, 4096)), 128, 0, h->stream>>>(n, L.ptr, L.col, L.val,
                                                                      h->cdense);
  MG_LAUNCH("k_dense_fill");
  double *Li = h->cinv + (size_t)n * n;
  MG_CUDA(cudaMemsetAsync(Li, 0, sizeof(double) * (size_t)n * n, h->stream));
  MG_CUDA(cudaMemsetAsync(h->cstat, 0, sizeof(int), h->stream));  // MGPBD_OK
  const int T = (n + kCT - 1) / kCT;
  for (int k = 0; k < T; ++k) {
    k_chol_panel<<<T, kCThreads, 0, h->stream>>>(n, T, k, h->cdense, Li, h->cstat);
    MG_LAUNCH("k_chol_panel");
    if (k + 1 < T) {
      k_chol_trail<<<dim3(T, T - k - 1), kCThreads, 0, h->stream>>>(n, k, h->cdense, Li,
                                                                    h->cstat);
      MG_LAUNCH("k_chol_trail");
    }
  }
  k_inv_gram<<<dim3(T, T), kCThreads, 0, h->stream>>>(n, T, Li, h->cinv, h->cstat);
  MG_LAUNCH("k_inv_gram");
  int st = 0;
  MG_CUDA(cudaMemcpyAsync(h->flag_host, h->cstat, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  MG_CUDA(cudaStreamSynchronize(h->stream));
  st = *h->flag_host;
  if (st != MGPBD_OK) {
    set_error("coarsest Cholesky: non-positive pivot");
    return MGPBD_E_SINGULAR;
  }
  return MGPBD_OK;
}

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------
// Lanes per row.  FP32 kernels are bandwidth-bound and take wide groups for
// coalescing.  FP64 arithmetic runs on few FP64 units on this part, so FP64
// kernels take 4-lane groups: a row of n entries then costs n + 4*2 FP64
// operations instead of n + 32*5 for a full-warp shuffle reduction.
static int group_rule(const Level &L, bool fp64) {
  double avg = L.n ? (double)L.nnz / L.n : 1.0;
  if (fp64) return 4;
  return avg <= 12 ? 4 : (avg <= 24 ? 8 : (avg <= 48 ? 16 : 32));
}

// lanes per row in effect: forced (mgpbd_set_lanes), else autotuned, else the rule
int group_for(const Handle *h, const Level &L, bool fp64) {
  const int f = fp64 ? h->force_csr64 : h->force_csr32;
  if (f) return f;
  int g = fp64 ? L.G64 : L.G32;
  return g ? g : group_rule(L, fp64);
}

static int row_blocks(int64_t rows, int G, int th = 256) {
  int64_t groups_per_block = th / G;
  int64_t b = (rows + groups_per_block - 1) / groups_per_block;
  int cap = 64 * num_sms();
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, cap));
}

#define DISPATCH_G(G, ...)                  \
  switch (G) {                              \
    case 4: { constexpr int GG = 4; __VA_ARGS__; } break;   \
    case 8: { constexpr int GG = 8; __VA_ARGS__; } break;   \
    case 16: { constexpr int GG = 16; __VA_ARGS__; } break; \
    default: { constexpr int GG = 32; __VA_ARGS__; } break; \
  }

template <class T>
static const T *vals(const Level &L);
template <>
const double *vals<double>(const Level &L) { return L.val; }
template <>
const float *vals<float>(const Level &L) { return L.val32; }
template <class T>
static const T *dinvs(const Level &L);
template <>
const double *dinvs<double>(const Level &L) { return L.dinv; }
template <>
const float *dinvs<float>(const Level &L) { return L.dinv32; }
template <class T>
static const T *Ps(const Level &L);
template <>
const double *Ps<double>(const Level &L) { return L.P; }
template <>
const float *Ps<float>(const Level &L) { return L.P32; }


// ---------------------------------------------------------------------------
// the V-cycle below level 0 in one cooperative launch
// ---------------------------------------------------------------------------
// Levels 1 .. coarsest of a V-cycle (weighted Jacobi, one column of P per
// aggregate) are small: as separate launches each step costs a launch's
// latency, not its bytes.  Here every block of one cooperative launch (all
// resident at once) runs the same steps over the same row bodies as the
// separate launches -- pre-sweeps, residual, restriction on the way down, the
// coarsest solve, prolongation and post-sweeps on the way up -- with a grid
// barrier between dependent steps.  No step reduces across rows, so the
// results are the same bits as the separate launches'.
// Grid-wide barrier of a cooperative launch, on one word: thread 0 of block
// 0 adds 2^31 - (blocks - 1), every other block's adds 1, so the top bit of
// the word flips exactly when the last block arrives; each block polls the
// word until its top bit differs from the value it found, at most `limit`
// polls.  False in every thread of a block whose wait ran out (the solve
// then fails with MGPBD_E_DEVICE_TIMEOUT; every other block gives up at its
// next barrier).  The word is reset to 0 between solves.
__device__ bool grid_barrier(unsigned int *bar, long long limit) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int add = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1) : 1u;
    __threadfence();
    const unsigned int old = atomicAdd(bar, add);
    ok = 1;
    long long polls = 0;
    while (((*(volatile unsigned int *)bar ^ old) & 0x80000000u) == 0) {
      if (polls++ >= limit) {
        ok = 0;
        break;
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

template <class T>
__global__ void __launch_bounds__(256) k_coarse_tail(TailDesc<T> d, unsigned int *bar,
                                                      long long limit, PcgScalars *sc) {
  if (is_done(sc)) return;  // the scalars do not change during this kernel
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  auto sync = [&]() -> bool {
    if (grid_barrier(bar, limit)) return true;
    if (threadIdx.x == 0) {
      sc->status = MGPBD_E_DEVICE_TIMEOUT;
      __threadfence();
      sc->done = 1;
    }
    return false;
  };
  T *cur[kMaxLevels];  // the buffer holding each level's iterate
  for (int l = d.first; l < d.coarsest; ++l) {
    const TailLevel<T> &L = d.lev[l];
    T *x = L.x, *x2 = L.x2;  // x holds the first sweep from zero
    for (int s = 1; s < d.sweeps; ++s) {
      DISPATCH_G(L.G, (jacobi_rows<GG, T>(w0, nw, L.n, L.ptr, L.col, L.val, L.dinv, L.omega,
                                          L.b, x, x2)));
      if (!sync()) return;
      T *t = x;
      x = x2;
      x2 = t;
    }
    DISPATCH_G(L.G, (resid_rows<GG, T>(w0, nw, L.n, L.ptr, L.col, L.val, L.b, x, L.r)));
    if (!sync()) return;
    const TailLevel<T> &Lc = d.lev[l + 1];
    const bool c_jac = l + 1 < d.coarsest;  // the coarse level's first sweep rides along
    restrict_aggs<T>(w0, nw, L.n_agg, 1, L.mptr, L.mrow, L.P, L.r, Lc.b,
                     c_jac ? Lc.dinv : nullptr, Lc.omega, c_jac ? Lc.x : nullptr);
    if (!sync()) return;
    cur[l] = x;
  }
  const TailLevel<T> &C = d.lev[d.coarsest];
  coarse_rows<T>(w0, nw, C.n, d.cinv, C.b, C.x);
  const T *xc = C.x;
  for (int l = d.coarsest - 1; l >= d.first; --l) {
    if (!sync()) return;
    const TailLevel<T> &L = d.lev[l];
    T *x = cur[l], *x2 = x == L.x ? L.x2 : L.x;
    prolong_rows<T>(blockIdx.x, gridDim.x, L.n, L.agg, L.P, xc, x);
    for (int s = 0; s < d.sweeps; ++s) {
      if (!sync()) return;
      DISPATCH_G(L.G, (jacobi_rows<GG, T>(w0, nw, L.n, L.ptr, L.col, L.val, L.dinv, L.omega,
                                          L.b, x, x2)));
      T *t = x;
      x = x2;
      x2 = t;
    }
    xc = x;
  }
}

// The tail applies from level `first` down: Jacobi smoothing, one column of
// P per aggregate, at least one level above the coarsest, and a level small
// enough that two blocks per SM cover its rows in about one pass (larger
// levels keep their own full-width launches; the tail then starts below them).
constexpr int kTailMaxRows = 16384;
static bool tail_applies(const Handle *h, int first) {
  return h->tail && h->p.smoother == MGPBD_SMOOTH_JACOBI && h->p.nk_vectors == 1 &&
         h->p.smooth_sweeps >= 1 && first >= 1 && first < h->L - 1 &&
         h->lev[first].n <= kTailMaxRows;
}

// level `first`'s result lies in x after an even number of buffer swaps (2
// sweeps - 1 of them), else in x2
template <class T>
static T *tail_result(Handle *h, int first) {
  Level &L = h->lev[first];
  return (T *)((2 * h->p.smooth_sweeps - 1) % 2 == 0 ? L.x : L.x2);
}

template <class T>
static mgpbd_status launch_tail(Handle *h, int first) {
  TailDesc<T> d;
  memset(&d, 0, sizeof(d));
  d.first = first;
  d.coarsest = h->L - 1;
  d.sweeps = h->p.smooth_sweeps;
  d.cinv = h->cinv;
  for (int l = first; l <= d.coarsest; ++l) {
    const Level &L = h->lev[l];
    TailLevel<T> &t = d.lev[l];
    t.n = L.n;
    t.G = group_for(h, L, sizeof(T) == 8);
    t.n_agg = L.n_agg;
    t.omega = (T)L.omega;
    t.ptr = L.ptr;
    t.col = L.col;
    t.val = vals<T>(L);
    t.dinv = dinvs<T>(L);
    t.x = (T *)L.x;
    t.x2 = (T *)L.x2;
    t.b = (T *)L.b;
    t.r = (T *)L.r;
    t.agg = L.agg;
    t.P = Ps<T>(L);
    t.mptr = L.mptr;
    t.mrow = L.mrow;
  }
  // at most two blocks per SM: every barrier waits for each block
  const int blocks = std::min(wave_blocks((const void *)k_coarse_tail<T>, 256), 2 * num_sms());
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(256);
  cfg.stream = h->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  MG_CUDA(cudaLaunchKernelEx(&cfg, k_coarse_tail<T>, d, h->gbar, h->wait_limit, h->sc));
  MG_LAUNCH("k_coarse_tail");
  return MGPBD_OK;
}

// ---------------------------------------------------------------------------
// batched PCG of a cohort: every step one launch for every member
// ---------------------------------------------------------------------------
#define COHORT_BLOCK                                                              \
  const CohortBlock cb_ = blk[blockIdx.x];                                        \
  if (is_done(cb_.sc)) return;                                                    \
  const CohortMember &M = mem[cb_.k];                                             \
  const int vb = cb_.vb, vn = cb_.vn

__global__ void kb_xr(const CohortMember *mem, const CohortBlock *blk) {
  COHORT_BLOCK;
  xr_update_body<float>(vb, vn, M.m, M.x, M.r, M.p, M.q, M.c_rr, M.b0, M.dinv0, M.om0, M.x0);
}

__global__ void kb_restrict0(const CohortMember *mem, const CohortBlock *blk) {
  COHORT_BLOCK;
  const TailLevel<float> &L1 = M.tail.lev[1];
  const bool c_jac = M.tail.coarsest > 1;  // level 1 smooths: its first sweep rides along
  restrict_aggs<float>(VG_WARPS(vb, vn), M.n_agg0, 1, M.mptr0, M.mrow0, M.P0, M.r0, L1.b,
                       c_jac ? L1.dinv : nullptr, L1.omega, c_jac ? L1.x : nullptr);
}

__global__ void kb_prolong0(const CohortMember *mem, const CohortBlock *blk) {
  COHORT_BLOCK;
  prolong_rows<float>(vb, vn, M.m, M.agg0, M.P0, M.xc1, M.x20);
}

__global__ void kb_pupdate(const CohortMember *mem, const CohortBlock *blk) {
  COHORT_BLOCK;
  p_update_body(vb, vn, M.m, M.p, M.z, M.sc);
}

// The V-cycle below level 0 of every member in one cooperative launch, depth
// by depth: at depth d the members whose coarsest level is deeper pre-smooth,
// take the residual and restrict; a member whose coarsest level is d solves
// it there; on the way back up each member prolongs and post-smooths its
// levels.  The warps (and, for the prolongation, the blocks) are split among
// the members in contiguous shares, so each warp reads one member's record and
// works only on its rows, and the members' small levels run side by side.  A
// member's own steps run in its standalone order over the same row bodies
// (no row's arithmetic depends on the warp that takes it), so its results are
// its standalone bits.
__global__ void __launch_bounds__(256) kb_tail(const CohortMember *mem, int K, int maxc,
                                                unsigned int *bar, long long limit) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  // this warp's member, its index among the member's warps and their number
  const int k = (int)((w * K) / nw);
  const int64_t w_lo = ((int64_t)k * nw + K - 1) / K, w_hi = ((int64_t)(k + 1) * nw + K - 1) / K;
  const int64_t lw = w - w_lo, nlw = w_hi - w_lo;
  // the same split of the blocks for the prolongation
  const int kb = (int)(((int64_t)blockIdx.x * K) / gridDim.x);
  const int64_t b_lo = ((int64_t)kb * gridDim.x + K - 1) / K,
                b_hi = ((int64_t)(kb + 1) * gridDim.x + K - 1) / K;
  unsigned long long act = 0;  // members still iterating (the same in every block)
  for (int j = 0; j < K; ++j)
    if (!is_done(mem[j].sc)) act |= 1ull << j;
  if (!act) return;
  auto sync = [&]() -> bool {
    if (grid_barrier(bar, limit)) return true;
    if (threadIdx.x == 0)
      for (int j = 0; j < K; ++j)
        if (act >> j & 1) {
          mem[j].sc->status = MGPBD_E_DEVICE_TIMEOUT;
          __threadfence();
          mem[j].sc->done = 1;
        }
    return false;
  };
  const bool mine = act >> k & 1;           // this warp's member iterates
  const TailDesc<float> &T = mem[k].tail;  // its levels
  const int ck = T.coarsest;
  const bool mine_b = act >> kb & 1;
  const TailDesc<float> &Tb = mem[kb].tail;
  auto jacobi = [&](const TailLevel<float> &L, const float *x, float *xn) {
    DISPATCH_G(L.G, (jacobi_rows<GG, float>(lw, nlw, L.n, L.ptr, L.col, L.val, L.dinv, L.omega,
                                            L.b, x, xn)));
  };
  for (int d = 1; d <= maxc; ++d) {
    if (mine && d < ck) jacobi(T.lev[d], T.lev[d].x, T.lev[d].x2);  // the pre-sweep after the first
    if (!sync()) return;
    if (mine && d < ck) {
      const TailLevel<float> &L = T.lev[d];
      DISPATCH_G(L.G, (resid_rows<GG, float>(lw, nlw, L.n, L.ptr, L.col, L.val, L.b, L.x2, L.r)));
    } else if (mine && d == ck) {
      coarse_rows<float>(lw, nlw, T.lev[d].n, T.cinv, T.lev[d].b, T.lev[d].x);
    }
    if (!sync()) return;
    if (d == maxc) break;
    if (mine && d < ck) {
      const TailLevel<float> &L = T.lev[d], &Lc = T.lev[d + 1];
      const bool c_jac = d + 1 < ck;
      restrict_aggs<float>(lw, nlw, L.n_agg, 1, L.mptr, L.mrow, L.P, L.r, Lc.b,
                           c_jac ? Lc.dinv : nullptr, Lc.omega, c_jac ? Lc.x : nullptr);
    }
    if (!sync()) return;
  }
  for (int d = maxc - 1; d >= 1; --d) {
    if (mine_b && d < Tb.coarsest) {
      const TailLevel<float> &L = Tb.lev[d], &Lc = Tb.lev[d + 1];
      const float *xc = d + 1 == Tb.coarsest ? Lc.x : Lc.x2;  // the coarser level's result
      prolong_rows<float>(blockIdx.x - b_lo, b_hi - b_lo, L.n, L.agg, L.P, xc, L.x2);
    }
    if (!sync()) return;
    for (int s = 0; s < 2; ++s) {
      if (mine && d < ck)
        jacobi(T.lev[d], s == 0 ? T.lev[d].x2 : T.lev[d].x, s == 0 ? T.lev[d].x : T.lev[d].x2);
      if ((d > 1 || s == 0) && !sync()) return;
    }
  }
}

__global__ void kb_gather(const CohortMember *mem, int K, PcgScalars *out) {
  for (int k = threadIdx.x; k < K; k += blockDim.x) out[k] = *mem[k].sc;
}

// ---- host side -------------------------------------------------------------
bool cohort_eligible(const Handle *h) {
  const mgpbd_params &p = h->p;
  return p.precision == MGPBD_MIXED && p.level0_op == 1 && !p.ap_split &&
         p.smoother == MGPBD_SMOOTH_JACOBI &&
         p.smooth_sweeps == 2 && p.nk_vectors == 1 && p.linear_solver == 0 && h->have_setup &&
         h->L >= 2 && h->m > 0;
}

Cohort::~Cohort() {
  if (graph) cudaGraphExecDestroy(graph);
  if (d_mem) cudaFree(d_mem);
  if (d_blk) cudaFree(d_blk);
  if (d_sc) cudaFree(d_sc);
  if (bar) cudaFree(bar);
  if (h_sc) cudaFreeHost(h_sc);
}

// Member records and block tables for the handles in c->hs (all eligible,
// all on c->stream).  Rebuilt when a member joins or leaves or its device
// arrays change (a new setup).
mgpbd_status cohort_build(Cohort *c) {
  const int K = (int)c->hs.size();
  if (K > kCohortMax) {
    set_error("cohort: more than 64 instances");
    return MGPBD_E_INVALID;
  }
  if (K > c->cap) {
    if (c->d_mem) cudaFree(c->d_mem);
    if (c->d_sc) cudaFree(c->d_sc);
    if (c->h_sc) cudaFreeHost(c->h_sc);
    c->d_mem = nullptr;
    c->d_sc = nullptr;
    c->h_sc = nullptr;
    c->cap = 0;
    MG_CUDA(cudaMalloc(&c->d_mem, sizeof(CohortMember) * kCohortMax));
    MG_CUDA(cudaMalloc(&c->d_sc, sizeof(PcgScalars) * kCohortMax));
    MG_CUDA(cudaMallocHost(&c->h_sc, sizeof(PcgScalars) * kCohortMax));
    c->cap = kCohortMax;
  }
  if (!c->bar) {
    MG_CUDA(cudaMalloc(&c->bar, 16 * sizeof(unsigned int)));
    MG_CUDA(cudaMemsetAsync(c->bar, 0, 16 * sizeof(unsigned int), c->stream));
  }
  std::vector<CohortMember> mem((size_t)K);
  c->maxc = 1;
  c->gens.assign(K, 0);
  for (int k = 0; k < K; ++k) {
    Handle *h = c->hs[k];
    CohortMember &M = mem[k];
    memset(&M, 0, sizeof(M));
    const Level &L0 = h->lev[0];
    M.m = h->m;
    M.N = h->N;
    M.E = h->E;
    M.gv64 = h->force_vert64 ? h->force_vert64 : h->mf_g64;
    M.gv32 = h->force_vert32 ? h->force_vert32 : h->mf_g32;
    M.edge = h->edge;
    M.tet = h->tet;
    M.vorder = h->vorder;
    M.vptr = h->vptr;
    M.vrow = h->vrow;
    M.ginc64 = h->ginc64;
    M.w = h->w;
    M.gd = h->gd;
    M.gt = h->gt;
    M.at = h->alpha_t;
    M.ginc4 = h->ginc4;
    M.w32 = h->w32;
    M.gd32 = h->gd32;
    M.gt32 = h->gt32;
    M.at32 = h->at32;
    M.u64 = h->u64;
    M.u32 = h->u32;
    M.x = h->dl;
    M.r = h->pr;
    M.z = h->pz;
    M.p = h->pp;
    M.q = h->pq;
    M.sc = h->sc;
    M.c_pq = make_ctx(h, DOT_PQ);
    M.c_rr = make_ctx(h, DOT_RR);
    M.c_rz = make_ctx(h, DOT_RZ);
    M.b0 = (float *)L0.b;
    M.x0 = (float *)L0.x;
    M.x20 = (float *)L0.x2;
    M.r0 = (float *)L0.r;
    M.dinv0 = L0.dinv32;
    M.om0 = (float)L0.omega;
    M.n_agg0 = L0.n_agg;
    M.mptr0 = L0.mptr;
    M.mrow0 = L0.mrow;
    M.P0 = L0.P32;
    M.agg0 = L0.agg;
    TailDesc<float> &T = M.tail;
    T.first = 1;
    T.coarsest = h->L - 1;
    T.sweeps = h->p.smooth_sweeps;
    T.cinv = h->cinv;
    for (int l = 1; l <= T.coarsest; ++l) {
      const Level &L = h->lev[l];
      TailLevel<float> &t = T.lev[l];
      t.n = L.n;
      t.G = group_for(h, L, false);
      t.n_agg = L.n_agg;
      t.omega = (float)L.omega;
      t.ptr = L.ptr;
      t.col = L.col;
      t.val = L.val32;
      t.dinv = L.dinv32;
      t.x = (float *)L.x;
      t.x2 = (float *)L.x2;
      t.b = (float *)L.b;
      t.r = (float *)L.r;
      t.agg = L.agg;
      t.P = L.P32;
      t.mptr = L.mptr;
      t.mrow = L.mrow;
    }
    M.xc1 = T.coarsest > 1 ? T.lev[1].x2 : T.lev[1].x;
    c->maxc = std::max(c->maxc, T.coarsest);
    mf_cohort_grids(h, M.grid);
    const int m = h->m;
    M.grid[CS_XR] = std::min(dot_grid(m), wave_blocks((const void *)k_xr_update<float>, kDotThreads));
    M.grid[CS_RESTRICT] = blocks_for((int64_t)L0.n_agg * 32, 256);
    M.grid[CS_PROLONG] = blocks_for((m + kProlongRows - 1) / kProlongRows, 256);
    M.grid[CS_PUPD] = blocks_for(std::max(1, (m / 2 + 1) / 2), 256);
    c->gens[k] = h->gen;
  }
  c->gv32 = mem.empty() ? 0 : mem[0].gv32;
  for (const CohortMember &M : mem)
    if (M.gv32 != c->gv32) c->gv32 = 0;
  // per step, each member's blocks in member order: (member, index, count)
  std::vector<CohortBlock> blk;
  for (int s = 0; s < CS_STEPS; ++s) {
    c->blk_off[s] = (int)blk.size();
    for (int k = 0; k < K; ++k)
      for (int b = 0; b < mem[k].grid[s]; ++b)
        blk.push_back(CohortBlock{k, b, mem[k].grid[s], 0, mem[k].sc, nullptr});
    c->blocks[s] = (int)blk.size() - c->blk_off[s];
  }
  if (blk.size() > c->blk_cap) {
    if (c->d_blk) cudaFree(c->d_blk);
    c->d_blk = nullptr;
    c->blk_cap = 0;
    MG_CUDA(cudaMalloc(&c->d_blk, sizeof(CohortBlock) * blk.size()));
    c->blk_cap = blk.size();
  }
  MG_CUDA(cudaMemcpyAsync(c->d_mem, mem.data(), sizeof(CohortMember) * K, cudaMemcpyHostToDevice,
                          c->stream));
  MG_CUDA(cudaMemcpyAsync(c->d_blk, blk.data(), sizeof(CohortBlock) * blk.size(),
                          cudaMemcpyHostToDevice, c->stream));
  MG_CUDA(cudaStreamSynchronize(c->stream));
  c->K = K;
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  return MGPBD_OK;
}

// true when a member's device arrays changed since the build
bool cohort_stale(const Cohort *c) {
  if ((int)c->hs.size() != c->K) return true;
  for (int k = 0; k < c->K; ++k)
    if (c->gens[k] != c->hs[k]->gen) return true;
  return false;
}

// one batched PCG iteration (the launch sequence of pcg_iteration for the
// configuration every member has)
static mgpbd_status cohort_iteration(Cohort *c) {
  const int K = c->K;
  cudaStream_t st = c->stream;
  const CohortMember *m = c->d_mem;
  auto blk = [&](int step) { return c->d_blk + c->blk_off[step]; };
  auto mf = [&](int step, int sel) {
    return mf_cohort_step(step, sel, m, blk(step), c->blocks[step], c->gv32, st);
  };
  MG_TRY(mf(CS_VERT64, 0));
  MG_TRY(mf(CS_ROW_PQ, 0));
  kb_xr<<<c->blocks[CS_XR], kDotThreads, 0, st>>>(m, blk(CS_XR));
  MG_LAUNCH("kb_xr");
  MG_TRY(mf(CS_VERT32, 0));
  MG_TRY(mf(CS_ROW, 0));
  MG_TRY(mf(CS_VERT32, 1));
  MG_TRY(mf(CS_ROW, 1));
  kb_restrict0<<<c->blocks[CS_RESTRICT], 256, 0, st>>>(m, blk(CS_RESTRICT));
  MG_LAUNCH("kb_restrict0");
  {
    const int blocks = std::min(wave_blocks((const void *)kb_tail, 256), 2 * num_sms());
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(256);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    MG_CUDA(cudaLaunchKernelEx(&cfg, kb_tail, m, K, c->maxc, c->bar, c->wait_limit));
    MG_LAUNCH("kb_tail");
  }
  kb_prolong0<<<c->blocks[CS_PROLONG], 256, 0, st>>>(m, blk(CS_PROLONG));
  MG_LAUNCH("kb_prolong0");
  MG_TRY(mf(CS_VERT32, 1));
  MG_TRY(mf(CS_ROW, 2));
  MG_TRY(mf(CS_VERT32, 0));
  MG_TRY(mf(CS_ROW_FINAL, 0));
  kb_pupdate<<<c->blocks[CS_PUPD], 256, 0, st>>>(m, blk(CS_PUPD));
  MG_LAUNCH("kb_pupdate");
  return MGPBD_OK;
}

// `iters` batched PCG iterations of every member (captured into a CUDA graph
// once per build and replayed), then every member's scalars into c->h_sc
// (synchronises)
mgpbd_status cohort_chunk(Cohort *c, int iters) {
  if (c->K == 0) return MGPBD_OK;
  if (!c->graph || c->graph_iters != iters) {
    if (c->graph) {
      cudaGraphExecDestroy(c->graph);
      c->graph = nullptr;
    }
    cudaGraph_t gr = nullptr;
    unsigned long long n0 = __atomic_load_n(&g_launches, __ATOMIC_RELAXED);
    MG_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    mgpbd_status cs = MGPBD_OK;
    for (int k = 0; k < iters && cs >= 0; ++k) cs = cohort_iteration(c);
    cudaError_t ce = cudaStreamEndCapture(c->stream, &gr);
    c->graph_kernels = __atomic_load_n(&g_launches, __ATOMIC_RELAXED) - n0;
    __atomic_fetch_sub(&g_launches, c->graph_kernels, __ATOMIC_RELAXED);
    if (cs < 0) {
      if (gr) cudaGraphDestroy(gr);
      return cs;
    }
    MG_CUDA(ce);
    ce = cudaGraphInstantiate(&c->graph, gr, 0);
    cudaGraphDestroy(gr);
    MG_CUDA(ce);
    c->graph_iters = iters;
  }
  MG_CUDA(cudaGraphLaunch(c->graph, c->stream));
  __atomic_fetch_add(&g_launches, c->graph_kernels, __ATOMIC_RELAXED);
  kb_gather<<<1, 64, 0, c->stream>>>(c->d_mem, c->K, c->d_sc);
  MG_LAUNCH("kb_gather");
  MG_CUDA(cudaMemcpyAsync(c->h_sc, c->d_sc, sizeof(PcgScalars) * c->K, cudaMemcpyDeviceToHost,
                          c->stream));
  MG_CUDA(cudaStreamSynchronize(c->stream));
  return MGPBD_OK;
}

// V-cycle on level l in precision T: L.b -> L.x (zero start).  On level 0 of
// a top V-cycle, `x0_ready` says the first Jacobi sweep is already in L.x,
// and `top` lets the last matrix-free sweep write z in FP64 (and r.z)
// instead of L.x; `*z_written` then reports that it did.
template <class T>
static mgpbd_status vcycle_level(Handle *h, int l, const T *b_in, bool x0_ready = false,
                                 const TopOut *top = nullptr, bool *z_written = nullptr) {
  Level &L = h->lev[l];
  const PcgScalars *sc = h->sc;
  const int n = L.n;
  T *x = (T *)L.x;
  if (l == h->L - 1) {
    k_coarse_apply<T><<<blocks_for((int64_t)n * 32, 256), 256, 0, h->stream>>>(n, h->cinv, b_in, x,
                                                                                sc);
    MG_LAUNCH("k_coarse_apply");
    return MGPBD_OK;
  }
  const int G = group_for(h, L, sizeof(T) == 8);
  const T om = (T)L.omega;
  const T *val = vals<T>(L);
  const T *dinv = dinvs<T>(L);
  T *x2 = (T *)L.x2, *r = (T *)L.r;
  const bool mf = l == 0 && h->p.level0_op == 1;  // matrix-free level-0 products
  const bool gs = h->p.smoother == MGPBD_SMOOTH_MCGS;
  // multicolour Gauss-Seidel: forward colours before the coarse correction,
  // reverse colours after (symmetric smoothing, Sec. 4.5)
  auto gs_sweeps = [&](bool reverse) -> mgpbd_status {
    const int nc = L.n_colors;
    for (int s = 0; s < h->p.smooth_sweeps; ++s)
      for (int k = 0; k < nc; ++k) {
        int c = reverse ? nc - 1 - k : k;
        int64_t off = L.hcptr[c], cnt = L.hcptr[c + 1] - off;
        if (cnt == 0) continue;
        DISPATCH_G(G, (k_gs_colour<GG, T><<<row_blocks(cnt, GG), 256, 0, h->stream>>>(
                          (int)cnt, L.crow + off, L.ptr, L.col, val, dinv, b_in, x, sc)));
        MG_LAUNCH("k_gs_colour");
      }
    return MGPBD_OK;
  };
  // Chebyshev smoother on [lambda_min_est, safety * lambda_max] with
  // smooth_sweeps products; coefficients follow from the lazily estimated
  // lambda_max of the setup (Sec. 4.5)
  const bool cheb = h->p.smoother == MGPBD_SMOOTH_CHEBYSHEV;
  auto apply = [&](const T *v, T *y) -> mgpbd_status {
    if (mf) return mf_level0<T>(h, kMfApply, v, b_in, dinv, om, y);
    DISPATCH_G(G, (k_spmv_plain<GG, T><<<row_blocks(n, GG), 256, 0, h->stream>>>(
                      n, L.ptr, L.col, val, v, y, sc)));
    MG_LAUNCH("k_spmv_plain");
    return MGPBD_OK;
  };
  // (from_zero: x = 0 on entry, so A x = 0 needs no product)
  auto cheb_smooth = [&](bool from_zero) -> mgpbd_status {
    const double lo = h->p.lambda_min_est, hi = h->p.power_safety * L.lmax;
    const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
    double rho = 1.0 / sigma;
    T *t = (T *)L.t, *d = x2;
    if (!from_zero) MG_TRY(apply(x, t));
    k_cheb_start<T><<<blocks_for(n, 256), 256, 0, h->stream>>>(
        n, b_in, from_zero ? nullptr : t, dinv, (T)(1.0 / theta), r, d, x, sc);
    MG_LAUNCH("k_cheb_start");
    for (int k = 1; k < h->p.smooth_sweeps; ++k) {
      MG_TRY(apply(d, t));
      double rho2 = 1.0 / (2.0 * sigma - rho);
      k_cheb_step<T><<<blocks_for(n, 256), 256, 0, h->stream>>>(
          n, t, dinv, (T)(rho2 * rho), (T)(2.0 * rho2 / delta), r, d, x, sc);
      MG_LAUNCH("k_cheb_step");
      rho = rho2;
    }
    return MGPBD_OK;
  };
  if (cheb) {
    MG_TRY(cheb_smooth(true));
  } else if (gs) {
    MG_CUDA(cudaMemsetAsync(x, 0, sizeof(T) * n, h->stream));
    MG_TRY(gs_sweeps(false));
  } else if (!x0_ready) {
    k_jacobi0<T><<<blocks_for(n, 256), 256, 0, h->stream>>>(n, b_in, dinv, om, x, sc);
    MG_LAUNCH("k_jacobi0");
  }
  for (int s = 1; s < h->p.smooth_sweeps && !gs && !cheb; ++s) {
    if (l == 0) MG_TRY(prof_begin(h));
    if (mf) {
      MG_TRY(mf_level0<T>(h, kMfSweep, x, b_in, dinv, om, x2));
    } else {
      DISPATCH_G(G, (k_jacobi<GG, T><<<row_blocks(n, GG), 256, 0, h->stream>>>(
                        n, L.ptr, L.col, val, dinv, om, b_in, x, x2, sc)));
      MG_LAUNCH("k_jacobi");
    }
    if (l == 0) MG_TRY(prof_end(h));
    std::swap(x, x2);
  }
  Level &Lc = h->lev[l + 1];
  // the coarse level's first Jacobi sweep from zero rides on the restriction
  const bool c_jac = !gs && !cheb && l + 2 < h->L;
  const int nk = h->p.nk_vectors;
  if (mf && L.mpos && nk == 1) {
    // the residual written in member order, the restriction streaming it
    MG_TRY(mf_level0<T>(h, kMfResidMember, x, b_in, dinv, om, r));
    k_restrict_member<T><<<blocks_for((int64_t)L.n_agg * 32, 256), 256, 0, h->stream>>>(
        L.n_agg, L.mptr, (const T *)L.Pm, r, (T *)Lc.b, sc, c_jac ? dinvs<T>(Lc) : nullptr,
        (T)Lc.omega, c_jac ? (T *)Lc.x : nullptr);
    MG_LAUNCH("k_restrict_member");
  } else if (mf) {
    MG_TRY(mf_level0<T>(h, kMfResid, x, b_in, dinv, om, r));
    k_restrict<T><<<blocks_for((int64_t)L.n_agg * 32, 256), 256, 0, h->stream>>>(
        L.n_agg, nk, L.mptr, L.mrow, Ps<T>(L), r, (T *)Lc.b, sc, c_jac ? dinvs<T>(Lc) : nullptr,
        (T)Lc.omega, c_jac ? (T *)Lc.x : nullptr);
    MG_LAUNCH("k_restrict");
  } else {
    DISPATCH_G(G, (k_resid<GG, T><<<row_blocks(n, GG), 256, 0, h->stream>>>(n, L.ptr, L.col, val,
                                                                           b_in, x, r, sc)));
    MG_LAUNCH("k_resid");
    k_restrict<T><<<blocks_for((int64_t)L.n_agg * 32, 256), 256, 0, h->stream>>>(
        L.n_agg, nk, L.mptr, L.mrow, Ps<T>(L), r, (T *)Lc.b, sc, c_jac ? dinvs<T>(Lc) : nullptr,
        (T)Lc.omega, c_jac ? (T *)Lc.x : nullptr);
    MG_LAUNCH("k_restrict");
  }
  const T *xc = (const T *)Lc.x;  // where the coarser level leaves its result
  if (tail_applies(h, l + 1)) {
    MG_TRY(launch_tail<T>(h, l + 1));
    xc = tail_result<T>(h, l + 1);
  } else {
    MG_TRY(vcycle_level<T>(h, l + 1, (const T *)Lc.b, c_jac));
  }
  if (nk == 1)
    k_prolong<T><<<blocks_for((n + kProlongRows - 1) / kProlongRows, 256), 256, 0, h->stream>>>(
        n, L.agg, Ps<T>(L), xc, x, sc);
  else
    k_prolong_k<T><<<blocks_for(n, 256), 256, 0, h->stream>>>(n, nk, L.agg, Ps<T>(L),
                                                              (const T *)Lc.x, x, sc);
  MG_LAUNCH("k_prolong");
  if (gs) MG_TRY(gs_sweeps(true));
  if (cheb) MG_TRY(cheb_smooth(false));
  bool zw = false;
  for (int s = 0; s < h->p.smooth_sweeps && !gs && !cheb; ++s) {
    if (mf && top && s + 1 == h->p.smooth_sweeps) {
      MG_TRY(mf_level0_final<T>(h, x, b_in, dinv, om, *top));
      zw = true;
      break;
    }
    if (l == 0) MG_TRY(prof_begin(h));
    if (mf) {
      MG_TRY(mf_level0<T>(h, kMfSweep, x, b_in, dinv, om, x2));
    } else {
      DISPATCH_G(G, (k_jacobi<GG, T><<<row_blocks(n, GG), 256, 0, h->stream>>>(
                        n, L.ptr, L.col, val, dinv, om, b_in, x, x2, sc)));
      MG_LAUNCH("k_jacobi");
    }
    if (l == 0) MG_TRY(prof_end(h));
    std::swap(x, x2);
  }
  if (z_written) *z_written = zw;
  if (x != (T *)L.x && !zw) {  // keep the result in L.x
    MG_CUDA(cudaMemcpyAsync(L.x, x, sizeof(T) * n, cudaMemcpyDeviceToDevice, h->stream));
  }
  return MGPBD_OK;
}

static mgpbd_status launch_dot(Handle *h, const double *x, const double *y, int64_t n, int mode,
                               int check_done, double *out = nullptr) {
  DotCtx c = make_ctx(h, mode, out);
  k_dot<<<std::min(dot_grid(n), wave_blocks((const void *)k_dot, kDotThreads)), kDotThreads, 0,
          h->stream>>>(n, x, y, c, check_done);
  MG_LAUNCH("k_dot");
  return MGPBD_OK;
}

// level 0 starts its V-cycle with a Jacobi sweep from zero (not the coarsest)
static bool top_jacobi(const Handle *h) {
  return h->p.smoother == MGPBD_SMOOTH_JACOBI && h->L > 1 && h->p.smooth_sweeps >= 1;
}

// z = V(r) on level 0, FP64 in and out.  `prepared`: the PCG update already
// wrote the V-cycle's right-hand side in its precision and, with the Jacobi
// smoother, the first sweep (k_xr_update).  dot_mode >= 0 folds r.z into the
// PCG scalars, inside the last matrix-free sweep when there is one.
static mgpbd_status vcycle_top(Handle *h, const double *r, double *z, bool prepared,
                               int dot_mode) {
  Level &L = h->lev[0];
  const int m = h->m;
  const bool jac = top_jacobi(h);
  TopOut o;
  o.r = r;
  o.z = z;
  o.dot = dot_mode >= 0;
  o.c = make_ctx(h, o.dot ? dot_mode : DOT_STORE);
  bool zw = false;
  if (h->p.precision == MGPBD_MIXED) {
    if (!prepared) {
      k_top_prep<float><<<blocks_for(m, 256), 256, 0, h->stream>>>(
          m, r, (float *)L.b, L.dinv32, (float)L.omega, jac ? (float *)L.x : nullptr, h->sc);
      MG_LAUNCH("k_top_prep");
    }
    MG_TRY(vcycle_level<float>(h, 0, (const float *)L.b, jac, &o, &zw));
    if (!zw) {
      k_convert<float, double><<<blocks_for(m, 256), 256, 0, h->stream>>>(m, (const float *)L.x,
                                                                          z, h->sc);
      MG_LAUNCH("k_convert");
    }
  } else {
    if (!prepared && jac) {
      k_top_prep<double><<<blocks_for(m, 256), 256, 0, h->stream>>>(m, r, nullptr, L.dinv, L.omega,
                                                                    (double *)L.x, h->sc);
      MG_LAUNCH("k_top_prep");
    }
    MG_TRY(vcycle_level<double>(h, 0, r, jac, &o, &zw));
    if (!zw) {
      k_convert<double, double><<<blocks_for(m, 256), 256, 0, h->stream>>>(
          m, (const double *)L.x, z, h->sc);
      MG_LAUNCH("k_convert");
    }
  }
  if (o.dot && !zw) MG_TRY(launch_dot(h, r, z, m, dot_mode, 1));
  return MGPBD_OK;
}

mgpbd_status vcycle_apply(Handle *h, const double *d_r, double *d_z) {
  k_pcg_init<<<1, 1, 0, h->stream>>>(h->sc, h->gbar);
  MG_LAUNCH("k_pcg_init");
  return vcycle_top(h, d_r, d_z, false, -1);
}

// y = A x at level 0 in one of the forms of the PCG recurrence's product:
// 0 FP64 CSR, 1 FP64 matrix-free, 2 matrix-free from float-float pairs
mgpbd_status apply_level0(Handle *h, int form, const double *x, double *y) {
  const int m = h->m;
  const Level &L = h->lev[0];
  k_pcg_init<<<1, 1, 0, h->stream>>>(h->sc, h->gbar);
  MG_LAUNCH("k_pcg_init");
  DotCtx c = make_ctx(h, DOT_STORE, &h->sc->tr2);  // x.Ax lands in a scratch scalar
  if (form == 0) {
    const int G = group_for(h, L, true);
    DISPATCH_G(G, (k_spmv_pq<GG, double, double>
                   <<<std::min(row_blocks(m, GG),
                               wave_blocks((const void *)k_spmv_pq<GG, double, double>, 256)),
                      256, 0, h->stream>>>(m, L.ptr, L.col, L.val, x, y, c)));
    MG_LAUNCH("k_spmv_pq");
    return MGPBD_OK;
  }
  if (form == 2) MG_TRY(mf_split(h, x, h->p_df, m));
  return mf_apply_pq_form(h, form == 2, x, y, c);
}

mgpbd_status dot_dd(Handle *h, const double *x, const double *y, int64_t n, double *d_out) {
  return launch_dot(h, x, y, n, DOT_STORE, 0, d_out);
}

// one PCG iteration (kernels return early once `done` is set)
static mgpbd_status pcg_iteration(Handle *h, double *x) {
  Level &L = h->lev[0];
  const int m = h->m;
  double *r = h->pr, *z = h->pz, *p = h->pp, *q = h->pq;
  const int G = group_for(h, L, true);
  DotCtx cpq = make_ctx(h, DOT_PQ);
  // A.p is part of the Krylov recurrence, not of the preconditioner, and stays
  // FP64 in both modes: rounding A's values to FP32 perturbs entries of size
  // ~1e4 by ~1e-3, far above alpha~ (~1e-7), and the FP32 operator is then
  // numerically indefinite on the stiff workloads (p.Ap <= 0).
  // (params.ap_split: the matrix-free product from float-float pairs, with
  // residual replacement in pcg_solve)
  MG_TRY(prof_begin(h, PROF_AP));
  if (h->p.level0_op == 1) {
    MG_TRY(mf_apply_pq(h, p, q, cpq));
  } else {
    DISPATCH_G(G, (k_spmv_pq<GG, double, double>
                   <<<std::min(row_blocks(m, GG),
                               wave_blocks((const void *)k_spmv_pq<GG, double, double>, 256)),
                      256, 0, h->stream>>>(m, L.ptr, L.col, L.val, p, q, cpq)));
    MG_LAUNCH("k_spmv_pq");
  }
  MG_TRY(prof_end(h, PROF_AP));
  // the update also starts the V-cycle (right-hand side, first Jacobi sweep)
  const bool jac = top_jacobi(h);
  if (h->p.precision == MGPBD_MIXED)
    k_xr_update<float><<<std::min(dot_grid(m), wave_blocks((const void *)k_xr_update<float>,
                                                           kDotThreads)),
                         kDotThreads, 0, h->stream>>>(
        m, x, r, p, q, make_ctx(h, DOT_RR), (float *)L.b, L.dinv32, (float)L.omega,
        jac ? (float *)L.x : nullptr);
  else
    k_xr_update<double><<<std::min(dot_grid(m), wave_blocks((const void *)k_xr_update<double>,
                                                            kDotThreads)),
                          kDotThreads, 0, h->stream>>>(
        m, x, r, p, q, make_ctx(h, DOT_RR), nullptr, L.dinv, L.omega,
        jac ? (double *)L.x : nullptr);
  MG_LAUNCH("k_xr_update");
  MG_TRY(vcycle_top(h, r, z, true, DOT_RZ));
  k_p_update<<<blocks_for(std::max(1, (m / 2 + 1) / 2), 256), 256, 0, h->stream>>>(
      m, p, z, h->sc, h->p.ap_split ? h->p_df : nullptr);
  MG_LAUNCH("k_p_update");
  return MGPBD_OK;
}

// start of MGPCG: x = 0, r = b, |b|^2, z = V(r), r.z, p = z
mgpbd_status pcg_begin(Handle *h, const double *b, double *x) {
  const int m = h->m;
  MG_CUDA(cudaEventRecord(h->ev0, h->stream));
  double *r = h->pr, *z = h->pz, *p = h->pp;
  h->pcg_k = -1;
  for (int ch = 0; ch < PROF_CH; ++ch) h->pev_used[ch] = 0;
  k_pcg_init<<<1, 1, 0, h->stream>>>(h->sc, h->gbar);
  MG_LAUNCH("k_pcg_init");
  MG_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * m, h->stream));
  MG_CUDA(cudaMemcpyAsync(r, b, sizeof(double) * m, cudaMemcpyDeviceToDevice, h->stream));
  MG_TRY(launch_dot(h, b, b, m, DOT_BNORM, 0));
  MG_TRY(vcycle_top(h, r, z, false, DOT_RZ0));
  MG_CUDA(cudaMemcpyAsync(p, z, sizeof(double) * m, cudaMemcpyDeviceToDevice, h->stream));
  h->n_replace = 0;
  if (h->p.ap_split) MG_TRY(mf_split(h, p, h->p_df, m));
  return MGPBD_OK;
}

mgpbd_status pcg_solve(Handle *h, const double *b, double *x, mgpbd_solve_info *info) {
  const int m = h->m;
  memset(info, 0, sizeof(*info));
  if (m == 0) return MGPBD_OK;
  MG_TRY(pcg_begin(h, b, x));
  const int chunk = 8;
  int launched = 0;
  // Chunks of PCG iterations replay a captured CUDA graph (one launch instead
  // of ~33 per iteration); the graph is re-captured when the hierarchy, the
  // output array or the profiling switch changes.  With profiling on, the
  // graph carries event-record nodes around the level-0 sweeps, read back
  // after every replay.
  // (the legacy default stream cannot be captured: graphs need the caller's own stream)
  const bool graphs = h->p.use_graphs && h->stream != nullptr &&
                      h->stream != cudaStreamLegacy && h->stream != cudaStreamPerThread;
  // Residual replacement (params.ap_split): the recursive residual drifts
  // from b - A x by the rounding of every A.p, ~2^-46 relative in the pair
  // form against 2^-53 in FP64.  Whenever |r| has fallen tenfold since the
  // start or the last replacement, r is recomputed as b - A x in FP64 between
  // two chunks (the reliable-update scheme for CG: only r is replaced, the
  // search direction and the scalars carry on), so the drift that remains at
  // convergence is that of the iterations after the last replacement, made
  // on residuals at most ten times the final one.
  double rr_ref = -1.0;
  while (launched < h->p.pcg_maxiter) {
    int c = std::min(chunk, h->p.pcg_maxiter - launched);
    const bool replay = graphs && c == chunk;
    if (replay) {
      if (!h->pcg_graph || h->graph_gen != h->gen || h->graph_x != x || h->graph_chunk != c ||
          h->graph_prof != h->prof) {
        if (h->pcg_graph) {
          cudaGraphExecDestroy(h->pcg_graph);
          h->pcg_graph = nullptr;
        }
        if (h->prof) MG_TRY(prof_reserve_graph(h, c * 2 * std::max(1, h->p.smooth_sweeps) + 8));
        cudaGraph_t gr = nullptr;
        unsigned long long n0 = __atomic_load_n(&g_launches, __ATOMIC_RELAXED);
        for (int ch = 0; ch < PROF_CH; ++ch) h->gev_used[ch] = 0;
        MG_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        h->capturing = true;
        mgpbd_status cs = MGPBD_OK;
        for (int k = 0; k < c && cs >= 0; ++k) {
          h->pcg_k = k;
          cs = pcg_iteration(h, x);
        }
        h->capturing = false;
        cudaError_t ce = cudaStreamEndCapture(h->stream, &gr);
        // captured launches run at each replay, not now: count them there
        h->graph_kernels = __atomic_load_n(&g_launches, __ATOMIC_RELAXED) - n0;
        __atomic_fetch_sub(&g_launches, h->graph_kernels, __ATOMIC_RELAXED);
        if (cs < 0) {
          if (gr) cudaGraphDestroy(gr);
          return cs;
        }
        MG_CUDA(ce);
        ce = cudaGraphInstantiate(&h->pcg_graph, gr, 0);
        cudaGraphDestroy(gr);
        MG_CUDA(ce);
        h->graph_gen = h->gen;
        h->graph_x = x;
        h->graph_chunk = c;
        h->graph_prof = h->prof;
      }
      MG_CUDA(cudaGraphLaunch(h->pcg_graph, h->stream));
      __atomic_fetch_add(&g_launches, h->graph_kernels, __ATOMIC_RELAXED);
    } else {
      for (int k = 0; k < c; ++k) {
        h->pcg_k = launched + k;
        MG_TRY(pcg_iteration(h, x));
      }
    }
    launched += c;
    MG_CUDA(cudaMemcpyAsync(h->sc_host, h->sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost,
                            h->stream));
    MG_CUDA(cudaStreamSynchronize(h->stream));
    if (replay && h->graph_prof) MG_TRY(prof_harvest_graph(h, launched - c));
    if (h->sc_host->done) break;
    if (h->p.ap_split && h->p.level0_op == 1) {
      const double rr = h->sc_host->rr;
      if (rr_ref < 0.0) rr_ref = h->sc_host->bnorm2;
      if (rr <= 1e-2 * rr_ref) {
        MG_TRY(mf_residual64(h, x, b, h->pr));
        rr_ref = rr;
        h->n_replace++;
      }
    }
  }
  return pcg_finish(h, b, x, info);
}

// end of MGPCG: the FP64 true residual |b - A x|, the scalars, the solve's
// time and status (synchronises)
mgpbd_status pcg_finish(Handle *h, const double *b, double *x, mgpbd_solve_info *info) {
  const int m = h->m;
  memset(info, 0, sizeof(*info));
  k_true_resid<<<std::min(row_blocks(m, 4), wave_blocks((const void *)k_true_resid, 256)), 256, 0,
                 h->stream>>>(
      m, h->lev[0].ptr, h->lev[0].col, h->lev[0].val, x, b, make_ctx(h, DOT_TR));
  MG_LAUNCH("k_true_resid");
  MG_CUDA(cudaMemcpyAsync(h->sc_host, h->sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost,
                          h->stream));
  MG_CUDA(cudaEventRecord(h->ev1, h->stream));
  MG_CUDA(cudaStreamSynchronize(h->stream));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, h->ev0, h->ev1);
  h->ms_solve += ms;
  const PcgScalars &s = *h->sc_host;
  MG_TRY(prof_harvest(h, s.iters));
  double bn = sqrt(s.bnorm2);
  info->pcg_iters = s.iters;
  info->bnorm = bn;
  info->rel_res = bn > 0 ? sqrt(s.rr) / bn : 0.0;
  info->true_rel_res = bn > 0 ? sqrt(s.tr2) / bn : 0.0;
  info->replacements = h->n_replace;
  info->status = s.done ? s.status : MGPBD_W_NOT_CONVERGED;
  if (bn == 0.0) info->status = MGPBD_OK;
  h->last_pcg_iters = s.iters;
  if (info->status == MGPBD_E_BREAKDOWN) set_error("PCG breakdown (p.Ap <= 0, r.z <= 0 or NaN)");
  if (info->status == MGPBD_E_DEVICE_TIMEOUT)
    set_error("a grid barrier of the coarse V-cycle kernel waited longer than its limit");
  return info->status;
}

// ---------------------------------------------------------------------------
// autotuner: lanes per row of the row kernels, per level and precision
// ---------------------------------------------------------------------------
// Reads up to 256 MB of the level-0 matrix values, so that a kernel timed by
// the autotuner starts from the cache state it meets inside a V-cycle (its
// data evicted by the level-0 passes), not hot from its previous repetition.
__global__ void k_evict(const ulonglong2 *p, int64_t n, int *sink) {
  unsigned long long acc = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const ulonglong2 v = p[i];
    acc ^= v.x ^ v.y;
  }
  if (acc == 0x5eed5eed5eed5eedull) *sink = 1;  // keeps the loads
}

mgpbd_status evict_l2(Handle *h) {
  const Level &L = h->lev[0];
  const int64_t n = std::min<int64_t>(L.nnz / 2, (256ll << 20) / 16);
  if (n <= 0 || !L.val) return MGPBD_OK;
  k_evict<<<std::min<int64_t>(4 * num_sms(), (n + 255) / 256), 256, 0, h->stream>>>(
      reinterpret_cast<const ulonglong2 *>(L.val), n, reinterpret_cast<int *>(h->partials + 4096 + 15));
  MG_LAUNCH("k_evict");
  return MGPBD_OK;
}

template <class T>
static mgpbd_status time_resid(Handle *h, const Level &L, int G, const T *val, const T *b,
                               const T *x, T *r, float *ms_out) {
  const int n = L.n;
  float best = 1e30f;
  for (int rep = 0; rep < 5; ++rep) {
    MG_TRY(evict_l2(h));
    MG_CUDA(cudaEventRecord(h->ev0, h->stream));
    DISPATCH_G(G, (k_resid<GG, T><<<row_blocks(n, GG), 256, 0, h->stream>>>(n, L.ptr, L.col, val,
                                                                           b, x, r, nullptr)));
    MG_LAUNCH("k_resid(tune)");
    MG_CUDA(cudaEventRecord(h->ev1, h->stream));
    MG_CUDA(cudaEventSynchronize(h->ev1));
    float ms = 0.f;
    MG_CUDA(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    best = std::min(best, ms);
  }
  *ms_out = best;
  return MGPBD_OK;
}

// Times the residual kernel (the access pattern of every row kernel) with
// 4, 8, 16 and 32 lanes per row on each level, in the V-cycle precision, and
// on level 0 in FP64 for A.p; keeps the fastest.  Runs after a setup when
// params.autotune is set.
mgpbd_status autotune_levels(Handle *h) {
  const bool mixed = h->p.precision == MGPBD_MIXED;
  for (int l = 0; l + 1 < h->L || (l == 0 && h->L >= 1); ++l) {
    Level &L = h->lev[l];
    if (L.n == 0) break;
    const int cands[4] = {4, 8, 16, 32};
    float best = 1e30f;
    int bestG = group_rule(L, !mixed);
    for (int c = 0; c < 4; ++c) {
      float ms = 0.f;
      if (mixed)
        MG_TRY(time_resid<float>(h, L, cands[c], L.val32, (const float *)L.b, (const float *)L.x,
                                 (float *)L.r, &ms));
      else
        MG_TRY(time_resid<double>(h, L, cands[c], L.val, (const double *)L.b,
                                  (const double *)L.x, (double *)L.r, &ms));
      if (ms < best) {
        best = ms;
        bestG = cands[c];
      }
    }
    if (mixed) L.G32 = bestG;
    else L.G64 = bestG;
    if (l == 0 && mixed) {  // FP64 A.p on level 0
      float b64 = 1e30f;
      int g64 = 4;
      for (int c = 0; c < 4; ++c) {
        float ms = 0.f;
        MG_TRY(time_resid<double>(h, L, cands[c], L.val, h->pr, h->pz, h->pq, &ms));
        if (ms < b64) {
          b64 = ms;
          g64 = cands[c];
        }
      }
      L.G64 = g64;
    }
    if (l + 1 >= h->L) break;
  }
  if (h->p.level0_op == 1) MG_TRY(mf_autotune(h));
  return MGPBD_OK;
}

// ---------------------------------------------------------------------------
// the conversions of the mixed-precision path on caller vectors
// ---------------------------------------------------------------------------
__global__ void k_convert_pair(int64_t n, const double *a64, float *b32, const float *a32,
                              double *b64) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (a64) b32[i] = f64_to_f32(a64[i]);
    if (a32) b64[i] = f32_to_f64(a32[i]);
  }
}

}  // namespace mg

extern "C" mgpbd_status mgpbd_convert(const double *d_in64, float *d_out32, const float *d_in32,
                                      double *d_out64, int64_t n, void *stream) {
  using namespace mg;
  if (n < 0 || (!d_in64) != (!d_out32) || (!d_in32) != (!d_out64)) {
    set_error("mgpbd_convert: n < 0 or an input without its output");
    return MGPBD_E_INVALID;
  }
  if (n == 0 || (!d_in64 && !d_in32)) return MGPBD_OK;
  k_convert_pair<<<(int)std::min<int64_t>((n + 255) / 256, 65535), 256, 0,
                   (cudaStream_t)stream>>>(n, d_in64, d_out32, d_in32, d_out64);
  MG_LAUNCH("k_convert_pair");
  return MGPBD_OK;
}

namespace mg {

// ---------------------------------------------------------------------------
// XPBD's local step (eq. 4): dl_j = b_j / A_jj for every constraint at once
// ---------------------------------------------------------------------------
__global__ void k_xpbd_step(int m, const int64_t *ptr, const double *val, const double *b,
                            double *dl) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x)
    dl[j] = b[j] / val[ptr[j + 1] - 1];
}

mgpbd_status xpbd_step(Handle *h, mgpbd_solve_info *info) {
  memset(info, 0, sizeof(*info));
  if (h->m == 0) return MGPBD_OK;
  const Level &L = h->lev[0];
  double *d_bn = h->partials + 4096 + 6;
  MG_TRY(dot_dd(h, h->b, h->b, h->m, d_bn));
  k_xpbd_step<<<blocks_for(h->m, 256), 256, 0, h->stream>>>(h->m, L.ptr, L.val, h->b, h->dl);
  MG_LAUNCH("k_xpbd_step");
  double bn2 = 0.0;
  MG_CUDA(cudaMemcpyAsync(&bn2, d_bn, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  MG_CUDA(cudaStreamSynchronize(h->stream));
  info->bnorm = sqrt(bn2);
  info->pcg_iters = 1;
  info->status = MGPBD_OK;
  return MGPBD_OK;
}

// ---------------------------------------------------------------------------
// power method for lambda_max(D^-1 A) (Sec. 4.5)
// ---------------------------------------------------------------------------
__global__ void k_pow_init(int n, uint64_t seed, int l, double *y) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    y[i] = u01(h64(hkey(seed, l, i)));
}

// z_i = (A y)_i / A_ii
__global__ void k_pow_apply(int n, const int64_t *ptr, const int32_t *col, const double *val,
                            const double *y, double *z) {
  GROUP_ROWS(4, n) {
    double s = valid ? row_dot<4, double, double, double>(ptr, col, val, y, (int)i, g) : 0.0;
    s = group_sum<4>(s);
    if (valid && g == 0) z[i] = s / val[ptr[i + 1] - 1];
  }
}

// lam = |z|/|y|; y = z/|z|  (s[0] = z.z, s[1] = y.y)
__global__ void k_pow_scale(int n, const double *z, double *y, const double *s, double *lam) {
  double nz = sqrt(s[0]), ny = sqrt(s[1]);
  if (blockIdx.x == 0 && threadIdx.x == 0) *lam = nz / ny;
  if (!(nz > 0.0)) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    y[i] = z[i] / nz;
}

mgpbd_status power_method(Handle *h, int l) {
  Level &L = h->lev[l];
  const int n = L.n;
  double *y = h->pp, *z = h->pq;
  double *s = h->partials + 4096;  // 3 scalars after the partial area used by dots
  k_pow_init<<<blocks_for(n, 256), 256, 0, h->stream>>>(n, h->p.seed_pow, l, y);
  MG_LAUNCH("k_pow_init");
  for (int it = 0; it < h->p.power_iters; ++it) {
    k_pow_apply<<<row_blocks(n, 4), 256, 0, h->stream>>>(
        n, L.ptr, L.col, L.val, y, z);
    MG_LAUNCH("k_pow_apply");
    MG_TRY(launch_dot(h, z, z, n, DOT_STORE, 0, s));
    MG_TRY(launch_dot(h, y, y, n, DOT_STORE, 0, s + 1));
    k_pow_scale<<<blocks_for(n, 256), 256, 0, h->stream>>>(n, z, y, s, s + 2);
    MG_LAUNCH("k_pow_scale");
  }
  double lam = 0.0;
  MG_CUDA(cudaMemcpyAsync(&lam, s + 2, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  MG_CUDA(cudaStreamSynchronize(h->stream));
  L.lmax = lam;
  L.omega = 2.0 / (h->p.power_safety * lam + h->p.lambda_min_est);
  return MGPBD_OK;
}

}  // namespace mg
