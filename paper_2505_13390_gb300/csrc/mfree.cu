// Matrix-free application of the level-0 operator A = grad C M^-1 grad C^T
// + alpha~ (Eq. 3), the "matrix-free" direction of the paper's future work
// (Sec. 6).  The assembled CSR matrix is still built every global iteration
// for the setup and the Galerkin products; this path replaces the level-0
// products inside MGPCG (A.p and the V-cycle's sweeps and residual) with two
// passes over the constraint Jacobian:
//
//   vertex pass  u_v = w_v * sum_{j incident to v} g_{j,v} x_j       (3-vector)
//   row pass     y_i = sum_{slots s of i} g_{i,s} . u_{v_s} + alpha~_i x_i
//
// which is A x term for term (A_ij = sum over shared v of w_v g_{i,v}.g_{j,v}).
// The vertex pass reads the gradients in incidence order from `ginc`, a copy
// laid out per (vertex, incident row) that is rebuilt once per global
// iteration, so both passes stream their inputs; in FP32 each incidence is
// one 16-byte record (gradient and row id).  Per product on the 1.65M-tet
// block this moves about 0.4 GB (FP32) / 0.8 GB (FP64) instead of 3.1 /
// 4.7 GB for the CSR pass, and about 4x fewer FP64 multiply-adds.

#include <algorithm>
#include <numeric>
#include <vector>

#include "cohort.cuh"
#include "common.cuh"
#include "reduce.cuh"

namespace mg {

constexpr int kMfVertexLanes = 8;
// u = W J^T x: three values per vertex for the FP32 and FP64 passes (a
// fourth, unused slot made the FP32 row pass 2% slower: its gathers of u
// then cover a third more lines), four (x, y, z, unused) for the pair
// form, whose row pass gathers a vertex's high and low parts with one
// 16-byte load each
constexpr int kUStride = 3, kUStrideDf = 4;

// slot of vertex v in each incident row (create time)
__global__ void k_vslot(int N, int E, const int32_t *edge, const int32_t *tet, const int64_t *vptr,
                        const int32_t *vrow, uint8_t *vslot) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x) {
    for (int64_t q = vptr[v]; q < vptr[v + 1]; ++q) {
      int j = vrow[q];
      int s;
      if (j < E) {
        s = edge[2 * (int64_t)j] == v ? 0 : 1;
      } else {
        const int32_t *t = tet + 4 * (int64_t)(j - E);
        s = t[0] == v ? 0 : (t[1] == v ? 1 : (t[2] == v ? 2 : 3));
      }
      vslot[q] = (uint8_t)s;
    }
  }
}

// gradients in incidence order: FP64 (row ids apart) and optionally FP32
// packed with the row id, one 16-byte load per incidence
__global__ void k_mf_prep(int N, int E, const int64_t *vptr, const int32_t *vrow,
                          const uint8_t *vslot, const double *gd, const double *gt, double *g64,
                          float4 *g4) {
  GROUP_ROWS(kMfVertexLanes, N) {
    if (!valid) continue;
    for (int64_t q = vptr[i] + g; q < vptr[i + 1]; q += kMfVertexLanes) {
      int j = vrow[q];
      int s = vslot[q];
      double a0, a1, a2;
      if (j < E) {
        const double *n = gd + 3 * (int64_t)j;
        double sg = s == 0 ? 1.0 : -1.0;
        a0 = sg * n[0];
        a1 = sg * n[1];
        a2 = sg * n[2];
      } else {
        const double *t = gt + 12 * (int64_t)(j - E) + 3 * s;
        a0 = t[0];
        a1 = t[1];
        a2 = t[2];
      }
      if (g64) {
        g64[3 * q] = a0;
        g64[3 * q + 1] = a1;
        g64[3 * q + 2] = a2;
      }
      if (g4)
        g4[q] = make_float4(f64_to_f32(a0), f64_to_f32(a1), f64_to_f32(a2), __int_as_float(j));
    }
  }
}

__global__ void k_to_f32_mf(int64_t n, const double *a, float *b) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    b[k] = f64_to_f32(a[k]);
}

// vertex pass: u_v = w_v * sum_q ginc_q * x_{row(q)}, G lanes per vertex.
// Each lane loads four incidences before it uses them (four gathers in
// flight); the sum order is the plain lane-strided order.
template <int G>
__device__ __forceinline__ void mf_vertex64_rows(int64_t w0, int64_t nw, int N,
                                                 const int32_t *vorder, const int64_t *vptr,
                                                 const int32_t *vrow, const double *ginc,
                                                 const double *w, const double *x, double *u) {
  GROUP_ROWS_OVER(G, N, w0, nw) {
    double a0 = 0, a1 = 0, a2 = 0;
    const int v = valid ? vorder[i] : 0;
    if (valid) {
      int64_t q = vptr[v] + g;
      const int64_t e = vptr[v + 1];
      for (; q + 3 * G < e; q += 4 * G) {
        double xv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) xv[k] = x[vrow[q + k * G]];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const double *gq = ginc + 3 * (q + k * G);
          a0 = fma(gq[0], xv[k], a0);
          a1 = fma(gq[1], xv[k], a1);
          a2 = fma(gq[2], xv[k], a2);
        }
      }
      for (; q < e; q += G) {
        const double xa = x[vrow[q]];
        a0 = fma(ginc[3 * q], xa, a0);
        a1 = fma(ginc[3 * q + 1], xa, a1);
        a2 = fma(ginc[3 * q + 2], xa, a2);
      }
    }
    double s = group_sum3<G>(a0, a1, a2, g);
    const int comp = group_sum3_component<G>(g);
    if (valid && comp < 3 && (g & (G / 4 - 1)) == 0) u[kUStride * (int64_t)v + comp] = w[v] * s;
  }
}

template <int G>
__global__ void k_mf_vertex64(int N, const int32_t *vorder, const int64_t *vptr,
                              const int32_t *vrow, const double *ginc, const double *w,
                              const double *x, double *u, const PcgScalars *sc) {
  if (sc && is_done(sc)) return;
  mf_vertex64_rows<G>(HW_WARPS, N, vorder, vptr, vrow, ginc, w, x, u);
}

template <int G>
__device__ __forceinline__ void mf_vertex32_rows(int64_t w0, int64_t nw, int N,
                                                 const int32_t *vorder, const int64_t *vptr,
                                                 const float4 *ginc, const float *w,
                                                 const float *x, float *u) {
  GROUP_ROWS_OVER(G, N, w0, nw) {
    float a0 = 0, a1 = 0, a2 = 0;
    const int v = valid ? vorder[i] : 0;
    if (valid) {
      int64_t q = vptr[v] + g;
      const int64_t e = vptr[v + 1];
      for (; q + 3 * G < e; q += 4 * G) {
        float4 ev[4];
        float xv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) ev[k] = ginc[q + k * G];
#pragma unroll
        for (int k = 0; k < 4; ++k) xv[k] = x[__float_as_int(ev[k].w)];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          a0 = fmaf(ev[k].x, xv[k], a0);
          a1 = fmaf(ev[k].y, xv[k], a1);
          a2 = fmaf(ev[k].z, xv[k], a2);
        }
      }
      for (; q < e; q += G) {
        const float4 ea = ginc[q];
        const float xa = x[__float_as_int(ea.w)];
        a0 = fmaf(ea.x, xa, a0);
        a1 = fmaf(ea.y, xa, a1);
        a2 = fmaf(ea.z, xa, a2);
      }
    }
    float s = group_sum3<G>(a0, a1, a2, g);
    const int comp = group_sum3_component<G>(g);
    if (valid && comp < 3 && (g & (G / 4 - 1)) == 0) u[kUStride * (int64_t)v + comp] = w[v] * s;
  }
}

template <int G>
__global__ void __launch_bounds__(256, 8)
    k_mf_vertex32(int N, const int32_t *vorder, const int64_t *vptr, const float4 *ginc,
                  const float *w, const float *x, float *u, const PcgScalars *sc) {
  if (sc && is_done(sc)) return;
  mf_vertex32_rows<G>(HW_WARPS, N, vorder, vptr, ginc, w, x, u);
}

// 16-byte loads of the pair form's row pass (all arrays 256-byte aligned by
// the arena): a vertex's three slots of u, and a tet row's twelve gradient
// values.  (The FP32 and FP64 row passes keep scalar loads: with these, the
// FP32 sweep needed more registers and ran slower.)
__device__ __forceinline__ void ld_u(const float *u, int v, float &a, float &b, float &c) {
  const float4 t = reinterpret_cast<const float4 *>(u)[v];
  a = t.x;
  b = t.y;
  c = t.z;
}
__device__ __forceinline__ void ld_g12(const float *g, float *o) {
  const float4 *q = reinterpret_cast<const float4 *>(g);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float4 t = q[k];
    o[4 * k] = t.x;
    o[4 * k + 1] = t.y;
    o[4 * k + 2] = t.z;
    o[4 * k + 3] = t.w;
  }
}

// ---------------------------------------------------------------------------
// A.p from float-float pairs (params.ap_split).  Every FP64 operand of the
// product is held as a pair (h, l) of binary32 numbers with a = h + l to 48
// bits (df_split).  A product of two pairs takes its rounding error from one
// FMA (Dekker's product, the FMA form) and adds the two cross terms; sums
// use Knuth's two-sum, whose error term is exact.  Every step issues on the
// FP32 pipe; one product carries about 2^-46 relative error, a sum of n
// terms about n 2^-47 of the sum of their magnitudes.
// ---------------------------------------------------------------------------
struct DF {
  float h, l;
};

// s + e == a + b exactly (Knuth's two-sum, no ordering condition)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// acc += (gh + gl) (xh + xl); the term gl xl lies below 2^-47 of the product
__device__ __forceinline__ void df_fma(DF &acc, float gh, float gl, float xh, float xl) {
  const float p = __fmul_rn(gh, xh);
  float e = __fmaf_rn(gh, xh, -p);  // gh xh - p, exactly
  e = __fmaf_rn(gh, xl, e);
  e = __fmaf_rn(gl, xh, e);
  float s, t;
  two_sum(acc.h, p, s, t);
  acc.h = s;
  acc.l = __fadd_rn(acc.l, __fadd_rn(t, e));
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
  float s, t;
  two_sum(a.h, b.h, s, t);
  return DF{s, __fadd_rn(__fadd_rn(a.l, b.l), t)};
}

// the pair with its low part below half a unit in the last place of h
__device__ __forceinline__ DF df_norm(DF a) {
  float s, t;
  two_sum(a.h, a.l, s, t);
  return DF{s, t};
}

__device__ __forceinline__ DF shfl_xor_df(DF v, int o) {
  return DF{__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)};
}

// group_sum3 (reduce.cuh) for pairs: the same exchange pattern, with the
// pairwise sums taken by df_add
template <int G>
__device__ __forceinline__ DF group_sum3_df(DF a0, DF a1, DF a2, int g) {
  static_assert(G >= 4 && G <= 32, "group of 4..32 lanes");
  constexpr int o1 = G / 2, o2 = G / 4;
  const bool h1 = (g & o1) != 0, h2 = (g & o2) != 0;
  const DF z{0.f, 0.f};
  DF k0 = h1 ? a2 : a0, k1 = h1 ? z : a1;
  const DF s0 = h1 ? a0 : a2, s1 = h1 ? a1 : z;
  k0 = df_add(k0, shfl_xor_df(s0, o1));
  k1 = df_add(k1, shfl_xor_df(s1, o1));
  DF k = h2 ? k1 : k0;
  const DF s = h2 ? k0 : k1;
  k = df_add(k, shfl_xor_df(s, o2));
#pragma unroll
  for (int o = o2 / 2; o > 0; o >>= 1) k = df_add(k, shfl_xor_df(k, o));
  return k;
}

// vertex pass of the pair product: u_v = w_v * sum_q g_q x_row(q) with the
// high parts of g (and the row id) from the FP32 incidence records and the
// low parts from `glo` (three per incidence); x and the result as pairs
template <int G>
__device__ __forceinline__ void mf_vertex_df_rows(int64_t w0, int64_t nw, int N,
                                                  const int32_t *vorder, const int64_t *vptr,
                                                  const float4 *ginc, const float *glo,
                                                  const float *wh, const float *wl,
                                                  const float2 *x, float *uh, float *ul) {
  GROUP_ROWS_OVER(G, N, w0, nw) {
    DF a0{0.f, 0.f}, a1{0.f, 0.f}, a2{0.f, 0.f};
    const int v = valid ? vorder[i] : 0;
    if (valid) {
      int64_t q = vptr[v] + g;
      const int64_t e = vptr[v + 1];
      for (; q + 3 * G < e; q += 4 * G) {
        float4 ev[4];
        float2 xv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) ev[k] = ginc[q + k * G];
#pragma unroll
        for (int k = 0; k < 4; ++k) xv[k] = x[__float_as_int(ev[k].w)];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float *lo = glo + 3 * (q + k * G);
          df_fma(a0, ev[k].x, lo[0], xv[k].x, xv[k].y);
          df_fma(a1, ev[k].y, lo[1], xv[k].x, xv[k].y);
          df_fma(a2, ev[k].z, lo[2], xv[k].x, xv[k].y);
        }
      }
      for (; q < e; q += G) {
        const float4 ea = ginc[q];
        const float2 xa = x[__float_as_int(ea.w)];
        const float *lo = glo + 3 * q;
        df_fma(a0, ea.x, lo[0], xa.x, xa.y);
        df_fma(a1, ea.y, lo[1], xa.x, xa.y);
        df_fma(a2, ea.z, lo[2], xa.x, xa.y);
      }
    }
    const DF s = group_sum3_df<G>(a0, a1, a2, g);
    const int comp = group_sum3_component<G>(g);
    if (valid && comp < 3 && (g & (G / 4 - 1)) == 0) {
      DF r{0.f, 0.f};
      df_fma(r, wh[v], wl[v], s.h, s.l);
      r = df_norm(r);
      uh[kUStrideDf * (int64_t)v + comp] = r.h;
      ul[kUStrideDf * (int64_t)v + comp] = r.l;
    }
  }
}

template <int G>
__global__ void k_mf_vertex_df(int N, const int32_t *vorder, const int64_t *vptr,
                               const float4 *ginc, const float *glo, const float *wh,
                               const float *wl, const float2 *x, float *uh, float *ul,
                               const PcgScalars *sc) {
  if (sc && is_done(sc)) return;
  mf_vertex_df_rows<G>(HW_WARPS, N, vorder, vptr, ginc, glo, wh, wl, x, uh, ul);
}

// row pass of the pair product: q_i = sum_s g_{i,s}.u_{v_s} + alpha~_i p_i,
// written in FP64 (h + l is exact there), with p.q folded into the PCG
// scalars (each thread's share summed as a pair, the block sums in FP64)
__global__ void __launch_bounds__(256, 4) k_mf_row_df(int E, int m, const int32_t *edge, const int32_t *tet,
                            const float *gdh, const float *gdl, const float *gth,
                            const float *gtl, const float *uh, const float *ul, const float *ath,
                            const float *atl, const float2 *p, double *q, DotCtx c) {
  if (is_done(c.sc)) return;
  DF dot{0.f, 0.f};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    DF y{0.f, 0.f};
    if (i < E) {
      const int2 e = reinterpret_cast<const int2 *>(edge)[i];
      float ah[3], al[3], bh[3], bl[3];
      ld_u(uh, e.x, ah[0], ah[1], ah[2]);
      ld_u(ul, e.x, al[0], al[1], al[2]);
      ld_u(uh, e.y, bh[0], bh[1], bh[2]);
      ld_u(ul, e.y, bl[0], bl[1], bl[2]);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const DF d = df_add(DF{ah[k], al[k]}, DF{-bh[k], -bl[k]});
        df_fma(y, gdh[3 * i + k], gdl[3 * i + k], d.h, d.l);
      }
    } else {
      const int4 t4 = reinterpret_cast<const int4 *>(tet)[i - E];
      const int t[4] = {t4.x, t4.y, t4.z, t4.w};
      float gh[12], gl[12];
      ld_g12(gth + 12 * (i - E), gh);
      ld_g12(gtl + 12 * (i - E), gl);
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        float h[3], l[3];
        ld_u(uh, t[s], h[0], h[1], h[2]);
        ld_u(ul, t[s], l[0], l[1], l[2]);
#pragma unroll
        for (int k = 0; k < 3; ++k) df_fma(y, gh[3 * s + k], gl[3 * s + k], h[k], l[k]);
      }
    }
    const float2 pi = p[i];
    df_fma(y, ath[i], atl[i], pi.x, pi.y);
    y = df_norm(y);
    q[i] = f32_to_f64(y.h) + f32_to_f64(y.l);
    df_fma(dot, pi.x, pi.y, y.h, y.l);
  }
  block_dot_finish(f32_to_f64(dot.h) + f32_to_f64(dot.l), c);
}

// low parts lo = RN32(a - hi) of FP64 values whose high parts are already
// stored (hi = RN32(a)); incidence records hold theirs in .x .y .z
__global__ void k_df_lo(int64_t n, const double *a, const float *hi, float *lo) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    lo[k] = f64_to_f32(a[k] - f32_to_f64(hi[k]));
}

__global__ void k_df_lo_inc(int64_t ninc, const double *g64, const float4 *g4, float *lo) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < ninc;
       k += (int64_t)gridDim.x * blockDim.x) {
    const float4 h = g4[k];
    lo[3 * k] = f64_to_f32(g64[3 * k] - f32_to_f64(h.x));
    lo[3 * k + 1] = f64_to_f32(g64[3 * k + 1] - f32_to_f64(h.y));
    lo[3 * k + 2] = f64_to_f32(g64[3 * k + 2] - f32_to_f64(h.z));
  }
}

// p as pairs (the start of a solve; later the p update writes them)
__global__ void k_df_split(int64_t n, const double *a, float2 *out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    out[k] = df_split(a[k]);
}

enum {
  MF_SWEEP = kMfSweep,
  MF_RESID = kMfResid,
  MF_APPLY_DOT = 2,
  MF_APPLY = kMfApply,
  MF_SWEEP_Z = 4,
  MF_SWEEP_ZDOT = 5,
  MF_RESID_MEMBER = kMfResidMember
};

// row pass: y_i = sum_s g_{i,s}.u_{v_s} + alpha~_i x_i, then
//   MF_SWEEP      out = x + omega D^-1 (b - y)
//   MF_RESID      out = b - y
//   MF_APPLY_DOT  out = y, with x.y folded into the PCG scalars (DOT_PQ)
//   MF_SWEEP_Z    z = x + omega D^-1 (b - y) widened to FP64
//   MF_SWEEP_ZDOT the same, with r.z folded into the PCG scalars
//   MF_RESID_MEMBER out[pos_i] = b - y for rows in an aggregate (the
//                 residual in member order, for the restriction)
template <class T, int MODE>
__device__ __forceinline__ void mf_row_body(int vb, int vn, int E, int m, const int32_t *edge,
                                            const int32_t *tet, const T *gd, const T *gt,
                                            const T *u, const T *at, const T *x, const T *b,
                                            const T *dinv, T omega, T *out, const DotCtx &c,
                                            double *z, const double *rr,
                                            const int32_t *pos = nullptr) {
  double acc = 0.0;
  for (int64_t i = vb * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)vn * blockDim.x) {
    T y;
    if (i < E) {
      const T *n = gd + 3 * i;
      const T *ua = u + kUStride * (int64_t)edge[2 * i];
      const T *ub = u + kUStride * (int64_t)edge[2 * i + 1];
      y = n[0] * (ua[0] - ub[0]);
      y = fma(n[1], ua[1] - ub[1], y);
      y = fma(n[2], ua[2] - ub[2], y);
    } else {
      const int32_t *t = tet + 4 * (i - E);
      const T *gg = gt + 12 * (i - E);
      y = 0;
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const T *uv = u + kUStride * (int64_t)t[s];
        y = fma(gg[3 * s], uv[0], y);
        y = fma(gg[3 * s + 1], uv[1], y);
        y = fma(gg[3 * s + 2], uv[2], y);
      }
    }
    T xi = x[i];
    y = fma(at[i], xi, y);
    if (MODE == MF_SWEEP) out[i] = fma(omega, (b[i] - y) * dinv[i], xi);
    else if (MODE == MF_RESID) out[i] = b[i] - y;
    else if (MODE == MF_RESID_MEMBER) {
      const int32_t q = pos[i];
      if (q >= 0) out[q] = b[i] - y;
    }
    else if (MODE == MF_APPLY) out[i] = y;
    else if (MODE == MF_APPLY_DOT) {
      out[i] = y;
      acc = fma(widen(xi), widen(y), acc);
    } else {
      double zi = widen(fma(omega, (b[i] - y) * dinv[i], xi));
      z[i] = zi;
      if (MODE == MF_SWEEP_ZDOT) acc = fma(rr[i], zi, acc);
    }
  }
  if (MODE == MF_APPLY_DOT || MODE == MF_SWEEP_ZDOT) block_dot_finish_vg(acc, c, vb, vn);
}

template <class T, int MODE>
__global__ void k_mf_row(int E, int m, const int32_t *edge, const int32_t *tet, const T *gd,
                         const T *gt, const T *u, const T *at, const T *x, const T *b,
                         const T *dinv, T omega, T *out, DotCtx c, double *z = nullptr,
                         const double *rr = nullptr, const int32_t *pos = nullptr) {
  if (is_done(c.sc)) return;
  mf_row_body<T, MODE>(blockIdx.x, gridDim.x, E, m, edge, tet, gd, gt, u, at, x, b, dinv, omega,
                       out, c, z, rr, pos);
}

// ---------------------------------------------------------------------------
mgpbd_status mf_create(Handle *h) {
  if (h->vslot || h->m == 0) return MGPBD_OK;
  const int64_t ninc = 2 * (int64_t)h->E + 4 * (int64_t)h->T;
  const bool mixed = h->p.precision == MGPBD_MIXED;
  MG_TRY(alloc_n(h->arena, &h->vslot, (size_t)ninc));
  MG_TRY(alloc_n(h->arena, &h->ginc64, 3 * (size_t)ninc));
  MG_TRY(alloc_n(h->arena, &h->u64, kUStride * (size_t)h->N));
  if (mixed) {
    MG_TRY(alloc_n(h->arena, &h->ginc4, (size_t)ninc));
    MG_TRY(alloc_n(h->arena, &h->gd32, 3 * (size_t)h->E));
    MG_TRY(alloc_n(h->arena, &h->gt32, 12 * (size_t)h->T));
    MG_TRY(alloc_n(h->arena, &h->at32, (size_t)h->m));
    MG_TRY(alloc_n(h->arena, &h->w32, (size_t)h->N));
    MG_TRY(alloc_n(h->arena, &h->u32, kUStride * (size_t)h->N));
    k_to_f32_mf<<<blocks_for(h->m, 256), 256, 0, h->stream>>>(h->m, h->alpha_t, h->at32);
    MG_LAUNCH("k_to_f32_mf(alpha)");
    k_to_f32_mf<<<blocks_for(h->N, 256), 256, 0, h->stream>>>(h->N, h->w, h->w32);
    MG_LAUNCH("k_to_f32_mf(w)");
  }
  if (h->p.ap_split) {
    MG_TRY(alloc_n(h->arena, &h->ginc_lo, 3 * (size_t)ninc));
    MG_TRY(alloc_n(h->arena, &h->gd_lo, 3 * (size_t)h->E));
    MG_TRY(alloc_n(h->arena, &h->gt_lo, 12 * (size_t)h->T));
    MG_TRY(alloc_n(h->arena, &h->at_lo, (size_t)h->m));
    MG_TRY(alloc_n(h->arena, &h->w_lo, (size_t)h->N));
    MG_TRY(alloc_n(h->arena, &h->u_hi, kUStrideDf * (size_t)h->N));
    MG_TRY(alloc_n(h->arena, &h->u_lo, kUStrideDf * (size_t)h->N));
    MG_TRY(alloc_n(h->arena, &h->p_df, (size_t)h->m));
    MG_CUDA(cudaMemsetAsync(h->p_df, 0, sizeof(float2) * (size_t)h->m, h->stream));
    k_df_lo<<<blocks_for(h->m, 256), 256, 0, h->stream>>>(h->m, h->alpha_t, h->at32, h->at_lo);
    MG_LAUNCH("k_df_lo(alpha)");
    k_df_lo<<<blocks_for(h->N, 256), 256, 0, h->stream>>>(h->N, h->w, h->w32, h->w_lo);
    MG_LAUNCH("k_df_lo(w)");
  }
  k_vslot<<<blocks_for(h->N, 128), 128, 0, h->stream>>>(h->N, h->E, h->edge, h->tet, h->vptr,
                                                       h->vrow, h->vslot);
  MG_LAUNCH("k_vslot");
  // Vertex-pass order: within windows of kOrderWindow consecutive vertices,
  // by incidence count (then id).  A G-lane group loops over its vertex's
  // incidences, so a warp costs its longest vertex; neighbouring vertices of
  // the tet lattice alternate between two degrees, and grouping equal
  // degrees inside a window removes that waste while the warp's vertices stay
  // close in the mesh (the gathers keep their locality).
  constexpr int kOrderWindow = 256;
  std::vector<int64_t> vp((size_t)h->N + 1);
  MG_CUDA(cudaMemcpyAsync(vp.data(), h->vptr, sizeof(int64_t) * vp.size(), cudaMemcpyDeviceToHost,
                          h->stream));
  MG_CUDA(cudaStreamSynchronize(h->stream));
  std::vector<int32_t> ord((size_t)h->N);
  std::iota(ord.begin(), ord.end(), 0);
  for (int64_t w0 = 0; w0 < h->N; w0 += kOrderWindow) {
    auto first = ord.begin() + w0, last = ord.begin() + std::min<int64_t>(h->N, w0 + kOrderWindow);
    std::stable_sort(first, last, [&](int32_t a, int32_t b) {
      return vp[a + 1] - vp[a] > vp[b + 1] - vp[b];
    });
  }
  MG_TRY(alloc_n(h->arena, &h->vorder, (size_t)h->N));
  MG_CUDA(cudaMemcpyAsync(h->vorder, ord.data(), sizeof(int32_t) * ord.size(),
                          cudaMemcpyHostToDevice, h->stream));
  MG_CUDA(cudaStreamSynchronize(h->stream));
  return MGPBD_OK;
}

// Row-pass grid: one thread per row up to 8,192 blocks, then grid-stride.  On
// the 3.68M-row block (14,375 blocks of rows) the cap measured 0.7% faster
// per PCG iteration than 4,096 blocks and 2% faster than one block per 256
// rows.
static int mf_grid(int64_t rows, int threads) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((rows + threads - 1) / threads, 8192));
}

mgpbd_status mf_prepare(Handle *h) {
  if (h->m == 0) return MGPBD_OK;
  MG_TRY(mf_create(h));
  const bool mixed = h->p.precision == MGPBD_MIXED;
  int64_t groups = (int64_t)h->N;
  int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(
                   (groups * kMfVertexLanes + 255) / 256, 64 * (int64_t)num_sms()));
  k_mf_prep<<<blocks, 256, 0, h->stream>>>(h->N, h->E, h->vptr, h->vrow, h->vslot, h->gd, h->gt,
                                          h->ginc64, mixed ? h->ginc4 : nullptr);
  MG_LAUNCH("k_mf_prep");
  if (mixed) {
    k_to_f32_mf<<<blocks_for(3 * (int64_t)h->E, 256), 256, 0, h->stream>>>(3 * (int64_t)h->E,
                                                                         h->gd, h->gd32);
    MG_LAUNCH("k_to_f32_mf(gd)");
    k_to_f32_mf<<<blocks_for(12 * (int64_t)h->T, 256), 256, 0, h->stream>>>(12 * (int64_t)h->T,
                                                                           h->gt, h->gt32);
    MG_LAUNCH("k_to_f32_mf(gt)");
  }
  if (h->p.ap_split) {
    const int64_t ninc = 2 * (int64_t)h->E + 4 * (int64_t)h->T;
    k_df_lo_inc<<<blocks_for(ninc, 256), 256, 0, h->stream>>>(ninc, h->ginc64, h->ginc4,
                                                             h->ginc_lo);
    MG_LAUNCH("k_df_lo_inc");
    k_df_lo<<<blocks_for(3 * (int64_t)h->E, 256), 256, 0, h->stream>>>(3 * (int64_t)h->E, h->gd,
                                                                      h->gd32, h->gd_lo);
    MG_LAUNCH("k_df_lo(gd)");
    k_df_lo<<<blocks_for(12 * (int64_t)h->T, 256), 256, 0, h->stream>>>(
        12 * (int64_t)h->T, h->gt, h->gt32, h->gt_lo);
    MG_LAUNCH("k_df_lo(gt)");
  }
  return MGPBD_OK;
}

static int mf_vertex_blocks(const Handle *h, int G) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)h->N * G + 255) / 256,
                                                      64 * (int64_t)num_sms()));
}

#define MF_G_DISPATCH(G, launch) \
  switch (G) {                   \
    case 4: {                    \
      constexpr int GG = 4;      \
      launch;                    \
    } break;                     \
    case 16: {                   \
      constexpr int GG = 16;     \
      launch;                    \
    } break;                     \
    default: {                   \
      constexpr int GG = 8;      \
      launch;                    \
    } break;                     \
  }

// ---------------------------------------------------------------------------
// the same passes for every instance of a cohort in one launch
// ---------------------------------------------------------------------------
#define COHORT_BLOCK                                                              \
  const CohortBlock cb_ = blk[blockIdx.x];                                        \
  if (is_done(cb_.sc)) return;                                                    \
  const CohortMember &M = mem[cb_.k];                                             \
  const int vb = cb_.vb, vn = cb_.vn

__global__ void kb_vertex64(const CohortMember *mem, const CohortBlock *blk) {
  COHORT_BLOCK;
  MF_G_DISPATCH(M.gv64, (mf_vertex64_rows<GG>(VG_WARPS(vb, vn), M.N, M.vorder, M.vptr, M.vrow,
                                               M.ginc64, M.w, M.p, M.u64)));
}

// every member with G lanes per vertex (the usual case), with the standalone
// kernel's register budget
template <int G>
__global__ void __launch_bounds__(256, 8)
    kb_vertex32(const CohortMember *mem, const CohortBlock *blk, int sel) {
  COHORT_BLOCK;
  mf_vertex32_rows<G>(VG_WARPS(vb, vn), M.N, M.vorder, M.vptr, M.ginc4, M.w32,
                      sel ? M.x20 : M.x0, M.u32);
}

// members with different lanes per vertex: the shape is chosen per block
__global__ void __launch_bounds__(256, 4)
    kb_vertex32_any(const CohortMember *mem, const CohortBlock *blk, int sel) {
  COHORT_BLOCK;
  MF_G_DISPATCH(M.gv32, (mf_vertex32_rows<GG>(VG_WARPS(vb, vn), M.N, M.vorder, M.vptr, M.ginc4,
                                               M.w32, sel ? M.x20 : M.x0, M.u32)));
}

__global__ void kb_row_pq(const CohortMember *mem, const CohortBlock *blk) {
  COHORT_BLOCK;
  mf_row_body<double, MF_APPLY_DOT>(vb, vn, M.E, M.m, M.edge, M.tet, M.gd, M.gt, M.u64, M.at,
                                    M.p, nullptr, nullptr, 0.0, M.q, M.c_pq, nullptr, nullptr);
}

// sel 0: pre-sweep x0 -> x20; 1: residual x20 -> r0; 2: post-sweep x20 -> x0
__global__ void kb_row(const CohortMember *mem, const CohortBlock *blk, int sel) {
  COHORT_BLOCK;
  DotCtx c{};
  c.sc = M.sc;
  if (sel == 1)
    mf_row_body<float, MF_RESID>(vb, vn, M.E, M.m, M.edge, M.tet, M.gd32, M.gt32, M.u32, M.at32,
                                 M.x20, M.b0, M.dinv0, M.om0, M.r0, c, nullptr, nullptr);
  else
    mf_row_body<float, MF_SWEEP>(vb, vn, M.E, M.m, M.edge, M.tet, M.gd32, M.gt32, M.u32, M.at32,
                                 sel == 0 ? M.x0 : M.x20, M.b0, M.dinv0, M.om0,
                                 sel == 0 ? M.x20 : M.x0, c, nullptr, nullptr);
}

__global__ void kb_row_final(const CohortMember *mem, const CohortBlock *blk) {
  COHORT_BLOCK;
  mf_row_body<float, MF_SWEEP_ZDOT>(vb, vn, M.E, M.m, M.edge, M.tet, M.gd32, M.gt32, M.u32,
                                    M.at32, M.x0, M.b0, M.dinv0, M.om0, nullptr, M.c_rz, M.z,
                                    M.r);
}

void mf_cohort_grids(const Handle *h, int grid[CS_STEPS]) {
  const int g64 = h->force_vert64 ? h->force_vert64 : h->mf_g64;
  const int g32 = h->force_vert32 ? h->force_vert32 : h->mf_g32;
  MF_G_DISPATCH(g64, (grid[CS_VERT64] = mf_vertex_blocks(h, GG)));
  MF_G_DISPATCH(g32, (grid[CS_VERT32] = mf_vertex_blocks(h, GG)));
  grid[CS_ROW_PQ] = std::min(mf_grid(h->m, 256),
                             wave_blocks((const void *)k_mf_row<double, MF_APPLY_DOT>, 256));
  grid[CS_ROW] = mf_grid(h->m, 256);
  grid[CS_ROW_FINAL] = std::min(mf_grid(h->m, 256),
                                wave_blocks((const void *)k_mf_row<float, MF_SWEEP_ZDOT>, 256));
}

mgpbd_status mf_cohort_step(int which, int sel, const CohortMember *d_mem,
                            const CohortBlock *d_blk, int blocks, int gv32, cudaStream_t st) {
  switch (which) {
    case CS_VERT64:
      kb_vertex64<<<blocks, 256, 0, st>>>(d_mem, d_blk);
      break;
    case CS_ROW_PQ:
      kb_row_pq<<<blocks, 256, 0, st>>>(d_mem, d_blk);
      break;
    case CS_VERT32:
      if (gv32 == 4 || gv32 == 8 || gv32 == 16) {
        MF_G_DISPATCH(gv32, (kb_vertex32<GG><<<blocks, 256, 0, st>>>(d_mem, d_blk, sel)));
      } else {
        kb_vertex32_any<<<blocks, 256, 0, st>>>(d_mem, d_blk, sel);
      }
      break;
    case CS_ROW:
      kb_row<<<blocks, 256, 0, st>>>(d_mem, d_blk, sel);
      break;
    default:
      kb_row_final<<<blocks, 256, 0, st>>>(d_mem, d_blk);
      break;
  }
  MG_LAUNCH("kb_mf");
  return MGPBD_OK;
}

// u = W J^T x (FP64: u64; FP32: u32); G = 0 takes the tuned lanes per vertex
static mgpbd_status mf_vertex(Handle *h, const double *x, int G = 0, bool check_done = true) {
  if (G == 0) G = h->force_vert64 ? h->force_vert64 : h->mf_g64;
  const PcgScalars *sc = check_done ? h->sc : nullptr;
  MF_G_DISPATCH(G, (k_mf_vertex64<GG><<<mf_vertex_blocks(h, GG), 256, 0, h->stream>>>(
                       h->N, h->vorder, h->vptr, h->vrow, h->ginc64, h->w, x, h->u64, sc)));
  MG_LAUNCH("k_mf_vertex64");
  return MGPBD_OK;
}

static mgpbd_status mf_vertex(Handle *h, const float *x, int G = 0, bool check_done = true) {
  if (G == 0) G = h->force_vert32 ? h->force_vert32 : h->mf_g32;
  const PcgScalars *sc = check_done ? h->sc : nullptr;
  MF_G_DISPATCH(G, (k_mf_vertex32<GG><<<mf_vertex_blocks(h, GG), 256, 0, h->stream>>>(
                       h->N, h->vorder, h->vptr, h->ginc4, h->w32, x, h->u32, sc)));
  MG_LAUNCH("k_mf_vertex32");
  return MGPBD_OK;
}

// u = W J^T x from pairs (params.ap_split): high parts into u_hi, low parts
// into u_lo; the lanes of the FP64 vertex pass, whose place it takes
static mgpbd_status mf_vertex(Handle *h, const float2 *x, int G = 0, bool check_done = true) {
  if (G == 0) G = h->force_vert64 ? h->force_vert64 : h->mf_g64;
  const PcgScalars *sc = check_done ? h->sc : nullptr;
  MF_G_DISPATCH(G, (k_mf_vertex_df<GG><<<mf_vertex_blocks(h, GG), 256, 0, h->stream>>>(
                       h->N, h->vorder, h->vptr, h->ginc4, h->ginc_lo, h->w32, h->w_lo, x,
                       h->u_hi, h->u_lo, sc)));
  MG_LAUNCH("k_mf_vertex_df");
  return MGPBD_OK;
}

// Times the vertex pass with 4, 8 and 16 lanes per vertex in each precision
// the solve uses and keeps the fastest (params.autotune); with ap_split the
// A.p's lanes are timed on its pair form.
mgpbd_status mf_autotune(Handle *h) {
  if (h->m == 0 || !h->vslot) return MGPBD_OK;
  auto pick = [&](auto *x, int *out) -> mgpbd_status {
    const int cands[3] = {4, 8, 16};
    float best = 1e30f;
    for (int c = 0; c < 3; ++c) {
      for (int rep = 0; rep < 5; ++rep) {
        MG_TRY(evict_l2(h));
        MG_CUDA(cudaEventRecord(h->ev0, h->stream));
        MG_TRY(mf_vertex(h, x, cands[c], false));
        MG_CUDA(cudaEventRecord(h->ev1, h->stream));
        MG_CUDA(cudaEventSynchronize(h->ev1));
        float ms = 0.f;
        MG_CUDA(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
        if (ms < best) {
          best = ms;
          *out = cands[c];
        }
      }
    }
    return MGPBD_OK;
  };
  if (h->p.ap_split)
    MG_TRY(pick((const float2 *)h->p_df, &h->mf_g64));
  else
    MG_TRY(pick((const double *)h->pr, &h->mf_g64));
  if (h->p.precision == MGPBD_MIXED) MG_TRY(pick((const float *)h->lev[0].b, &h->mf_g32));
  return MGPBD_OK;
}

// A.p with p.Ap folded into the PCG scalars: in FP64, or (pairs) from the
// pairs of p that the p update wrote beside it
mgpbd_status mf_apply_pq_form(Handle *h, bool pairs, const double *p, double *q,
                              const DotCtx &c) {
  if (pairs) {
    MG_TRY(mf_vertex(h, (const float2 *)h->p_df));
    const int grid =
        std::min(mf_grid(h->m, 256), wave_blocks((const void *)k_mf_row_df, 256));
    k_mf_row_df<<<grid, 256, 0, h->stream>>>(h->E, h->m, h->edge, h->tet, h->gd32, h->gd_lo,
                                             h->gt32, h->gt_lo, h->u_hi, h->u_lo, h->at32,
                                             h->at_lo, h->p_df, q, c);
    MG_LAUNCH("k_mf_row_df(A.p)");
    return MGPBD_OK;
  }
  MG_TRY(mf_vertex(h, p));
  const int grid = std::min(mf_grid(h->m, 256),
                            wave_blocks((const void *)k_mf_row<double, MF_APPLY_DOT>, 256));
  k_mf_row<double, MF_APPLY_DOT><<<grid, 256, 0, h->stream>>>(
      h->E, h->m, h->edge, h->tet, h->gd, h->gt, h->u64, h->alpha_t, p, nullptr, nullptr, 0.0, q,
      c);
  MG_LAUNCH("k_mf_row(A.p)");
  return MGPBD_OK;
}

mgpbd_status mf_apply_pq(Handle *h, const double *p, double *q, const DotCtx &c) {
  return mf_apply_pq_form(h, h->p.ap_split != 0, p, q, c);
}

// r = b - A x in FP64 (the residual replacement that accompanies the pair
// form of A.p)
mgpbd_status mf_residual64(Handle *h, const double *x, const double *b, double *r) {
  MG_TRY(mf_vertex(h, x, 0, false));
  DotCtx c{};
  c.sc = h->sc;
  k_mf_row<double, MF_RESID><<<mf_grid(h->m, 256), 256, 0, h->stream>>>(
      h->E, h->m, h->edge, h->tet, h->gd, h->gt, h->u64, h->alpha_t, x, b, nullptr, 0.0, r, c);
  MG_LAUNCH("k_mf_row(b - A x)");
  return MGPBD_OK;
}

// pairs of an FP64 vector (p at the start of a solve)
mgpbd_status mf_split(Handle *h, const double *a, float2 *out, int64_t n) {
  k_df_split<<<blocks_for(n, 256), 256, 0, h->stream>>>(n, a, out);
  MG_LAUNCH("k_df_split");
  return MGPBD_OK;
}

// level-0 sweep or residual of the V-cycle in its precision
template <class T>
mgpbd_status mf_level0(Handle *h, int mode, const T *x, const T *b, const T *dinv, T omega,
                       T *out);

template <>
mgpbd_status mf_level0<float>(Handle *h, int mode, const float *x, const float *b,
                              const float *dinv, float omega, float *out) {
  MG_TRY(mf_vertex(h, x));
  DotCtx c{};
  c.sc = h->sc;
  if (mode == MF_SWEEP)
    k_mf_row<float, MF_SWEEP><<<mf_grid(h->m, 256), 256, 0, h->stream>>>(
        h->E, h->m, h->edge, h->tet, h->gd32, h->gt32, h->u32, h->at32, x, b, dinv, omega, out, c);
  else if (mode == MF_APPLY)
    k_mf_row<float, MF_APPLY><<<mf_grid(h->m, 256), 256, 0, h->stream>>>(
        h->E, h->m, h->edge, h->tet, h->gd32, h->gt32, h->u32, h->at32, x, b, dinv, omega, out, c);
  else if (mode == MF_RESID_MEMBER)
    k_mf_row<float, MF_RESID_MEMBER><<<mf_grid(h->m, 256), 256, 0, h->stream>>>(
        h->E, h->m, h->edge, h->tet, h->gd32, h->gt32, h->u32, h->at32, x, b, dinv, omega, out, c,
        nullptr, nullptr, h->lev[0].mpos);
  else
    k_mf_row<float, MF_RESID><<<mf_grid(h->m, 256), 256, 0, h->stream>>>(
        h->E, h->m, h->edge, h->tet, h->gd32, h->gt32, h->u32, h->at32, x, b, dinv, omega, out, c);
  MG_LAUNCH("k_mf_row(f32)");
  return MGPBD_OK;
}

template <>
mgpbd_status mf_level0<double>(Handle *h, int mode, const double *x, const double *b,
                               const double *dinv, double omega, double *out) {
  MG_TRY(mf_vertex(h, x));
  DotCtx c{};
  c.sc = h->sc;
  if (mode == MF_SWEEP)
    k_mf_row<double, MF_SWEEP><<<mf_grid(h->m, 256), 256, 0, h->stream>>>(
        h->E, h->m, h->edge, h->tet, h->gd, h->gt, h->u64, h->alpha_t, x, b, dinv, omega, out, c);
  else if (mode == MF_APPLY)
    k_mf_row<double, MF_APPLY><<<mf_grid(h->m, 256), 256, 0, h->stream>>>(
        h->E, h->m, h->edge, h->tet, h->gd, h->gt, h->u64, h->alpha_t, x, b, dinv, omega, out, c);
  else if (mode == MF_RESID_MEMBER)
    k_mf_row<double, MF_RESID_MEMBER><<<mf_grid(h->m, 256), 256, 0, h->stream>>>(
        h->E, h->m, h->edge, h->tet, h->gd, h->gt, h->u64, h->alpha_t, x, b, dinv, omega, out, c,
        nullptr, nullptr, h->lev[0].mpos);
  else
    k_mf_row<double, MF_RESID><<<mf_grid(h->m, 256), 256, 0, h->stream>>>(
        h->E, h->m, h->edge, h->tet, h->gd, h->gt, h->u64, h->alpha_t, x, b, dinv, omega, out, c);
  MG_LAUNCH("k_mf_row(f64)");
  return MGPBD_OK;
}

template <class T>
mgpbd_status mf_level0_final(Handle *h, const T *x, const T *b, const T *dinv, T omega,
                             const TopOut &o) {
  const bool dbl = sizeof(T) == 8;
  MG_TRY(mf_vertex(h, x));
  const T *gd = dbl ? (const T *)h->gd : (const T *)h->gd32;
  const T *gt = dbl ? (const T *)h->gt : (const T *)h->gt32;
  const T *u = dbl ? (const T *)h->u64 : (const T *)h->u32;
  const T *at = dbl ? (const T *)h->alpha_t : (const T *)h->at32;
  DotCtx c = o.c;
  c.sc = h->sc;
  if (o.dot)
    k_mf_row<T, MF_SWEEP_ZDOT><<<std::min(mf_grid(h->m, 256),
                                          wave_blocks((const void *)k_mf_row<T, MF_SWEEP_ZDOT>,
                                                      256)),
                                 256, 0, h->stream>>>(
        h->E, h->m, h->edge, h->tet, gd, gt, u, at, x, b, dinv, omega, nullptr, c, o.z, o.r);
  else
    k_mf_row<T, MF_SWEEP_Z><<<mf_grid(h->m, 256), 256, 0, h->stream>>>(
        h->E, h->m, h->edge, h->tet, gd, gt, u, at, x, b, dinv, omega, nullptr, c, o.z, o.r);
  MG_LAUNCH("k_mf_row(final sweep)");
  return MGPBD_OK;
}

template mgpbd_status mf_level0_final<float>(Handle *, const float *, const float *, const float *,
                                             float, const TopOut &);
template mgpbd_status mf_level0_final<double>(Handle *, const double *, const double *,
                                              const double *, double, const TopOut &);

}  // namespace mg
