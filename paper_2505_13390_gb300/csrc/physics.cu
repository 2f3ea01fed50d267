// Per-vertex and per-constraint kernels of Algorithm 1: rest shape,
// semi-implicit Euler prologue, constraint values and gradients, the values
// of A on the fixed pattern, and the dx / lambda / x update (eq. 5).
//
// Arithmetic is spelled out operation by operation (the library is built
// without FMA contraction), so that these kernels give the IEEE-754 result
// of the formulas as written:
//   distance  C = |d| - L0, |d| = sqrt(fma(dz,dz, fma(dy,dy, dx*dx))),
//             n = d/|d| (n = 0 if |d| = 0), gradients n and -n
//   volume    e_k = x_k - x_0, V = fma(e1z,c23z, fma(e1y,c23y, e1x*c23x))/6,
//             g1 = (e2 x e3)/6, g2 = (e3 x e1)/6, g3 = (e1 x e2)/6,
//             g0 = -((g1 + g2) + g3)
//   ARAP      (Sec. 5.3) C = |F - R|_F^2, F = Ds B with B = Dm^-1 (rows of B:
//             (e2 x e3, e3 x e1, e1 x e2) / det Dm at rest),
//             F_ac = fma(d3_a,B_2c, fma(d2_a,B_1c, d1_a*B_0c)); R by 20 Newton steps
//             R <- 0.5 * (R + R^-T) from R = F, R^-T = [c1 x c2, c2 x c0, c0 x c1] / det
//             (columns c_k of R); det F = 0 gives C = 0 and zero gradient;
//             C = sum over (a, c) row-major of fma(D_ac, D_ac, .), D = F - R;
//             g_k = 2 D B^T e_k (k = 1..3), g0 = -((g1 + g2) + g3)
//   A_ij      sum over shared vertices (ascending id) acc = fma(w_v, g_i.g_j, acc),
//             g_i.g_j = fma(gz_i,gz_j, fma(gy_i,gy_j, gx_i*gx_j)); A_ii + alpha~ last
#include "common.cuh"

namespace mg {

__device__ __forceinline__ double dist_eval(const double *xa, const double *xb, double L0,
                                            double n[3]) {
  double d0 = xa[0] - xb[0], d1 = xa[1] - xb[1], d2 = xa[2] - xb[2];
  double len = sqrt(fma(d2, d2, fma(d1, d1, d0 * d0)));
  if (len > 0.0) {
    n[0] = d0 / len;
    n[1] = d1 / len;
    n[2] = d2 / len;
  } else {
    n[0] = n[1] = n[2] = 0.0;
  }
  return len - L0;
}

__device__ __forceinline__ void cross3(const double *a, const double *b, double *c) {
  double t1, t2;
  t1 = a[1] * b[2]; t2 = a[2] * b[1]; c[0] = t1 - t2;
  t1 = a[2] * b[0]; t2 = a[0] * b[2]; c[1] = t1 - t2;
  t1 = a[0] * b[1]; t2 = a[1] * b[0]; c[2] = t1 - t2;
}

__device__ __forceinline__ double tet_eval(const double *x0, const double *x1, const double *x2,
                                           const double *x3, double V0, double g[12]) {
  double e1[3], e2[3], e3[3], c23[3], c31[3], c12[3];
  for (int k = 0; k < 3; ++k) {
    e1[k] = x1[k] - x0[k];
    e2[k] = x2[k] - x0[k];
    e3[k] = x3[k] - x0[k];
  }
  cross3(e2, e3, c23);
  cross3(e3, e1, c31);
  cross3(e1, e2, c12);
  for (int k = 0; k < 3; ++k) {
    g[3 + k] = c23[k] / 6.0;
    g[6 + k] = c31[k] / 6.0;
    g[9 + k] = c12[k] / 6.0;
    g[k] = -((g[3 + k] + g[6 + k]) + g[9 + k]);
  }
  double V = fma(e1[2], c23[2], fma(e1[1], c23[1], e1[0] * c23[0])) / 6.0;
  return V - V0;
}

constexpr int kArapPolarIters = 20;

__device__ void arap_rest(const double *x0, const double *x1, const double *x2,
                          const double *x3, double *B) {
  double e1[3], e2[3], e3[3], c[3][3];
  for (int k = 0; k < 3; ++k) {
    e1[k] = x1[k] - x0[k];
    e2[k] = x2[k] - x0[k];
    e3[k] = x3[k] - x0[k];
  }
  cross3(e2, e3, c[0]);
  cross3(e3, e1, c[1]);
  cross3(e1, e2, c[2]);
  const double det = fma(e1[2], c[0][2], fma(e1[1], c[0][1], e1[0] * c[0][0]));
  for (int r = 0; r < 3; ++r)
    for (int k = 0; k < 3; ++k) B[3 * r + k] = det != 0.0 ? c[r][k] / det : 0.0;
}

__device__ double arap_eval(const double *x0, const double *x1, const double *x2,
                            const double *x3, const double *B, double g[12]) {
  double d[3][3];  // d[k] = x_{k+1} - x_0, column k of Ds
  for (int a = 0; a < 3; ++a) {
    d[0][a] = x1[a] - x0[a];
    d[1][a] = x2[a] - x0[a];
    d[2][a] = x3[a] - x0[a];
  }
  double F[3][3], R[3][3];
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c)
      F[a][c] = fma(d[2][a], B[6 + c], fma(d[1][a], B[3 + c], d[0][a] * B[c]));
  double col[3][3], x12[3];
  for (int k = 0; k < 3; ++k)
    for (int a = 0; a < 3; ++a) col[k][a] = F[a][k];
  cross3(col[1], col[2], x12);
  const double detF = fma(col[0][2], x12[2], fma(col[0][1], x12[1], col[0][0] * x12[0]));
  if (detF == 0.0) {
    for (int k = 0; k < 12; ++k) g[k] = 0.0;
    return 0.0;
  }
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) R[a][c] = F[a][c];
  for (int it = 0; it < kArapPolarIters; ++it) {
    double cc[3][3], dual[3][3];
    for (int k = 0; k < 3; ++k)
      for (int a = 0; a < 3; ++a) cc[k][a] = R[a][k];
    cross3(cc[1], cc[2], dual[0]);
    cross3(cc[2], cc[0], dual[1]);
    cross3(cc[0], cc[1], dual[2]);
    const double det = fma(cc[0][2], dual[0][2], fma(cc[0][1], dual[0][1], cc[0][0] * dual[0][0]));
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
      const double t = fma(D[a][2], B[3 * k + 2], fma(D[a][1], B[3 * k + 1], D[a][0] * B[3 * k]));
      g[3 * (k + 1) + a] = 2.0 * t;
    }
  for (int a = 0; a < 3; ++a) g[a] = -((g[3 + a] + g[6 + a]) + g[9 + a]);
  return C;
}

__device__ __forceinline__ void load3(const double *p, double *o) {
  o[0] = p[0];
  o[1] = p[1];
  o[2] = p[2];
}

// ---------------------------------------------------------------------------
__global__ void k_rest(int E, int T, const int32_t *edge, const int32_t *tet, const double *X,
                       double *L0, double *V0, double *Dminv) {
  int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = tid; j < (int64_t)E + T; j += stride) {
    if (j < E) {
      double a[3], b[3], n[3];
      load3(X + 3 * (int64_t)edge[2 * j], a);
      load3(X + 3 * (int64_t)edge[2 * j + 1], b);
      L0[j] = dist_eval(a, b, 0.0, n);
    } else {
      int64_t t = j - E;
      const int32_t *q = tet + 4 * t;
      double p0[3], p1[3], p2[3], p3[3], g[12];
      load3(X + 3 * (int64_t)q[0], p0);
      load3(X + 3 * (int64_t)q[1], p1);
      load3(X + 3 * (int64_t)q[2], p2);
      load3(X + 3 * (int64_t)q[3], p3);
      V0[t] = tet_eval(p0, p1, p2, p3, 0.0, g);
      if (Dminv) arap_rest(p0, p1, p2, p3, Dminv + 9 * t);
    }
  }
}

mgpbd_status rest_shape(Handle *h) {
  if (h->m == 0) return MGPBD_OK;
  k_rest<<<blocks_for(h->m, 256), 256, 0, h->stream>>>(h->E, h->T, h->edge, h->tet, h->rest,
                                                       h->L0, h->V0, h->Dminv);
  MG_LAUNCH("k_rest");
  return MGPBD_OK;
}

// ---------------------------------------------------------------------------
// Alg. 1 prologue: free vertices v += dt g, x_old = x, x += dt v;
// pinned vertices (w = 0) keep x and get v = 0.  lambda = 0.
__global__ void k_begin_frame(int N, double dt, double g0, double g1, double g2, const double *w,
                              double *x, double *v, double *xold) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    double *xi = x + 3 * (int64_t)i, *vi = v + 3 * (int64_t)i, *oi = xold + 3 * (int64_t)i;
    double gg[3] = {g0, g1, g2};
    for (int k = 0; k < 3; ++k) oi[k] = xi[k];
    if (w[i] == 0.0) {
      vi[0] = vi[1] = vi[2] = 0.0;
      continue;
    }
    for (int k = 0; k < 3; ++k) {
      double t = dt * gg[k];
      double vk = vi[k] + t;
      vi[k] = vk;
      double t2 = dt * vk;
      xi[k] = xi[k] + t2;
    }
  }
}

mgpbd_status launch_begin_frame(Handle *h) {
  k_begin_frame<<<blocks_for(h->N, 256), 256, 0, h->stream>>>(
      h->N, h->p.dt, h->p.gravity[0], h->p.gravity[1], h->p.gravity[2], h->w, h->x, h->v, h->xold);
  MG_LAUNCH("k_begin_frame");
  if (h->m) MG_CUDA(cudaMemsetAsync(h->lambda, 0, sizeof(double) * h->m, h->stream));
  return MGPBD_OK;
}

// Alg. 1 epilogue: v = (x - x_old) / dt
__global__ void k_end_frame(int64_t n3, double dt, const double *x, const double *xold,
                            double *v) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n3;
       q += (int64_t)gridDim.x * blockDim.x)
    v[q] = (x[q] - xold[q]) / dt;
}

mgpbd_status launch_end_frame(Handle *h) {
  int64_t n3 = 3 * (int64_t)h->N;
  k_end_frame<<<blocks_for(n3, 256), 256, 0, h->stream>>>(n3, h->p.dt, h->x, h->xold, h->v);
  MG_LAUNCH("k_end_frame");
  return MGPBD_OK;
}

// ---------------------------------------------------------------------------
// Alg. 1: C and grad C; eq. 3: b = -C - alpha~ lambda
__global__ void k_eval(int E, int T, const int32_t *edge, const int32_t *tet, const double *x,
                       const double *L0, const double *V0, const double *Dminv,
                       const double *alpha_t, const double *lambda, double *C, double *b,
                       double *gd, double *gt) {
  int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = tid; j < (int64_t)E + T; j += stride) {
    double c;
    if (j < E) {
      double a[3], bb[3], n[3];
      load3(x + 3 * (int64_t)edge[2 * j], a);
      load3(x + 3 * (int64_t)edge[2 * j + 1], bb);
      c = dist_eval(a, bb, L0[j], n);
      gd[3 * j] = n[0];
      gd[3 * j + 1] = n[1];
      gd[3 * j + 2] = n[2];
    } else {
      int64_t t = j - E;
      const int32_t *q = tet + 4 * t;
      double p0[3], p1[3], p2[3], p3[3], g[12];
      load3(x + 3 * (int64_t)q[0], p0);
      load3(x + 3 * (int64_t)q[1], p1);
      load3(x + 3 * (int64_t)q[2], p2);
      load3(x + 3 * (int64_t)q[3], p3);
      c = Dminv ? arap_eval(p0, p1, p2, p3, Dminv + 9 * t, g) : tet_eval(p0, p1, p2, p3, V0[t], g);
      double *o = gt + 12 * t;
      for (int k = 0; k < 12; ++k) o[k] = g[k];
    }
    C[j] = c;
    double t = alpha_t[j] * lambda[j];
    b[j] = (-c) - t;
  }
}

mgpbd_status launch_eval(Handle *h) {
  if (h->m == 0) return MGPBD_OK;
  k_eval<<<blocks_for(h->m, 256), 256, 0, h->stream>>>(h->E, h->T, h->edge, h->tet, h->x, h->L0,
                                                       h->V0, h->Dminv, h->alpha_t, h->lambda,
                                                       h->C, h->b, h->gd, h->gt);
  MG_LAUNCH("k_eval");
  return MGPBD_OK;
}

// ---------------------------------------------------------------------------
// gradient of row j at slot s
__device__ __forceinline__ void row_grad(int j, int s, int E, const double *gd, const double *gt,
                                         double g[3]) {
  if (j < E) {
    const double *n = gd + 3 * (int64_t)j;
    if (s == 0) {
      g[0] = n[0]; g[1] = n[1]; g[2] = n[2];
    } else {
      g[0] = -n[0]; g[1] = -n[1]; g[2] = -n[2];
    }
  } else {
    const double *t = gt + 12 * (int64_t)(j - E) + 3 * s;
    g[0] = t[0]; g[1] = t[1]; g[2] = t[2];
  }
}

__device__ __forceinline__ double gdot(const double *a, const double *b) {
  return fma(a[2], b[2], fma(a[1], b[1], a[0] * b[0]));
}

// Values of A (eq. 3, Sec. 4.2 formulas); one warp per row, lanes over the
// row's off-diagonals; lane 0 also forms the diagonal.  Also writes 1/A_ii
// and, in mixed precision, the FP32 mirrors.
__global__ void k_assemble(int m, int E, const int32_t *edge, const int32_t *tet, const double *w,
                           const double *gd, const double *gt, const double *alpha_t,
                           const int64_t *ptr, const int32_t *col, const uint16_t *map,
                           double *val, double *dinv, float *val32, float *dinv32) {
  const int lane = threadIdx.x & 31;
  int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t ii = warp; ii < m; ii += nwarps) {
    int i = (int)ii;
    int32_t v[4];
    int c;
    if (i < E) {
      v[0] = edge[2 * (int64_t)i];
      v[1] = edge[2 * (int64_t)i + 1];
      v[2] = v[3] = 0;
      c = 2;
    } else {
      const int32_t *t = tet + 4 * (int64_t)(i - E);
      v[0] = t[0]; v[1] = t[1]; v[2] = t[2]; v[3] = t[3];
      c = 4;
    }
    double gi[4][3], wi[4];
    for (int s = 0; s < 4; ++s) {
      if (s < c) {
        row_grad(i, s, E, gd, gt, gi[s]);
        wi[s] = w[v[s]];
      } else {
        gi[s][0] = gi[s][1] = gi[s][2] = 0.0;
        wi[s] = 0.0;
      }
    }
    int64_t s0 = ptr[i], e = ptr[i + 1] - 1;
    for (int64_t k = s0 + lane; k < e; k += 32) {
      int j = col[k];
      unsigned code = map[k];
      int ns = code & 3;
      double acc = 0.0;
      for (int p = 0; p < ns; ++p) {
        int si = (code >> (2 + 4 * p)) & 3, sj = (code >> (4 + 4 * p)) & 3;
        double gj[3];
        row_grad(j, sj, E, gd, gt, gj);
        acc = fma(wi[si], gdot(gi[si], gj), acc);
      }
      val[k] = acc;
      if (val32) val32[k] = f64_to_f32(acc);
    }
    if (lane == 0) {
      double acc = 0.0;
      for (int s = 0; s < c; ++s) acc = fma(wi[s], gdot(gi[s], gi[s]), acc);
      double d = acc + alpha_t[i];
      val[e] = d;
      dinv[i] = 1.0 / d;
      if (val32) {
        val32[e] = f64_to_f32(d);
        dinv32[i] = f64_to_f32(1.0 / d);
      }
    }
  }
}

mgpbd_status launch_assemble(Handle *h) {
  if (h->m == 0) return MGPBD_OK;
  Level &L = h->lev[0];
  const int th = 256;
  int64_t warps = h->m;
  int blocks = blocks_for(warps * 32, th);
  k_assemble<<<blocks, th, 0, h->stream>>>(h->m, h->E, h->edge, h->tet, h->w, h->gd, h->gt,
                                            h->alpha_t, L.ptr, L.col, h->map, L.val, L.dinv,
                                            L.val32, L.dinv32);
  MG_LAUNCH("k_assemble");
  return MGPBD_OK;
}

// ---------------------------------------------------------------------------
// eq. 5: dx_v = w_v * sum_{j incident to v, ascending} fma(g_{j,v}, dl_j, .)
__global__ void k_dx(int N, int E, const int32_t *edge, const int32_t *tet, const int64_t *vptr,
                     const int32_t *vrow, const double *gd, const double *gt, const double *dl,
                     const double *w, double *dx) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x) {
    double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0;
    for (int64_t q = vptr[v]; q < vptr[v + 1]; ++q) {
      int j = vrow[q];
      int s;
      if (j < E) {
        s = edge[2 * (int64_t)j] == v ? 0 : 1;
      } else {
        const int32_t *t = tet + 4 * (int64_t)(j - E);
        s = t[0] == v ? 0 : (t[1] == v ? 1 : (t[2] == v ? 2 : 3));
      }
      double g[3];
      row_grad(j, s, E, gd, gt, g);
      double d = dl[j];
      acc0 = fma(g[0], d, acc0);
      acc1 = fma(g[1], d, acc1);
      acc2 = fma(g[2], d, acc2);
    }
    double wv = w[v];
    double *o = dx + 3 * (int64_t)v;
    o[0] = wv * acc0;
    o[1] = wv * acc1;
    o[2] = wv * acc2;
  }
}

// x = fma(omega, dx, base)   (base may alias x)
__global__ void k_apply_x(int64_t n3, double omega, const double *dx, const double *base,
                          double *x) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n3;
       q += (int64_t)gridDim.x * blockDim.x)
    x[q] = fma(omega, dx[q], base[q]);
}

__global__ void k_add(int64_t n, const double *a, double *y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = y[i] + a[i];
}

// Alg. 1 update: lambda += dl, x = fma(omega, dx, x).  With backtracking the
// step starts at omega_x and halves while |b| at the new state is not below
// the current |b|, at most `backtrack` times (the last trial is kept).
mgpbd_status launch_update(Handle *h, mgpbd_solve_info *info) {
  info->omega = h->p.omega_x;
  info->bnorm_after = -1.0;
  if (h->m == 0) return MGPBD_OK;
  const int64_t n3 = 3 * (int64_t)h->N;
  k_dx<<<blocks_for(h->N, 128), 128, 0, h->stream>>>(h->N, h->E, h->edge, h->tet, h->vptr,
                                                    h->vrow, h->gd, h->gt, h->dl, h->w, h->dx);
  MG_LAUNCH("k_dx");
  k_add<<<blocks_for(h->m, 256), 256, 0, h->stream>>>(h->m, h->dl, h->lambda);
  MG_LAUNCH("k_add");
  double om = h->p.omega_x;
  if (h->p.backtrack <= 0) {
    k_apply_x<<<blocks_for(n3, 256), 256, 0, h->stream>>>(n3, om, h->dx, h->x, h->x);
    MG_LAUNCH("k_apply_x");
    return MGPBD_OK;
  }
  MG_CUDA(cudaMemcpyAsync(h->xbak, h->x, sizeof(double) * n3, cudaMemcpyDeviceToDevice,
                          h->stream));
  double *d_nb = h->partials + 4096 + 4;  // scratch scalar after the dot partials
  double nb = 0.0;
  for (int t = 0; t <= h->p.backtrack; ++t) {
    k_apply_x<<<blocks_for(n3, 256), 256, 0, h->stream>>>(n3, om, h->dx, h->xbak, h->x);
    MG_LAUNCH("k_apply_x");
    MG_TRY(launch_eval(h));
    MG_TRY(dot_dd(h, h->b, h->b, h->m, d_nb));
    MG_CUDA(cudaMemcpyAsync(&nb, d_nb, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    MG_CUDA(cudaStreamSynchronize(h->stream));
    nb = sqrt(nb);
    if (nb < info->bnorm || t == h->p.backtrack) break;
    om = om * 0.5;
  }
  info->omega = om;
  info->bnorm_after = nb;
  return MGPBD_OK;
}

}  // namespace mg
