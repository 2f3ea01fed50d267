// Lazy UA-AMG setup (Sec. 4.1-4.3, setup-pipeline figure of the paper) and the Galerkin
// re-form of Sec. 4.4, on the device.
//
//   near-kernel  B_0: nk_sweeps weighted-Jacobi sweeps on A x = 0 from
//                x0_i = u_i * max|A_ij| (Sec. 4.3), row sums in storage order
//   filter       off-diagonal A_ij strong unless |A_ij| < theta_s sqrt(|A_ii||A_jj|)
//   aggregate    deterministic MIS-2 rule; rows without a strong neighbour
//                are left alone (no aggregate, zero row of P); roots = greedy
//                distance-2 independent set of the strength graph in decreasing
//                priority h64(key(seed_agg, l, i)), computed here by parallel
//                rounds (a row becomes a root when it has the highest
//                priority among undecided rows within distance 2); strong
//                neighbours of a root join it; the rest join the aggregate of
//                their strongest pass-1 neighbour (ties: smaller aggregate
//                id, then smaller neighbour index)
//   inject       P_i = B_i / |B_agg|, next near-kernel B_{l+1}[a] = |B_agg|
//                (k = 1 QR), |B_agg| summed over members in ascending order;
//                with k > 1 vectors a modified Gram-Schmidt QR per aggregate
//                (k columns of P, k unknowns per coarse aggregate)
//   Galerkin     A_{l+1} = P^T A_l P; entry (a,b), b >= a, accumulates
//                fma(P_i*A_ij, P_j, acc) over member rows i of a ascending and
//                row i's storage order; entries with b < a copy (b,a)
//   colouring    Jones-Plassmann rounds: a row takes the smallest colour absent
//                among its higher-priority neighbours once those are coloured
//   smoother     omega_l = 2 / (safety * lambda_max(D^-1 A_l) + lambda_min_est)
// All integer decisions and the values they depend on follow the same
// operation order as a plain sequential FP64 program, so aggregates, P, B and
// colours are reproducible bit for bit.
#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace mg {

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ double diag_at(const int64_t *ptr, const double *val, int i) {
  return val[ptr[i + 1] - 1];
}

// lexicographic (pri, idx) max over a warp; idx < 0 means "none"
__device__ __forceinline__ void warp_best(uint64_t &pri, int &idx) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    uint64_t p2 = __shfl_xor_sync(0xffffffffu, pri, o);
    int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
    bool better = i2 >= 0 && (idx < 0 || p2 > pri || (p2 == pri && i2 > idx));
    if (better) {
      pri = p2;
      idx = i2;
    }
  }
}

#define WARP_LOOP(nrows)                                                        \
  const int lane = threadIdx.x & 31;                                            \
  const int64_t nwarps_ = ((int64_t)gridDim.x * blockDim.x) >> 5;               \
  for (int64_t row_ = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;   \
       row_ < (nrows); row_ += nwarps_)

static inline int warp_blocks(int64_t rows, int th = 256) { return blocks_for(rows * 32, th); }

// ---------------------------------------------------------------------------
// near-kernel (Sec. 4.3)
// ---------------------------------------------------------------------------
__global__ void k_absmax(int64_t nnz, const double *val, unsigned long long *out) {
  double m = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
       k += (int64_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs(val[k]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

__global__ void k_nk_init(int n, uint64_t seed, const unsigned long long *amax_bits, double *x) {
  double amax = __longlong_as_double((long long)*amax_bits);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    x[i] = u01(h64(hkey(seed, 0, i))) * amax;
}

// row sum in storage order: s = fma(A_ij, x_j, s), folded sequentially
__device__ __forceinline__ double row_dot_canonical(const int64_t s0, const int64_t e,
                                                    const int32_t *col, const double *val,
                                                    const double *x, int lane) {
  double s = 0.0;
  for (int64_t base = s0; base < e; base += 32) {
    int64_t k = base + lane;
    double a = 0.0, xv = 0.0;
    if (k < e) {
      a = val[k];
      xv = x[col[k]];
    }
    int cnt = (int)min((int64_t)32, e - base);
    for (int t = 0; t < cnt; ++t) {
      double at = __shfl_sync(0xffffffffu, a, t);
      double xt = __shfl_sync(0xffffffffu, xv, t);
      if (lane == 0) s = fma(at, xt, s);
    }
  }
  return __shfl_sync(0xffffffffu, s, 0);
}

__global__ void k_nk_sweep(int n, const int64_t *ptr, const int32_t *col, const double *val,
                           double omega, const double *x, double *xn) {
  WARP_LOOP(n) {
    int i = (int)row_;
    int64_t s0 = ptr[i], e = ptr[i + 1];
    double s = row_dot_canonical(s0, e, col, val, x, lane);
    if (lane == 0) xn[i] = fma(-omega, s / val[e - 1], x[i]);
  }
}

// ---------------------------------------------------------------------------
// strength filter (Sec. 4.1)
// ---------------------------------------------------------------------------
// also initialises the MIS-2 state: rows without a strong off-diagonal are
// left alone (state 2: never a root, no aggregate), the others undecided (0)
__global__ void k_strength(int n, const int64_t *ptr, const int32_t *col, const double *val,
                           double theta, uint8_t *S, uint8_t *state) {
  WARP_LOOP(n) {
    int i = (int)row_;
    int64_t s0 = ptr[i], e = ptr[i + 1] - 1;
    double aii = fabs(val[e]);
    int any = 0;
    for (int64_t k = s0 + lane; k < e; k += 32) {
      int j = col[k];
      double prod = aii * fabs(diag_at(ptr, val, j));
      double thr = theta * sqrt(prod);
      uint8_t st = fabs(val[k]) >= thr ? 1 : 0;
      S[k] = st;
      any |= st;
    }
    any = __any_sync(0xffffffffu, any);
    if (lane == 0) {
      S[e] = 0;
      state[i] = any ? 0 : 2;
    }
  }
}

// ---------------------------------------------------------------------------
// MIS-2 rounds
// state: 0 undecided, 1 root, 2 excluded
// ---------------------------------------------------------------------------
__global__ void k_mis_m1(int n, const int64_t *ptr, const int32_t *col, const uint8_t *S,
                         const uint8_t *state, uint64_t seed, int l, uint64_t *m1p, int *m1i) {
  WARP_LOOP(n) {
    int i = (int)row_;
    uint64_t bp = 0;
    int bi = -1;
    if (lane == 0 && state[i] == 0) {
      bp = h64(hkey(seed, l, i));
      bi = i;
    }
    int64_t s0 = ptr[i], e = ptr[i + 1] - 1;
    for (int64_t k = s0 + lane; k < e; k += 32) {
      if (!S[k]) continue;
      int j = col[k];
      if (state[j] != 0) continue;
      uint64_t pj = h64(hkey(seed, l, j));
      if (bi < 0 || pj > bp || (pj == bp && j > bi)) {
        bp = pj;
        bi = j;
      }
    }
    warp_best(bp, bi);
    if (lane == 0) {
      m1p[i] = bp;
      m1i[i] = bi;
    }
  }
}

__global__ void k_mis_m2(int n, const int64_t *ptr, const int32_t *col, const uint8_t *S,
                         const uint64_t *m1p, const int *m1i, uint8_t *state) {
  WARP_LOOP(n) {
    int i = (int)row_;
    uint64_t bp = 0;
    int bi = -1;
    if (lane == 0) {
      bp = m1p[i];
      bi = m1i[i];
    }
    int64_t s0 = ptr[i], e = ptr[i + 1] - 1;
    for (int64_t k = s0 + lane; k < e; k += 32) {
      if (!S[k]) continue;
      int j = col[k];
      int ij = m1i[j];
      if (ij < 0) continue;
      uint64_t pj = m1p[j];
      if (bi < 0 || pj > bp || (pj == bp && ij > bi)) {
        bp = pj;
        bi = ij;
      }
    }
    warp_best(bp, bi);
    if (lane == 0 && state[i] == 0 && bi == i) state[i] = 1;
  }
}

__global__ void k_mis_e1(int n, const int64_t *ptr, const int32_t *col, const uint8_t *S,
                         const uint8_t *state, uint8_t *e1) {
  WARP_LOOP(n) {
    int i = (int)row_;
    int hit = 0;
    int64_t s0 = ptr[i], e = ptr[i + 1] - 1;
    for (int64_t k = s0 + lane; k < e; k += 32)
      if (S[k] && state[col[k]] == 1) hit = 1;
    hit = __any_sync(0xffffffffu, hit);
    if (lane == 0) e1[i] = (uint8_t)(hit || state[i] == 1);
  }
}

__global__ void k_mis_e2(int n, const int64_t *ptr, const int32_t *col, const uint8_t *S,
                         const uint8_t *e1, uint8_t *state, int *remaining) {
  WARP_LOOP(n) {
    int i = (int)row_;
    if (state[i] != 0) continue;
    int hit = 0;
    int64_t s0 = ptr[i], e = ptr[i + 1] - 1;
    for (int64_t k = s0 + lane; k < e; k += 32)
      if (S[k] && e1[col[k]]) hit = 1;
    hit = __any_sync(0xffffffffu, hit) || e1[i];
    if (lane == 0) {
      if (hit) state[i] = 2;
      else atomicAdd(remaining, 1);
    }
  }
}

__global__ void k_root_flags(int n, const uint8_t *state, uint8_t *root, int64_t *flag64) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    uint8_t r = state[i] == 1;
    root[i] = r;
    flag64[i] = r;
  }
}

__global__ void k_agg_pass1(int n, const int64_t *ptr, const int32_t *col, const uint8_t *S,
                            const uint8_t *root, const int64_t *ids, int *p1) {
  WARP_LOOP(n) {
    int i = (int)row_;
    int a = -1;
    if (root[i]) {
      a = (int)ids[i];
    } else {
      int64_t s0 = ptr[i], e = ptr[i + 1] - 1;
      for (int64_t k = s0 + lane; k < e; k += 32) {
        int j = col[k];
        if (S[k] && root[j]) a = (int)ids[j];  // at most one root is adjacent (MIS-2)
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a = max(a, __shfl_xor_sync(0xffffffffu, a, o));
    }
    if (lane == 0) p1[i] = a;
  }
}

// pass 2: strongest pass-1 neighbour; key (|A_ij| desc, aggregate asc, j asc).
// Rows without a strong neighbour stay alone (agg = -1).
__global__ void k_agg_pass2(int n, const int64_t *ptr, const int32_t *col, const double *val,
                            const uint8_t *S, const int *p1, int32_t *agg, int *bad) {
  WARP_LOOP(n) {
    int i = (int)row_;
    int mine = p1[i];
    if (mine >= 0) {
      if (lane == 0) agg[i] = mine;
      continue;
    }
    unsigned long long bs = 0;
    int ba = -1, bw = -1, strong = 0;
    int64_t s0 = ptr[i], e = ptr[i + 1] - 1;
    for (int64_t k = s0 + lane; k < e; k += 32) {
      if (!S[k]) continue;
      strong = 1;
      int w = col[k];
      int a = p1[w];
      if (a < 0) continue;
      unsigned long long s = (unsigned long long)__double_as_longlong(fabs(val[k]));
      if (ba < 0 || s > bs || (s == bs && (a < ba || (a == ba && w < bw)))) {
        bs = s;
        ba = a;
        bw = w;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long s2 = __shfl_xor_sync(0xffffffffu, bs, o);
      int a2 = __shfl_xor_sync(0xffffffffu, ba, o);
      int w2 = __shfl_xor_sync(0xffffffffu, bw, o);
      if (a2 >= 0 && (ba < 0 || s2 > bs || (s2 == bs && (a2 < ba || (a2 == ba && w2 < bw))))) {
        bs = s2;
        ba = a2;
        bw = w2;
      }
    }
    strong = __any_sync(0xffffffffu, strong);
    if (lane == 0) {
      agg[i] = ba;
      if (ba < 0 && strong) atomicExch(bad, 1);
    }
  }
}

// ---------------------------------------------------------------------------
// aggregate member lists (ascending rows)
// ---------------------------------------------------------------------------
__global__ void k_mem_count(int n, const int32_t *agg, unsigned long long *cnt) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if (agg[i] >= 0) atomicAdd(&cnt[agg[i]], 1ull);
}

__global__ void k_mem_fill(int n, const int32_t *agg, const int64_t *mptr,
                           unsigned long long *fill, int32_t *tmp) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (agg[i] < 0) continue;
    unsigned long long pos = atomicAdd(&fill[agg[i]], 1ull);
    tmp[mptr[agg[i]] + (int64_t)pos] = i;
  }
}

// rank sort inside each aggregate (members are distinct), warp per aggregate
__global__ void k_mem_sort(int na, const int64_t *mptr, const int32_t *tmp, int32_t *mrow,
                           int *max_members) {
  WARP_LOOP(na) {
    int a = (int)row_;
    int64_t s0 = mptr[a], e = mptr[a + 1];
    int64_t len = e - s0;
    for (int64_t q = s0 + lane; q < e; q += 32) {
      int32_t me = tmp[q];
      int64_t rank = 0;
      for (int64_t t = s0; t < e; ++t) rank += tmp[t] < me;
      mrow[s0 + rank] = me;
    }
    if (lane == 0) atomicMax(max_members, (int)len);
  }
}

// ---------------------------------------------------------------------------
// injection (k = 1): P_i = B_i / |B_a|, B_{l+1}[a] = |B_a|
// ---------------------------------------------------------------------------
__global__ void k_inject(int na, const int64_t *mptr, const int32_t *mrow, const double *B,
                         double *P, double *Bc) {
  WARP_LOOP(na) {
    int a = (int)row_;
    int64_t s0 = mptr[a], e = mptr[a + 1];
    double acc = 0.0;
    for (int64_t base = s0; base < e; base += 32) {
      int64_t q = base + lane;
      double bi = q < e ? B[mrow[q]] : 0.0;
      int cnt = (int)min((int64_t)32, e - base);
      for (int t = 0; t < cnt; ++t) {
        double bt = __shfl_sync(0xffffffffu, bi, t);
        if (lane == 0) acc = fma(bt, bt, acc);
      }
    }
    acc = __shfl_sync(0xffffffffu, acc, 0);
    double nrm = sqrt(acc);
    double sz = (double)(e - s0);
    for (int64_t q = s0 + lane; q < e; q += 32) {
      int i = mrow[q];
      P[i] = nrm > 0.0 ? B[i] / nrm : 1.0 / sqrt(sz);
    }
    if (lane == 0) Bc[a] = nrm;
  }
}

// ---------------------------------------------------------------------------
// Galerkin pattern: block per coarse row, shared-memory hash set of columns
// ---------------------------------------------------------------------------
constexpr int kHash = 8192;
constexpr int kHashList = 4000;  // unique columns per coarse row (static smem < 48 KB)

__device__ __forceinline__ void hash_insert(int *tab, int key, int *n_unique) {
  unsigned hsh = ((unsigned)key * 2654435761u) & (kHash - 1);
  for (int probe = 0; probe < kHash; ++probe) {
    int old = atomicCAS(&tab[hsh], -1, key);
    if (old == -1) {
      atomicAdd(n_unique, 1);
      return;
    }
    if (old == key) return;
    hsh = (hsh + 1) & (kHash - 1);
  }
}

__global__ void k_gal_pattern(int na, const int64_t *mptr, const int32_t *mrow,
                              const int64_t *ptr, const int32_t *col, const int32_t *agg,
                              int64_t *cnt, const int64_t *cptr, int32_t *ccol, int *overflow) {
  __shared__ int tab[kHash];
  __shared__ int n_unique;
  __shared__ int n_list;
  __shared__ int list[kHashList];
  for (int a = blockIdx.x; a < na; a += gridDim.x) {
    for (int t = threadIdx.x; t < kHash; t += blockDim.x) tab[t] = -1;
    if (threadIdx.x == 0) {
      n_unique = 0;
      n_list = 0;
    }
    __syncthreads();
    for (int64_t q = mptr[a]; q < mptr[a + 1]; ++q) {
      int i = mrow[q];
      for (int64_t k = ptr[i] + threadIdx.x; k < ptr[i + 1]; k += blockDim.x) {
        int b = agg[col[k]];
        if (b >= 0 && b != a && n_unique < kHashList) hash_insert(tab, b, &n_unique);
      }
    }
    __syncthreads();
    if (n_unique >= kHashList) {
      if (threadIdx.x == 0) atomicExch(overflow, 1);
      __syncthreads();
      continue;
    }
    if (!ccol) {
      if (threadIdx.x == 0) cnt[a] = n_unique + 1;
      __syncthreads();
      continue;
    }
    for (int t = threadIdx.x; t < kHash; t += blockDim.x)
      if (tab[t] >= 0) list[atomicAdd(&n_list, 1)] = tab[t];
    __syncthreads();
    int u = n_list;
    int64_t base = cptr[a];
    for (int t = threadIdx.x; t < u; t += blockDim.x) {
      int me = list[t], rank = 0;
      for (int s = 0; s < u; ++s) rank += list[s] < me;
      ccol[base + rank] = me;
    }
    if (threadIdx.x == 0) ccol[base + u] = a;  // diagonal last
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Galerkin values, canonical order (warp per coarse row, shared accumulators)
// ---------------------------------------------------------------------------
__global__ void k_gal_values(int na, const int64_t *mptr, const int32_t *mrow,
                             const int64_t *ptr, const int32_t *col, const double *val,
                             const int32_t *agg, const double *P, const int64_t *cptr,
                             const int32_t *ccol, double *cval, int maxlen) {
  extern __shared__ unsigned char smem_raw[];
  const int wib = threadIdx.x >> 5;
  double *acc = reinterpret_cast<double *>(smem_raw) + (size_t)wib * maxlen;
  int *cols = reinterpret_cast<int *>(reinterpret_cast<double *>(smem_raw) +
                                      (size_t)(blockDim.x >> 5) * maxlen) +
              (size_t)wib * maxlen;
  WARP_LOOP(na) {
    int a = (int)row_;
    int64_t cb = cptr[a];
    int len = (int)(cptr[a + 1] - cb);
    for (int t = lane; t < len; t += 32) {
      acc[t] = 0.0;
      cols[t] = ccol[cb + t];
    }
    __syncwarp();
    for (int64_t q = mptr[a]; q < mptr[a + 1]; ++q) {
      int i = mrow[q];
      double pi = P[i];
      int64_t s0 = ptr[i], e = ptr[i + 1];
      for (int64_t base = s0; base < e; base += 32) {
        int64_t k = base + lane;
        int slot = -1;
        double tt = 0.0, pj = 0.0;
        if (k < e) {
          int j = col[k];
          int b = agg[j];
          if (b >= a) {
            tt = pi * val[k];
            pj = P[j];
            if (b == a) {
              slot = len - 1;
            } else {
              int lo = 0, hi = len - 1;
              while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (cols[mid] < b) lo = mid + 1;
                else hi = mid;
              }
              slot = lo;
            }
          }
        }
        int cnt = (int)min((int64_t)32, e - base);
        for (int t = 0; t < cnt; ++t) {
          int st = __shfl_sync(0xffffffffu, slot, t);
          double tv = __shfl_sync(0xffffffffu, tt, t);
          double pv = __shfl_sync(0xffffffffu, pj, t);
          if (lane == 0 && st >= 0) acc[st] = fma(tv, pv, acc[st]);
        }
      }
    }
    __syncwarp();
    for (int t = lane; t < len; t += 32)
      if (cols[t] >= a) cval[cb + t] = acc[t];
    __syncwarp();
  }
}

__global__ void k_gal_mirror(int na, const int64_t *cptr, const int32_t *ccol, double *cval) {
  WARP_LOOP(na) {
    int a = (int)row_;
    int64_t s0 = cptr[a], e = cptr[a + 1] - 1;
    for (int64_t k = s0 + lane; k < e; k += 32) {
      int b = ccol[k];
      if (b >= a) continue;
      int64_t lo = cptr[b], hi = cptr[b + 1] - 1;
      while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (ccol[mid] < a) lo = mid + 1;
        else hi = mid;
      }
      cval[k] = cval[lo];
    }
  }
}

// 1/A_ii and FP32 mirrors of a level
__global__ void k_level_aux(int n, const int64_t *ptr, const double *val, double *dinv,
                            float *dinv32) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double d = val[ptr[i + 1] - 1];
    double r = 1.0 / d;
    dinv[i] = r;
    if (dinv32) dinv32[i] = f64_to_f32(r);
  }
}

__global__ void k_to_f32(int64_t n, const double *a, float *b) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    b[k] = f64_to_f32(a[k]);
}

// ---------------------------------------------------------------------------
// Jones-Plassmann colouring
// ---------------------------------------------------------------------------
__global__ void k_jp_round(int n, const int64_t *ptr, const int32_t *col, uint64_t seed, int l,
                           int32_t *color, int *remaining) {
  WARP_LOOP(n) {
    int i = (int)row_;
    if (((volatile int32_t *)color)[i] >= 0) continue;
    uint64_t pi = h64(hkey(seed, l, i));
    int64_t s0 = ptr[i], e = ptr[i + 1] - 1;
    int wait = 0;
    for (int64_t k = s0 + lane; k < e; k += 32) {
      int j = col[k];
      uint64_t pj = h64(hkey(seed, l, j));
      if ((pj > pi || (pj == pi && j > i)) && ((volatile int32_t *)color)[j] < 0) wait = 1;
    }
    if (__any_sync(0xffffffffu, wait)) {
      if (lane == 0) atomicAdd(remaining, 1);
      continue;
    }
    int c = -1;
    for (int base = 0; c < 0; base += 64) {
      unsigned long long used = 0;
      for (int64_t k = s0 + lane; k < e; k += 32) {
        int j = col[k];
        uint64_t pj = h64(hkey(seed, l, j));
        if (pj > pi || (pj == pi && j > i)) {
          int cj = ((volatile int32_t *)color)[j];
          if (cj >= base && cj < base + 64) used |= 1ull << (cj - base);
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) used |= __shfl_xor_sync(0xffffffffu, used, o);
      if (~used) c = base + __ffsll((long long)~used) - 1;
    }
    if (lane == 0) ((volatile int32_t *)color)[i] = c;
  }
}

__global__ void k_max_i32(int n, const int32_t *a, int *out) {
  int m = -1;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    m = max(m, a[i]);
  atomicMax(out, m);
}

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------
static mgpbd_status read_int(Handle *h, const int *d, int *out) {
  MG_CUDA(cudaMemcpyAsync(h->flag_host, d, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  MG_CUDA(cudaStreamSynchronize(h->stream));
  *out = *h->flag_host;
  return MGPBD_OK;
}

static size_t tsize(const Handle *h) { return h->p.precision == MGPBD_MIXED ? 4 : 8; }

// Level 0's member order (matrix-free operator, one column of P): pos_i =
// the position of row i in the member list (-1 before: rows in no
// aggregate), and P in member order in the V-cycle's precision.  The
// level-0 residual is then written, and restricted, in member order: the
// restriction streams P and r instead of gathering them row by row, with
// the same products summed in the same order.
__global__ void k_member_order(int na, const int64_t *mptr, const int32_t *mrow, const double *P,
                               const float *P32, double *Pm64, float *Pm32, int32_t *pos) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < na; a += gridDim.x * blockDim.x)
    for (int64_t q = mptr[a]; q < mptr[a + 1]; ++q) {
      const int i = mrow[q];
      pos[i] = (int32_t)q;
      if (Pm64) Pm64[q] = P[i];
      else Pm32[q] = P32[i];
    }
}

static mgpbd_status member_order_level0(Handle *h) {
  Level &L = h->lev[0];
  const bool mixed = h->p.precision == MGPBD_MIXED;
  if (!L.mpos) {
    MG_TRY(alloc_n(h->arena, &L.mpos, (size_t)L.n));
    MG_TRY(h->arena.alloc(&L.Pm, tsize(h) * (size_t)L.n));
  }
  MG_CUDA(cudaMemsetAsync(L.mpos, 0xff, sizeof(int32_t) * (size_t)L.n, h->stream));
  k_member_order<<<blocks_for(L.n_agg, 128), 128, 0, h->stream>>>(
      L.n_agg, L.mptr, L.mrow, L.P, L.P32, mixed ? nullptr : (double *)L.Pm,
      mixed ? (float *)L.Pm : nullptr, L.mpos);
  MG_LAUNCH("k_member_order");
  return MGPBD_OK;
}

// n-sized and nnz-sized buffers of a level, grown on demand
static mgpbd_status ensure_level(Handle *h, int l, int n, int64_t nnz) {
  Level &L = h->lev[l];
  bool mixed = h->p.precision == MGPBD_MIXED;
  if (n > L.cap_n) {
    int cap = std::max(n, L.cap_n + L.cap_n / 4);
    if (l > 0) {
      h->arena.release(L.ptr);
      h->arena.release(L.dinv);
      h->arena.release(L.dinv32);
      L.dinv32 = nullptr;
      MG_TRY(alloc_n(h->arena, &L.ptr, (size_t)cap + 1));
      MG_TRY(alloc_n(h->arena, &L.dinv, (size_t)cap));
      if (mixed) MG_TRY(alloc_n(h->arena, &L.dinv32, (size_t)cap));
    }
    void *olds[] = {L.agg, L.root, L.P, L.P32, L.B, L.pdead, L.mptr, L.mrow, L.color, L.crow,
                    L.x, L.x2, L.b, L.r, L.t, L.gbptr};
    for (void *o : olds) h->arena.release(o);
    L.P32 = nullptr;
    L.crow = nullptr;
    L.pdead = nullptr;
    L.gbptr = nullptr;
    const size_t k = (size_t)h->p.nk_vectors;
    MG_TRY(alloc_n(h->arena, &L.agg, (size_t)cap));
    MG_TRY(alloc_n(h->arena, &L.root, (size_t)cap));
    MG_TRY(alloc_n(h->arena, &L.P, (size_t)cap * k));
    if (mixed) MG_TRY(alloc_n(h->arena, &L.P32, (size_t)cap * k));
    MG_TRY(alloc_n(h->arena, &L.B, (size_t)cap * k));
    if (k > 1) {
      MG_TRY(alloc_n(h->arena, &L.pdead, (size_t)cap * k));
      MG_TRY(alloc_n(h->arena, &L.gbptr, (size_t)cap + 1));
    }
    MG_TRY(alloc_n(h->arena, &L.mptr, (size_t)cap + 1));
    MG_TRY(alloc_n(h->arena, &L.mrow, (size_t)cap));
    MG_TRY(alloc_n(h->arena, &L.color, (size_t)cap));
    MG_TRY(h->arena.alloc(&L.x, tsize(h) * cap));
    MG_TRY(h->arena.alloc(&L.x2, tsize(h) * cap));
    MG_TRY(h->arena.alloc(&L.b, tsize(h) * cap));
    MG_TRY(h->arena.alloc(&L.r, tsize(h) * cap));
    MG_TRY(h->arena.alloc(&L.t, tsize(h) * cap));
    L.cap_n = cap;
  }
  if (l > 0 && nnz > L.cap_nnz) {
    int64_t cap = std::max(nnz, L.cap_nnz + L.cap_nnz / 4);
    h->arena.release(L.col);
    h->arena.release(L.val);
    h->arena.release(L.val32);
    L.val32 = nullptr;
    MG_TRY(alloc_n(h->arena, &L.col, (size_t)cap));
    MG_TRY(alloc_n(h->arena, &L.val, (size_t)cap));
    if (mixed) MG_TRY(alloc_n(h->arena, &L.val32, (size_t)cap));
    L.cap_nnz = cap;
  }
  L.n = n;
  if (l > 0) L.nnz = nnz;
  return MGPBD_OK;
}

mgpbd_status level_precision_copies(Handle *h, int l) {
  Level &L = h->lev[l];
  if (L.n == 0) return MGPBD_OK;
  k_level_aux<<<blocks_for(L.n, 256), 256, 0, h->stream>>>(L.n, L.ptr, L.val, L.dinv, L.dinv32);
  MG_LAUNCH("k_level_aux");
  if (L.val32 && l > 0) {
    k_to_f32<<<blocks_for(L.nnz, 256), 256, 0, h->stream>>>(L.nnz, L.val, L.val32);
    MG_LAUNCH("k_to_f32");
  }
  return MGPBD_OK;
}

// The largest dynamic shared memory a Galerkin launch requests.  The limit a
// kernel may request is one setting per kernel for the whole process, so it is
// raised once to this bound (under a mutex, before the first launch), never
// per launch: per launch, one thread could lower it between another thread's
// setting and that thread's launch, which then fails.
constexpr int kGalerkinSmemMax = 200 * 1024;

__global__ void k_gal_values_k(int na, int k, const int64_t *mptr, const int32_t *mrow,
                               const int64_t *ptr, const int32_t *col, const double *val,
                               const int32_t *agg, const double *P, const int64_t *bptr,
                               const int32_t *bcol, const int64_t *cptr, double *cval,
                               int maxblk, double *acc_global);

static mgpbd_status galerkin_smem_limits() {
  static std::mutex mu;
  static bool done = false;
  std::lock_guard<std::mutex> lock(mu);
  if (done) return MGPBD_OK;
  MG_CUDA(cudaFuncSetAttribute(k_gal_values, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               kGalerkinSmemMax));
  MG_CUDA(cudaFuncSetAttribute(k_gal_values_k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               kGalerkinSmemMax));
  done = true;
  return MGPBD_OK;
}

static mgpbd_status galerkin_values(Handle *h, int l) {
  Level &L = h->lev[l], &Lc = h->lev[l + 1];
  int maxlen = std::max(L.max_coarse_row, 1);
  int warps = maxlen > 1536 ? 1 : (maxlen > 384 ? 2 : 4);
  size_t smem = (size_t)warps * maxlen * (sizeof(double) + sizeof(int));
  if (smem > (size_t)kGalerkinSmemMax) {
    set_error("Galerkin: coarse row too long for shared memory");
    return MGPBD_E_SETUP;
  }
  MG_TRY(galerkin_smem_limits());
  int blocks = (int)std::min<int64_t>((L.n_agg + warps - 1) / warps, 1 << 20);
  k_gal_values<<<blocks, warps * 32, smem, h->stream>>>(L.n_agg, L.mptr, L.mrow, L.ptr, L.col,
                                                       L.val, L.agg, L.P, Lc.ptr, Lc.col, Lc.val,
                                                       maxlen);
  MG_LAUNCH("k_gal_values");
  k_gal_mirror<<<warp_blocks(L.n_agg), 256, 0, h->stream>>>(L.n_agg, Lc.ptr, Lc.col, Lc.val);
  MG_LAUNCH("k_gal_mirror");
  return level_precision_copies(h, l + 1);
}

static mgpbd_status colour_level(Handle *h, int l) {
  Level &L = h->lev[l];
  MG_CUDA(cudaMemsetAsync(L.color, 0xff, sizeof(int32_t) * L.n, h->stream));
  for (int round = 0; round < 100000; ++round) {
    MG_CUDA(cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream));
    k_jp_round<<<warp_blocks(L.n), 256, 0, h->stream>>>(L.n, L.ptr, L.col, h->p.seed_col, l,
                                                        L.color, h->flag);
    MG_LAUNCH("k_jp_round");
    int rem = 0;
    MG_TRY(read_int(h, h->flag, &rem));
    if (rem == 0) break;
  }
  MG_CUDA(cudaMemsetAsync(h->flag, 0xff, sizeof(int), h->stream));
  k_max_i32<<<blocks_for(L.n, 256), 256, 0, h->stream>>>(L.n, L.color, h->flag);
  MG_LAUNCH("k_max_i32");
  int mx = -1;
  MG_TRY(read_int(h, h->flag, &mx));
  L.n_colors = mx + 1;
  return MGPBD_OK;
}

// rows grouped by colour for the multicolour Gauss-Seidel sweeps
__global__ void k_col_count(int n, const int32_t *color, unsigned long long *cnt) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    atomicAdd(&cnt[color[i]], 1ull);
}

__global__ void k_col_fill(int n, const int32_t *color, const int64_t *cptr,
                           unsigned long long *fill, int32_t *crow) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    unsigned long long pos = atomicAdd(&fill[color[i]], 1ull);
    crow[cptr[color[i]] + (int64_t)pos] = i;
  }
}

static mgpbd_status colour_groups(Handle *h, int l) {
  Level &L = h->lev[l];
  const int nc = L.n_colors;
  if (!L.crow) MG_TRY(alloc_n(h->arena, &L.crow, (size_t)L.cap_n));
  MG_TRY(ensure_tmp(h, sizeof(int64_t) * (2 * (size_t)nc + 2)));
  unsigned long long *cnt = (unsigned long long *)h->tmp;
  int64_t *dptr = (int64_t *)h->tmp + nc + 1;
  MG_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int64_t) * nc, h->stream));
  k_col_count<<<blocks_for(L.n, 256), 256, 0, h->stream>>>(L.n, L.color, cnt);
  MG_LAUNCH("k_col_count");
  std::vector<int64_t> c((size_t)nc);
  MG_CUDA(cudaMemcpyAsync(c.data(), cnt, sizeof(int64_t) * nc, cudaMemcpyDeviceToHost, h->stream));
  MG_CUDA(cudaStreamSynchronize(h->stream));
  L.hcptr.assign((size_t)nc + 1, 0);
  for (int k = 0; k < nc; ++k) L.hcptr[k + 1] = L.hcptr[k] + c[k];
  MG_CUDA(cudaMemcpyAsync(dptr, L.hcptr.data(), sizeof(int64_t) * (nc + 1), cudaMemcpyHostToDevice,
                          h->stream));
  MG_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int64_t) * nc, h->stream));
  k_col_fill<<<blocks_for(L.n, 256), 256, 0, h->stream>>>(L.n, L.color, dptr, cnt, L.crow);
  MG_LAUNCH("k_col_fill");
  MG_CUDA(cudaStreamSynchronize(h->stream));
  return MGPBD_OK;
}

// strength filter + MIS-2 aggregation of a CSR (the rows of a level, or its
// nodes): agg, root and the number of aggregates
static mgpbd_status mis2_aggregate(Handle *h, int l, int n, int64_t nnz, const int64_t *ptr,
                                   const int32_t *col, const double *val, int32_t *agg,
                                   uint8_t *root, int64_t *na_out) {
  const int th = 256;
  // scratch: state u8 | e1 u8 | m1p u64 | m1i i32 | p1 i32 | flags i64 | ids i64 (n+1)
  size_t off_state = 0, off_e1 = (size_t)n, off_m1p = ((2 * (size_t)n + 15) / 16) * 16;
  size_t off_m1i = off_m1p + 8 * (size_t)n, off_p1 = off_m1i + 4 * (size_t)n;
  size_t off_f = ((off_p1 + 4 * (size_t)n + 15) / 16) * 16, off_ids = off_f + 8 * (size_t)n;
  size_t need = off_ids + 8 * ((size_t)n + 1);
  MG_TRY(ensure_tmp(h, need));
  // with k > 1 unknowns per aggregate a coarse level can hold more nonzeros
  // than level 0, for which the strength mask was sized
  if (nnz > h->cap_S) {
    h->arena.release(h->S);
    h->S = nullptr;
    MG_TRY(alloc_n(h->arena, &h->S, (size_t)nnz));
    h->cap_S = nnz;
  }
  char *base = (char *)h->tmp;
  uint8_t *state = (uint8_t *)(base + off_state), *e1 = (uint8_t *)(base + off_e1);
  uint64_t *m1p = (uint64_t *)(base + off_m1p);
  int *m1i = (int *)(base + off_m1i), *p1 = (int *)(base + off_p1);
  int64_t *f64 = (int64_t *)(base + off_f), *ids = (int64_t *)(base + off_ids);
  k_strength<<<warp_blocks(n), th, 0, h->stream>>>(n, ptr, col, val, h->p.theta_s, h->S, state);
  MG_LAUNCH("k_strength");
  for (int round = 0;; ++round) {
    if (round > 100000) {
      set_error("MIS-2 did not terminate");
      return MGPBD_E_SETUP;
    }
    k_mis_m1<<<warp_blocks(n), th, 0, h->stream>>>(n, ptr, col, h->S, state, h->p.seed_agg, l,
                                                   m1p, m1i);
    MG_LAUNCH("k_mis_m1");
    k_mis_m2<<<warp_blocks(n), th, 0, h->stream>>>(n, ptr, col, h->S, m1p, m1i, state);
    MG_LAUNCH("k_mis_m2");
    k_mis_e1<<<warp_blocks(n), th, 0, h->stream>>>(n, ptr, col, h->S, state, e1);
    MG_LAUNCH("k_mis_e1");
    MG_CUDA(cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream));
    k_mis_e2<<<warp_blocks(n), th, 0, h->stream>>>(n, ptr, col, h->S, e1, state, h->flag);
    MG_LAUNCH("k_mis_e2");
    int rem = 0;
    MG_TRY(read_int(h, h->flag, &rem));
    if (rem == 0) break;
  }
  k_root_flags<<<blocks_for(n, th), th, 0, h->stream>>>(n, state, root, f64);
  MG_LAUNCH("k_root_flags");
  MG_TRY(scan_counts(h, f64, ids, n));
  int64_t na = 0;
  MG_TRY(read_i64(h, ids + n, &na));
  k_agg_pass1<<<warp_blocks(n), th, 0, h->stream>>>(n, ptr, col, h->S, root, ids, p1);
  MG_LAUNCH("k_agg_pass1");
  MG_CUDA(cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream));
  k_agg_pass2<<<warp_blocks(n), th, 0, h->stream>>>(n, ptr, col, val, h->S, p1, agg, h->flag);
  MG_LAUNCH("k_agg_pass2");
  int bad = 0;
  MG_TRY(read_int(h, h->flag, &bad));
  if (bad) {
    set_error("aggregation left a row unassigned");
    return MGPBD_E_SETUP;
  }
  *na_out = na;
  return MGPBD_OK;
}

// node matrix of a level with k unknowns per node: the Frobenius norm of each
// k x k block of the node pattern (off-diagonal nodes ascending, the node
// itself last), summed over rows p ascending and their storage order
__global__ void k_node_norms(int nn, int k, const int64_t *ptr, const int32_t *col,
                             const double *val, const int64_t *nptr, const int32_t *ncol,
                             double *nval) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < nn; a += gridDim.x * blockDim.x) {
    const int64_t base = nptr[a];
    const int deg = (int)(nptr[a + 1] - base), noff = deg - 1;
    for (int t = 0; t < deg; ++t) nval[base + t] = 0.0;
    for (int p = 0; p < k; ++p) {
      const int64_t r = (int64_t)a * k + p;
      for (int64_t e = ptr[r]; e < ptr[r + 1]; ++e) {
        const int b = col[e] / k;
        int t = noff;
        if (b != a) {
          int lo = 0, hi = noff;
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (ncol[base + mid] < b) lo = mid + 1;
            else hi = mid;
          }
          t = lo;
        }
        const double v = val[e];
        nval[base + t] = fma(v, v, nval[base + t]);
      }
    }
    for (int t = 0; t < deg; ++t) nval[base + t] = sqrt(nval[base + t]);
  }
}

__global__ void k_expand_nodes(int n, int k, const int32_t *nagg, const uint8_t *nroot,
                               int32_t *agg, uint8_t *root) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    agg[i] = nagg[i / k];
    root[i] = nroot[i / k];
  }
}

// aggregation of level l: fills L.agg, L.root, L.n_agg and the member lists
// (L.n_agg = 0 when the level does not coarsen).  With k > 1 unknowns per
// node, coarse levels aggregate whole nodes: the node matrix comes from the
// aggregate pattern the level was built from (level l-1's gbptr/gbcol).
static mgpbd_status aggregate_level(Handle *h, int l) {
  Level &L = h->lev[l];
  const int n = L.n;
  const int th = 256;
  const int k = h->p.nk_vectors;
  int64_t na = 0;
  int units = n;
  if (k > 1 && l > 0) {
    const Level &Lp = h->lev[l - 1];
    const int nn = n / k;
    units = nn;
    int64_t nnz_n = 0;
    MG_TRY(read_i64(h, Lp.gbptr + nn, &nnz_n));
    double *nval = nullptr;
    int32_t *nagg = nullptr;
    uint8_t *nroot = nullptr;
    MG_TRY(alloc_n(h->arena, &nval, (size_t)nnz_n));
    MG_TRY(alloc_n(h->arena, &nagg, (size_t)nn));
    MG_TRY(alloc_n(h->arena, &nroot, (size_t)nn));
    k_node_norms<<<blocks_for(nn, 128), 128, 0, h->stream>>>(nn, k, L.ptr, L.col, L.val, Lp.gbptr,
                                                            Lp.gbcol, nval);
    MG_LAUNCH("k_node_norms");
    mgpbd_status st =
        mis2_aggregate(h, l, nn, nnz_n, Lp.gbptr, Lp.gbcol, nval, nagg, nroot, &na);
    if (st >= 0) {
      k_expand_nodes<<<blocks_for(n, th), th, 0, h->stream>>>(n, k, nagg, nroot, L.agg, L.root);
      MG_LAUNCH("k_expand_nodes");
    }
    h->arena.release(nval);
    h->arena.release(nagg);
    h->arena.release(nroot);
    MG_TRY(st);
  } else {
    MG_TRY(mis2_aggregate(h, l, n, L.nnz, L.ptr, L.col, L.val, L.agg, L.root, &na));
  }
  L.n_agg = (int)na;
  if (na == 0 || na == units) {  // nothing to coarsen; caller stops here
    L.n_agg = 0;
    return MGPBD_OK;
  }
  // member lists (over rows)
  MG_TRY(ensure_tmp(h, sizeof(int64_t) * (2 * (size_t)n + 2)));
  int64_t *f64 = (int64_t *)h->tmp, *ids = f64 + n + 1;
  unsigned long long *cnt = (unsigned long long *)f64;  // reuse (na <= n)
  MG_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int64_t) * na, h->stream));
  k_mem_count<<<blocks_for(n, th), th, 0, h->stream>>>(n, L.agg, cnt);
  MG_LAUNCH("k_mem_count");
  MG_TRY(scan_counts(h, (const int64_t *)cnt, L.mptr, na));
  MG_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int64_t) * na, h->stream));
  int32_t *tmpm = (int32_t *)ids;  // reuse (n int32 fit in n+1 int64)
  k_mem_fill<<<blocks_for(n, th), th, 0, h->stream>>>(n, L.agg, L.mptr, cnt, tmpm);
  MG_LAUNCH("k_mem_fill");
  MG_CUDA(cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream));
  k_mem_sort<<<warp_blocks(na), th, 0, h->stream>>>((int)na, L.mptr, tmpm, L.mrow, h->flag);
  MG_LAUNCH("k_mem_sort");
  MG_TRY(read_int(h, h->flag, &L.max_members));
  return MGPBD_OK;
}

static mgpbd_status galerkin_pattern(Handle *h, int l) {
  Level &L = h->lev[l];
  const int na = L.n_agg;
  MG_TRY(ensure_tmp(h, sizeof(int64_t) * ((size_t)na + 1)));
  int64_t *cnt = (int64_t *)h->tmp;
  MG_CUDA(cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream));
  int blocks = std::min(na, 65535);
  k_gal_pattern<<<blocks, 256, 0, h->stream>>>(na, L.mptr, L.mrow, L.ptr, L.col, L.agg, cnt,
                                               nullptr, nullptr, h->flag);
  MG_LAUNCH("k_gal_pattern(count)");
  int ovf = 0;
  MG_TRY(read_int(h, h->flag, &ovf));
  if (ovf) {
    set_error("Galerkin pattern: coarse row has too many columns");
    return MGPBD_E_SETUP;
  }
  // coarse ptr (level l+1): allocate n-sized buffers first
  Level &Lc = h->lev[l + 1];
  MG_TRY(ensure_level(h, l + 1, na, 0));
  MG_TRY(scan_counts(h, cnt, Lc.ptr, na));
  int64_t cnnz = 0;
  MG_TRY(read_i64(h, Lc.ptr + na, &cnnz));
  MG_TRY(ensure_level(h, l + 1, na, cnnz));
  // longest coarse row
  {
    std::vector<int64_t> hp((size_t)na + 1);
    MG_CUDA(cudaMemcpyAsync(hp.data(), Lc.ptr, sizeof(int64_t) * (na + 1), cudaMemcpyDeviceToHost,
                            h->stream));
    MG_CUDA(cudaStreamSynchronize(h->stream));
    int64_t mx = 0;
    for (int a = 0; a < na; ++a) mx = std::max(mx, hp[a + 1] - hp[a]);
    L.max_coarse_row = (int)mx;
  }
  k_gal_pattern<<<blocks, 256, 0, h->stream>>>(na, L.mptr, L.mrow, L.ptr, L.col, L.agg, nullptr,
                                               Lc.ptr, Lc.col, h->flag);
  MG_LAUNCH("k_gal_pattern(fill)");
  return MGPBD_OK;
}

// ---------------------------------------------------------------------------
// k > 1 near-kernel vectors (Sec. 4.3): the tentative prolongator of each
// aggregate from a QR factorisation of its block of B, and P^T A P with k
// unknowns per aggregate, in the canonical order of the k = 1 kernels.
// ---------------------------------------------------------------------------
constexpr double kQrDrop = 1e-6;  // a column below this share of |B_a[:,c]| is dropped

__global__ void k_set_col(int n, int k, int c, const double *v, double *B) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    B[(int64_t)i * k + c] = v[i];
}

// Modified Gram-Schmidt with one re-orthogonalisation pass per aggregate,
// one thread per aggregate, members in ascending order (the order of the
// FP64 sums is that of the definition): P rows take Q, the next level's
// near-kernel rows (a, d) take R[d][:], dead (dropped) columns are zero.
__global__ void k_inject_k(int na, int k, const int64_t *mptr, const int32_t *mrow,
                           const double *B, double *P, uint8_t *pdead, double *Bc, double *v) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < na; a += gridDim.x * blockDim.x) {
    const int64_t q0 = mptr[a], q1 = mptr[a + 1];
    double *R = Bc + (int64_t)a * k * k;
    for (int c = 0; c < k; ++c) {
      for (int64_t q = q0; q < q1; ++q) v[q] = B[(int64_t)mrow[q] * k + c];
      for (int pass = 0; pass < 2; ++pass)
        for (int d = 0; d < c; ++d) {
          double r = 0.0;
          for (int64_t q = q0; q < q1; ++q) r = fma(P[(int64_t)mrow[q] * k + d], v[q], r);
          R[d * k + c] = pass ? R[d * k + c] + r : r;
          for (int64_t q = q0; q < q1; ++q) v[q] = fma(-r, P[(int64_t)mrow[q] * k + d], v[q]);
        }
      double nb = 0.0, nv = 0.0;
      for (int64_t q = q0; q < q1; ++q) {
        const double bq = B[(int64_t)mrow[q] * k + c];
        nb = fma(bq, bq, nb);
        nv = fma(v[q], v[q], nv);
      }
      const double nrm = sqrt(nv);
      const bool live = nv > 0.0 && nrm > kQrDrop * sqrt(nb);
      for (int64_t q = q0; q < q1; ++q) P[(int64_t)mrow[q] * k + c] = live ? v[q] / nrm : 0.0;
      R[c * k + c] = live ? nrm : 0.0;
      pdead[(int64_t)a * k + c] = live ? 0 : 1;
    }
  }
}

// the k-unknown coarse pattern from the aggregate pattern (off-diagonal
// aggregates ascending, the diagonal last): row (a, p) = a*k+p holds the
// columns b*k+q of a's aggregates ascending (a included) with (a, p) moved last
__global__ void k_expand_count(int na, int k, const int64_t *bptr, int64_t *cnt) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < (int64_t)na * k;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(r / k);
    cnt[r] = (bptr[a + 1] - bptr[a]) * k;
  }
}

__device__ __forceinline__ int sorted_block(const int32_t *off, int noff, int sa, int a, int s) {
  return s < sa ? off[s] : (s == sa ? a : off[s - 1]);
}

__global__ void k_expand_fill(int na, int k, const int64_t *bptr, const int32_t *bcol,
                              const int64_t *cptr, int32_t *ccol) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < (int64_t)na * k;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(r / k);
    const int32_t *off = bcol + bptr[a];
    const int noff = (int)(bptr[a + 1] - bptr[a]) - 1;
    int sa = 0;  // position of a among its aggregates in ascending order
    while (sa < noff && off[sa] < a) ++sa;
    int64_t w = cptr[r];
    for (int s = 0; s <= noff; ++s) {
      const int b = sorted_block(off, noff, sa, a, s);
      for (int q = 0; q < k; ++q) {
        const int64_t c = (int64_t)b * k + q;
        if (c != r) ccol[w++] = (int32_t)c;
      }
    }
    ccol[w] = (int32_t)r;
  }
}

// Values of the k-unknown coarse operator: warp per aggregate a, lanes over
// the k x k pairs (p, q); each pair's sums run over member rows i of a in
// ascending order and row i's storage order, acc = fma(P_ip * A_ij, P_jq,
// acc), as in the definition.  Only entries (b, q) >= (a, p) are formed.
__global__ void k_gal_values_k(int na, int k, const int64_t *mptr, const int32_t *mrow,
                               const int64_t *ptr, const int32_t *col, const double *val,
                               const int32_t *agg, const double *P, const int64_t *bptr,
                               const int32_t *bcol, const int64_t *cptr, double *cval,
                               int maxblk, double *acc_global) {
  extern __shared__ unsigned char smem_raw[];
  const int wib = threadIdx.x >> 5;
  const int64_t per = (int64_t)k * maxblk * k;
  // accumulators: shared memory, or a global slot per warp for long block rows
  double *acc = acc_global
                    ? acc_global + ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * per
                    : reinterpret_cast<double *>(smem_raw) + (size_t)wib * per;
  WARP_LOOP(na) {
    const int a = (int)row_;
    const int32_t *off = bcol + bptr[a];
    const int noff = (int)(bptr[a + 1] - bptr[a]) - 1;
    const int nb = noff + 1;
    int sa = 0;
    while (sa < noff && off[sa] < a) ++sa;
    const int width = nb * k;
    for (int t = lane; t < k * width; t += 32) acc[t] = 0.0;
    __syncwarp();
    for (int64_t m = mptr[a]; m < mptr[a + 1]; ++m) {
      const int i = mrow[m];
      for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e) {
        const int j = col[e];
        const int b = agg[j];
        if (b < a) continue;  // uniform over the warp
        int sb;
        if (b == a) {
          sb = sa;
        } else {
          int lo = 0, hi = noff;
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (off[mid] < b) lo = mid + 1;
            else hi = mid;
          }
          sb = lo < sa ? lo : lo + 1;
        }
        const double aij = val[e];
        for (int pq = lane; pq < k * k; pq += 32) {
          const int p = pq / k, q = pq % k;
          if (b == a && q < p) continue;
          const double t = P[(int64_t)i * k + p] * aij;
          double *cell = acc + p * width + sb * k + q;
          *cell = fma(t, P[(int64_t)j * k + q], *cell);
        }
      }
    }
    __syncwarp();
    for (int p = 0; p < k; ++p) {
      const int64_t r = (int64_t)a * k + p;
      const int64_t rb = cptr[r], len = cptr[r + 1] - rb;
      for (int t = lane; t < width; t += 32) {
        const int s = t / k, q = t % k;
        const int64_t c = (int64_t)sorted_block(off, noff, sa, a, s) * k + q;
        if (c < r) continue;
        const int64_t pos = c == r ? len - 1 : t - 1;
        cval[rb + pos] = acc[p * width + t];
      }
    }
    __syncwarp();
  }
}

__global__ void k_dead_diag(int64_t nc, const uint8_t *pdead, const int64_t *cptr, double *cval) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nc;
       r += (int64_t)gridDim.x * blockDim.x)
    if (pdead[r]) cval[cptr[r + 1] - 1] = 1.0;
}

// aggregate pattern of level l+1 (kept in L.gbptr/gbcol), then the k-unknown
// pattern in level l+1
static mgpbd_status galerkin_pattern_k(Handle *h, int l) {
  Level &L = h->lev[l];
  Level &Lc = h->lev[l + 1];
  const int k = h->p.nk_vectors, na = L.n_agg;
  MG_TRY(galerkin_pattern(h, l));  // aggregate pattern, in level l+1's arrays for now
  int64_t bnnz = 0;
  MG_TRY(read_i64(h, Lc.ptr + na, &bnnz));
  if (bnnz > L.cap_gb) {
    h->arena.release(L.gbcol);
    L.gbcol = nullptr;
    MG_TRY(alloc_n(h->arena, &L.gbcol, (size_t)bnnz));
    L.cap_gb = bnnz;
  }
  MG_CUDA(cudaMemcpyAsync(L.gbptr, Lc.ptr, sizeof(int64_t) * ((size_t)na + 1),
                          cudaMemcpyDeviceToDevice, h->stream));
  MG_CUDA(cudaMemcpyAsync(L.gbcol, Lc.col, sizeof(int32_t) * (size_t)bnnz,
                          cudaMemcpyDeviceToDevice, h->stream));
  const int64_t nc = (int64_t)na * k;
  MG_TRY(ensure_level(h, l + 1, (int)nc, 0));
  MG_TRY(ensure_tmp(h, sizeof(int64_t) * ((size_t)nc + 1)));
  int64_t *cnt = (int64_t *)h->tmp;
  k_expand_count<<<blocks_for(nc, 256), 256, 0, h->stream>>>(na, k, L.gbptr, cnt);
  MG_LAUNCH("k_expand_count");
  MG_TRY(scan_counts(h, cnt, Lc.ptr, nc));
  MG_TRY(ensure_level(h, l + 1, (int)nc, bnnz * k * k));
  k_expand_fill<<<blocks_for(nc, 256), 256, 0, h->stream>>>(na, k, L.gbptr, L.gbcol, Lc.ptr,
                                                            Lc.col);
  MG_LAUNCH("k_expand_fill");
  return MGPBD_OK;
}

static mgpbd_status galerkin_values_k(Handle *h, int l) {
  Level &L = h->lev[l], &Lc = h->lev[l + 1];
  const int k = h->p.nk_vectors;
  const int maxblk = std::max(L.max_coarse_row, 1);
  const size_t per = sizeof(double) * (size_t)k * maxblk * k;
  int warps = (int)std::max<size_t>(1, std::min<size_t>(4, (160 * 1024) / per));
  size_t smem = (size_t)warps * per;
  int blocks = (int)std::min<int64_t>((L.n_agg + warps - 1) / warps, 1 << 20);
  double *acc_global = nullptr;
  if (smem > 160 * 1024) {
    // block rows too long for shared memory: 256 warps with a global slot each
    warps = 4;
    blocks = (int)std::min<int64_t>((L.n_agg + warps - 1) / warps, 64);
    MG_TRY(ensure_tmp(h, per * (size_t)blocks * warps));
    acc_global = (double *)h->tmp;
    smem = 0;
  }
  MG_TRY(galerkin_smem_limits());
  k_gal_values_k<<<blocks, warps * 32, smem, h->stream>>>(L.n_agg, k, L.mptr, L.mrow, L.ptr,
                                                         L.col, L.val, L.agg, L.P, L.gbptr,
                                                         L.gbcol, Lc.ptr, Lc.val, maxblk,
                                                         acc_global);
  MG_LAUNCH("k_gal_values_k");
  const int64_t nc = (int64_t)L.n_agg * k;
  k_gal_mirror<<<warp_blocks(nc), 256, 0, h->stream>>>((int)nc, Lc.ptr, Lc.col, Lc.val);
  MG_LAUNCH("k_gal_mirror");
  k_dead_diag<<<blocks_for(nc, 256), 256, 0, h->stream>>>(nc, L.pdead, Lc.ptr, Lc.val);
  MG_LAUNCH("k_dead_diag");
  return level_precision_copies(h, l + 1);
}

mgpbd_status amg_setup(Handle *h) {
  if (h->m == 0) {
    h->L = 1;
    h->have_setup = true;
    h->n_setups++;
    return MGPBD_OK;
  }
  Level &L0 = h->lev[0];
  MG_TRY(ensure_level(h, 0, h->m, L0.nnz));
  const int th = 256;
  // near-kernel on level 0 (Sec. 4.3)
  {
    unsigned long long *amax = (unsigned long long *)h->flag;
    MG_CUDA(cudaMemsetAsync(amax, 0, sizeof(unsigned long long), h->stream));
    k_absmax<<<std::min(blocks_for(L0.nnz, th), 4 * num_sms()), th, 0, h->stream>>>(L0.nnz, L0.val,
                                                                                    amax);
    MG_LAUNCH("k_absmax");
    // vector c (of k) from the generator stream seed_nk + c; B is m x k
    const int k = h->p.nk_vectors;
    MG_TRY(ensure_tmp(h, sizeof(double) * (size_t)h->m * (k > 1 ? 2 : 1)));
    for (int c = 0; c < k; ++c) {
      double *xa = k > 1 ? (double *)h->tmp : L0.B;
      double *xb = k > 1 ? (double *)h->tmp + h->m : (double *)h->tmp;
      k_nk_init<<<blocks_for(h->m, th), th, 0, h->stream>>>(h->m, h->p.seed_nk + (uint64_t)c,
                                                            amax, xa);
      MG_LAUNCH("k_nk_init");
      for (int s = 0; s < h->p.nk_sweeps; ++s) {
        k_nk_sweep<<<warp_blocks(h->m), th, 0, h->stream>>>(h->m, L0.ptr, L0.col, L0.val,
                                                            h->p.nk_omega, xa, xb);
        MG_LAUNCH("k_nk_sweep");
        MG_CUDA(cudaMemcpyAsync(xa, xb, sizeof(double) * h->m, cudaMemcpyDeviceToDevice,
                                h->stream));
      }
      if (k > 1) {
        k_set_col<<<blocks_for(h->m, th), th, 0, h->stream>>>(h->m, k, c, xa, L0.B);
        MG_LAUNCH("k_set_col");
      }
    }
  }
  int l = 0;
  for (;;) {
    Level &L = h->lev[l];
    if (L.n < h->p.coarse_max || l == h->p.max_levels - 1 || l == kMaxLevels - 1) break;
    MG_TRY(aggregate_level(h, l));
    if (L.n_agg == 0 || L.n_agg == L.n) break;
    const int k = h->p.nk_vectors;
    if (k == 1) {
      MG_TRY(galerkin_pattern(h, l));
      Level &Lc = h->lev[l + 1];
      MG_CUDA(cudaMemsetAsync(L.P, 0, sizeof(double) * L.n, h->stream));  // left-alone rows
      k_inject<<<warp_blocks(L.n_agg), th, 0, h->stream>>>(L.n_agg, L.mptr, L.mrow, L.B, L.P,
                                                           Lc.B);
      MG_LAUNCH("k_inject");
    } else {
      MG_TRY(galerkin_pattern_k(h, l));
      Level &Lc = h->lev[l + 1];
      MG_CUDA(cudaMemsetAsync(L.P, 0, sizeof(double) * L.n * k, h->stream));
      MG_CUDA(cudaMemsetAsync(Lc.B, 0, sizeof(double) * Lc.n * k, h->stream));
      MG_TRY(ensure_tmp(h, sizeof(double) * (size_t)L.n));
      k_inject_k<<<blocks_for(L.n_agg, 128), 128, 0, h->stream>>>(
          L.n_agg, k, L.mptr, L.mrow, L.B, L.P, L.pdead, Lc.B, (double *)h->tmp);
      MG_LAUNCH("k_inject_k");
    }
    if (L.P32) {
      k_to_f32<<<blocks_for((int64_t)L.n * k, th), th, 0, h->stream>>>((int64_t)L.n * k, L.P,
                                                                       L.P32);
      MG_LAUNCH("k_to_f32(P)");
    }
    if (l == 0 && k == 1 && h->p.level0_op == 1) MG_TRY(member_order_level0(h));
    MG_TRY(k == 1 ? galerkin_values(h, l) : galerkin_values_k(h, l));
    ++l;
  }
  h->L = l + 1;
  if (h->lev[h->L - 1].n > 4096) {
    set_error("AMG setup: coarsest level has more than 4096 rows");
    return MGPBD_E_SETUP;
  }
  for (int q = 0; q + 1 < h->L; ++q) {
    // the multicolour ordering is needed by the Gauss-Seidel smoother only
    if (h->p.smoother == MGPBD_SMOOTH_MCGS || h->want_colors) MG_TRY(colour_level(h, q));
    else h->lev[q].n_colors = 0;
    if (h->p.smoother == MGPBD_SMOOTH_MCGS) MG_TRY(colour_groups(h, q));
    MG_TRY(power_method(h, q));
  }
  h->lev[h->L - 1].n_colors = 0;
  if (h->p.autotune) MG_TRY(autotune_levels(h));
  h->have_setup = true;
  h->n_setups++;
  h->gen++;  // new hierarchy: captured PCG graphs are stale
  MG_CUDA(cudaStreamSynchronize(h->stream));
  return MGPBD_OK;
}

mgpbd_status galerkin_reform(Handle *h) {
  for (int l = 0; l + 1 < h->L; ++l)
    MG_TRY(h->p.nk_vectors == 1 ? galerkin_values(h, l) : galerkin_values_k(h, l));
  return MGPBD_OK;
}

}  // namespace mg
