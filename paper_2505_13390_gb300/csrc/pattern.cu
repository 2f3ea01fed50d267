// Fixed CSR pattern of A = grad C M^-1 grad C^T + alpha~ (Sec. 4.2: three
// fixed-length arrays, off-diagonal terms first and the diagonal last), its
// assembly map, and the vertex -> row incidence used by the position update
// (eq. 5).  Built once at create time on the device.
//
// Row i's off-diagonals are the rows j != i that share at least one vertex
// with i (pinned vertices included: the pattern depends on topology only),
// in ascending j.  The assembly map of an off-diagonal lists the shared
// vertices in ascending vertex id as (slot in i, slot in j) pairs packed in a
// uint16: bits 0-1 the count, pair p at bits 2+4p and 4+4p.
#include "common.cuh"

namespace mg {

// ---------------------------------------------------------------------------
// exclusive scan of int64 counts (out has n+1 entries, out[n] = total)
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t *warp_tot, int64_t *total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) warp_tot[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int64_t s = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
    int64_t si = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t t = __shfl_up_sync(0xffffffffu, si, o);
      if (lane >= o) si += t;
    }
    warp_tot[lane] = si - s;
    if (lane == 31) *total = si;
  }
  __syncthreads();
  int64_t r = warp_tot[wid] + inc - v;
  __syncthreads();
  return r;
}

__global__ void k_tile_sums(const int64_t *in, int64_t n, int64_t *sums) {
  __shared__ int64_t wt[32];
  __shared__ int64_t tot;
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t s = 0;
  for (int k = 0; k < kScanItems; ++k)
    if (base + k < n) s += in[base + k];
  block_excl_scan(s, wt, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_tile_scan(const int64_t *in, int64_t n, const int64_t *offs, int64_t *out) {
  __shared__ int64_t wt[32];
  __shared__ int64_t tot;
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t s = 0;
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = base + k < n ? in[base + k] : 0;
    s += v[k];
  }
  int64_t e = block_excl_scan(s, wt, &tot) + (offs ? offs[blockIdx.x] : 0);
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = e;
    e += v[k];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) out[n] = e;
}

static mgpbd_status scan_rec(Handle *h, const int64_t *in, int64_t *out, int64_t n,
                             int64_t *scratch, size_t scratch_n) {
  int64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles <= 1) {
    k_tile_scan<<<1, kScanThreads, 0, h->stream>>>(in, n, nullptr, out);
    MG_LAUNCH("k_tile_scan");
    return MGPBD_OK;
  }
  if ((size_t)(2 * (tiles + 1)) > scratch_n) {
    set_error("scan scratch too small");
    return MGPBD_E_INVALID;
  }
  int64_t *sums = scratch, *offs = scratch + tiles + 1;
  k_tile_sums<<<(unsigned)tiles, kScanThreads, 0, h->stream>>>(in, n, sums);
  MG_LAUNCH("k_tile_sums");
  MG_TRY(scan_rec(h, sums, offs, tiles, scratch + 2 * (tiles + 1), scratch_n - 2 * (tiles + 1)));
  k_tile_scan<<<(unsigned)tiles, kScanThreads, 0, h->stream>>>(in, n, offs, out);
  MG_LAUNCH("k_tile_scan");
  return MGPBD_OK;
}

mgpbd_status scan_counts(Handle *h, const int64_t *counts, int64_t *out, int64_t n) {
  if (n == 0) {
    MG_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), h->stream));
    return MGPBD_OK;
  }
  // scratch for the tile sums lives in its own small allocation so callers may
  // pass h->tmp as `counts`
  int64_t tiles = (n + kScanTile - 1) / kScanTile;
  size_t need = (size_t)(4 * (tiles + 2) + 64);
  int64_t *scratch = nullptr;
  MG_TRY(alloc_n(h->arena, &scratch, need));
  mgpbd_status s = scan_rec(h, counts, out, n, scratch, need);
  cudaStreamSynchronize(h->stream);
  h->arena.release(scratch);
  return s;
}

// ---------------------------------------------------------------------------
// vertex -> incident rows
// ---------------------------------------------------------------------------
__device__ __forceinline__ int row_verts(int j, int E, const int32_t *edge, const int32_t *tet,
                                         int32_t v[4]) {
  if (j < E) {
    v[0] = edge[2 * (int64_t)j];
    v[1] = edge[2 * (int64_t)j + 1];
    return 2;
  }
  const int32_t *t = tet + 4 * (int64_t)(j - E);
  v[0] = t[0];
  v[1] = t[1];
  v[2] = t[2];
  v[3] = t[3];
  return 4;
}

__global__ void k_inc_count(int m, int E, const int32_t *edge, const int32_t *tet,
                            unsigned long long *cnt) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
    int32_t v[4];
    int c = row_verts(j, E, edge, tet, v);
    for (int k = 0; k < c; ++k) atomicAdd(&cnt[v[k]], 1ull);
  }
}

__global__ void k_inc_fill(int m, int E, const int32_t *edge, const int32_t *tet,
                           const int64_t *vptr, unsigned long long *fill, int32_t *vrow) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
    int32_t v[4];
    int c = row_verts(j, E, edge, tet, v);
    for (int k = 0; k < c; ++k) {
      unsigned long long pos = atomicAdd(&fill[v[k]], 1ull);
      vrow[vptr[v[k]] + (int64_t)pos] = j;
    }
  }
}

// insertion sort of each vertex's incident rows (short lists)
__global__ void k_inc_sort(int N, const int64_t *vptr, int32_t *vrow) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x) {
    int64_t s = vptr[v], e = vptr[v + 1];
    for (int64_t a = s + 1; a < e; ++a) {
      int32_t key = vrow[a];
      int64_t b = a - 1;
      while (b >= s && vrow[b] > key) {
        vrow[b + 1] = vrow[b];
        --b;
      }
      vrow[b + 1] = key;
    }
  }
}

mgpbd_status build_incidence(Handle *h) {
  const int N = h->N, m = h->m, E = h->E;
  MG_TRY(alloc_n(h->arena, &h->vptr, (size_t)N + 1));
  MG_TRY(alloc_n(h->arena, &h->vrow, 2 * (size_t)h->E + 4 * (size_t)h->T));
  MG_TRY(ensure_tmp(h, sizeof(unsigned long long) * (size_t)N));
  unsigned long long *cnt = (unsigned long long *)h->tmp;
  MG_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * N, h->stream));
  const int th = 256;
  if (m > 0) {
    k_inc_count<<<blocks_for(m, th), th, 0, h->stream>>>(m, E, h->edge, h->tet, cnt);
    MG_LAUNCH("k_inc_count");
  }
  MG_TRY(scan_counts(h, (const int64_t *)cnt, h->vptr, N));
  MG_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * N, h->stream));
  if (m > 0) {
    k_inc_fill<<<blocks_for(m, th), th, 0, h->stream>>>(m, E, h->edge, h->tet, h->vptr, cnt,
                                                        h->vrow);
    MG_LAUNCH("k_inc_fill");
  }
  k_inc_sort<<<blocks_for(N, th), th, 0, h->stream>>>(N, h->vptr, h->vrow);
  MG_LAUNCH("k_inc_sort");
  return MGPBD_OK;
}

// ---------------------------------------------------------------------------
// pattern: k-way merge of the (sorted) incidence lists of row i's vertices
// ---------------------------------------------------------------------------
struct Merge {
  int c;
  int64_t pos[4], end[4];
  __device__ __forceinline__ void init(int cnt, const int32_t v[4], const int64_t *vptr) {
    c = cnt;
    for (int s = 0; s < 4; ++s) {
      pos[s] = s < c ? vptr[v[s]] : 0;
      end[s] = s < c ? vptr[v[s] + 1] : 0;
    }
  }
  // next distinct row id (INT_MAX when done) and the mask of i's slots it came from
  __device__ __forceinline__ int next(const int32_t *vrow, int *mask) {
    int best = 0x7fffffff;
    for (int s = 0; s < c; ++s)
      if (pos[s] < end[s]) {
        int r = vrow[pos[s]];
        if (r < best) best = r;
      }
    int mk = 0;
    if (best != 0x7fffffff)
      for (int s = 0; s < c; ++s)
        if (pos[s] < end[s] && vrow[pos[s]] == best) {
          mk |= 1 << s;
          ++pos[s];
        }
    *mask = mk;
    return best;
  }
};

__global__ void k_row_count(int m, int E, const int32_t *edge, const int32_t *tet,
                            const int64_t *vptr, const int32_t *vrow, int64_t *cnt) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    int32_t v[4];
    int c = row_verts(i, E, edge, tet, v);
    Merge mg;
    mg.init(c, v, vptr);
    int64_t n = 0;
    int mask;
    for (int j = mg.next(vrow, &mask); j != 0x7fffffff; j = mg.next(vrow, &mask))
      if (j != i) ++n;
    cnt[i] = n + 1;  // + diagonal
  }
}

__global__ void k_row_fill(int m, int E, const int32_t *edge, const int32_t *tet,
                           const int64_t *vptr, const int32_t *vrow, const int64_t *ptr,
                           int32_t *col, uint16_t *map) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    int32_t v[4];
    int c = row_verts(i, E, edge, tet, v);
    Merge mg;
    mg.init(c, v, vptr);
    int64_t k = ptr[i];
    int mask;
    for (int j = mg.next(vrow, &mask); j != 0x7fffffff; j = mg.next(vrow, &mask)) {
      if (j == i) continue;
      int32_t w[4];
      int cj = row_verts(j, E, edge, tet, w);
      int sv[4], si[4], sj[4], ns = 0;
      for (int s = 0; s < c; ++s) {
        if (!(mask >> s & 1)) continue;
        int t = 0;
        while (t < cj && w[t] != v[s]) ++t;
        sv[ns] = v[s];
        si[ns] = s;
        sj[ns] = t;
        ++ns;
      }
      for (int a = 1; a < ns; ++a)  // ascending vertex id
        for (int b = a; b > 0 && sv[b - 1] > sv[b]; --b) {
          int t0 = sv[b]; sv[b] = sv[b - 1]; sv[b - 1] = t0;
          int t1 = si[b]; si[b] = si[b - 1]; si[b - 1] = t1;
          int t2 = sj[b]; sj[b] = sj[b - 1]; sj[b - 1] = t2;
        }
      if (ns > 3) ns = 3;
      unsigned code = (unsigned)ns;
      for (int p = 0; p < ns; ++p) code |= (unsigned)(si[p] << (2 + 4 * p)) | (unsigned)(sj[p] << (4 + 4 * p));
      col[k] = j;
      map[k] = (uint16_t)code;
      ++k;
    }
    col[k] = i;  // diagonal last
    map[k] = 0;
  }
}

mgpbd_status build_pattern(Handle *h) {
  const int m = h->m, E = h->E;
  Level &L = h->lev[0];
  L.n = m;
  MG_TRY(alloc_n(h->arena, &L.ptr, (size_t)m + 1));
  MG_TRY(ensure_tmp(h, sizeof(int64_t) * ((size_t)m + 1)));
  int64_t *cnt = (int64_t *)h->tmp;
  const int th = 128;
  if (m > 0) {
    k_row_count<<<blocks_for(m, th), th, 0, h->stream>>>(m, E, h->edge, h->tet, h->vptr, h->vrow,
                                                         cnt);
    MG_LAUNCH("k_row_count");
  }
  MG_TRY(scan_counts(h, cnt, L.ptr, m));
  int64_t nnz = 0;
  MG_TRY(read_i64(h, L.ptr + m, &nnz));
  L.nnz = nnz;
  MG_TRY(alloc_n(h->arena, &L.col, (size_t)nnz));
  MG_TRY(alloc_n(h->arena, &h->map, (size_t)nnz));
  MG_TRY(alloc_n(h->arena, &L.val, (size_t)nnz));
  MG_TRY(alloc_n(h->arena, &L.dinv, (size_t)m));
  MG_TRY(alloc_n(h->arena, &h->S, (size_t)nnz));
  h->cap_S = nnz;
  if (h->p.precision == MGPBD_MIXED) {
    MG_TRY(alloc_n(h->arena, &L.val32, (size_t)nnz));
    MG_TRY(alloc_n(h->arena, &L.dinv32, (size_t)m));
  }
  if (m > 0) {
    k_row_fill<<<blocks_for(m, th), th, 0, h->stream>>>(m, E, h->edge, h->tet, h->vptr, h->vrow,
                                                        L.ptr, L.col, h->map);
    MG_LAUNCH("k_row_fill");
  }
  return MGPBD_OK;
}

}  // namespace mg
