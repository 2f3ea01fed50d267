// C ABI of the GB300 MGPBD library: handle lifecycle, state I/O, the
// Algorithm 1 driver (frame prologue, global iterations, epilogue) and the
// inspection getters.  Compute happens in the kernels of pattern.cu
// (incidence, CSR pattern), physics.cu (constraints, assembly, updates),
// setup.cu (AMG setup and Galerkin products), solve.cu (MGPCG, V-cycle,
// smoothers) and mfree.cu (matrix-free level-0 products); serve.cu holds the
// multi-instance service and noalloc.cu the allocation-free residual.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <iterator>
#include <mutex>
#include <string>
#include <unordered_map>

#include "common.cuh"

namespace mg {

static thread_local std::string g_err;
unsigned long long g_launches = 0;

static mgpbd_status grow_events(std::vector<cudaEvent_t> &ev, std::vector<int> &it, int pairs) {
  if ((int)ev.size() >= 2 * pairs) return MGPBD_OK;
  size_t old = ev.size();
  size_t want = std::max<size_t>({(size_t)2048, 2 * old, 2 * (size_t)pairs});
  ev.resize(want);
  it.resize(want / 2);
  for (size_t k = old; k < want; ++k) MG_CUDA(cudaEventCreate(&ev[k]));
  return MGPBD_OK;
}

// events for a chunk's graph are created before capture begins (`pairs`
// per channel)
mgpbd_status prof_reserve_graph(Handle *h, int pairs) {
  for (int ch = 0; ch < PROF_CH; ++ch) MG_TRY(grow_events(h->gev[ch], h->gev_iter[ch], pairs));
  return MGPBD_OK;
}

mgpbd_status prof_begin(Handle *h, int ch) {
  if (!h->prof || !(h->prof_mask & (1 << ch))) return MGPBD_OK;
  if (h->capturing) {
    if (h->gev_used[ch] + 1 > (int)h->gev[ch].size() / 2) {
      set_error("profiling: event pool of the captured chunk is too small");
      return MGPBD_E_INVALID;
    }
    MG_CUDA(cudaEventRecordWithFlags(h->gev[ch][2 * h->gev_used[ch]], h->stream,
                                     cudaEventRecordExternal));
    return MGPBD_OK;
  }
  MG_TRY(grow_events(h->pev[ch], h->pev_iter[ch], h->pev_used[ch] + 1));
  MG_CUDA(cudaEventRecord(h->pev[ch][2 * h->pev_used[ch]], h->stream));
  return MGPBD_OK;
}

mgpbd_status prof_end(Handle *h, int ch) {
  if (!h->prof || !(h->prof_mask & (1 << ch))) return MGPBD_OK;
  if (h->capturing) {
    MG_CUDA(cudaEventRecordWithFlags(h->gev[ch][2 * h->gev_used[ch] + 1], h->stream,
                                     cudaEventRecordExternal));
    h->gev_iter[ch][h->gev_used[ch]] = h->pcg_k;
    h->gev_used[ch]++;
    return MGPBD_OK;
  }
  MG_CUDA(cudaEventRecord(h->pev[ch][2 * h->pev_used[ch] + 1], h->stream));
  h->pev_iter[ch][h->pev_used[ch]] = h->pcg_k;
  h->pev_used[ch]++;
  return MGPBD_OK;
}

// Whether the timed launch of PCG iteration `it` ran in a solve that took
// `iters` iterations: iteration k's A.p runs before its convergence test,
// its V-cycle after it (kernels return at once after the solve has finished).
static bool prof_ran(int ch, int it, int iters) {
  return ch == PROF_AP ? it <= iters - 1 : it <= iters - 2;
}

// after a replay of the chunk that starts at PCG iteration first_iter (the
// host has synchronised and copied the scalars)
mgpbd_status prof_harvest_graph(Handle *h, int first_iter) {
  const PcgScalars &s = *h->sc_host;
  for (int ch = 0; ch < PROF_CH; ++ch)
    for (int k = 0; k < h->gev_used[ch]; ++k) {
      const int it = first_iter + h->gev_iter[ch][k];
      if (s.done && !prof_ran(ch, it, s.iters)) continue;
      float ms = 0.f;
      MG_CUDA(cudaEventElapsedTime(&ms, h->gev[ch][2 * k], h->gev[ch][2 * k + 1]));
      h->prof_ms[ch] += ms;
      h->prof_n[ch]++;
    }
  return MGPBD_OK;
}

mgpbd_status prof_harvest(Handle *h, int iters) {
  if (!h->prof) return MGPBD_OK;
  for (int ch = 0; ch < PROF_CH; ++ch) {
    for (int k = 0; k < h->pev_used[ch]; ++k) {
      if (!prof_ran(ch, h->pev_iter[ch][k], iters)) continue;
      float ms = 0.f;
      MG_CUDA(cudaEventSynchronize(h->pev[ch][2 * k + 1]));
      MG_CUDA(cudaEventElapsedTime(&ms, h->pev[ch][2 * k], h->pev[ch][2 * k + 1]));
      h->prof_ms[ch] += ms;
      h->prof_n[ch]++;
    }
    h->pev_used[ch] = 0;
  }
  return MGPBD_OK;
}

void set_error(const std::string &msg) { g_err = msg; }

mgpbd_status cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
  cudaGetLastError();  // a failed call must not resurface at the next launch check
  char buf[512];
  snprintf(buf, sizeof(buf), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  set_error(buf);
  return e == cudaErrorMemoryAllocation ? MGPBD_E_OOM : MGPBD_E_CUDA;
}

void Arena::use_workspace(void *p, size_t n) {
  base = static_cast<char *>(p);
  cap = n & ~(size_t)255;
  holes.clear();
  if (cap) holes.emplace(0, cap);
}

mgpbd_status Arena::alloc(void **p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 16;
  n = (n + 255) & ~(size_t)255;  // keep every buffer 256-byte aligned
  if (base) {
    auto it = holes.begin();
    while (it != holes.end() && it->second < n) ++it;
    if (it == holes.end()) {
      char buf[160];
      snprintf(buf, sizeof(buf),
               "workspace of %zu bytes exhausted: %zu more bytes needed with %zu live", cap, n,
               bytes);
      set_error(buf);
      return MGPBD_E_BUDGET;
    }
    const size_t off = it->first, len = it->second;
    holes.erase(it);
    if (len > n) holes.emplace(off + n, len - n);
    *p = base + off;
  } else {
    cudaError_t e = cudaMallocAsync(p, n, stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      *p = nullptr;
      char buf[128];
      snprintf(buf, sizeof(buf), "device allocation of %zu bytes failed: %s", n,
               cudaGetErrorString(e));
      set_error(buf);
      return MGPBD_E_OOM;
    }
  }
  bytes += n;
  peak = std::max(peak, bytes);
  live.emplace_back(*p, n);
  return MGPBD_OK;
}

void Arena::release(void *p) {
  if (!p) return;
  size_t n = 0;
  for (auto it = live.begin(); it != live.end(); ++it)
    if (it->first == p) {
      n = it->second;
      bytes -= n;
      live.erase(it);
      break;
    }
  if (!base) {
    cudaFreeAsync(p, stream);
    return;
  }
  if (!n) return;  // not an array of this arena
  size_t off = static_cast<size_t>(static_cast<char *>(p) - base), len = n;
  auto next = holes.lower_bound(off);
  if (next != holes.end() && off + len == next->first) {  // merge with the range after
    len += next->second;
    next = holes.erase(next);
  }
  if (next != holes.begin()) {  // merge with the range before
    auto prev = std::prev(next);
    if (prev->first + prev->second == off) {
      off = prev->first;
      len += prev->second;
      holes.erase(prev);
    }
  }
  holes.emplace(off, len);
}

void Arena::release_all() {
  if (!base)
    for (auto &q : live) cudaFreeAsync(q.first, stream);
  live.clear();
  bytes = 0;
  if (base) use_workspace(base, cap);
  cudaStreamSynchronize(stream);
}

int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

int wave_blocks(const void *kernel, int threads) {
  static std::mutex mu;
  static std::unordered_map<const void *, int> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(kernel);
  if (it != cache.end()) return it->second;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess ||
      per_sm <= 0) {
    cudaGetLastError();
    per_sm = 1;
  }
  const int n = per_sm * num_sms();
  cache.emplace(kernel, n);
  return n;
}

mgpbd_status ensure_tmp(Handle *h, size_t bytes) {
  if (h->tmp_bytes >= bytes) return MGPBD_OK;
  if (h->tmp) {
    MG_CUDA(cudaStreamSynchronize(h->stream));
    h->arena.release(h->tmp);
    h->tmp = nullptr;
    h->tmp_bytes = 0;
  }
  size_t want = std::max(bytes, (size_t)1 << 20);
  MG_TRY(h->arena.alloc(&h->tmp, want));
  h->tmp_bytes = want;
  return MGPBD_OK;
}

mgpbd_status read_i64(Handle *h, const int64_t *d, int64_t *out) {
  MG_CUDA(cudaMemcpyAsync(out, d, sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream));
  MG_CUDA(cudaStreamSynchronize(h->stream));
  return MGPBD_OK;
}

static mgpbd_status copy_out(Handle *h, void *dst, const void *src, size_t bytes, int mem) {
  if (!dst || bytes == 0) return MGPBD_OK;
  if (!src) {
    set_error("requested array is not available (no setup yet?)");
    return MGPBD_E_INVALID;
  }
  MG_CUDA(cudaMemcpyAsync(dst, src, bytes,
                          mem == MGPBD_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                          h->stream));
  if (mem == MGPBD_MEM_HOST) MG_CUDA(cudaStreamSynchronize(h->stream));
  return MGPBD_OK;
}

static mgpbd_status check_params(const mgpbd_params *p) {
  if (!(p->dt > 0.0) || p->max_iter < 0 || p->pcg_maxiter < 1 || p->nk_sweeps < 0 ||
      p->smooth_sweeps < 1 || p->power_iters < 1 || p->coarse_max < 1 || p->max_levels < 1 ||
      p->max_levels > kMaxLevels || (p->precision != MGPBD_FP64 && p->precision != MGPBD_MIXED) ||
      (p->smoother != MGPBD_SMOOTH_JACOBI && p->smoother != MGPBD_SMOOTH_MCGS &&
       p->smoother != MGPBD_SMOOTH_CHEBYSHEV) ||
      !(p->theta_s >= 0.0) || p->backtrack < 0 ||
      (p->autotune != 0 && p->autotune != 1) || (p->level0_op != 0 && p->level0_op != 1) ||
      (p->use_graphs != 0 && p->use_graphs != 1) ||
      (p->linear_solver != 0 && p->linear_solver != 1) || p->nk_vectors < 1 ||
      p->nk_vectors > 8 || (p->ap_split != 0 && p->ap_split != 1) ||
      (p->ap_split == 1 && (p->precision != MGPBD_MIXED || p->level0_op != 1)) ||
      !(p->pcg_rtol >= 0.0) || !(p->power_safety > 0.0)) {
    set_error("invalid mgpbd_params");
    return MGPBD_E_INVALID;
  }
  return MGPBD_OK;
}

static void destroy(Handle *h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  h->arena.release_all();
  if (h->sc_host) cudaFreeHost(h->sc_host);
  if (h->flag_host) cudaFreeHost(h->flag_host);
  for (int ch = 0; ch < PROF_CH; ++ch) {
    for (cudaEvent_t e : h->pev[ch]) cudaEventDestroy(e);
    for (cudaEvent_t e : h->gev[ch]) cudaEventDestroy(e);
  }
  if (h->pcg_graph) cudaGraphExecDestroy(h->pcg_graph);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  delete h;
}

static mgpbd_status create(const mgpbd_mesh_desc *md, const mgpbd_params *p, void *stream,
                           void *ws, size_t ws_bytes, Handle **out) {
  *out = nullptr;
  if (!md || !p || md->n_verts <= 0 || md->n_dist < 0 || md->n_tet < 0 || !md->rest_pos ||
      !md->inv_mass || (md->n_dist > 0 && !md->dist) || (md->n_tet > 0 && !md->tet) ||
      (md->n_dist + md->n_tet > 0 && !md->alpha) || md->tet_kind < 0 || md->tet_kind > 1) {
    set_error("invalid mesh descriptor");
    return MGPBD_E_INVALID;
  }
  if ((int64_t)md->n_dist + md->n_tet >= (int64_t)1 << 31) {
    set_error("too many constraint rows");
    return MGPBD_E_INVALID;
  }
  MG_TRY(check_params(p));
  // host-side validation of indices (rows must reference distinct vertices)
  for (int64_t j = 0; j < md->n_dist; ++j) {
    int a = md->dist[2 * j], b = md->dist[2 * j + 1];
    if (a < 0 || a >= md->n_verts || b < 0 || b >= md->n_verts || a == b) {
      set_error("distance pair out of range or degenerate");
      return MGPBD_E_INVALID;
    }
  }
  for (int64_t t = 0; t < md->n_tet; ++t) {
    const int32_t *q = md->tet + 4 * t;
    for (int k = 0; k < 4; ++k) {
      if (q[k] < 0 || q[k] >= md->n_verts) {
        set_error("tet vertex out of range");
        return MGPBD_E_INVALID;
      }
      for (int k2 = 0; k2 < k; ++k2)
        if (q[k] == q[k2]) {
          set_error("degenerate tet (repeated vertex)");
          return MGPBD_E_INVALID;
        }
    }
  }
  for (int64_t v = 0; v < md->n_verts; ++v)
    if (!(md->inv_mass[v] >= 0.0)) {
      set_error("inverse mass must be >= 0");
      return MGPBD_E_INVALID;
    }

  Handle *h = new Handle();
  h->stream = (cudaStream_t)stream;
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    set_error("create: cudaGetDevice failed");
    return MGPBD_E_CUDA;
  }
  h->arena.stream = h->stream;
  if (ws) h->arena.use_workspace(ws, ws_bytes);
  h->p = *p;
  h->N = md->n_verts;
  h->E = md->n_dist;
  h->T = md->n_tet;
  h->m = h->E + h->T;
  h->tet_kind = md->tet_kind;
  auto fail = [&](mgpbd_status s) {
    destroy(h);
    return s;
  };
  mgpbd_status s;
#define CK(expr)             \
  do {                       \
    s = (expr);              \
    if (s < 0) return fail(s); \
  } while (0)
  const int N = h->N, E = h->E, T = h->T, m = h->m;
  CK(alloc_n(h->arena, &h->rest, 3 * (size_t)N));
  CK(alloc_n(h->arena, &h->w, (size_t)N));
  CK(alloc_n(h->arena, &h->alpha_t, (size_t)m));
  CK(alloc_n(h->arena, &h->L0, (size_t)E));
  CK(alloc_n(h->arena, &h->V0, (size_t)T));
  if (h->tet_kind == 1) CK(alloc_n(h->arena, &h->Dminv, 9 * (size_t)T));
  CK(alloc_n(h->arena, &h->edge, 2 * (size_t)E));
  CK(alloc_n(h->arena, &h->tet, 4 * (size_t)T));
  CK(alloc_n(h->arena, &h->x, 3 * (size_t)N));
  CK(alloc_n(h->arena, &h->v, 3 * (size_t)N));
  CK(alloc_n(h->arena, &h->xold, 3 * (size_t)N));
  CK(alloc_n(h->arena, &h->lambda, (size_t)m));
  CK(alloc_n(h->arena, &h->C, (size_t)m));
  CK(alloc_n(h->arena, &h->b, (size_t)m));
  CK(alloc_n(h->arena, &h->dl, (size_t)m));
  CK(alloc_n(h->arena, &h->dx, 3 * (size_t)N));
  CK(alloc_n(h->arena, &h->xbak, 3 * (size_t)N));
  CK(alloc_n(h->arena, &h->gd, 3 * (size_t)E));
  CK(alloc_n(h->arena, &h->gt, 12 * (size_t)T));
  CK(alloc_n(h->arena, &h->pr, (size_t)m));
  CK(alloc_n(h->arena, &h->pz, (size_t)m));
  CK(alloc_n(h->arena, &h->pp, (size_t)m));
  CK(alloc_n(h->arena, &h->pq, (size_t)m));
  CK(alloc_n(h->arena, &h->sc, 1));
  CK(alloc_n(h->arena, &h->partials, 4096 + 16));
  CK(alloc_n(h->arena, &h->counter, 16));
  CK(alloc_n(h->arena, &h->gbar, 16));
  CK(alloc_n(h->arena, &h->flag, 16));
  CK(alloc_n(h->arena, &h->cstat, 4));
  if (cudaMallocHost((void **)&h->sc_host, sizeof(PcgScalars)) != cudaSuccess ||
      cudaMallocHost((void **)&h->flag_host, 16 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    set_error("pinned host allocation failed");
    return fail(MGPBD_E_OOM);
  }
  if (cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess) {
    set_error("cudaEventCreate failed");
    return fail(MGPBD_E_CUDA);
  }
  cudaStream_t st = h->stream;
  auto up = [&](void *d, const void *src, size_t bytes) -> mgpbd_status {
    if (!bytes) return MGPBD_OK;
    MG_CUDA(cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, st));
    return MGPBD_OK;
  };
  CK(up(h->rest, md->rest_pos, sizeof(double) * 3 * N));
  CK(up(h->x, md->rest_pos, sizeof(double) * 3 * N));
  CK(up(h->w, md->inv_mass, sizeof(double) * N));
  CK(up(h->edge, md->dist, sizeof(int32_t) * 2 * E));
  CK(up(h->tet, md->tet, sizeof(int32_t) * 4 * T));
  {
    // alpha~ = alpha / dt^2 (eq. 2), computed on the host in IEEE double
    std::vector<double> at((size_t)m);
    double dt2 = p->dt * p->dt;
    for (int j = 0; j < m; ++j) at[j] = md->alpha[j] / dt2;
    CK(up(h->alpha_t, at.data(), sizeof(double) * m));
    if (cudaStreamSynchronize(st) != cudaSuccess) return fail(MGPBD_E_CUDA);
  }
  if (cudaMemsetAsync(h->v, 0, sizeof(double) * 3 * N, st) != cudaSuccess ||
      cudaMemsetAsync(h->lambda, 0, sizeof(double) * m, st) != cudaSuccess ||
      cudaMemsetAsync(h->counter, 0, 16 * sizeof(unsigned), st) != cudaSuccess ||
      cudaMemsetAsync(h->gbar, 0, 16 * sizeof(unsigned), st) != cudaSuccess)
    return fail(MGPBD_E_CUDA);
  CK(rest_shape(h));
  CK(build_incidence(h));
  CK(build_pattern(h));
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    set_error("create: stream error");
    return fail(MGPBD_E_CUDA);
  }
#undef CK
  *out = h;
  return MGPBD_OK;
}

static mgpbd_status timed_begin(Handle *h) {
  MG_CUDA(cudaEventRecord(h->ev0, h->stream));
  return MGPBD_OK;
}
static mgpbd_status timed_end(Handle *h, double *acc) {
  MG_CUDA(cudaEventRecord(h->ev1, h->stream));
  MG_CUDA(cudaEventSynchronize(h->ev1));
  float ms = 0.f;
  MG_CUDA(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
  *acc += ms;
  return MGPBD_OK;
}

// The parts of one global iteration of Alg. 1 around its MGPCG solve.
// Before: C and grad C, assembly, the matrix-free arrays, the lazy setup when
// due (else the Galerkin re-form) and the coarsest factorisation.
mgpbd_status iterate_prepare(Handle *h, bool *due) {
  MG_TRY(launch_eval(h));
  MG_TRY(launch_assemble(h));
  if (h->p.level0_op == 1) MG_TRY(mf_prepare(h));
  *due = !h->have_setup || (h->p.setup_interval > 0 && h->it_global % h->p.setup_interval == 0);
  if (*due) {
    MG_TRY(timed_begin(h));
    MG_TRY(amg_setup(h));
    MG_TRY(timed_end(h, &h->ms_setup));
  } else {
    MG_TRY(galerkin_reform(h));
  }
  return coarsest_factor(h);
}

// After the solve (status st, inf): a breakdown on a reused hierarchy (omega
// or P built for an A that has since changed) sets up afresh for the current
// A and solves once more; then dlambda, lambda and x are applied (eq. 5).
mgpbd_status iterate_complete(Handle *h, mgpbd_status st, mgpbd_solve_info *inf, bool due,
                              mgpbd_solve_info *info) {
  if (st == MGPBD_E_BREAKDOWN && !due) {
    MG_TRY(timed_begin(h));
    MG_TRY(amg_setup(h));
    MG_TRY(timed_end(h, &h->ms_setup));
    MG_TRY(coarsest_factor(h));
    *inf = mgpbd_solve_info{};
    st = pcg_solve(h, h->b, h->dl, inf);
  }
  h->it_global++;
  if (st < 0) {
    h->last = *inf;
    if (info) *info = *inf;
    return st;
  }
  MG_TRY(launch_update(h, inf));
  h->last = *inf;
  if (info) *info = *inf;
  return inf->status;
}

// One global iteration of Alg. 1.
static mgpbd_status iterate(Handle *h, mgpbd_solve_info *info) {
  if (h->p.linear_solver == 1) {  // XPBD's local step (eq. 4)
    MG_TRY(launch_eval(h));
    MG_TRY(launch_assemble(h));
    mgpbd_solve_info inf{};
    MG_TRY(xpbd_step(h, &inf));
    h->it_global++;
    MG_TRY(launch_update(h, &inf));
    h->last = inf;
    if (info) *info = inf;
    return MGPBD_OK;
  }
  bool due = false;
  MG_TRY(iterate_prepare(h, &due));
  mgpbd_solve_info inf{};
  mgpbd_status st = pcg_solve(h, h->b, h->dl, &inf);
  return iterate_complete(h, st, &inf, due, info);
}

}  // namespace mg

using namespace mg;

struct mgpbd_handle : public Handle {};

static inline Handle *H(mgpbd_handle_t *h) { return reinterpret_cast<Handle *>(h); }

extern "C" {

const char *mgpbd_last_error(void) { return g_err.c_str(); }

mgpbd_status mgpbd_default_params(mgpbd_params *p) {
  if (!p) return MGPBD_E_INVALID;
  memset(p, 0, sizeof(*p));
  p->dt = 1.0 / 60.0;
  p->gravity[0] = 0.0;
  p->gravity[1] = -9.8;
  p->gravity[2] = 0.0;
  p->omega_x = 0.25;
  p->max_iter = 20;
  p->eps_b = 0.0;
  p->pcg_rtol = 1e-6;
  p->pcg_maxiter = 20000;
  p->setup_interval = 400;
  p->nk_sweeps = 3;
  p->nk_omega = 2.0 / 3.0;
  p->theta_s = 0.1;
  p->smoother = MGPBD_SMOOTH_JACOBI;
  p->smooth_sweeps = 2;
  p->lambda_min_est = 0.1;
  p->power_iters = 15;
  p->power_safety = 1.25;
  p->coarse_max = 400;
  p->max_levels = 8;
  p->precision = MGPBD_FP64;
  p->backtrack = 0;
  p->autotune = 0;
  p->level0_op = 0;
  p->use_graphs = 0;
  p->linear_solver = 0;
  p->nk_vectors = 1;
  p->ap_split = 0;
  p->seed_nk = 3;
  p->seed_agg = 4;
  p->seed_col = 5;
  p->seed_pow = 7;
  return MGPBD_OK;
}

mgpbd_status mgpbd_create(const mgpbd_mesh_desc *mesh, const mgpbd_params *p, void *stream,
                          mgpbd_handle_t **out) {
  if (!out) {
    set_error("out is NULL");
    return MGPBD_E_INVALID;
  }
  Handle *h = nullptr;
  mgpbd_status s = create(mesh, p, stream, nullptr, 0, &h);
  *out = reinterpret_cast<mgpbd_handle_t *>(h);
  return s;
}

mgpbd_status mgpbd_create_in_workspace(const mgpbd_mesh_desc *mesh, const mgpbd_params *p,
                                       void *d_workspace, size_t bytes, void *stream,
                                       mgpbd_handle_t **out) {
  if (!out) {
    set_error("out is NULL");
    return MGPBD_E_INVALID;
  }
  *out = nullptr;
  if (!d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) & 255) || bytes < 256) {
    set_error("workspace must be a non-NULL, 256-byte aligned device buffer of >= 256 bytes");
    return MGPBD_E_INVALID;
  }
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, d_workspace) != cudaSuccess ||
      attr.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    set_error("workspace is not device memory");
    return MGPBD_E_INVALID;
  }
  Handle *h = nullptr;
  mgpbd_status s = create(mesh, p, stream, d_workspace, bytes, &h);
  *out = reinterpret_cast<mgpbd_handle_t *>(h);
  return s;
}

void mgpbd_destroy(mgpbd_handle_t *h) { destroy(H(h)); }

mgpbd_status mgpbd_set_state(mgpbd_handle_t *hh, const double *x, const double *v, int mem) {
  Handle *h = H(hh);
  if (!h) return MGPBD_E_INVALID;
  cudaMemcpyKind k = mem == MGPBD_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  size_t bytes = sizeof(double) * 3 * (size_t)h->N;
  if (x) MG_CUDA(cudaMemcpyAsync(h->x, x, bytes, k, h->stream));
  if (v) MG_CUDA(cudaMemcpyAsync(h->v, v, bytes, k, h->stream));
  if (mem == MGPBD_MEM_HOST) MG_CUDA(cudaStreamSynchronize(h->stream));
  return MGPBD_OK;
}

mgpbd_status mgpbd_get_state(mgpbd_handle_t *hh, double *x, double *v, int mem) {
  Handle *h = H(hh);
  if (!h) return MGPBD_E_INVALID;
  size_t bytes = sizeof(double) * 3 * (size_t)h->N;
  MG_TRY(copy_out(h, x, h->x, bytes, mem));
  MG_TRY(copy_out(h, v, h->v, bytes, mem));
  return MGPBD_OK;
}

mgpbd_status mgpbd_begin_frame(mgpbd_handle_t *hh) {
  Handle *h = H(hh);
  if (!h) return MGPBD_E_INVALID;
  return launch_begin_frame(h);
}

mgpbd_status mgpbd_end_frame(mgpbd_handle_t *hh) {
  Handle *h = H(hh);
  if (!h) return MGPBD_E_INVALID;
  return launch_end_frame(h);
}

mgpbd_status mgpbd_iterate(mgpbd_handle_t *hh, mgpbd_solve_info *info) {
  Handle *h = H(hh);
  if (!h) return MGPBD_E_INVALID;
  return iterate(h, info);
}

mgpbd_status mgpbd_step(mgpbd_handle_t *hh, int n_frames) {
  Handle *h = H(hh);
  if (!h || n_frames < 0) return MGPBD_E_INVALID;
  mgpbd_status worst = MGPBD_OK;
  for (int f = 0; f < n_frames; ++f) {
    MG_TRY(launch_begin_frame(h));
    for (int it = 0; it < h->p.max_iter; ++it) {
      mgpbd_solve_info inf{};
      mgpbd_status s = iterate(h, &inf);
      if (s < 0) return s;
      if (s > worst) worst = s;
      if (inf.bnorm < h->p.eps_b) break;
    }
    MG_TRY(launch_end_frame(h));
  }
  MG_CUDA(cudaStreamSynchronize(h->stream));
  return worst;
}

mgpbd_status mgpbd_eval_assemble(mgpbd_handle_t *hh) {
  Handle *h = H(hh);
  if (!h) return MGPBD_E_INVALID;
  MG_TRY(launch_eval(h));
  MG_TRY(launch_assemble(h));
  if (h->p.level0_op == 1) MG_TRY(mf_prepare(h));
  return MGPBD_OK;
}

mgpbd_status mgpbd_setup(mgpbd_handle_t *hh) {
  Handle *h = H(hh);
  if (!h) return MGPBD_E_INVALID;
  return amg_setup(h);
}

mgpbd_status mgpbd_prepare_solve(mgpbd_handle_t *hh) {
  Handle *h = H(hh);
  if (!h) return MGPBD_E_INVALID;
  if (!h->have_setup) MG_TRY(amg_setup(h));
  else MG_TRY(galerkin_reform(h));
  MG_TRY(coarsest_factor(h));
  MG_CUDA(cudaStreamSynchronize(h->stream));
  return MGPBD_OK;
}

mgpbd_status mgpbd_solve(mgpbd_handle_t *hh, const double *d_b, double *d_dl,
                         mgpbd_solve_info *info) {
  Handle *h = H(hh);
  if (!h || !d_b || !d_dl) return MGPBD_E_INVALID;
  if (!h->have_setup) {
    set_error("mgpbd_solve: no hierarchy (call mgpbd_prepare_solve first)");
    return MGPBD_E_INVALID;
  }
  mgpbd_solve_info inf{};
  mgpbd_status s = pcg_solve(h, d_b, d_dl, &inf);
  if (info) *info = inf;
  return s;
}

mgpbd_status mgpbd_vcycle(mgpbd_handle_t *hh, const double *d_r, double *d_z) {
  Handle *h = H(hh);
  if (!h || !d_r || !d_z || !h->have_setup) return MGPBD_E_INVALID;
  MG_TRY(vcycle_apply(h, d_r, d_z));
  MG_CUDA(cudaStreamSynchronize(h->stream));
  return MGPBD_OK;
}

mgpbd_status mgpbd_apply(mgpbd_handle_t *hh, const double *d_x, double *d_y, int form) {
  Handle *h = H(hh);
  if (!h || (h->m > 0 && (!d_x || !d_y)) || form < 0 || form > 2) return MGPBD_E_INVALID;
  if (h->m == 0) return MGPBD_OK;
  if (!h->lev[0].val || (form >= 1 && (h->p.level0_op != 1 || !h->vslot)) ||
      (form == 2 && !h->p.ap_split)) {
    set_error("mgpbd_apply: this form of A is not prepared on the instance");
    return MGPBD_E_INVALID;
  }
  MG_TRY(apply_level0(h, form, d_x, d_y));
  MG_CUDA(cudaStreamSynchronize(h->stream));
  return MGPBD_OK;
}

mgpbd_status mgpbd_stats(mgpbd_handle_t *hh, mgpbd_stats_t *s) {
  Handle *h = H(hh);
  if (!h || !s) return MGPBD_E_INVALID;
  MG_CUDA(cudaStreamSynchronize(h->stream));
  memset(s, 0, sizeof(*s));
  s->levels = h->L;
  s->n_setups = h->n_setups;
  s->global_iters = h->it_global;
  double tot = 0;
  for (int l = 0; l < h->L; ++l) tot += (double)h->lev[l].nnz;
  s->op_complexity = h->L && h->lev[0].nnz ? tot / (double)h->lev[0].nnz : 0.0;
  s->device_bytes = h->arena.bytes;
  s->peak_device_bytes = h->arena.peak;
  s->ms_setup = h->ms_setup;
  s->ms_galerkin = h->ms_galerkin;
  s->ms_solve = h->ms_solve;
  s->ms_other = h->ms_other;
  return MGPBD_OK;
}

mgpbd_status mgpbd_set_colouring(mgpbd_handle_t *hh, int enable) {
  Handle *h = H(hh);
  if (!h) return MGPBD_E_INVALID;
  h->want_colors = enable != 0;
  return MGPBD_OK;
}

mgpbd_status mgpbd_profile(mgpbd_handle_t *hh, int enable) {
  Handle *h = H(hh);
  if (!h) return MGPBD_E_INVALID;
  MG_CUDA(cudaStreamSynchronize(h->stream));
  if (enable < 0 || enable > 3) return MGPBD_E_INVALID;
  h->prof = enable != 0;
  h->prof_mask = enable;
  h->gen++;  // a captured graph records the channels of its capture
  for (int ch = 0; ch < PROF_CH; ++ch) {
    h->pev_used[ch] = 0;
    h->prof_ms[ch] = 0.0;
    h->prof_n[ch] = 0;
  }
  return MGPBD_OK;
}

mgpbd_status mgpbd_profile_read(mgpbd_handle_t *hh, double *total_ms, int64_t *launches,
                                double *bytes_per_launch) {
  Handle *h = H(hh);
  if (!h) return MGPBD_E_INVALID;
  MG_CUDA(cudaStreamSynchronize(h->stream));
  if (total_ms) *total_ms = h->prof_ms[PROF_SWEEP];
  if (launches) *launches = h->prof_n[PROF_SWEEP];
  if (bytes_per_launch) {
    const Level &L = h->lev[0];
    double vb = h->p.precision == MGPBD_MIXED ? 4.0 : 8.0;
    if (h->p.level0_op == 1) {
      // matrix-free sweep: vertex pass (row ids and incidence-ordered
      // gradients, row pointers, x and w once, u written) and row pass
      // (row gradients, vertex ids, u once, alpha~, x, b, 1/A_ii, x_new)
      double ninc = 2.0 * h->E + 4.0 * h->T;
      *bytes_per_launch = ninc * (4.0 + 3.0 * vb) + (h->N + 1.0) * 8.0 + (double)h->m * vb +
                          h->N * vb + 3.0 * h->N * vb + h->E * (3.0 * vb + 8.0) +
                          h->T * (12.0 * vb + 16.0) + 3.0 * h->N * vb + 5.0 * h->m * vb;
    } else {
      // CSR sweep: values and column indices once, row pointers, and four
      // vectors (x, b, 1/A_ii, x_new)
      *bytes_per_launch = (double)L.nnz * (vb + 4.0) + (double)L.n * (8.0 + 4.0 * vb);
    }
  }
  return MGPBD_OK;
}

mgpbd_status mgpbd_profile_read_ap(mgpbd_handle_t *hh, double *total_ms, int64_t *launches,
                                   double *bytes_per_launch) {
  Handle *h = H(hh);
  if (!h) return MGPBD_E_INVALID;
  MG_CUDA(cudaStreamSynchronize(h->stream));
  if (total_ms) *total_ms = h->prof_ms[PROF_AP];
  if (launches) *launches = h->prof_n[PROF_AP];
  if (bytes_per_launch) {
    const Level &L = h->lev[0];
    if (h->p.level0_op == 1) {
      // vertex pass: per incidence a row id and an 8-byte value per gradient
      // component (FP64, or FP32 high and low parts); row pointers, order, p
      // and w once, u written.  Row pass: row gradients and vertex ids, u
      // once, alpha~, p and q.  Every value is 8 bytes in both forms.
      double ninc = 2.0 * h->E + 4.0 * h->T;
      *bytes_per_launch = ninc * 28.0 + (h->N + 1.0) * 8.0 + h->N * 4.0 + (double)h->m * 8.0 +
                          h->N * 8.0 + 3.0 * h->N * 8.0 + h->E * 32.0 + h->T * 112.0 +
                          3.0 * h->N * 8.0 + 3.0 * h->m * 8.0;
    } else {
      // FP64 CSR product: values and columns once, row pointers, p once, q
      *bytes_per_launch = (double)L.nnz * 12.0 + (double)L.n * 24.0;
    }
  }
  return MGPBD_OK;
}

unsigned long long mgpbd_launch_count(void) { return g_launches; }

mgpbd_status mgpbd_sizes(mgpbd_handle_t *hh, int *n_verts, int *n_rows, int64_t *nnz) {
  Handle *h = H(hh);
  if (!h) return MGPBD_E_INVALID;
  if (n_verts) *n_verts = h->N;
  if (n_rows) *n_rows = h->m;
  if (nnz) *nnz = h->lev[0].nnz;
  return MGPBD_OK;
}

mgpbd_status mgpbd_level_info_get(mgpbd_handle_t *hh, int level, mgpbd_level_info *info) {
  Handle *h = H(hh);
  if (!h || !info || level < 0 || level >= std::max(h->L, 1)) return MGPBD_E_INVALID;
  const Level &L = h->lev[level];
  info->n = L.n;
  info->nnz = L.nnz;
  info->n_agg = level + 1 < h->L ? L.n_agg : 0;
  info->n_colors = L.n_colors;
  info->lmax = L.lmax;
  info->omega = L.omega;
  info->lanes_fp32 = L.G32;
  info->lanes_fp64 = L.G64;
  return MGPBD_OK;
}

mgpbd_status mgpbd_set_lanes(mgpbd_handle_t *hh, int csr32, int csr64, int vert32, int vert64) {
  Handle *h = H(hh);
  auto csr_ok = [](int g) { return g == 0 || g == 4 || g == 8 || g == 16 || g == 32; };
  auto vert_ok = [](int g) { return g == 0 || g == 4 || g == 8 || g == 16; };
  if (!h || !csr_ok(csr32) || !csr_ok(csr64) || !vert_ok(vert32) || !vert_ok(vert64)) {
    set_error("mgpbd_set_lanes: lanes per CSR row must be 0, 4, 8, 16 or 32 and lanes per "
              "vertex 0, 4, 8 or 16");
    return MGPBD_E_INVALID;
  }
  h->force_csr32 = csr32;
  h->force_csr64 = csr64;
  h->force_vert32 = vert32;
  h->force_vert64 = vert64;
  h->gen++;  // a captured PCG graph holds the previous shapes
  return MGPBD_OK;
}

mgpbd_status mgpbd_set_coarse_tail(mgpbd_handle_t *hh, int enable) {
  Handle *h = H(hh);
  if (!h || (enable != 0 && enable != 1)) return MGPBD_E_INVALID;
  h->tail = enable == 1;
  h->gen++;  // a captured PCG graph holds the other form
  return MGPBD_OK;
}

mgpbd_status mgpbd_set_wait_limit(mgpbd_handle_t *hh, long long polls) {
  Handle *h = H(hh);
  if (!h || polls < 0) return MGPBD_E_INVALID;
  h->wait_limit = polls;
  h->gen++;  // the limit is a launch argument of captured graphs
  return MGPBD_OK;
}

mgpbd_status mgpbd_get_lanes(mgpbd_handle_t *hh, int level, int *csr32, int *csr64, int *vert32,
                             int *vert64) {
  Handle *h = H(hh);
  if (!h || level < 0 || level >= std::max(h->L, 1)) return MGPBD_E_INVALID;
  const Level &L = h->lev[level];
  if (csr32) *csr32 = group_for(h, L, false);
  if (csr64) *csr64 = group_for(h, L, true);
  if (vert32) *vert32 = h->force_vert32 ? h->force_vert32 : h->mf_g32;
  if (vert64) *vert64 = h->force_vert64 ? h->force_vert64 : h->mf_g64;
  return MGPBD_OK;
}

mgpbd_status mgpbd_get_matrix(mgpbd_handle_t *hh, int level, int64_t *ptr, int32_t *col,
                              double *val, int mem) {
  Handle *h = H(hh);
  if (!h || level < 0 || level >= std::max(h->L, 1)) return MGPBD_E_INVALID;
  const Level &L = h->lev[level];
  MG_TRY(copy_out(h, ptr, L.ptr, sizeof(int64_t) * ((size_t)L.n + 1), mem));
  MG_TRY(copy_out(h, col, L.col, sizeof(int32_t) * (size_t)L.nnz, mem));
  MG_TRY(copy_out(h, val, L.val, sizeof(double) * (size_t)L.nnz, mem));
  return MGPBD_OK;
}

mgpbd_status mgpbd_get_map(mgpbd_handle_t *hh, uint16_t *map, int mem) {
  Handle *h = H(hh);
  if (!h) return MGPBD_E_INVALID;
  return copy_out(h, map, h->map, sizeof(uint16_t) * (size_t)h->lev[0].nnz, mem);
}

mgpbd_status mgpbd_get_incidence(mgpbd_handle_t *hh, int64_t *vptr, int32_t *vrow, int mem) {
  Handle *h = H(hh);
  if (!h) return MGPBD_E_INVALID;
  MG_TRY(copy_out(h, vptr, h->vptr, sizeof(int64_t) * ((size_t)h->N + 1), mem));
  MG_TRY(copy_out(h, vrow, h->vrow, sizeof(int32_t) * (2 * (size_t)h->E + 4 * (size_t)h->T), mem));
  return MGPBD_OK;
}

mgpbd_status mgpbd_get_aggregates(mgpbd_handle_t *hh, int level, int32_t *agg, uint8_t *root,
                                  double *P, double *B, int mem) {
  Handle *h = H(hh);
  if (!h || !h->have_setup || level < 0 || level >= h->L) return MGPBD_E_INVALID;
  const Level &L = h->lev[level];
  size_t n = (size_t)L.n, nk = n * (size_t)h->p.nk_vectors;
  if (level + 1 < h->L) {
    MG_TRY(copy_out(h, agg, L.agg, sizeof(int32_t) * n, mem));
    MG_TRY(copy_out(h, root, L.root, n, mem));
    MG_TRY(copy_out(h, P, L.P, sizeof(double) * nk, mem));
  }
  if (L.B) MG_TRY(copy_out(h, B, L.B, sizeof(double) * nk, mem));
  return MGPBD_OK;
}

mgpbd_status mgpbd_get_colors(mgpbd_handle_t *hh, int level, int32_t *color, int mem) {
  Handle *h = H(hh);
  if (!h || !h->have_setup || level < 0 || level >= h->L) return MGPBD_E_INVALID;
  const Level &L = h->lev[level];
  if (!L.color || L.n_colors <= 0) {
    set_error("no colouring: enable it with mgpbd_set_colouring before the setup");
    return MGPBD_E_INVALID;
  }
  return copy_out(h, color, L.color, sizeof(int32_t) * (size_t)L.n, mem);
}

mgpbd_status mgpbd_get_constraints(mgpbd_handle_t *hh, double *C, double *b, double *gd,
                                   double *gt, int mem) {
  Handle *h = H(hh);
  if (!h) return MGPBD_E_INVALID;
  MG_TRY(copy_out(h, C, h->C, sizeof(double) * (size_t)h->m, mem));
  MG_TRY(copy_out(h, b, h->b, sizeof(double) * (size_t)h->m, mem));
  MG_TRY(copy_out(h, gd, h->gd, sizeof(double) * 3 * (size_t)h->E, mem));
  MG_TRY(copy_out(h, gt, h->gt, sizeof(double) * 12 * (size_t)h->T, mem));
  return MGPBD_OK;
}

mgpbd_status mgpbd_get_lambda(mgpbd_handle_t *hh, double *lambda, double *dlambda, int mem) {
  Handle *h = H(hh);
  if (!h) return MGPBD_E_INVALID;
  MG_TRY(copy_out(h, lambda, h->lambda, sizeof(double) * (size_t)h->m, mem));
  MG_TRY(copy_out(h, dlambda, h->dl, sizeof(double) * (size_t)h->m, mem));
  return MGPBD_OK;
}

}  // extern "C"
