// Continuous-batching service of many simulation instances on one GPU.
//
// The paper runs one instance at a time; this layer serves step requests
// (one request = one frame of Alg. 1 for one instance) for many instances of
// different meshes.  Instance state stays on the device between its
// requests while memory allows.  Admission is by a device-memory budget:
// an instance is made resident only if its bytes fit, after evicting idle
// resident instances (least recently used first; their positions and
// velocities go to host memory and come back when they are next admitted).
// Up to `max_active` instances step at the same time, each on its own CUDA
// stream driven by its own worker thread, so their kernels overlap on the
// GPU and requests that arrive while others run are admitted as soon as a
// worker and memory are free.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"

namespace mg {

struct Instance {
  std::vector<double> rest, w, alpha, x, v;
  std::vector<int32_t> dist, tet;
  mgpbd_mesh_desc desc{};
  mgpbd_params p{};
  mgpbd_handle_t *h = nullptr;  // resident when not null
  cudaStream_t stream = nullptr;
  size_t est_bytes = 0, bytes = 0;
  bool busy = false;
  double last_used = 0.0;
  std::deque<int> pending;  // request indices in arrival order
};

struct Batch {
  mgpbd_batch_config cfg{};
  std::vector<Instance> inst;
  std::mutex mu;
  std::condition_variable cv;
  size_t resident = 0;  // bytes held by resident instances (reserved estimate while loading)
};

// upper estimate of an instance's device bytes from its mesh (before create):
// per nonzero of A (bounded by the sum over rows of their vertices' degrees)
// the column, FP64 and FP32 values, assembly map and strength mask; per row,
// vertex and incidence entry the vectors, gradients and matrix-free arrays;
// the dense coarsest factor and inverse (3 n_c^2 doubles, n_c below
// coarse_max or the whole system when it is smaller)
static size_t estimate_bytes_desc(const mgpbd_mesh_desc *d, const mgpbd_params *p) {
  const int N = d->n_verts, E = d->n_dist, T = d->n_tet;
  std::vector<int64_t> deg((size_t)N, 0);
  for (int64_t j = 0; j < 2 * (int64_t)E; ++j) deg[d->dist[j]]++;
  for (int64_t j = 0; j < 4 * (int64_t)T; ++j) deg[d->tet[j]]++;
  double nnz = 0.0;
  for (int64_t j = 0; j < 2 * (int64_t)E; ++j) nnz += (double)deg[d->dist[j]];
  for (int64_t j = 0; j < 4 * (int64_t)T; ++j) nnz += (double)deg[d->tet[j]];
  double m = (double)E + T, ninc = 2.0 * E + 4.0 * T;
  double b = nnz * (4 + 8 + 4 + 2 + 1) + m * 400.0 + N * 200.0 + ninc * 48.0 + (2 << 20);
  const double nc = std::min(m, (double)std::max(p->coarse_max, 1));
  b += 24.0 * nc * nc;
  return (size_t)b;
}

static size_t estimate_bytes(const Instance &in) { return estimate_bytes_desc(&in.desc, &in.p); }

static double now_s(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// drops the instance's handle and stream (its device state is lost)
static void drop_handle(Instance &in) {
  if (in.h) mgpbd_destroy(in.h);
  in.h = nullptr;
  if (in.stream) cudaStreamDestroy(in.stream);
  in.stream = nullptr;
}

// Creates the instance on the device from its host state.  On any failure
// nothing stays resident: a handle whose state was never loaded must not be
// stepped by a later request.
static mgpbd_status make_resident(Instance &in) {
  if (in.h) return MGPBD_OK;
  MG_CUDA(cudaStreamCreateWithFlags(&in.stream, cudaStreamNonBlocking));
  mgpbd_status s = mgpbd_create(&in.desc, &in.p, in.stream, &in.h);
  if (s >= 0) s = mgpbd_set_state(in.h, in.x.data(), in.v.data(), MGPBD_MEM_HOST);
  if (s < 0) {
    drop_handle(in);
    return s;
  }
  return MGPBD_OK;
}

// Moves the instance's state to host memory and frees its device memory.  If
// the state cannot be read back, the handle stays resident (its device state
// is the only current copy) and the error is returned.
static mgpbd_status evict(Instance &in) {
  if (!in.h) return MGPBD_OK;
  mgpbd_status s = mgpbd_get_state(in.h, in.x.data(), in.v.data(), MGPBD_MEM_HOST);
  if (s < 0) return s;
  drop_handle(in);
  return MGPBD_OK;
}

// one request: `frames` frames of Alg. 1 on one instance
static mgpbd_status run_request(Instance &in, int frames, mgpbd_step_result *r) {
  mgpbd_status worst = MGPBD_OK;
  for (int f = 0; f < frames; ++f) {
    MG_TRY(mgpbd_begin_frame(in.h));
    for (int it = 0; it < in.p.max_iter; ++it) {
      mgpbd_solve_info info{};
      mgpbd_status s = mgpbd_iterate(in.h, &info);
      r->global_iters++;
      r->pcg_iters += info.pcg_iters;
      if (s < 0) return s;
      worst = std::max(worst, s);
      if (info.bnorm < in.p.eps_b) break;
    }
    MG_TRY(mgpbd_end_frame(in.h));
  }
  MG_CUDA(cudaStreamSynchronize(in.stream));
  return worst;
}

}  // namespace mg

using namespace mg;

struct mgpbd_batch : public Batch {};

extern "C" {

mgpbd_status mgpbd_workspace_size(const mgpbd_mesh_desc *md, const mgpbd_params *p,
                                  size_t *bytes) {
  if (!md || !p || !bytes || md->n_verts <= 0 || md->n_dist < 0 || md->n_tet < 0 ||
      (md->n_dist > 0 && !md->dist) || (md->n_tet > 0 && !md->tet)) {
    set_error("mgpbd_workspace_size: invalid mesh descriptor");
    return MGPBD_E_INVALID;
  }
  for (int64_t j = 0; j < 2 * (int64_t)md->n_dist; ++j)
    if (md->dist[j] < 0 || md->dist[j] >= md->n_verts) {
      set_error("mgpbd_workspace_size: distance vertex out of range");
      return MGPBD_E_INVALID;
    }
  for (int64_t j = 0; j < 4 * (int64_t)md->n_tet; ++j)
    if (md->tet[j] < 0 || md->tet[j] >= md->n_verts) {
      set_error("mgpbd_workspace_size: tet vertex out of range");
      return MGPBD_E_INVALID;
    }
  *bytes = estimate_bytes_desc(md, p);
  return MGPBD_OK;
}

mgpbd_status mgpbd_batch_create(const mgpbd_batch_config *cfg, mgpbd_batch_t **out) {
  if (!cfg || !out || cfg->max_active < 1 || cfg->hbm_budget == 0) {
    set_error("mgpbd_batch_create: invalid configuration");
    return MGPBD_E_INVALID;
  }
  Batch *b = new Batch();
  b->cfg = *cfg;
  *out = reinterpret_cast<mgpbd_batch_t *>(b);
  num_sms();  // query once before worker threads exist
  return MGPBD_OK;
}

mgpbd_status mgpbd_batch_add_instance(mgpbd_batch_t *bb, const mgpbd_mesh_desc *md,
                                      const mgpbd_params *p, const double *x0, const double *v0,
                                      int *id) {
  Batch *b = reinterpret_cast<Batch *>(bb);
  if (!b || !md || !p || !id || md->n_verts <= 0 || md->n_dist < 0 || md->n_tet < 0) {
    set_error("mgpbd_batch_add_instance: invalid argument");
    return MGPBD_E_INVALID;
  }
  Instance in;
  const int N = md->n_verts, E = md->n_dist, T = md->n_tet;
  in.rest.assign(md->rest_pos, md->rest_pos + 3 * (size_t)N);
  in.w.assign(md->inv_mass, md->inv_mass + (size_t)N);
  if (E) in.dist.assign(md->dist, md->dist + 2 * (size_t)E);
  if (T) in.tet.assign(md->tet, md->tet + 4 * (size_t)T);
  if (E + T) in.alpha.assign(md->alpha, md->alpha + (size_t)E + T);
  in.x.assign(x0 ? x0 : md->rest_pos, (x0 ? x0 : md->rest_pos) + 3 * (size_t)N);
  in.v.assign(3 * (size_t)N, 0.0);
  if (v0) in.v.assign(v0, v0 + 3 * (size_t)N);
  in.p = *p;
  std::lock_guard<std::mutex> lock(b->mu);
  b->inst.push_back(std::move(in));
  Instance &r = b->inst.back();
  r.desc.n_verts = N;
  r.desc.rest_pos = r.rest.data();
  r.desc.inv_mass = r.w.data();
  r.desc.n_dist = E;
  r.desc.dist = E ? r.dist.data() : nullptr;
  r.desc.n_tet = T;
  r.desc.tet = T ? r.tet.data() : nullptr;
  r.desc.alpha = (E + T) ? r.alpha.data() : nullptr;
  r.desc.tet_kind = md->tet_kind;
  r.est_bytes = estimate_bytes(r);
  *id = (int)b->inst.size() - 1;
  // descriptors of earlier instances stay valid: vectors own their storage and
  // std::vector<Instance> moves the element vectors without reallocating them
  for (Instance &q : b->inst) {
    q.desc.rest_pos = q.rest.data();
    q.desc.inv_mass = q.w.data();
    q.desc.dist = q.desc.n_dist ? q.dist.data() : nullptr;
    q.desc.tet = q.desc.n_tet ? q.tet.data() : nullptr;
    q.desc.alpha = (q.desc.n_dist + q.desc.n_tet) ? q.alpha.data() : nullptr;
  }
  return MGPBD_OK;
}

mgpbd_status mgpbd_batch_run(mgpbd_batch_t *bb, const mgpbd_step_request *req, int n_req,
                             mgpbd_step_result *res) {
  Batch *b = reinterpret_cast<Batch *>(bb);
  if (!b || n_req < 0 || (n_req && (!req || !res))) return MGPBD_E_INVALID;
  for (int i = 0; i < n_req; ++i)
    if (req[i].instance < 0 || req[i].instance >= (int)b->inst.size() || req[i].frames < 1) {
      set_error("mgpbd_batch_run: request names an unknown instance or no frames");
      return MGPBD_E_INVALID;
    }
  int dev = 0;
  MG_CUDA(cudaGetDevice(&dev));
  std::vector<int> order((size_t)n_req);
  for (int i = 0; i < n_req; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int c) { return req[a].arrival_s < req[c].arrival_s; });
  for (int i = 0; i < n_req; ++i) {
    memset(&res[i], 0, sizeof(res[i]));
    res[i].id = req[i].id;
    res[i].instance = req[i].instance;
    res[i].arrival_s = req[i].arrival_s;
    res[i].start_s = res[i].finish_s = -1.0;
  }
  auto t0 = std::chrono::steady_clock::now();
  std::deque<int> jobs;  // requests whose instance is resident/being loaded, ready to run
  int done = 0, next_arrival = 0, active = 0;
  bool stop = false;
  mgpbd_status first_err = MGPBD_OK;

  auto worker = [&]() {
    cudaSetDevice(dev);
    std::unique_lock<std::mutex> lock(b->mu);
    for (;;) {
      b->cv.wait(lock, [&] { return stop || !jobs.empty(); });
      if (jobs.empty() && stop) return;
      int k = jobs.front();
      jobs.pop_front();
      Instance &in = b->inst[req[k].instance];
      lock.unlock();
      res[k].start_s = now_s(t0);
      mgpbd_status s = make_resident(in);
      if (s >= 0) s = run_request(in, req[k].frames, &res[k]);
      res[k].finish_s = now_s(t0);
      res[k].status = s;
      size_t held = 0;
      if (in.h) {
        mgpbd_stats_t st{};
        mgpbd_stats(in.h, &st);
        held = st.device_bytes;
      }
      lock.lock();
      if (s < 0 && first_err >= 0) first_err = s;
      // replace the admission estimate by the measured bytes
      b->resident = b->resident - in.bytes + held;
      in.bytes = held;
      in.busy = false;
      in.last_used = now_s(t0);
      --active;
      ++done;
      b->cv.notify_all();
    }
  };

  std::vector<std::thread> pool;
  for (int t = 0; t < b->cfg.max_active; ++t) pool.emplace_back(worker);

  std::unique_lock<std::mutex> lock(b->mu);
  while (done < n_req) {
    double now = now_s(t0);
    while (next_arrival < n_req && req[order[next_arrival]].arrival_s <= now) {
      int k = order[next_arrival++];
      b->inst[req[k].instance].pending.push_back(k);
    }
    // admit: earliest pending request of an idle instance, while memory and
    // workers allow
    for (;;) {
      if (active >= b->cfg.max_active) break;
      int best = -1;
      for (size_t i = 0; i < b->inst.size(); ++i) {
        Instance &in = b->inst[i];
        if (in.busy || in.pending.empty()) continue;
        if (best < 0 || req[in.pending.front()].arrival_s <
                            req[b->inst[best].pending.front()].arrival_s)
          best = (int)i;
      }
      if (best < 0) break;
      Instance &in = b->inst[best];
      if (!in.h) {
        size_t need = in.bytes ? in.bytes : in.est_bytes;
        if (need > b->cfg.hbm_budget) {  // can never fit: fail the request
          int k = in.pending.front();
          in.pending.pop_front();
          res[k].status = MGPBD_E_BUDGET;
          res[k].start_s = res[k].finish_s = now_s(t0);
          if (first_err >= 0) first_err = MGPBD_E_BUDGET;
          ++done;
          set_error("mgpbd_batch_run: an instance needs more memory than the budget");
          continue;
        }
        while (b->resident + need > b->cfg.hbm_budget) {
          int victim = -1;
          for (size_t i = 0; i < b->inst.size(); ++i) {
            Instance &q = b->inst[i];
            // busy first: a busy instance's handle is being written by its
            // worker outside the lock, so it must not be read here
            if (q.busy || !q.h || (int)i == best) continue;
            if (victim < 0 || q.last_used < b->inst[victim].last_used) victim = (int)i;
          }
          if (victim < 0) break;
          Instance &q = b->inst[victim];
          mgpbd_status s = evict(q);
          if (s < 0) {  // still resident (its state could not be read back)
            if (first_err >= 0) first_err = s;
            break;
          }
          b->resident -= q.bytes;
          q.bytes = 0;
        }
        if (b->resident + need > b->cfg.hbm_budget && active > 0) break;  // wait for memory
        b->resident += need;  // reserved until the worker measures the real size
        in.bytes = need;
      }
      int k = in.pending.front();
      in.pending.pop_front();
      in.busy = true;
      ++active;
      jobs.push_back(k);
      b->cv.notify_all();
    }
    if (done >= n_req) break;
    double wait = 0.05;
    if (next_arrival < n_req) wait = std::min(wait, std::max(0.0, req[order[next_arrival]].arrival_s - now));
    b->cv.wait_for(lock, std::chrono::duration<double>(wait));
  }
  stop = true;
  b->cv.notify_all();
  lock.unlock();
  for (auto &t : pool) t.join();
  return first_err;
}

mgpbd_status mgpbd_batch_get_state(mgpbd_batch_t *bb, int id, double *x, double *v) {
  Batch *b = reinterpret_cast<Batch *>(bb);
  if (!b || id < 0 || id >= (int)b->inst.size()) return MGPBD_E_INVALID;
  Instance &in = b->inst[id];
  if (in.h) MG_TRY(mgpbd_get_state(in.h, in.x.data(), in.v.data(), MGPBD_MEM_HOST));
  if (x) memcpy(x, in.x.data(), sizeof(double) * in.x.size());
  if (v) memcpy(v, in.v.data(), sizeof(double) * in.v.size());
  return MGPBD_OK;
}

mgpbd_status mgpbd_batch_resident(mgpbd_batch_t *bb, int *n_resident, size_t *bytes) {
  Batch *b = reinterpret_cast<Batch *>(bb);
  if (!b) return MGPBD_E_INVALID;
  int n = 0;
  for (Instance &in : b->inst) n += in.h != nullptr;
  if (n_resident) *n_resident = n;
  if (bytes) *bytes = b->resident;
  return MGPBD_OK;
}

void mgpbd_batch_destroy(mgpbd_batch_t *bb) {
  Batch *b = reinterpret_cast<Batch *>(bb);
  if (!b) return;
  for (Instance &in : b->inst) evict(in);
  delete b;
}

}  // extern "C"
