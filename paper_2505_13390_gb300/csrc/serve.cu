// Continuous-batching service of many simulation instances on one GPU.
//
// The paper runs one instance at a time; this layer serves step requests
// (one request = `frames` frames of Alg. 1 for one instance) for many
// instances of different meshes, as a request loop: mgpbd_batch_admit
// submits a request at any time, also while others run, and
// mgpbd_batch_tick returns the requests that finished since the previous
// tick.  Instance state stays on the device between its requests while
// memory allows.  Admission is by a device-memory budget: an instance is
// made resident only if its bytes fit, after evicting idle resident
// instances (least recently used first; their positions and velocities go to
// host memory and come back when they are next admitted).  Up to
// `max_active` requests run at the same time, each on its instance's own
// CUDA stream driven by one of `max_active` worker threads, so their kernels
// overlap on the GPU.  A dispatcher runs under the batch lock whenever a
// request arrives or a worker finishes: it starts the earliest queued
// request whose instance is idle while a worker and memory are free.
// mgpbd_batch_run replays a list of timed requests through the same loop.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "cohort.cuh"
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
  bool busy = false;  // a worker steps it (or a state read holds it)
  double last_used = 0.0;
};

struct Req {
  int ticket, instance, frames;
  double arrival;  // seconds on the batch's clock
};

struct Batch {
  mgpbd_batch_config cfg{};
  int device = 0;
  std::chrono::steady_clock::time_point t0;  // the batch's clock starts at create
  // instances are held by pointer: adding one never moves another
  std::vector<std::unique_ptr<Instance>> inst;
  std::mutex mu;
  std::condition_variable cv_work;  // workers wait for jobs
  std::condition_variable cv_done;  // tick and state reads wait for results
  size_t resident = 0;  // bytes held by resident instances (reserved estimate while loading)
  int next_ticket = 0;
  std::deque<Req> queue;  // submitted, not started, in arrival order
  std::deque<Req> jobs;   // started, waiting for a worker
  int running = 0;        // requests in `jobs` or in a worker
  std::vector<mgpbd_step_result> finished;  // not yet returned by a tick
  bool stop = false;
  std::vector<std::thread> workers;
  // cohort mode: the stream of the batched launches (only the stepping thread
  // uses it; instances keep their own streams)
  cudaStream_t cohort_stream = nullptr;
  unsigned long long submitted = 0;  // requests submitted so far
  // cohort mode: rounds of the stepping thread, batched PCG iterations
  // launched, and the wall time spent in the batched chunks and in the
  // instances' own work between solves
  long long rounds = 0, batched_iters = 0;
  double chunk_s = 0.0, phase_s = 0.0;
  std::string last_err;  // text of the most recent failed request's error
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
  // float-float A.p: low parts of the gradients (incidence and row order),
  // alpha~ and w, u's low part, p as pairs
  if (p->ap_split) b += ninc * 12.0 + (double)E * 12.0 + (double)T * 48.0 + m * 12.0 + N * 40.0;
  const double nc = std::min(m, (double)std::max(p->coarse_max, 1));
  b += 24.0 * nc * nc;
  return (size_t)b;
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
  // served instances run beside each other: a cooperative coarse tail would
  // wait for every SM, so their V-cycles keep separate launches (the cohort
  // form has its own batched tail)
  if (s >= 0) s = mgpbd_set_coarse_tail(in.h, 0);
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

static double clock_s(const Batch *b) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - b->t0).count();
}

// a request that never ran (its instance can never fit)
static void fail_request(Batch *b, const Req &q, mgpbd_status s) {
  mgpbd_step_result r{};
  r.id = q.ticket;
  r.instance = q.instance;
  r.status = s;
  r.arrival_s = q.arrival;
  r.start_s = r.finish_s = clock_s(b);
  b->finished.push_back(r);
  b->cv_done.notify_all();
}

// Starts queued requests while a worker and memory are free (lock held).
// Queue order is arrival order; a request whose instance is busy waits, and
// so do the later requests of that instance, so each instance's requests run
// in submission order.
static void dispatch(Batch *b) {
  while (b->running < b->cfg.max_active) {
    auto it = b->queue.begin();
    for (; it != b->queue.end(); ++it)
      if (!b->inst[it->instance]->busy) break;
    if (it == b->queue.end()) return;
    const Req q = *it;
    Instance &in = *b->inst[q.instance];
    if (!in.h) {
      const size_t need = in.bytes ? in.bytes : in.est_bytes;
      if (need > b->cfg.hbm_budget) {  // can never fit: fail the request
        b->queue.erase(it);
        fail_request(b, q, MGPBD_E_BUDGET);
        continue;
      }
      mgpbd_status evict_err = MGPBD_OK;
      while (b->resident + need > b->cfg.hbm_budget) {
        int victim = -1;
        for (size_t i = 0; i < b->inst.size(); ++i) {
          const Instance &v = *b->inst[i];
          if (v.busy || !v.h || (int)i == q.instance) continue;
          if (victim < 0 || v.last_used < b->inst[victim]->last_used) victim = (int)i;
        }
        if (victim < 0) break;
        Instance &v = *b->inst[victim];
        mgpbd_status s = evict(v);
        if (s < 0) {  // still resident: its state could not be read back
          evict_err = s;
          break;
        }
        b->resident -= v.bytes;
        v.bytes = 0;
      }
      if (b->resident + need > b->cfg.hbm_budget) {
        if (b->running > 0) return;  // memory frees up when a request finishes
        b->queue.erase(it);          // nothing runs and nothing more can be evicted
        fail_request(b, q, evict_err < 0 ? evict_err : MGPBD_E_BUDGET);
        continue;
      }
      b->resident += need;  // reserved until the worker measures the real size
      in.bytes = need;
    }
    b->queue.erase(it);
    in.busy = true;
    ++b->running;
    b->jobs.push_back(q);
    b->cv_work.notify_one();
  }
}

static void worker(Batch *b) {
  cudaSetDevice(b->device);
  std::unique_lock<std::mutex> lock(b->mu);
  for (;;) {
    b->cv_work.wait(lock, [&] { return b->stop || !b->jobs.empty(); });
    if (b->jobs.empty()) return;  // stopping
    const Req q = b->jobs.front();
    b->jobs.pop_front();
    Instance &in = *b->inst[q.instance];
    lock.unlock();
    mgpbd_step_result r{};
    r.id = q.ticket;
    r.instance = q.instance;
    r.arrival_s = q.arrival;
    r.start_s = clock_s(b);
    mgpbd_status s = make_resident(in);
    if (s >= 0) s = run_request(in, q.frames, &r);
    size_t held = 0;
    if (in.h) {
      mgpbd_stats_t st{};
      mgpbd_stats(in.h, &st);
      held = st.device_bytes;
    }
    r.finish_s = clock_s(b);
    r.status = s;
    const std::string msg = s < 0 ? std::string(mgpbd_last_error()) : std::string();
    lock.lock();
    if (s < 0) b->last_err = "request " + std::to_string(q.ticket) + ": " + msg;
    b->resident = b->resident - in.bytes + held;  // the measured size replaces the estimate
    in.bytes = held;
    in.busy = false;
    in.last_used = r.finish_s;
    --b->running;
    b->finished.push_back(r);
    dispatch(b);
    b->cv_done.notify_all();
  }
}

// ---- cohort mode ------------------------------------------------------------
// One stepping thread runs every started request.  Each round it advances
// the requests that are between solves (frame prologue, C, A, setup or
// Galerkin re-form, coarsest factorisation, the solve's start) with their
// own launches on their own streams, then runs eight PCG iterations of every
// solving instance as one launch per step on the batch's cohort stream
// (which first waits for each member's start), then finishes the solves that
// have converged (true residual, position update, frame epilogue).  Only the
// stepping thread uses the cohort stream, so no other thread's work can fall
// into its graph capture.  Instances whose configuration the batched kernels
// do not cover solve alone, one global iteration per round.  An instance's
// arithmetic is its standalone solve's, bit for bit, whatever else runs.
struct CohortRun {
  Req q;
  Instance *in;
  mgpbd_step_result r;
  int frame = 0, it = 0;     // frame of the request and global iteration within it
  bool frame_open = false;   // begin_frame ran for `frame`
  bool solving = false;      // a batched solve is in progress
  bool due = false;          // the iteration set up afresh (breakdown retry rule)
  bool done = false;
  mgpbd_status worst = MGPBD_OK;
  cudaEvent_t started = nullptr;  // recorded after the solve's start
};

// counts one finished global iteration and closes the frame or the request
static void cohort_advance(CohortRun &c, const mgpbd_solve_info &inf, mgpbd_status st) {
  c.r.global_iters++;
  c.r.pcg_iters += inf.pcg_iters;
  if (st < 0) {
    c.worst = st;
    c.done = true;
    return;
  }
  c.worst = std::max(c.worst, st);
  c.it++;
  if (c.it >= c.in->p.max_iter || inf.bnorm < c.in->p.eps_b) {
    mgpbd_status e = mgpbd_end_frame(c.in->h);
    if (e < 0) {
      c.worst = e;
      c.done = true;
      return;
    }
    c.frame++;
    c.it = 0;
    c.frame_open = false;
    if (c.frame >= c.q.frames) c.done = true;
  }
}

// the part of a global iteration before its solve; starts a batched solve or
// runs the whole iteration alone
static void cohort_prepare(CohortRun &c) {
  Handle *h = reinterpret_cast<Handle *>(c.in->h);
  if (!c.frame_open) {
    mgpbd_status e = mgpbd_begin_frame(c.in->h);
    if (e < 0) {
      c.worst = e;
      c.done = true;
      return;
    }
    c.frame_open = true;
  }
  if (h->p.max_iter <= 0) {  // a frame without iterations
    cohort_advance(c, mgpbd_solve_info{}, MGPBD_OK);
    return;
  }
  if (h->p.linear_solver == 0) {
    mgpbd_status e = iterate_prepare(h, &c.due);
    if (e < 0) {
      c.r.global_iters++;
      c.worst = e;
      c.done = true;
      return;
    }
    if (cohort_eligible(h)) {
      e = h->m > 0 ? pcg_begin(h, h->b, h->dl) : MGPBD_OK;
      if (e < 0) {
        c.worst = e;
        c.done = true;
        return;
      }
      c.solving = true;
      return;
    }
    mgpbd_solve_info inf{}, info{};
    mgpbd_status st = pcg_solve(h, h->b, h->dl, &inf);
    st = iterate_complete(h, st, &inf, c.due, &info);
    cohort_advance(c, info, st);
    return;
  }
  mgpbd_solve_info info{};
  mgpbd_status st = mgpbd_iterate(c.in->h, &info);
  cohort_advance(c, info, st);
}

static void cohort_stepper(Batch *b) {
  cudaSetDevice(b->device);
  Cohort co;
  co.stream = b->cohort_stream;
  std::vector<CohortRun> runs;
  unsigned long long seen = 0;
  std::unique_lock<std::mutex> lock(b->mu);
  for (;;) {
    dispatch(b);
    seen = b->submitted;
    if (runs.empty() && b->jobs.empty()) {
      b->cv_work.wait(lock, [&] { return b->stop || !b->jobs.empty() || b->submitted != seen; });
      if (b->stop && b->jobs.empty()) return;
      continue;
    }
    std::vector<CohortRun> fresh;
    while (!b->jobs.empty()) {
      CohortRun c;
      c.q = b->jobs.front();
      b->jobs.pop_front();
      c.in = b->inst[c.q.instance].get();
      c.r = mgpbd_step_result{};
      c.r.id = c.q.ticket;
      c.r.instance = c.q.instance;
      c.r.arrival_s = c.q.arrival;
      c.r.start_s = clock_s(b);
      fresh.push_back(c);
    }
    lock.unlock();
    for (CohortRun &c : fresh) {
      mgpbd_status e = make_resident(*c.in);
      if (e >= 0 && cudaEventCreateWithFlags(&c.started, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        e = MGPBD_E_CUDA;
      }
      if (e < 0) {
        c.worst = e;
        c.done = true;
      }
      runs.push_back(c);
    }
    // requests between solves: the next global iteration up to its solve
    const double t_phase0 = clock_s(b);
    for (CohortRun &c : runs)
      if (!c.done && !c.solving) cohort_prepare(c);
    double t_chunk = 0.0;
    // the batched chunk over every instance that is solving
    std::vector<Handle *> members;
    for (CohortRun &c : runs)
      if (!c.done && c.solving) members.push_back(reinterpret_cast<Handle *>(c.in->h));
    if (!members.empty()) {
      mgpbd_status e = MGPBD_OK;
      if (members != co.hs || cohort_stale(&co)) {
        co.hs = members;
        e = cohort_build(&co);
      }
      // the chunk follows each member's own work (its solve's start)
      for (CohortRun &c : runs)
        if (e >= 0 && !c.done && c.solving &&
            (cudaEventRecord(c.started, c.in->stream) != cudaSuccess ||
             cudaStreamWaitEvent(b->cohort_stream, c.started, 0) != cudaSuccess))
          e = cuda_fail(cudaGetLastError(), "cohort: ordering a member's start", __FILE__,
                        __LINE__);
      const double t0 = clock_s(b);
      if (e >= 0) e = cohort_chunk(&co, 8);
      t_chunk = clock_s(b) - t0;
      for (CohortRun &c : runs) {
        if (c.done || !c.solving) continue;
        Handle *h = reinterpret_cast<Handle *>(c.in->h);
        if (e < 0) {
          c.worst = e;
          c.done = true;
          continue;
        }
        const int k = (int)(std::find(co.hs.begin(), co.hs.end(), h) - co.hs.begin());
        if (!co.h_sc[k].done) continue;
        c.solving = false;
        mgpbd_solve_info inf{}, info{};
        mgpbd_status st = pcg_finish(h, h->b, h->dl, &inf);
        st = iterate_complete(h, st, &inf, c.due, &info);
        cohort_advance(c, info, st);
      }
    }
    const double t_round = clock_s(b) - t_phase0;
    // finished requests leave
    std::vector<CohortRun> left;
    std::vector<std::pair<CohortRun, size_t>> fin;
    for (CohortRun &c : runs) {
      if (!c.done) {
        left.push_back(c);
        continue;
      }
      size_t held = 0;
      if (c.in->h) {
        mgpbd_stats_t st{};
        mgpbd_stats(c.in->h, &st);
        held = st.device_bytes;
      }
      if (c.started) cudaEventDestroy(c.started);
      c.r.finish_s = clock_s(b);
      c.r.status = c.worst;
      if (c.worst < 0) {
        std::lock_guard<std::mutex> g(b->mu);
        b->last_err = "request " + std::to_string(c.q.ticket) + ": " + mgpbd_last_error();
      }
      fin.emplace_back(c, held);
    }
    runs.swap(left);
    if (runs.empty()) co.hs.clear();  // no member holds a handle that may be evicted
    lock.lock();
    b->rounds++;
    if (!members.empty()) b->batched_iters += 8;
    b->chunk_s += t_chunk;
    b->phase_s += t_round - t_chunk;
    for (auto &f : fin) {
      Instance &in = *f.first.in;
      b->resident = b->resident - in.bytes + f.second;
      in.bytes = f.second;
      in.busy = false;
      in.last_used = f.first.r.finish_s;
      --b->running;
      b->finished.push_back(f.first.r);
    }
    if (!fin.empty()) b->cv_done.notify_all();
  }
}

// Moves up to `max` finished results that `want` accepts into `out`, in
// finishing order, waiting up to wait_s seconds for the first one (lock held
// by the caller through `lock`).
template <class Pred>
static int take_results(Batch *b, std::unique_lock<std::mutex> &lock, double wait_s,
                        mgpbd_step_result *out, int max, Pred want) {
  auto any = [&] {
    for (const auto &r : b->finished)
      if (want(r)) return true;
    return false;
  };
  if (wait_s > 0 && !any())
    b->cv_done.wait_for(lock, std::chrono::duration<double>(wait_s), any);
  int k = 0;
  for (auto it = b->finished.begin(); it != b->finished.end() && k < max;) {
    if (want(*it)) {
      out[k++] = *it;
      it = b->finished.erase(it);
    } else {
      ++it;
    }
  }
  return k;
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
  if (!cfg || !out || cfg->max_active < 1 || cfg->max_active > 256 || cfg->hbm_budget == 0 ||
      (cfg->cohort != 0 && cfg->cohort != 1) || (cfg->cohort && cfg->max_active > kCohortMax)) {
    set_error("mgpbd_batch_create: invalid configuration");
    return MGPBD_E_INVALID;
  }
  *out = nullptr;
  num_sms();  // query once before worker threads exist
  Batch *b = new Batch();
  b->cfg = *cfg;
  b->t0 = std::chrono::steady_clock::now();
  if (cudaGetDevice(&b->device) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    set_error("mgpbd_batch_create: cudaGetDevice failed");
    return MGPBD_E_CUDA;
  }
  if (cfg->cohort) {
    if (cudaStreamCreateWithFlags(&b->cohort_stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete b;
      set_error("mgpbd_batch_create: cudaStreamCreate failed");
      return MGPBD_E_CUDA;
    }
    b->workers.emplace_back(cohort_stepper, b);
  } else {
    for (int t = 0; t < cfg->max_active; ++t) b->workers.emplace_back(worker, b);
  }
  *out = reinterpret_cast<mgpbd_batch_t *>(b);
  return MGPBD_OK;
}

mgpbd_status mgpbd_batch_add_instance(mgpbd_batch_t *bb, const mgpbd_mesh_desc *md,
                                      const mgpbd_params *p, const double *x0, const double *v0,
                                      int *id) {
  Batch *b = reinterpret_cast<Batch *>(bb);
  if (!b || !md || !p || !id || md->n_verts <= 0 || md->n_dist < 0 || md->n_tet < 0 ||
      !md->rest_pos || !md->inv_mass || (md->n_dist > 0 && !md->dist) ||
      (md->n_tet > 0 && !md->tet) || (md->n_dist + md->n_tet > 0 && !md->alpha)) {
    set_error("mgpbd_batch_add_instance: invalid argument");
    return MGPBD_E_INVALID;
  }
  size_t est = 0;
  MG_TRY(mgpbd_workspace_size(md, p, &est));  // also range-checks the indices
  auto in = std::make_unique<Instance>();
  const int N = md->n_verts, E = md->n_dist, T = md->n_tet;
  in->rest.assign(md->rest_pos, md->rest_pos + 3 * (size_t)N);
  in->w.assign(md->inv_mass, md->inv_mass + (size_t)N);
  if (E) in->dist.assign(md->dist, md->dist + 2 * (size_t)E);
  if (T) in->tet.assign(md->tet, md->tet + 4 * (size_t)T);
  if (E + T) in->alpha.assign(md->alpha, md->alpha + (size_t)E + T);
  in->x.assign(x0 ? x0 : md->rest_pos, (x0 ? x0 : md->rest_pos) + 3 * (size_t)N);
  in->v.assign(3 * (size_t)N, 0.0);
  if (v0) in->v.assign(v0, v0 + 3 * (size_t)N);
  in->p = *p;
  in->desc.n_verts = N;
  in->desc.rest_pos = in->rest.data();
  in->desc.inv_mass = in->w.data();
  in->desc.n_dist = E;
  in->desc.dist = E ? in->dist.data() : nullptr;
  in->desc.n_tet = T;
  in->desc.tet = T ? in->tet.data() : nullptr;
  in->desc.alpha = (E + T) ? in->alpha.data() : nullptr;
  in->desc.tet_kind = md->tet_kind;
  in->est_bytes = est;
  std::lock_guard<std::mutex> lock(b->mu);
  b->inst.push_back(std::move(in));
  *id = (int)b->inst.size() - 1;
  return MGPBD_OK;
}

mgpbd_status mgpbd_batch_admit(mgpbd_batch_t *bb, int instance, int frames, int *ticket) {
  Batch *b = reinterpret_cast<Batch *>(bb);
  if (!b || !ticket || frames < 1) {
    set_error("mgpbd_batch_admit: invalid argument");
    return MGPBD_E_INVALID;
  }
  std::lock_guard<std::mutex> lock(b->mu);
  if (instance < 0 || instance >= (int)b->inst.size()) {
    set_error("mgpbd_batch_admit: unknown instance");
    return MGPBD_E_INVALID;
  }
  Req q{b->next_ticket++, instance, frames, clock_s(b)};
  b->queue.push_back(q);
  *ticket = q.ticket;
  b->submitted++;
  dispatch(b);
  b->cv_work.notify_all();
  return MGPBD_OK;
}

mgpbd_status mgpbd_batch_tick(mgpbd_batch_t *bb, double wait_s, mgpbd_step_result *res, int max,
                              int *n) {
  Batch *b = reinterpret_cast<Batch *>(bb);
  if (!b || !n || max < 0 || (max > 0 && !res) || !(wait_s >= 0.0)) {
    set_error("mgpbd_batch_tick: invalid argument");
    return MGPBD_E_INVALID;
  }
  std::unique_lock<std::mutex> lock(b->mu);
  *n = take_results(b, lock, max > 0 ? wait_s : 0.0, res, max,
                    [](const mgpbd_step_result &) { return true; });
  return MGPBD_OK;
}

mgpbd_status mgpbd_batch_counts(mgpbd_batch_t *bb, int *queued, int *running, int *unreported,
                                double *clock) {
  Batch *b = reinterpret_cast<Batch *>(bb);
  if (!b) return MGPBD_E_INVALID;
  std::lock_guard<std::mutex> lock(b->mu);
  if (queued) *queued = (int)b->queue.size();
  if (running) *running = b->running;
  if (unreported) *unreported = (int)b->finished.size();
  if (clock) *clock = clock_s(b);
  return MGPBD_OK;
}

const char *mgpbd_batch_error(mgpbd_batch_t *bb) {
  Batch *b = reinterpret_cast<Batch *>(bb);
  if (!b) return "";
  thread_local std::string copy;
  std::lock_guard<std::mutex> lock(b->mu);
  copy = b->last_err;
  return copy.c_str();
}

mgpbd_status mgpbd_batch_cohort_stats(mgpbd_batch_t *bb, int64_t *rounds, int64_t *batched_iters,
                                      double *chunk_s, double *other_s) {
  Batch *b = reinterpret_cast<Batch *>(bb);
  if (!b) return MGPBD_E_INVALID;
  std::lock_guard<std::mutex> lock(b->mu);
  if (rounds) *rounds = b->rounds;
  if (batched_iters) *batched_iters = b->batched_iters;
  if (chunk_s) *chunk_s = b->chunk_s;
  if (other_s) *other_s = b->phase_s;
  return MGPBD_OK;
}

mgpbd_status mgpbd_batch_run(mgpbd_batch_t *bb, const mgpbd_step_request *req, int n_req,
                             mgpbd_step_result *res) {
  Batch *b = reinterpret_cast<Batch *>(bb);
  if (!b || n_req < 0 || (n_req && (!req || !res))) return MGPBD_E_INVALID;
  {
    std::lock_guard<std::mutex> lock(b->mu);
    for (int i = 0; i < n_req; ++i)
      if (req[i].instance < 0 || req[i].instance >= (int)b->inst.size() || req[i].frames < 1) {
        set_error("mgpbd_batch_run: request names an unknown instance or no frames");
        return MGPBD_E_INVALID;
      }
  }
  std::vector<int> order((size_t)n_req);
  for (int i = 0; i < n_req; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int c) { return req[a].arrival_s < req[c].arrival_s; });
  std::unordered_map<int, int> index;  // ticket -> request
  const double t_run = clock_s(b);
  int next = 0, got = 0;
  mgpbd_status first_err = MGPBD_OK;
  std::vector<mgpbd_step_result> buf(64);
  while (got < n_req) {
    while (next < n_req && req[order[next]].arrival_s <= clock_s(b) - t_run) {
      const int k = order[next++];
      int ticket = -1;
      MG_TRY(mgpbd_batch_admit(bb, req[k].instance, req[k].frames, &ticket));
      index[ticket] = k;
    }
    double wait = 0.05;
    if (next < n_req)
      wait = std::min(wait, std::max(0.0, req[order[next]].arrival_s - (clock_s(b) - t_run)));
    int n = 0;
    {
      std::unique_lock<std::mutex> lock(b->mu);
      n = take_results(b, lock, wait, buf.data(), (int)buf.size(),
                       [&](const mgpbd_step_result &r) { return index.count(r.id) != 0; });
    }
    for (int j = 0; j < n; ++j) {
      const int k = index[buf[j].id];
      mgpbd_step_result r = buf[j];
      r.id = req[k].id;
      r.arrival_s -= t_run;
      r.start_s -= t_run;
      r.finish_s -= t_run;
      res[k] = r;
      if (r.status < 0 && first_err >= 0) first_err = r.status;
      ++got;
    }
  }
  return first_err;
}

mgpbd_status mgpbd_batch_get_state(mgpbd_batch_t *bb, int id, double *x, double *v) {
  Batch *b = reinterpret_cast<Batch *>(bb);
  if (!b) return MGPBD_E_INVALID;
  std::unique_lock<std::mutex> lock(b->mu);
  if (id < 0 || id >= (int)b->inst.size()) return MGPBD_E_INVALID;
  Instance &in = *b->inst[id];
  b->cv_done.wait(lock, [&] { return !in.busy; });  // not while a worker steps it
  in.busy = true;
  lock.unlock();
  mgpbd_status s = MGPBD_OK;
  if (in.h) s = mgpbd_get_state(in.h, in.x.data(), in.v.data(), MGPBD_MEM_HOST);
  if (s >= 0) {
    if (x) memcpy(x, in.x.data(), sizeof(double) * in.x.size());
    if (v) memcpy(v, in.v.data(), sizeof(double) * in.v.size());
  }
  lock.lock();
  in.busy = false;
  dispatch(b);
  b->cv_done.notify_all();
  return s;
}

mgpbd_status mgpbd_batch_resident(mgpbd_batch_t *bb, int *n_resident, size_t *bytes) {
  Batch *b = reinterpret_cast<Batch *>(bb);
  if (!b) return MGPBD_E_INVALID;
  std::lock_guard<std::mutex> lock(b->mu);
  int n = 0;
  for (auto &in : b->inst) n += in->h != nullptr;
  if (n_resident) *n_resident = n;
  if (bytes) *bytes = b->resident;
  return MGPBD_OK;
}

void mgpbd_batch_destroy(mgpbd_batch_t *bb) {
  Batch *b = reinterpret_cast<Batch *>(bb);
  if (!b) return;
  {
    std::lock_guard<std::mutex> lock(b->mu);
    b->stop = true;
    b->queue.clear();  // requests that have not started are dropped
  }
  b->cv_work.notify_all();
  for (auto &t : b->workers) t.join();  // workers finish the jobs they hold first
  for (auto &in : b->inst) {
    evict(*in);
    drop_handle(*in);
  }
  if (b->cohort_stream) cudaStreamDestroy(b->cohort_stream);
  delete b;
}

}  // extern "C"
