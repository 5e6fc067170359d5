// lise_serve.cu -- a request loop over one GPU (lise_server_* in include/lise.h).
//
// Each request is one independent TDSLDA evolution (parameters, initial state,
// number of ABM steps).  Two host threads share the device:
//   stepper  for every active request whose previous chunk of steps has finished
//            on the GPU (event query), enqueue the next chunk (lise_step on the
//            request's own stream); a request whose last chunk finished moves to
//            the retire list.  It never blocks on the device, so the GPU stays fed.
//   service  (kServiceThreads of them, so that the host-side copies of several
//            requests proceed in parallel) retires finished requests (copy the final state to the request's
//            host buffer, E and N, free the context: stream-ordered frees, no
//            device-wide synchronisation) and admits queued requests while the sum
//            of their device footprints (lise_footprint_bytes) stays within the
//            budget and fewer than max_active are in flight: create the context
//            and enqueue the H2D copy and the series-expansion start without
//            waiting for the device.
//            Order: arrival (FIFO), or first fit with a bound on how often one
//            request may be passed over.
// Work of different requests overlaps on the device through their streams;
// every request runs the same deterministic kernels on its own buffers, so its
// result does not depend on what else is in flight.
// With batching on (lise_server_set_batching), the stepper steps the active requests of
// each FP32 compute precision and lattice size together through one lise_batch (shared
// launches over a device work table), rebuilt whenever a request joins (its series start
// has finished on the device) or leaves (its steps are done); the others are stepped one
// by one.  Groups of different lattice sizes advance independently (their own streams and
// chunk queues), so that a rebuild of one group does not hold up the others.  A batch's
// members advance by the same number of steps per turn, so every chunk is bounded by the
// member with the fewest steps left.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/lise.h"
#include "lise_internal.h"

namespace {

struct Request {
  long id = 0;
  lise_params p{};
  std::vector<double> v_static;
  double* host = nullptr;  // input state, then the final state (owned copy)
  bool pinned = false;     // page-locked (cudaHostAlloc) rather than malloc
  bool borrowed = false;   // caller's buffers instead of an owned copy:
  const double* src = nullptr;  //   initial state, read at admission
  double* dst = nullptr;        //   final state (may be null), written at completion
  size_t bytes = 0;
  double t0 = 0, dt = 0;
  int n_steps = 0, done_steps = 0;
  size_t footprint = 0;
  lise_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  bool ev_pending = false;
  cudaEvent_t ready_ev = nullptr;  // the series start has finished (batch membership)
  bool batched = false;            // stepped through a batch
  int status = LISE_OK;
  enum State { QUEUED, ACTIVE, DONE } state = QUEUED;
  int skipped = 0;  // times a later request was admitted ahead of this one
  lise_request_info info{};
};

}  // namespace

// Requests stepped together (one group per batchable precision and lattice size).  Up to two
// chunks of steps are queued on the batch's stream, so that the device never waits for the
// stepper between chunks; membership changes once the queue has drained.
struct BatchGroup {
  int precision = 0, N = 0;
  std::vector<Request*> members;
  lise_batch* batch = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};  // end of each queued chunk (a ring)
  int head = 0, queued = 0;                // next event slot, chunks not yet seen complete
};

struct lise_server {
  int device = 0;
  bool batching = false;
  std::vector<BatchGroup> groups;  // by (precision, lattice size), created on first use
  size_t budget = 0;
  int max_active = 1;
  int steps_per_turn = 1;
  int policy = LISE_ADMIT_FIFO;
  int max_skips = 0;
  std::mutex mu;
  std::condition_variable cv_service, cv_done;
  std::deque<Request*> queue;
  std::vector<Request*> active;   // stepped by the stepper
  std::vector<Request*> retire;   // finished stepping (or failed), for the service thread
  int in_flight = 0;              // admitted and not yet retired
  std::map<long, Request*> all;
  size_t used = 0, peak_used = 0;
  int peak_active = 0;
  long next_id = 1;
  bool stop = false;
  std::thread stepper;
  std::vector<std::thread> service;
  std::chrono::steady_clock::time_point t0;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  void run_stepper();
  void step_loop();
  void run_service();
};

namespace {

constexpr int kServiceThreads = 4;

void release_host(Request* r) {
  if (!r->host) return;
  if (r->pinned)
    cudaFreeHost(r->host);
  else
    std::free(r->host);
  r->host = nullptr;
}

// Final state, E, N; free the context and the request's budget share.
void finish(lise_server* s, Request* r) {
  int status = r->status;
  if (r->ctx) {
    double* out = r->borrowed ? r->dst : r->host;
    if (status == LISE_OK && out) status = lise_get_state(r->ctx, out);
    if (status == LISE_OK && !out) status = lise_sync(r->ctx);
    double t = 0;
    lise_get_time(r->ctx, &t);
    r->info.t = t;
    if (status == LISE_OK) status = lise_energy(r->ctx, &r->info.E, &r->info.N);
    lise_destroy(r->ctx);
    r->ctx = nullptr;
  }
  if (r->ev) cudaEventDestroy(r->ev);
  if (r->ready_ev) cudaEventDestroy(r->ready_ev);
  r->ready_ev = nullptr;
  if (r->stream) cudaStreamDestroy(r->stream);
  r->ev = nullptr;
  r->stream = nullptr;
  std::lock_guard<std::mutex> lk(s->mu);
  r->info.status = status;
  r->info.done_s = s->now();
  r->state = Request::DONE;
  s->used -= r->footprint;
  --s->in_flight;
  s->cv_done.notify_all();
}

// Context, stream and series start of an admitted request (service thread).
int admit(Request* r) {
  int rc = cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking) == cudaSuccess ? LISE_OK : LISE_ECUDA;
  if (rc == LISE_OK && cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming) != cudaSuccess) rc = LISE_ECUDA;
  if (rc == LISE_OK) {
    r->p.stream = r->stream;
    r->p.v_static = r->v_static.empty() ? nullptr : r->v_static.data();
    rc = lise_create(&r->p, &r->ctx);
  }
  if (rc == LISE_OK) rc = lise_set_state_enqueue(r->ctx, r->borrowed ? r->src : r->host, r->t0, r->dt);
  if (rc == LISE_OK && cudaEventCreateWithFlags(&r->ready_ev, cudaEventDisableTiming) != cudaSuccess) rc = LISE_ECUDA;
  if (rc == LISE_OK && cudaEventRecord(r->ready_ev, r->stream) != cudaSuccess) rc = LISE_ECUDA;
  return rc;
}

bool batchable(const Request* r) {
  return (r->p.precision == LISE_MIXED || r->p.precision == LISE_MIXED_STRICT) && !r->p.remove_phase &&
         !r->p.renormalize;
}

}  // namespace

void lise_server::run_stepper() {
  for (;;) {
    try {
      step_loop();  // returns when the server stops
      return;
    } catch (...) {
      // host containers could not grow: fail the requests in flight (the service threads
      // retire them) and carry on with the next ones rather than end the process
      for (auto& G : groups) {
        if (G.batch) lise_batch_destroy(G.batch);
        G.batch = nullptr;
        G.members.clear();
        G.queued = 0;
      }
      std::lock_guard<std::mutex> lk(mu);
      for (Request* r : active) {
        r->status = LISE_ENOMEM;
        r->batched = false;
        retire.push_back(r);
      }
      active.clear();
      cv_service.notify_all();
    }
  }
}

void lise_server::step_loop() {
  cudaSetDevice(device);
  std::vector<Request*> act;
  auto to_retire = [&](Request* r) {
    std::lock_guard<std::mutex> lk(mu);
    active.erase(std::find(active.begin(), active.end(), r));
    retire.push_back(r);
    cv_service.notify_one();
  };
  for (;;) {
    bool batching_now;
    {
      std::lock_guard<std::mutex> lk(mu);
      if (stop && queue.empty() && in_flight == 0) {
        for (auto& G : groups) {
          if (G.batch) lise_batch_destroy(G.batch);
          for (auto& e : G.ev) {
            if (e) cudaEventDestroy(e);
            e = nullptr;
          }
          G.batch = nullptr;
        }
        return;
      }
      act = active;
      batching_now = batching;
    }
    bool progressed = false;
    // a group for every (precision, lattice size) of a batchable active request
    if (batching_now)
      for (Request* r : act)
        if (batchable(r) &&
            std::none_of(groups.begin(), groups.end(),
                         [&](const BatchGroup& G) { return G.precision == r->p.precision && G.N == r->p.nx; })) {
          groups.emplace_back();
          groups.back().precision = r->p.precision;
          groups.back().N = r->p.nx;
        }
    // batched requests: up to two chunks queued per group; membership changes between chunks
    for (size_t gi = 0; gi < groups.size() && batching_now; ++gi) {
      BatchGroup& G = groups[gi];
      while (G.queued > 0) {  // chunks that have finished, oldest first
        const int tail = (G.head - G.queued + 2) % 2;
        const cudaError_t q = cudaEventQuery(G.ev[tail]);
        if (q == cudaErrorNotReady) break;
        --G.queued;
        if (q != cudaSuccess)
          for (Request* r : G.members) r->status = LISE_ECUDA;
      }
      // leaving: finished (all steps enqueued) or failed members; joining: requests whose
      // series start is done.  (A fresh snapshot: a request retired above may already be gone.)
      {
        std::lock_guard<std::mutex> lk(mu);
        act = active;
      }
      std::vector<Request*> keep, joined;
      for (Request* r : G.members)
        if (r->status == LISE_OK && r->done_steps < r->n_steps) keep.push_back(r);
      for (Request* r : act)
        if (!r->batched && batchable(r) && r->p.precision == G.precision && r->p.nx == G.N && r->status == LISE_OK &&
            r->done_steps < r->n_steps && !r->ev_pending && cudaEventQuery(r->ready_ev) == cudaSuccess)
          joined.push_back(r);
      const bool changed = keep.size() != G.members.size() || !joined.empty();
      if (changed || (!G.batch && !keep.empty())) {
        if (G.queued > 0) continue;  // the queued chunks finish first
        if (G.batch) lise_batch_destroy(G.batch);
        G.batch = nullptr;
        for (Request* r : G.members)
          if (std::find(keep.begin(), keep.end(), r) == keep.end()) {
            r->batched = false;
            to_retire(r);
          }
        for (Request* r : joined) r->batched = true;
        keep.insert(keep.end(), joined.begin(), joined.end());
        G.members = keep;
        progressed = true;
        if (!G.members.empty()) {
          std::vector<lise_ctx*> cs;
          for (Request* r : G.members) cs.push_back(r->ctx);
          const int rc = lise_batch_create(cs.data(), (int)cs.size(), &G.batch);
          if (rc != LISE_OK) {
            for (Request* r : G.members) r->status = rc;
            continue;  // retired at the next turn
          }
          for (auto& e : G.ev)
            if (!e && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) e = nullptr;
        }
      }
      if (!G.batch || G.members.empty() || G.queued >= 2 || !G.ev[G.head]) continue;
      int k = steps_per_turn;
      for (Request* r : G.members) k = std::min(k, r->n_steps - r->done_steps);
      int rc = lise_batch_step(G.batch, k);
      if (rc == LISE_OK && cudaEventRecord(G.ev[G.head], (cudaStream_t)lise_batch_stream(G.batch)) != cudaSuccess)
        rc = LISE_ECUDA;
      if (rc != LISE_OK) {
        for (Request* r : G.members) r->status = rc;
      } else {
        for (Request* r : G.members) r->done_steps += k;
        G.head ^= 1;
        ++G.queued;
      }
      progressed = true;
    }
    // requests stepped one by one (a fresh snapshot: the batch groups above may have retired
    // some of the earlier one's requests, which must not be touched again)
    {
      std::lock_guard<std::mutex> lk(mu);
      act = active;
    }
    for (Request* r : act) {
      if (r->batched) continue;
      if (batching_now && batchable(r) && r->status == LISE_OK && r->done_steps < r->n_steps && !r->ev_pending)
        continue;  // waits for its series start, then joins its batch group
      if (batching_now && batchable(r) && r->status != LISE_OK) {
        to_retire(r);
        progressed = true;
        continue;
      }
      if (r->ev_pending) {
        const cudaError_t q = cudaEventQuery(r->ev);
        if (q == cudaErrorNotReady) continue;
        r->ev_pending = false;
        if (q != cudaSuccess) r->status = LISE_ECUDA;
      }
      bool last = r->status != LISE_OK || r->done_steps >= r->n_steps;
      if (!last) {
        const int k = std::min(steps_per_turn, r->n_steps - r->done_steps);
        int rc = lise_step(r->ctx, k, r->dt);
        if (rc == LISE_OK && cudaEventRecord(r->ev, r->stream) != cudaSuccess) rc = LISE_ECUDA;
        if (rc != LISE_OK) {
          r->status = rc;
          last = true;
        } else {
          r->done_steps += k;
          r->ev_pending = true;
        }
      }
      if (last) to_retire(r);
      progressed = true;
    }
    if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(100));
  }
}

void lise_server::run_service() {
  cudaSetDevice(device);
  for (;;) {
    Request* done = nullptr;
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(mu);
      auto pick_next = [&]() -> std::deque<Request*>::iterator {
        if (queue.empty() || in_flight >= max_active) return queue.end();
        for (auto it = queue.begin(); it != queue.end(); ++it) {
          if (used + (*it)->footprint <= budget) return it;
          // FIFO, or a request already passed over max_skips times: nothing later may go first
          if (policy == LISE_ADMIT_FIFO || (*it)->skipped >= max_skips) break;
        }
        return queue.end();
      };
      cv_service.wait_for(lk, std::chrono::milliseconds(50), [&] {
        return stop || !retire.empty() || pick_next() != queue.end();
      });
      if (stop && queue.empty() && in_flight == 0) {
        cv_service.notify_all();
        return;
      }
      if (!retire.empty()) {  // retirements first: they return budget
        done = retire.back();
        retire.pop_back();
      } else {
        auto it = pick_next();
        if (it != queue.end()) {
          for (auto jt = queue.begin(); jt != it; ++jt) ++(*jt)->skipped;
          r = *it;
          queue.erase(it);
          used += r->footprint;
          peak_used = std::max(peak_used, used);
          ++in_flight;
          peak_active = std::max(peak_active, in_flight);
          r->state = Request::ACTIVE;
          r->info.admit_s = now();
        }
      }
    }
    if (done) {
      finish(this, done);
      cv_service.notify_all();  // budget returned: another thread may admit
    }
    if (r) {
      r->status = admit(r);
      std::lock_guard<std::mutex> lk(mu);
      if (r->status == LISE_OK)
        active.push_back(r);
      else
        retire.push_back(r);
    }
  }
}

extern "C" {

int lise_server_create(int device, size_t hbm_budget_bytes, int max_active, int steps_per_turn, lise_server** out) {
  if (!out || max_active < 1 || steps_per_turn < 1 || hbm_budget_bytes == 0) return LISE_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return LISE_EINVAL;
  lise_server* s = new (std::nothrow) lise_server();
  if (!s) return LISE_ENOMEM;
  s->device = device;
  s->budget = hbm_budget_bytes;
  s->max_active = max_active;
  s->steps_per_turn = steps_per_turn;
  s->t0 = std::chrono::steady_clock::now();
  // keep freed context memory in the device's pool for the next requests (up to the budget)
  cudaMemPool_t pool;
  if (cudaSetDevice(device) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    unsigned long long keep = hbm_budget_bytes;  // the attribute is a 64-bit unsigned value
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  s->stepper = std::thread([s] { s->run_stepper(); });
  for (int k = 0; k < kServiceThreads; ++k) s->service.emplace_back([s] { s->run_service(); });
  *out = s;
  return LISE_OK;
}

namespace {
int submit_common(lise_server* s, const lise_params* p, const double* psi, double* psi_out, bool borrow, double t0,
                  double dt, int n_steps, long* id_out) {
  if (!s || !p || !psi || !id_out || n_steps < 0 || !(dt != 0.0)) return LISE_EINVAL;
  const size_t fp = lise_footprint_bytes(p);
  if (fp == 0) return LISE_EINVAL;
  if (fp > s->budget) return LISE_ENOMEM;  // could never be admitted
  Request* r = new (std::nothrow) Request();
  if (!r) return LISE_ENOMEM;
  r->p = *p;
  r->p.device = s->device;
  r->p.hbm_budget_bytes = 0;
  const long nxyz = (long)p->nx * p->ny * p->nz;
  if (p->v_static) r->v_static.assign(p->v_static, p->v_static + nxyz);
  r->bytes = (size_t)p->n_qp * 2 * nxyz * 2 * sizeof(double);
  if (borrow) {
    r->borrowed = true;
    r->src = psi;
    r->dst = psi_out;
  } else {
    // pageable host copy: page-locking multi-GB buffers (cudaHostAlloc) stalls the
    // other threads' CUDA calls for seconds, which costs more than the slower copies
    r->host = static_cast<double*>(std::malloc(r->bytes));
    if (!r->host) {
      delete r;
      return LISE_ENOMEM;
    }
    std::memcpy(r->host, psi, r->bytes);
  }
  r->t0 = t0;
  r->dt = dt;
  r->n_steps = n_steps;
  r->footprint = fp;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      release_host(r);
      delete r;
      return LISE_ESTATE;
    }
    r->id = s->next_id++;
    r->info.submit_s = s->now();
    s->queue.push_back(r);
    s->all[r->id] = r;
    *id_out = r->id;
  }
  s->cv_service.notify_one();
  return LISE_OK;
}
}  // namespace

int lise_server_submit(lise_server* s, const lise_params* p, const double* psi, double t0, double dt, int n_steps,
                       long* id_out) {
  return submit_common(s, p, psi, nullptr, false, t0, dt, n_steps, id_out);
}

int lise_server_submit_borrowed(lise_server* s, const lise_params* p, const double* psi_in, double* psi_out, double t0,
                                double dt, int n_steps, long* id_out) {
  return submit_common(s, p, psi_in, psi_out, true, t0, dt, n_steps, id_out);
}

int lise_server_wait(lise_server* s, long id, double* psi_out, lise_request_info* info) {
  if (!s) return LISE_EINVAL;
  Request* r = nullptr;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return LISE_EINVAL;
    r = it->second;
    s->cv_done.wait(lk, [&] { return r->state == Request::DONE; });
    s->all.erase(it);
  }
  if (psi_out && !r->borrowed && r->info.status == LISE_OK) std::memcpy(psi_out, r->host, r->bytes);
  if (info) *info = r->info;
  const int status = r->info.status;
  release_host(r);
  delete r;
  return status;
}

int lise_server_poll(lise_server* s, long id, int* done) {
  if (!s || !done) return LISE_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) return LISE_EINVAL;
  *done = it->second->state == Request::DONE ? 1 : 0;
  return LISE_OK;
}

int lise_server_set_admission(lise_server* s, int policy, int max_skips) {
  if (!s || (policy != LISE_ADMIT_FIFO && policy != LISE_ADMIT_FIRST_FIT) || max_skips < 0) return LISE_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->policy = policy;
    s->max_skips = max_skips;
  }
  s->cv_service.notify_one();
  return LISE_OK;
}

int lise_server_set_batching(lise_server* s, int enable) {
  if (!s) return LISE_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->next_id != 1) return LISE_ESTATE;  // only before the first submission
  s->batching = enable != 0;
  return LISE_OK;
}

int lise_server_stats(lise_server* s, size_t* peak_used_bytes, int* peak_active) {
  if (!s) return LISE_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (peak_used_bytes) *peak_used_bytes = s->peak_used;
  if (peak_active) *peak_active = s->peak_active;
  return LISE_OK;
}

void lise_server_destroy(lise_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_service.notify_all();
  if (s->stepper.joinable()) s->stepper.join();
  for (auto& t : s->service)
    if (t.joinable()) t.join();
  for (auto& kv : s->all) {
    release_host(kv.second);
    delete kv.second;
  }
  delete s;
}

}  // extern "C"
