// lise_serve.cu -- a request loop over one GPU (lise_server_* in include/lise.h).
//
// Each request is one independent TDSLDA evolution (parameters, initial state,
// number of ABM steps).  A worker thread owns the device and repeats:
//   1. for every active request whose previous chunk of steps has finished on
//      the GPU, enqueue the next chunk (lise_step on the request's own stream);
//   2. retire requests whose last chunk has finished: copy the final state to
//      the request's host buffer, compute E and N, free its context (its HBM
//      budget share returns to the pool);
//   3. admit queued requests in arrival order while the sum of their device
//      footprints (lise_footprint_bytes) stays within the budget and fewer than
//      max_active are active: create the context and run lise_set_state (the
//      H2D copy and the series-expansion start).  Step chunks already enqueued
//      for other requests keep the GPU busy meanwhile.
// Work of different requests overlaps on the device through their streams;
// every request runs the same deterministic kernels on its own buffers, so its
// result does not depend on what else is in flight.
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

namespace {

struct Request {
  long id = 0;
  lise_params p{};
  std::vector<double> v_static;
  double* host = nullptr;  // input state, then the final state
  size_t bytes = 0;
  double t0 = 0, dt = 0;
  int n_steps = 0, done_steps = 0;
  size_t footprint = 0;
  lise_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  bool ev_pending = false;
  enum State { QUEUED, ACTIVE, DONE } state = QUEUED;
  lise_request_info info{};
};

}  // namespace

struct lise_server {
  int device = 0;
  size_t budget = 0;
  int max_active = 1;
  int steps_per_turn = 1;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::vector<Request*> active;
  std::map<long, Request*> all;
  size_t used = 0, peak_used = 0;
  int peak_active = 0;
  long next_id = 1;
  bool stop = false;
  std::thread worker;
  std::chrono::steady_clock::time_point t0;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  void run();
};

namespace {

void finish(lise_server* s, Request* r, int status) {
  if (r->ctx) {
    if (status == LISE_OK) status = lise_get_state(r->ctx, r->host);
    double t = 0;
    lise_get_time(r->ctx, &t);
    r->info.t = t;
    if (status == LISE_OK) status = lise_energy(r->ctx, &r->info.E, &r->info.N);
    lise_destroy(r->ctx);
    r->ctx = nullptr;
  }
  if (r->ev) cudaEventDestroy(r->ev);
  if (r->stream) cudaStreamDestroy(r->stream);
  r->ev = nullptr;
  r->stream = nullptr;
  std::lock_guard<std::mutex> lk(s->mu);
  r->info.status = status;
  r->info.done_s = s->now();
  r->state = Request::DONE;
  s->used -= r->footprint;
  for (size_t i = 0; i < s->active.size(); ++i)
    if (s->active[i] == r) {
      s->active.erase(s->active.begin() + i);
      break;
    }
  s->cv_done.notify_all();
}

}  // namespace

void lise_server::run() {
  cudaSetDevice(device);
  for (;;) {
    std::vector<Request*> act;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_work.wait(lk, [&] { return stop || !queue.empty() || !active.empty(); });
      if (stop && queue.empty() && active.empty()) return;
      act = active;
    }
    bool progressed = false;
    // 1-2: enqueue the next chunk of every request whose last chunk finished; retire finished ones
    for (Request* r : act) {
      if (r->ev_pending) {
        cudaError_t q = cudaEventQuery(r->ev);
        if (q == cudaErrorNotReady) continue;
        r->ev_pending = false;
        if (q != cudaSuccess) {
          finish(this, r, LISE_ECUDA);
          progressed = true;
          continue;
        }
      }
      if (r->done_steps >= r->n_steps) {
        finish(this, r, lise_sync(r->ctx));
        progressed = true;
        continue;
      }
      const int k = std::min(steps_per_turn, r->n_steps - r->done_steps);
      int rc = lise_step(r->ctx, k, r->dt);
      if (rc == LISE_OK && cudaEventRecord(r->ev, r->stream) != cudaSuccess) rc = LISE_ECUDA;
      if (rc != LISE_OK) {
        finish(this, r, rc);
      } else {
        r->done_steps += k;
        r->ev_pending = true;
      }
      progressed = true;
    }
    // 3: admission in arrival order under the budget
    for (;;) {
      Request* r = nullptr;
      {
        std::lock_guard<std::mutex> lk(mu);
        if (queue.empty() || (int)active.size() >= max_active || used + queue.front()->footprint > budget) break;
        r = queue.front();
        queue.pop_front();
        used += r->footprint;
        if (used > peak_used) peak_used = used;
        r->state = Request::ACTIVE;
        r->info.admit_s = now();
      }
      int rc = cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking) == cudaSuccess ? LISE_OK : LISE_ECUDA;
      if (rc == LISE_OK && cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming) != cudaSuccess) rc = LISE_ECUDA;
      if (rc == LISE_OK) {
        r->p.stream = r->stream;
        r->p.v_static = r->v_static.empty() ? nullptr : r->v_static.data();
        rc = lise_create(&r->p, &r->ctx);
      }
      if (rc == LISE_OK) rc = lise_set_state(r->ctx, r->host, r->t0, r->dt);
      {
        std::lock_guard<std::mutex> lk(mu);
        active.push_back(r);
        if ((int)active.size() > peak_active) peak_active = (int)active.size();
      }
      if (rc != LISE_OK) finish(this, r, rc);
      progressed = true;
    }
    if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(200));
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
  s->worker = std::thread([s] { s->run(); });
  *out = s;
  return LISE_OK;
}

int lise_server_submit(lise_server* s, const lise_params* p, const double* psi, double t0, double dt, int n_steps,
                       long* id_out) {
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
  r->host = static_cast<double*>(std::malloc(r->bytes));
  if (!r->host) {
    delete r;
    return LISE_ENOMEM;
  }
  std::memcpy(r->host, psi, r->bytes);
  r->t0 = t0;
  r->dt = dt;
  r->n_steps = n_steps;
  r->footprint = fp;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      std::free(r->host);
      delete r;
      return LISE_ESTATE;
    }
    r->id = s->next_id++;
    r->info.submit_s = s->now();
    s->queue.push_back(r);
    s->all[r->id] = r;
    *id_out = r->id;
  }
  s->cv_work.notify_one();
  return LISE_OK;
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
  if (psi_out && r->info.status == LISE_OK) std::memcpy(psi_out, r->host, r->bytes);
  if (info) *info = r->info;
  const int status = r->info.status;
  std::free(r->host);
  delete r;
  return status;
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
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto& kv : s->all) {
    std::free(kv.second->host);
    delete kv.second;
  }
  delete s;
}

}  // extern "C"
