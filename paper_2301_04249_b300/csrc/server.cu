// Continuous-batching server for independent core-hole propagations.
//
// Core holes are independent ("unique and can run simultaneously", Section 3),
// so the server runs many propagations at once on one GPU.  A scheduler thread
// admits queued requests (first come, first served) while a slot is free and
// their estimated device memory fits the budget; each admitted request gets its
// own context and stream, and the thread advances every running request with
// non-blocking polls, so work of different requests overlaps on the device and
// requests that arrive later join as soon as slots and memory free up.  A
// request that fails (bad input, non-convergence) is isolated: its context is
// destroyed and the others continue.  Results (C_0..C_n) stay on the device
// until the request completes and are then copied to host memory owned by the
// server until the caller reads them.  Requests with RTEOM_FLAG_GROUPED
// advance together: in each pass those that are ready (their previous
// micro-iteration finished) run one residual each with their ladder GEMMs in
// grouped persistent launches, so uneven requests share launches without
// waiting on one another.
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/rteom.h"
#include "common.cuh"

int rteom_internal_begin(rteom_ctx* c, int nsteps, double dt, double tol, int max_micro);
int rteom_internal_poll(rteom_ctx* c, bool* finished, int* waiting);
void rteom_internal_group_poll(rteom_ctx* const* cs, int n, int* rc, bool* done,
                               bool* progressed);
double rteom_internal_device_bytes(const rteom_ctx* c);

namespace {

using Clock = std::chrono::steady_clock;

double seconds_since(Clock::time_point t0) {
  return std::chrono::duration<double>(Clock::now() - t0).count();
}

// Host copies of one molecule's inputs, shared by the requests of a sweep
// over core holes and dropped once the last of them has built its context.
struct Inputs {
  std::vector<double> eps, L, t1, t2;
  bool has_t1 = false, has_t2 = false;
};

struct Request {
  long long id = 0;
  int O = 0, V = 0, nchol = 0, core = 0, flags = 0;
  std::shared_ptr<const Inputs> in;
  int nsteps = 0, max_micro = 1;
  double dt = 0.0, tol = 0.0;
  int status = RTEOM_REQ_QUEUED;
  int error = RTEOM_OK;
  std::string msg;
  rteom_ctx* ctx = nullptr;
  std::vector<double> C;
  double estimate = 0.0, charged = 0.0;
  double t_submit = 0.0, t_admit = -1.0, t_done = -1.0;
  bool cancel = false;
};

// Device bytes a context of this shape needs at its peak (set-up and the
// first residual, every constant tensor-core pack cached), from the host
// dry-run plan of rteom_plan_bytes, with 5 % and 256 MB of margin.  Whole
// bytes, so the admission ledger (doubles, all below 2^53) sums exactly and
// returns to zero when the last request leaves.
double estimate_bytes(int O, int V, int nchol, int precision, int flags = 0) {
  double b[3] = {0.0, 0.0, 0.0};
  if (rteom_plan_bytes(O, V, nchol, precision,
                       flags & (RTEOM_FLAG_LADDER_CHOLESKY | RTEOM_FLAG_ANDERSON |
                                RTEOM_FLAG_GROUPED), b) != RTEOM_OK)
    return 0.0;
  return std::ceil(1.05 * b[0]) + 256.0 * 1024 * 1024;
}

}  // namespace

struct rteom_server {
  int device = 0, precision = RTEOM_FP64, max_active = 1;
  double budget = 0.0, in_use = 0.0;
  Clock::time_point t0 = Clock::now();
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  std::deque<Request*> queue;
  std::vector<Request*> active;
  std::map<long long, std::unique_ptr<Request>> all;
  long long next_id = 1;
  long long n_done = 0, n_failed = 0;
  double steps_done = 0.0;
  std::string err;
  std::thread worker;

  void finish(Request* r, int status, int error, const std::string& msg) {
    // called by the worker without the lock held
    if (r->ctx) {
      if (status == RTEOM_REQ_DONE) {
        r->C.assign(2 * (size_t)(r->nsteps + 1), 0.0);
        int rc = rteom_get_cumulant(r->ctx, r->nsteps + 1, r->C.data(), nullptr);
        if (rc != RTEOM_OK) {
          status = RTEOM_REQ_FAILED;
          error = rc;
        }
      }
      rteom_destroy(r->ctx);
      r->ctx = nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    r->status = status;
    r->error = error;
    r->msg = msg;
    r->t_done = seconds_since(t0);
    in_use -= r->charged;
    r->charged = 0.0;
    if (status == RTEOM_REQ_DONE) {
      ++n_done;
      steps_done += r->nsteps;
    } else if (status == RTEOM_REQ_FAILED) {
      ++n_failed;
    }
    r->in.reset();  // a cancelled or failed request may still hold its inputs
    cv_done.notify_all();
  }

  void loop() {
    cudaSetDevice(device);
    std::vector<Request*> admitting;
    while (true) {
      admitting.clear();
      {
        std::unique_lock<std::mutex> lock(mu);
        if (active.empty() && queue.empty()) {
          if (stop) break;
          cv_work.wait(lock, [&] { return stop || !queue.empty(); });
          if (stop && queue.empty()) break;
        }
        while (!queue.empty() && (int)(active.size() + admitting.size()) < max_active) {
          Request* r = queue.front();
          if (r->cancel) {
            queue.pop_front();
            r->status = RTEOM_REQ_CANCELLED;
            r->t_done = seconds_since(t0);
            r->in.reset();
            cv_done.notify_all();
            continue;
          }
          // memory admission; a lone request is always tried (it may fail OOM)
          if (in_use + r->estimate > budget && !(active.empty() && admitting.empty())) break;
          queue.pop_front();
          r->charged = r->estimate;
          in_use += r->charged;
          r->status = RTEOM_REQ_RUNNING;
          r->t_admit = seconds_since(t0);
          admitting.push_back(r);
        }
      }
      for (Request* r : admitting) {
        const Inputs& in = *r->in;
        int rc = rteom_create(&r->ctx, r->O, r->V, r->nchol, in.eps.data(),
                              r->nchol ? in.L.data() : nullptr, in.has_t1 ? in.t1.data() : nullptr,
                              in.has_t2 ? in.t2.data() : nullptr, r->core, precision, r->flags,
                              nullptr);
        r->in.reset();  // the context holds its own device copies now
        if (rc != RTEOM_OK) {
          finish(r, RTEOM_REQ_FAILED, rc, rteom_last_error(nullptr));
          continue;
        }
        {
          // charge what the context really holds
          std::lock_guard<std::mutex> lock(mu);
          const double real = rteom_internal_device_bytes(r->ctx);
          in_use += real - r->charged;
          r->charged = real;
        }
        rc = rteom_internal_begin(r->ctx, r->nsteps, r->dt, r->tol, r->max_micro);
        if (rc != RTEOM_OK) {
          finish(r, RTEOM_REQ_FAILED, rc, rteom_last_error(r->ctx));
          continue;
        }
        std::lock_guard<std::mutex> lock(mu);
        active.push_back(r);
      }
      // advance every running request once, without blocking; requests with
      // RTEOM_FLAG_GROUPED advance together, the ladder GEMMs of those ready
      // in one grouped launch per round
      bool progressed = false;
      std::vector<Request*> snapshot, grouped;
      {
        std::lock_guard<std::mutex> lock(mu);
        snapshot = active;
      }
      auto retire = [&](Request* r, int status, int error, const std::string& msg) {
        {
          std::lock_guard<std::mutex> lock(mu);
          for (size_t k = 0; k < active.size(); ++k)
            if (active[k] == r) {
              active.erase(active.begin() + k);
              break;
            }
        }
        finish(r, status, error, msg);
        progressed = true;
      };
      for (Request* r : snapshot) {
        bool cancel;
        {
          std::lock_guard<std::mutex> lock(mu);
          cancel = r->cancel;
        }
        if (cancel) {
          retire(r, RTEOM_REQ_CANCELLED, RTEOM_OK, std::string());
          continue;
        }
        if (r->flags & RTEOM_FLAG_GROUPED) {
          grouped.push_back(r);
          continue;
        }
        bool fin = false;
        int waiting = 0;
        int rc = rteom_internal_poll(r->ctx, &fin, &waiting);
        progressed |= !waiting;
        if (rc != RTEOM_OK)
          retire(r, RTEOM_REQ_FAILED, rc, rteom_last_error(r->ctx));
        else if (fin)
          retire(r, RTEOM_REQ_DONE, RTEOM_OK, std::string());
      }
      if (!grouped.empty()) {
        const int n = (int)grouped.size();
        std::vector<rteom_ctx*> cs(n);
        std::vector<int> rcs(n, RTEOM_OK);
        std::unique_ptr<bool[]> fin(new bool[n]);
        for (int k = 0; k < n; ++k) cs[k] = grouped[k]->ctx;
        rteom_internal_group_poll(cs.data(), n, rcs.data(), fin.get(), &progressed);
        for (int k = 0; k < n; ++k) {
          if (rcs[k] != RTEOM_OK)
            retire(grouped[k], RTEOM_REQ_FAILED, rcs[k], rteom_last_error(grouped[k]->ctx));
          else if (fin[k])
            retire(grouped[k], RTEOM_REQ_DONE, RTEOM_OK, std::string());
        }
      }
      if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
  }
};

namespace {

std::shared_ptr<const Inputs> copy_inputs(int nocc, int nvir, int nchol, const double* eps,
                                          const double* L, const double* t1_gs,
                                          const double* t2_gs) {
  auto in = std::make_shared<Inputs>();
  const size_t nb = (size_t)nocc + nvir;
  in->eps.assign(eps, eps + nb);
  if (nchol) in->L.assign(L, L + (size_t)nchol * nb * nb);
  if (t1_gs) {
    in->t1.assign(t1_gs, t1_gs + (size_t)nocc * nvir);
    in->has_t1 = true;
  }
  if (t2_gs) {
    in->t2.assign(t2_gs, t2_gs + (size_t)nocc * nocc * nvir * nvir);
    in->has_t2 = true;
  }
  return in;
}

bool bad_request(const rteom_server* s, int nocc, int nvir, int nchol, const double* eps,
                 const double* L, int nsteps, double dt, double tol, int max_micro) {
  return !s || !eps || nocc < 1 || nvir < 1 || nchol < 0 || (nchol > 0 && !L) || nsteps < 0 ||
         !(dt > 0) || !(tol > 0) || max_micro < 1;
}

// Queue requests for the given core holes, all sharing one input copy.
void enqueue(rteom_server* s, int nocc, int nvir, int nchol, std::shared_ptr<const Inputs> in,
             const int* cores, int ncores, int flags, int nsteps, double dt, double tol,
             int max_micro, long long* ids) {
  const double est = estimate_bytes(nocc, nvir, nchol, s->precision, flags);
  std::vector<std::unique_ptr<Request>> rs;
  for (int k = 0; k < ncores; ++k) {
    std::unique_ptr<Request> r(new Request());
    r->O = nocc;
    r->V = nvir;
    r->nchol = nchol;
    r->core = cores[k];
    r->flags = flags;
    r->in = in;
    r->nsteps = nsteps;
    r->dt = dt;
    r->tol = tol;
    r->max_micro = max_micro;
    r->estimate = est;
    rs.push_back(std::move(r));
  }
  std::lock_guard<std::mutex> lock(s->mu);
  for (int k = 0; k < ncores; ++k) {
    Request* r = rs[k].get();
    r->id = s->next_id++;
    r->t_submit = seconds_since(s->t0);
    ids[k] = r->id;
    s->queue.push_back(r);
    s->all[r->id] = std::move(rs[k]);
  }
  s->cv_work.notify_all();
}

}  // namespace

extern "C" {

int rteom_server_create(rteom_server** out, double mem_budget_bytes, int max_active,
                        int precision) {
  if (!out) return RTEOM_ERR_ARG;
  *out = nullptr;
  if (max_active < 1 || mem_budget_bytes < 0 ||
      !rteom::valid_precision(precision))
    return RTEOM_ERR_ARG;
  std::unique_ptr<rteom_server> s(new rteom_server());
  if (cudaGetDevice(&s->device) != cudaSuccess) return RTEOM_ERR_CUDA;
  if (mem_budget_bytes == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return RTEOM_ERR_CUDA;
    mem_budget_bytes = 0.8 * (double)fr;
  }
  s->budget = mem_budget_bytes;
  s->max_active = max_active;
  s->precision = precision;
  rteom_server* raw = s.get();
  s->worker = std::thread([raw] { raw->loop(); });
  *out = s.release();
  return RTEOM_OK;
}

int rteom_server_submit(rteom_server* s, int nocc, int nvir, int nchol, const double* eps,
                        const double* L, const double* t1_gs, const double* t2_gs, int core_index,
                        int flags, int nsteps, double dt, double tol, int max_micro,
                        long long* request_id) {
  if (!request_id || bad_request(s, nocc, nvir, nchol, eps, L, nsteps, dt, tol, max_micro))
    return RTEOM_ERR_ARG;
  enqueue(s, nocc, nvir, nchol, copy_inputs(nocc, nvir, nchol, eps, L, t1_gs, t2_gs),
          &core_index, 1, flags, nsteps, dt, tol, max_micro, request_id);
  return RTEOM_OK;
}

int rteom_server_submit_sweep(rteom_server* s, int nocc, int nvir, int nchol, const double* eps,
                              const double* L, const double* t1_gs, const double* t2_gs,
                              const int* cores, int ncores, int flags, int nsteps, double dt,
                              double tol, int max_micro, long long* request_ids) {
  if (!request_ids || !cores || ncores < 1 ||
      bad_request(s, nocc, nvir, nchol, eps, L, nsteps, dt, tol, max_micro))
    return RTEOM_ERR_ARG;
  for (int k = 0; k < ncores; ++k)
    if (cores[k] < 0 || cores[k] >= nocc) return RTEOM_ERR_ARG;
  enqueue(s, nocc, nvir, nchol, copy_inputs(nocc, nvir, nchol, eps, L, t1_gs, t2_gs), cores,
          ncores, flags, nsteps, dt, tol, max_micro, request_ids);
  return RTEOM_OK;
}

int rteom_server_poll(rteom_server* s, long long id, int* status, int* error, double* C_out,
                      double* times) {
  if (!s) return RTEOM_ERR_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) return RTEOM_ERR_ARG;
  Request* r = it->second.get();
  if (status) *status = r->status;
  if (error) *error = r->error;
  if (C_out && r->status == RTEOM_REQ_DONE)
    std::copy(r->C.begin(), r->C.end(), C_out);
  if (times) {
    times[0] = r->t_submit;
    times[1] = r->t_admit;
    times[2] = r->t_done;
  }
  return RTEOM_OK;
}

int rteom_server_wait(rteom_server* s, long long id, double timeout_s) {
  if (!s) return RTEOM_ERR_ARG;
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) return RTEOM_ERR_ARG;
  Request* r = it->second.get();
  auto done = [&] {
    return r->status == RTEOM_REQ_DONE || r->status == RTEOM_REQ_FAILED ||
           r->status == RTEOM_REQ_CANCELLED;
  };
  if (timeout_s <= 0) {
    s->cv_done.wait(lock, done);
    return RTEOM_OK;
  }
  return s->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s), done)
             ? RTEOM_OK
             : RTEOM_ERR_STATE;
}

int rteom_server_cancel(rteom_server* s, long long id) {
  if (!s) return RTEOM_ERR_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) return RTEOM_ERR_ARG;
  it->second->cancel = true;
  s->cv_work.notify_all();
  return RTEOM_OK;
}

int rteom_server_stats(rteom_server* s, long long* queued, long long* running, long long* done,
                       long long* failed, double* mem_in_use, double* steps_done) {
  if (!s) return RTEOM_ERR_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  if (queued) *queued = (long long)s->queue.size();
  if (running) *running = (long long)s->active.size();
  if (done) *done = s->n_done;
  if (failed) *failed = s->n_failed;
  if (mem_in_use) *mem_in_use = s->in_use;
  if (steps_done) *steps_done = s->steps_done;
  return RTEOM_OK;
}

double rteom_server_estimate_bytes(int nocc, int nvir, int nchol, int precision) {
  return estimate_bytes(nocc, nvir, nchol, precision);
}

void rteom_server_destroy(rteom_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    for (auto& kv : s->all)
      if (kv.second->status == RTEOM_REQ_QUEUED || kv.second->status == RTEOM_REQ_RUNNING)
        kv.second->cancel = true;
    s->stop = true;
    s->cv_work.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  delete s;
}

}  // extern "C"
