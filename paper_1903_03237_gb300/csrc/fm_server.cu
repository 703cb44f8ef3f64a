// Serving loop for separation requests (continuous batching), host code.
//
// Requests arrive by fmnmf_server_submit (any thread) with their own mixture and shapes.
// A scheduler thread admits queued requests in arrival order while a slot is free and
// their device footprint (fmnmf_footprint: the context arena plus the Wiener output) fits
// the server's HBM budget, and keeps every admitted request's state resident in its own
// context (and stream).  Each admitted request advances in steps of iters_per_step
// iterations on its own stream, so the kernels of resident requests overlap on the
// device; the scheduler polls the streams (fmnmf_query) and enqueues a request's next
// step as soon as its previous one has finished, so no request waits for another's step,
// and requests that arrived meanwhile are admitted between polls.  A request that has run its
// iterations is separated (Eq. 3) into a host buffer, its context is destroyed, and its
// memory returns to the budget.  Each request computes exactly what a context running it
// alone computes: the kernels and their reduction orders do not depend on the mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fastmnmf.h"
#include "fm_launch.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
  uint64_t id = 0;
  int F = 0, T = 0, M = 0, N = 0, K = 0, n_iter = 0;
  uint64_t seed = 0;
  std::vector<float> X;     // host copy of the mixture (released once on the device)
  std::vector<float> out;   // separated images [N][F][T][M] complex64 (when done)
  double ll = 0.0;
  int state = FMNMF_JOB_QUEUED;
  fmnmf_status status = FMNMF_OK;
  std::string err;
  int iters_done = 0;
  int pending = 0;          // iterations of the step in flight
  size_t bytes = 0;
  fmnmf_ctx* ctx = nullptr;
  Clock::time_point t_submit, t_done;
};

fmnmf_status serr(fmnmf_status s, const char* fmt, ...) {
  char buf[384];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  fm::set_thread_error(buf);
  return s;
}

}  // namespace

struct fmnmf_server {
  fmnmf_server_opts o{};
  int device = 0;
  size_t budget = 0;
  std::mutex mu;
  std::condition_variable cv;       // scheduler wake-up (new request, stop)
  std::condition_variable done_cv;  // a request finished
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, std::unique_ptr<Job>> jobs;
  std::vector<Job*> active;
  size_t used = 0;
  uint64_t next_id = 1;
  long long completed = 0, failed = 0;
  bool stop = false;
  std::thread th;

  void finish(Job* j, int state, fmnmf_status st, const std::string& msg) {
    std::lock_guard<std::mutex> lk(mu);
    j->state = state;
    j->status = st;
    j->err = msg;
    j->t_done = Clock::now();
    used -= std::min(used, j->bytes);
    active.erase(std::remove(active.begin(), active.end(), j), active.end());
    if (state == FMNMF_JOB_DONE) ++completed; else ++failed;
    done_cv.notify_all();
  }

  void fail(Job* j, fmnmf_status st) {
    std::string msg = fmnmf_last_error(j->ctx);
    fmnmf_destroy(j->ctx);
    j->ctx = nullptr;
    finish(j, FMNMF_JOB_FAILED, st, msg);
  }

  // Enqueues the next step of j on its stream (asynchronous).
  void launch_step(Job* j) {
    const int k = std::min(o.iters_per_step, j->n_iter - j->iters_done);
    j->pending = k;
    fmnmf_status st = k > 0 ? fmnmf_iterate(j->ctx, k) : FMNMF_OK;
    if (st != FMNMF_OK) fail(j, st);
  }

  // The step of j has finished: account for it, and either separate and retire the
  // request or enqueue its next step.
  void step_done(Job* j, fmnmf_status st) {
    if (st != FMNMF_OK) { fail(j, st); return; }
    j->iters_done += j->pending;
    j->pending = 0;
    if (j->iters_done < j->n_iter) { launch_step(j); return; }
    j->out.resize((size_t)2 * j->N * j->F * j->T * j->M);
    st = fmnmf_separate(j->ctx, j->out.data(), 0);
    if (st == FMNMF_OK) st = fmnmf_loglik(j->ctx, &j->ll);
    if (st != FMNMF_OK) { fail(j, st); return; }
    fmnmf_destroy(j->ctx);
    j->ctx = nullptr;
    finish(j, FMNMF_JOB_DONE, FMNMF_OK, "");
  }

  void run() {
    cudaSetDevice(device);
    for (;;) {
      std::vector<Job*> admit, live;
      {
        std::unique_lock<std::mutex> lk(mu);
        if (active.empty())
          cv.wait_for(lk, std::chrono::milliseconds(2), [&] { return stop || !queue.empty(); });
        if (stop && active.empty()) break;
        while (!stop && !queue.empty() && (int)(active.size() + admit.size()) < o.max_active) {
          Job* j = jobs[queue.front()].get();
          if (used + j->bytes > budget) break;  // wait for memory to come back
          queue.pop_front();
          used += j->bytes;
          admit.push_back(j);
        }
      }
      for (Job* j : admit) {
        fmnmf_opts op;
        fmnmf_default_opts(&op);
        op.precision = o.precision;
        fmnmf_status st = fmnmf_init(&j->ctx, j->X.data(), 0, j->F, j->T, j->M, j->N, j->K, j->seed, &op);
        if (st != FMNMF_OK) {
          j->ctx = nullptr;
          finish(j, FMNMF_JOB_FAILED, st, fmnmf_last_error(nullptr));
          continue;
        }
        std::vector<float>().swap(j->X);
        {
          std::lock_guard<std::mutex> lk(mu);
          j->state = FMNMF_JOB_RUNNING;
          active.push_back(j);
        }
        launch_step(j);
      }
      {
        std::lock_guard<std::mutex> lk(mu);
        live = active;
      }
      bool progressed = !admit.empty();
      for (Job* j : live) {
        const fmnmf_status st = fmnmf_query(j->ctx);
        if (st == FMNMF_EBUSY) continue;
        progressed = true;
        step_done(j, st);
      }
      if (!progressed) {
        // nothing finished: sleep briefly unless a request arrives
        std::unique_lock<std::mutex> lk(mu);
        cv.wait_for(lk, std::chrono::microseconds(50), [&] { return stop || !queue.empty(); });
      }
    }
  }
};

extern "C" {

fmnmf_status fmnmf_server_create(const fmnmf_server_opts* opts, fmnmf_server** out) {
  if (!out) return serr(FMNMF_EINVAL, "server_create: out is NULL");
  *out = nullptr;
  auto* s = new fmnmf_server();
  if (opts) s->o = *opts;
  if (s->o.max_active <= 0) s->o.max_active = 16;
  if (s->o.iters_per_step <= 0) s->o.iters_per_step = 10;
  if (s->o.precision < FMNMF_PREC_FP32 || s->o.precision > FMNMF_PREC_TF32) {
    delete s;
    return serr(FMNMF_EINVAL, "server_create: unknown precision");
  }
  if (cudaGetDevice(&s->device) != cudaSuccess) { delete s; return serr(FMNMF_ECUDA, "server_create: no device"); }
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { delete s; return serr(FMNMF_ECUDA, "server_create: cudaMemGetInfo failed"); }
  s->budget = s->o.hbm_budget ? s->o.hbm_budget : (size_t)(0.7 * (double)fr);
  s->th = std::thread([s] { s->run(); });
  *out = s;
  return FMNMF_OK;
}

fmnmf_status fmnmf_server_submit(fmnmf_server* s, const void* X, int F, int T, int M, int N, int K, int n_iter,
                                 uint64_t seed, uint64_t* job) {
  if (!s || !X || !job) return serr(FMNMF_EINVAL, "server_submit: NULL argument");
  if (n_iter < 0) return serr(FMNMF_EINVAL, "server_submit: n_iter < 0");
  fmnmf_opts op;
  fmnmf_default_opts(&op);
  op.precision = s->o.precision;
  size_t bytes = 0;
  fmnmf_status st = fmnmf_footprint(F, T, M, N, K, &op, &bytes);
  if (st != FMNMF_OK) return st;
  if (bytes > s->budget)
    return serr(FMNMF_ENOMEM, "server_submit: request needs %zu bytes, the server budget is %zu", bytes, s->budget);
  auto j = std::make_unique<Job>();
  j->F = F; j->T = T; j->M = M; j->N = N; j->K = K; j->n_iter = n_iter; j->seed = seed; j->bytes = bytes;
  const float* x = (const float*)X;
  j->X.assign(x, x + (size_t)2 * F * T * M);
  j->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return serr(FMNMF_EBUSY, "server_submit: the server is stopping");
  j->id = s->next_id++;
  *job = j->id;
  s->queue.push_back(j->id);
  s->jobs.emplace(j->id, std::move(j));
  s->cv.notify_all();
  return FMNMF_OK;
}

fmnmf_status fmnmf_server_poll(fmnmf_server* s, uint64_t job, int* state, double* latency_s) {
  if (!s) return serr(FMNMF_EINVAL, "server_poll: NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(job);
  if (it == s->jobs.end()) return serr(FMNMF_EINVAL, "server_poll: unknown request %llu", (unsigned long long)job);
  Job* j = it->second.get();
  if (state) *state = j->state;
  if (latency_s)
    *latency_s = (j->state >= FMNMF_JOB_DONE)
                     ? std::chrono::duration<double>(j->t_done - j->t_submit).count() : -1.0;
  return FMNMF_OK;
}

fmnmf_status fmnmf_server_wait(fmnmf_server* s, uint64_t job, double timeout_s, int* state) {
  if (!s) return serr(FMNMF_EINVAL, "server_wait: NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(job);
  if (it == s->jobs.end()) return serr(FMNMF_EINVAL, "server_wait: unknown request %llu", (unsigned long long)job);
  Job* j = it->second.get();
  const bool ok = s->done_cv.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                      [&] { return j->state >= FMNMF_JOB_DONE; });
  if (state) *state = j->state;
  return ok ? FMNMF_OK : serr(FMNMF_ETIMEOUT, "server_wait: request %llu not finished", (unsigned long long)job);
}

fmnmf_status fmnmf_server_result(fmnmf_server* s, uint64_t job, void* out, double* loglik) {
  if (!s) return serr(FMNMF_EINVAL, "server_result: NULL server");
  std::unique_ptr<Job> j;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job);
    if (it == s->jobs.end()) return serr(FMNMF_EINVAL, "server_result: unknown request %llu", (unsigned long long)job);
    if (it->second->state < FMNMF_JOB_DONE) return serr(FMNMF_EBUSY, "server_result: request not finished");
    j = std::move(it->second);
    s->jobs.erase(it);
  }
  if (j->state == FMNMF_JOB_FAILED) return serr(j->status, "request %llu failed: %s", (unsigned long long)job, j->err.c_str());
  if (out) std::copy(j->out.begin(), j->out.end(), (float*)out);
  if (loglik) *loglik = j->ll;
  return FMNMF_OK;
}

fmnmf_status fmnmf_server_stats(fmnmf_server* s, long long* queued, long long* active, long long* completed,
                                long long* failed, size_t* bytes_in_use) {
  if (!s) return serr(FMNMF_EINVAL, "server_stats: NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  if (queued) *queued = (long long)s->queue.size();
  if (active) *active = (long long)s->active.size();
  if (completed) *completed = s->completed;
  if (failed) *failed = s->failed;
  if (bytes_in_use) *bytes_in_use = s->used;
  return FMNMF_OK;
}

fmnmf_status fmnmf_server_destroy(fmnmf_server* s) {
  if (!s) return FMNMF_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->queue.clear();
    s->cv.notify_all();
  }
  if (s->th.joinable()) s->th.join();
  for (auto& kv : s->jobs)
    if (kv.second->ctx) fmnmf_destroy(kv.second->ctx);
  delete s;
  return FMNMF_OK;
}

}  // extern "C"
