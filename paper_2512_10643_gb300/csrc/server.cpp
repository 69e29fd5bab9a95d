// Request scheduler: continuous batching of state-build + sampling jobs on
// one GPU (not a step of the paper's method; it serves the method's output).
//
// A fixed set of slots each owns a worker thread, a non-blocking CUDA stream
// and a library context.  Requests queue in arrival order; a free slot admits
// the first of the next ADMIT_WINDOW queued requests whose device-memory
// estimate (gbsmps_estimate_bytes) fits the budget left by the jobs already
// on the device, so small jobs flow past a large one that is waiting for
// memory, and a request that has been passed over STARVE_LIMIT times blocks
// later ones until it fits.  An admitted job runs the whole path on its
// slot's stream (Gamma in, MPS built and kept on the device, samples drawn,
// patterns copied out) through the public entry points, so its result does
// not depend on what else runs: the kernels of concurrent jobs only share the
// GPU.  With batch_max > 1 a slot takes up to batch_max admissible jobs at
// once and builds them in one batched call (gbsmps_build_batch), then samples
// each; under load this turns many small launches into few large ones.
// Completion times give the per-request latency (submit to done).
#include "gbsmps.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

namespace {

constexpr int ADMIT_WINDOW = 8;
constexpr int STARVE_LIMIT = 32;

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Job {
  int64_t id = 0;
  gbsmps_request req{};
  size_t est = 0;
  int passed_over = 0;
  gbsmps_job_info info{};
};

}  // namespace

struct gbsmps_server {
  int device = 0;
  gbsmps_server_opts opts{};
  size_t budget = 0, in_use = 0, peak = 0;
  double t0 = 0.0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Job>> queue;
  std::unordered_map<int64_t, std::shared_ptr<Job>> jobs;
  std::vector<std::thread> workers;
  std::vector<gbsmps_ctx_t> ctxs;
  std::vector<cudaStream_t> streams;
  bool stop = false;
  int64_t next_id = 1;
  int64_t submitted = 0, completed = 0, failed = 0, running = 0;
  double first_admit = -1.0, last_done = 0.0;
  double tensors = 0.0, samples = 0.0;
  std::vector<double> lat_ms;

  // the next admissible job, or null (called with mu held)
  std::shared_ptr<Job> pick() {
    const int n = std::min<int>(ADMIT_WINDOW, (int)queue.size());
    for (int k = 0; k < n; ++k) {
      auto& j = queue[k];
      if (j->est <= budget - in_use) {
        for (int i = 0; i < k; ++i) queue[i]->passed_over++;
        auto r = j;
        queue.erase(queue.begin() + k);
        return r;
      }
      if (j->passed_over >= STARVE_LIMIT) break;   // the oldest starved job goes first
    }
    return nullptr;
  }

  // a job's end: its memory returns to the budget, its record is final
  void finish(Job& j, int rc) {
    {
      std::lock_guard<std::mutex> lk(mu);
      in_use -= j.est;
      --running;
      j.info.t_done = now_s() - t0;
      j.info.error = rc;
      j.info.state = rc ? 3 : 2;
      if (rc) std::snprintf(j.info.detail, sizeof(j.info.detail), "%s", gbsmps_last_error_detail());
      if (rc) {
        ++failed;
      } else {
        ++completed;
        lat_ms.push_back(1e3 * (j.info.t_done - j.info.t_submit));
        tensors += j.req.N;
        samples += (double)j.req.samples;
      }
      last_done = std::max(last_done, j.info.t_done);
    }
    cv_done.notify_all();
    cv_work.notify_all();
  }

  int sample_one(Job& j, gbsmps_mps_t m) {
    int rc = GBSMPS_OK;
    if (j.req.samples > 0)
      rc = gbsmps_sample(m, j.req.samples, j.req.seed, j.req.counter0, nullptr, j.req.out,
                         j.req.flags, GBSMPS_MEM_HOST);
    const int rc2 = gbsmps_release(m);
    return rc ? rc : rc2;
  }

  void run(std::vector<std::shared_ptr<Job>>& js, int slot) {
    if (opts.simulate_s_per_tensor > 0.0) {
      double n = 0.0;
      for (auto& j : js) n += j->req.N;
      std::this_thread::sleep_for(std::chrono::duration<double>(opts.simulate_s_per_tensor * n));
      for (auto& j : js) {
        if (j->req.out) std::fill(j->req.out, j->req.out + (size_t)j->req.samples * j->req.N, (uint8_t)0);
        if (j->req.flags) std::fill(j->req.flags, j->req.flags + (size_t)j->req.samples, (uint8_t)0);
        finish(*j, GBSMPS_OK);
      }
      return;
    }
    if (js.size() == 1) {
      Job& j = *js[0];
      gbsmps_mps_t m = nullptr;
      int rc = gbsmps_build_from_cov(ctxs[slot], j.req.N, j.req.gamma, GBSMPS_MEM_HOST, &j.req.opts, &m);
      if (!rc) rc = sample_one(j, m);
      finish(j, rc);
      return;
    }
    const int n = (int)js.size();
    std::vector<int32_t> Ns(n);
    std::vector<const double*> gs(n);
    std::vector<gbsmps_opts> os(n);
    std::vector<gbsmps_mps_t> hs(n, nullptr);
    for (int k = 0; k < n; ++k) {
      Ns[k] = js[k]->req.N;
      gs[k] = js[k]->req.gamma;
      os[k] = js[k]->req.opts;
    }
    const int rc = gbsmps_build_batch(ctxs[slot], n, Ns.data(), gs.data(), GBSMPS_MEM_HOST, os.data(),
                                      hs.data());
    for (int k = 0; k < n; ++k) finish(*js[k], rc ? rc : sample_one(*js[k], hs[k]));
  }

  void worker(int slot) {
    if (opts.simulate_s_per_tensor <= 0.0) cudaSetDevice(device);
    for (;;) {
      std::vector<std::shared_ptr<Job>> js;
      {
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
          if (stop && queue.empty()) return;
          auto j = pick();
          if (j) { js.push_back(j); break; }
          cv_work.wait(lk);
        }
        // more admissible jobs ride along, up to batch_max: each admitted
        // job's estimate is reserved before the next one is looked for, so
        // a batch admits a job only while it still fits the budget
        in_use += js[0]->est;
        while ((int)js.size() < opts.batch_max) {
          auto j = pick();
          if (!j) break;
          in_use += j->est;
          js.push_back(j);
        }
        peak = std::max(peak, in_use);
        for (auto& j : js) {
          ++running;
          j->info.state = 1;
          j->info.slot = slot;
          j->info.batch = (int32_t)js.size();
          j->info.t_admit = now_s() - t0;
          if (first_admit < 0.0) first_admit = j->info.t_admit;
        }
      }
      run(js, slot);
    }
  }
};

extern "C" {

int gbsmps_server_opts_default(gbsmps_server_opts* o) {
  if (!o) return GBSMPS_ERR_ARG;
  o->slots = 4;
  o->hbm_budget = 0;
  o->simulate_s_per_tensor = 0.0;
  o->batch_max = 1;
  return GBSMPS_OK;
}

int gbsmps_server_create(int device, const gbsmps_server_opts* o, gbsmps_server_t* out) {
  if (!o || !out) return GBSMPS_ERR_ARG;
  if (o->slots < 1 || o->slots > 64) return GBSMPS_ERR_ARG;
  if (o->batch_max < 1 || o->batch_max > 64) return GBSMPS_ERR_ARG;
  auto srv = std::make_unique<gbsmps_server>();
  srv->device = device;
  srv->opts = *o;
  srv->t0 = now_s();
  if (o->simulate_s_per_tensor > 0.0) {
    if (o->hbm_budget == 0) return GBSMPS_ERR_ARG;
    srv->budget = o->hbm_budget;
  } else {
    if (cudaSetDevice(device) != cudaSuccess) return GBSMPS_ERR_ARG;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return GBSMPS_ERR_CUDA;
    const size_t cap = fr / 10 * 9;
    srv->budget = o->hbm_budget ? std::min(o->hbm_budget, cap) : fr / 5 * 4;
    for (int k = 0; k < o->slots; ++k) {
      cudaStream_t st = nullptr;
      if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        for (auto c : srv->ctxs) gbsmps_destroy(c);
        for (auto s2 : srv->streams) cudaStreamDestroy(s2);
        return GBSMPS_ERR_CUDA;
      }
      gbsmps_ctx_t c = nullptr;
      int rc = gbsmps_create(device, st, &c);
      if (rc) {
        cudaStreamDestroy(st);
        for (auto c2 : srv->ctxs) gbsmps_destroy(c2);
        for (auto s2 : srv->streams) cudaStreamDestroy(s2);
        return rc;
      }
      srv->streams.push_back(st);
      srv->ctxs.push_back(c);
    }
  }
  gbsmps_server* p = srv.get();
  for (int k = 0; k < o->slots; ++k) p->workers.emplace_back([p, k] { p->worker(k); });
  *out = srv.release();
  return GBSMPS_OK;
}

int gbsmps_server_submit(gbsmps_server_t srv, const gbsmps_request* req, int64_t* id) {
  if (!srv || !req || !id) return GBSMPS_ERR_ARG;
  if (req->N < 1 || req->samples < 0 || (req->samples > 0 && !req->out)) return GBSMPS_ERR_ARG;
  if (!req->gamma && srv->opts.simulate_s_per_tensor <= 0.0) return GBSMPS_ERR_ARG;
  const size_t est = gbsmps_estimate_bytes(req->N, &req->opts, req->samples);
  if (est == 0) return GBSMPS_ERR_ARG;
  auto j = std::make_shared<Job>();
  j->req = *req;
  j->est = est;
  j->info.hbm_bytes = est;
  j->info.slot = -1;
  j->info.batch = 0;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->stop) return GBSMPS_ERR_STATE;
    if (est > srv->budget) return GBSMPS_ERR_OOM;
    j->id = srv->next_id++;
    j->info.t_submit = now_s() - srv->t0;
    srv->queue.push_back(j);
    srv->jobs[j->id] = j;
    ++srv->submitted;
    *id = j->id;
  }
  srv->cv_work.notify_all();
  return GBSMPS_OK;
}

int gbsmps_server_wait(gbsmps_server_t srv, int64_t id, double timeout_s, gbsmps_job_info* info) {
  if (!srv) return GBSMPS_ERR_ARG;
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->jobs.find(id);
  if (it == srv->jobs.end()) return GBSMPS_ERR_ARG;
  auto j = it->second;
  auto done = [&] { return j->info.state >= 2; };
  if (timeout_s < 0.0) srv->cv_done.wait(lk, done);
  else if (!srv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done)) {
    if (info) *info = j->info;
    return GBSMPS_ERR_TIMEOUT;
  }
  if (info) *info = j->info;
  return j->info.error;
}

int gbsmps_server_drain(gbsmps_server_t srv, double timeout_s) {
  if (!srv) return GBSMPS_ERR_ARG;
  std::unique_lock<std::mutex> lk(srv->mu);
  auto idle = [&] { return srv->queue.empty() && srv->running == 0; };
  if (timeout_s < 0.0) srv->cv_done.wait(lk, idle);
  else if (!srv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), idle))
    return GBSMPS_ERR_TIMEOUT;
  return GBSMPS_OK;
}

int gbsmps_server_stats_read(gbsmps_server_t srv, gbsmps_server_stats* st) {
  if (!srv || !st) return GBSMPS_ERR_ARG;
  std::lock_guard<std::mutex> lk(srv->mu);
  *st = gbsmps_server_stats{};
  st->submitted = srv->submitted;
  st->completed = srv->completed;
  st->failed = srv->failed;
  st->running = srv->running;
  st->queued = (int64_t)srv->queue.size();
  std::vector<double> l = srv->lat_ms;
  std::sort(l.begin(), l.end());
  if (!l.empty()) {
    auto q = [&](double f) {   // nearest-rank quantile
      size_t k = (size_t)std::max(0.0, std::ceil(f * l.size()) - 1.0);
      return l[std::min(k, l.size() - 1)];
    };
    st->p50_ms = q(0.50);
    st->p99_ms = q(0.99);
    double s = 0.0;
    for (double v : l) s += v;
    st->mean_ms = s / l.size();
  }
  st->busy_s = srv->first_admit >= 0.0 ? srv->last_done - srv->first_admit : 0.0;
  st->tensors = srv->tensors;
  st->samples = srv->samples;
  st->hbm_in_use = srv->in_use;
  st->hbm_budget = srv->budget;
  st->hbm_peak = srv->peak;
  return GBSMPS_OK;
}

int gbsmps_server_destroy(gbsmps_server_t srv) {
  if (!srv) return GBSMPS_ERR_ARG;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
  }
  srv->cv_work.notify_all();
  for (auto& t : srv->workers) t.join();
  for (auto c : srv->ctxs) gbsmps_destroy(c);
  for (auto s : srv->streams) cudaStreamDestroy(s);
  delete srv;
  return GBSMPS_OK;
}

}  // extern "C"
