// Request server: continuous batching of reconstructions on one GPU.
//
// Clients submit reconstructions (any N, K, M, analysis prior, fixed or adaptive
// penalty) at any time.  A
// worker thread admits queued requests in arrival order as soon as an
// execution slot is free and the device memory they need fits the budget,
// gives each its own stream and plan, and drives all running requests in
// chunks of `check_every` iterations: every chunk ends with the residual
// check of Alg. 1's stopping rule (relative primal/dual residuals of
// Eq. paramS below tol) and is launched without waiting for the others, so the
// kernels of different requests overlap on the device.  A request finishes
// when it converges or reaches max_iter; its x is copied to the client's
// buffer, its plan is freed and the next queued request can enter.
//
// A request with the adaptive penalty of Eq. paramS has the rule applied at every
// check, as cip_iterate does; it keeps its own factor and setup buffers, since a
// change of rho forms both again.
//
// Requests that carry the same nonzero psf_key and the same (N, K, M, prior,
// rho, beta) share one factor: the first one forms it in a cached plan, later
// ones copy the packed factor instead of recomputing it.  Cached factors are
// evicted least-recently-used when memory is needed.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "../../include/cip.h"
#include "plan_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

enum { RQ_QUEUED = 0, RQ_RUNNING = 1, RQ_DONE = 2, RQ_FAILED = 3, RQ_CANCELLED = 4 };

struct Request {
  unsigned long long id = 0;
  cip_request r{};
  std::vector<float> h, y;
  int state = RQ_QUEUED;
  int status = CIP_OK;
  int iterations = 0;
  int chunk = 0;
  double resid[2] = {0, 0};
  double* pinned = nullptr;
  double t_submit = 0, t_admit = 0, t_done = 0;
  size_t bytes = 0;
  cip_plan* plan = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  bool cancel = false;
  std::string err;
};

struct CacheEntry {
  cip_plan* plan = nullptr;
  size_t bytes = 0;
  Clock::time_point used;
};

using CacheKey = std::tuple<unsigned long long, int, int, int, int, double, double>;

}  // namespace

struct cip_server {
  size_t budget = 0;
  int max_active = 16;
  int check_every = 10;
  int device = 0;
  Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<std::shared_ptr<Request>> queue;
  std::map<unsigned long long, std::shared_ptr<Request>> all;
  std::vector<std::shared_ptr<Request>> running;
  std::map<CacheKey, CacheEntry> cache;
  size_t used = 0;
  unsigned long long next_id = 1;
  std::atomic<bool> stop{false};
  std::thread worker;
  // pinned host slots (cip::kResidHost doubles each) for the residuals of running requests
  double* pinned = nullptr;
  // stream of the cached factor plans (they outlive the requests and their streams)
  cudaStream_t cache_stream = nullptr;
  std::vector<int> free_slots;
  // statistics
  double voxel_iters = 0;
  int cache_hits = 0, cache_misses = 0;
};

namespace {

double now_s(const cip_server* s) { return std::chrono::duration<double>(Clock::now() - s->t0).count(); }

CacheKey key_of(const cip_request& r) {
  return CacheKey(r.psf_key, r.N, r.K, r.M, r.prior, r.rho, r.beta);
}

bool adaptive(const cip_request& r) { return r.rho_tau > 0; }

// factor sharing: a nonzero psf_key on a fixed-penalty request
bool shares_factor(const cip_request& r) { return r.psf_key != 0 && !adaptive(r); }

size_t full_plan_bytes(const cip_request& r) {
  size_t b = cip_plan_bytes(r.N, r.K, r.M, CIP_F32, (cip_prior)r.prior);
  // the adaptive penalty also keeps the measurement spectra (K half spectra, 16 bytes per bin)
  if (adaptive(r)) b += (size_t)r.K * r.N * (r.N / 2 + 4) * 16;
  return b;
}

// evict least-recently-used cached factors until `need` more bytes fit; returns whether they fit
bool make_room(cip_server* s, size_t need) {
  while (s->used + need > s->budget && !s->cache.empty()) {
    auto victim = s->cache.begin();
    for (auto it = s->cache.begin(); it != s->cache.end(); ++it)
      if (it->second.used < victim->second.used) victim = it;
    cip_plan_destroy(victim->second.plan);
    s->used -= victim->second.bytes;
    s->cache.erase(victim);
  }
  return s->used + need <= s->budget;
}

void finish(cip_server* s, Request& q, int state, int status) {
  if (q.plan) cip_plan_destroy(q.plan);
  q.plan = nullptr;
  if (q.ev) cudaEventDestroy(q.ev);
  if (q.stream) cudaStreamDestroy(q.stream);
  q.ev = nullptr;
  q.stream = nullptr;
  std::vector<float>().swap(q.h);
  std::vector<float>().swap(q.y);
  q.t_done = now_s(s);
  q.status = status;
  std::lock_guard<std::mutex> lk(s->mu);
  if (q.pinned) s->free_slots.push_back((int)((q.pinned - s->pinned) / cip::kResidHost));
  q.pinned = nullptr;
  s->used -= q.bytes;
  q.state = state;
  s->cv.notify_all();
}

// plan creation and setup of an admitted request (on the worker thread)
cip_status setup(cip_server* s, Request& q) {
  cudaStream_t st = q.stream;
  cip_status r = cip_plan_create_on_stream(&q.plan, q.r.N, q.r.K, q.r.M, CIP_F32, nullptr, st);
  if (r != CIP_OK) {
    q.err = cip_last_error(nullptr);
    return r;
  }
  r = cip_set_prior(q.plan, (cip_prior)q.r.prior, q.r.lambda, q.r.rho, q.r.beta, st);
  if (r != CIP_OK) return r;
  if (adaptive(q.r)) {
    r = cip_set_rho_adaptation(q.plan, q.r.rho_tau, q.r.rho_mu);
    if (r != CIP_OK) return r;
  }
  cip_plan* src = nullptr;
  if (shares_factor(q.r)) {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->cache.find(key_of(q.r));
    if (it != s->cache.end()) {
      src = it->second.plan;
      it->second.used = Clock::now();
      s->cache_hits++;
    } else {
      s->cache_misses++;
    }
  }
  if (shares_factor(q.r) && !src) {
    // form the factor once in a cached plan
    // (set_psfs waits for the factor, so the request's stream may read it right after)
    cip_plan* cp = nullptr;
    cudaStream_t cs = s->cache_stream;
    r = cip_plan_create_on_stream(&cp, q.r.N, q.r.K, q.r.M, CIP_F32, nullptr, cs);
    if (r == CIP_OK) r = cip_set_prior(cp, (cip_prior)q.r.prior, q.r.lambda, q.r.rho, q.r.beta, cs);
    if (r == CIP_OK) r = cip_set_psfs(cp, q.h.data(), cs);
    if (r != CIP_OK) {
      if (cp) cip_plan_destroy(cp);
      return r;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    CacheEntry e;
    e.plan = cp;
    e.bytes = full_plan_bytes(q.r);
    e.used = Clock::now();
    s->used += e.bytes;
    s->cache[key_of(q.r)] = e;
    src = cp;
  }
  if (src) {
    r = cip::plan_adopt_factor(q.plan, src, st);
  } else {
    r = cip_set_psfs(q.plan, q.h.data(), st);
  }
  if (r != CIP_OK) return r;
  r = cip_set_measurements(q.plan, q.y.data(), st);
  if (r != CIP_OK) return r;
  if (!adaptive(q.r)) {  // an adaptive request forms its factor again whenever rho changes
    r = cip::plan_trim(q.plan);
    if (r != CIP_OK) return r;
  }
  std::vector<float>().swap(q.h);
  std::vector<float>().swap(q.y);
  return CIP_OK;
}

void launch_chunk(cip_server* s, Request& q) {
  const int left = q.r.max_iter - q.iterations;
  q.chunk = std::min(s->check_every, left);
  cip_status r = cip::plan_iterate_async(q.plan, q.chunk, q.stream, q.pinned, q.ev);
  if (r != CIP_OK) {
    q.err = cip_last_error(q.plan);
    finish(s, q, RQ_FAILED, r);
  }
}

void worker_main(cip_server* s) {
  cudaSetDevice(s->device);
  while (!s->stop.load()) {
    // admission: in arrival order, while a slot is free and the request fits the budget
    std::vector<std::shared_ptr<Request>> admitted;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      while (!s->queue.empty()) {
        auto q = s->queue.front();
        if (q->cancel) {
          s->queue.pop_front();
          q->state = RQ_CANCELLED;
          q->t_done = now_s(s);
          s->cv.notify_all();
          continue;
        }
        if ((int)(s->running.size() + admitted.size()) >= s->max_active) break;
        const size_t need = full_plan_bytes(q->r) * (shares_factor(q->r) ? 2 : 1);
        if (!make_room(s, need) && !(s->running.empty() && admitted.empty())) break;
        s->queue.pop_front();
        // setup needs the full footprint; it drops to the resident size after trimming
        q->bytes = full_plan_bytes(q->r);
        s->used += q->bytes;
        q->pinned = s->pinned + cip::kResidHost * s->free_slots.back();
        s->free_slots.pop_back();
        q->state = RQ_RUNNING;
        q->t_admit = now_s(s);
        admitted.push_back(q);
      }
    }
    for (auto& q : admitted) {
      cudaStreamCreateWithFlags(&q->stream, cudaStreamNonBlocking);
      cudaEventCreateWithFlags(&q->ev, cudaEventDisableTiming);
      cip_status r = setup(s, *q);
      if (r != CIP_OK) {
        if (q->err.empty()) q->err = q->plan ? cip_last_error(q->plan) : cip_last_error(nullptr);
        finish(s, *q, RQ_FAILED, r);
        continue;
      }
      {
        std::lock_guard<std::mutex> lk(s->mu);
        const size_t res = adaptive(q->r) ? full_plan_bytes(q->r)
                                          : cip::plan_resident_bytes(q->r.N, q->r.K, q->r.M, CIP_F32,
                                                                     (cip_prior)q->r.prior);
        s->used -= q->bytes;
        q->bytes = res;
        s->used += q->bytes;
        s->running.push_back(q);
      }
      launch_chunk(s, *q);
    }
    // progress of the running requests
    bool any = false;
    std::vector<std::shared_ptr<Request>> still;
    std::vector<std::shared_ptr<Request>> snapshot;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      snapshot = s->running;
    }
    for (auto& q : snapshot) {
      if (q->state != RQ_RUNNING) continue;
      if (cudaEventQuery(q->ev) != cudaSuccess) {
        still.push_back(q);
        continue;
      }
      any = true;
      q->iterations += q->chunk;
      q->resid[0] = q->pinned[cip::kResidHost - 2];
      q->resid[1] = q->pinned[cip::kResidHost - 1];
      {
        std::lock_guard<std::mutex> lk(s->mu);
        s->voxel_iters += (double)q->r.N * q->r.N * q->r.M * q->chunk;
      }
      const bool conv = q->r.tol > 0 && q->resid[0] < q->r.tol && q->resid[1] < q->r.tol;
      if (q->cancel) {
        finish(s, *q, RQ_CANCELLED, CIP_OK);
      } else if (conv || q->iterations >= q->r.max_iter) {
        cip_status r = cip_get_x(q->plan, q->r.x_out, q->stream);
        finish(s, *q, r == CIP_OK ? RQ_DONE : RQ_FAILED, r);
      } else {
        if (adaptive(q->r)) {
          // Eq. paramS at this check; a change of rho is enqueued ahead of the next chunk
          cip_status r = cip::plan_adapt_rho(q->plan, q->pinned, q->stream);
          if (r != CIP_OK) {
            q->err = cip_last_error(q->plan);
            finish(s, *q, RQ_FAILED, r);
            continue;
          }
        }
        launch_chunk(s, *q);
        if (q->state == RQ_RUNNING) still.push_back(q);
      }
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      std::vector<std::shared_ptr<Request>> keep;
      for (auto& q : s->running)
        if (q->state == RQ_RUNNING) keep.push_back(q);
      s->running.swap(keep);
    }
    if (!any && admitted.empty()) {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait_for(lk, std::chrono::microseconds(50));
    }
  }
}

}  // namespace

extern "C" {

cip_status cip_server_create(cip_server** out, size_t hbm_budget, int max_active, int check_every) {
  if (!out || hbm_budget == 0) return CIP_ERR_INVALID_ARG;
  cip_server* s = new cip_server();
  s->budget = hbm_budget;
  s->max_active = max_active > 0 ? max_active : 16;
  s->check_every = check_every > 0 ? check_every : 10;
  cudaGetDevice(&s->device);
  if (cudaMallocHost((void**)&s->pinned, cip::kResidHost * sizeof(double) * s->max_active) != cudaSuccess) {
    delete s;
    return CIP_ERR_OOM;
  }
  for (int i = s->max_active - 1; i >= 0; --i) s->free_slots.push_back(i);
  cudaStreamCreateWithFlags(&s->cache_stream, cudaStreamNonBlocking);
  s->t0 = Clock::now();
  s->worker = std::thread(worker_main, s);
  *out = s;
  return CIP_OK;
}

cip_status cip_server_submit(cip_server* s, const cip_request* r, unsigned long long* id) {
  if (!s || !r || !r->h || !r->y || !r->x_out) return CIP_ERR_INVALID_ARG;
  if (r->prior != CIP_PRIOR_TV && r->prior != CIP_PRIOR_DCT8 && r->prior != CIP_PRIOR_L1 &&
      r->prior != CIP_PRIOR_TV_ISO && r->prior != CIP_PRIOR_WDCT)
    return CIP_ERR_UNSUPPORTED;
  if (r->rho_tau != 0.0 && !(r->rho_tau > 1.0 && r->rho_mu > 1.0 && std::isfinite(r->rho_tau) &&
                             std::isfinite(r->rho_mu)))
    return CIP_ERR_INVALID_ARG;
  if (r->N < 64 || r->N > 2048 || (r->N & (r->N - 1)) || r->K < 1 || r->K > 16 || r->M < 1 || r->M > 16)
    return CIP_ERR_UNSUPPORTED;
  if (r->max_iter < 1) return CIP_ERR_INVALID_ARG;
  auto q = std::make_shared<Request>();
  q->r = *r;
  const size_t nn = (size_t)r->N * r->N;
  q->h.assign(r->h, r->h + (size_t)r->K * r->M * nn);
  q->y.assign(r->y, r->y + (size_t)r->K * nn);
  std::lock_guard<std::mutex> lk(s->mu);
  if (full_plan_bytes(*r) > s->budget) return CIP_ERR_OOM;
  q->id = s->next_id++;
  q->t_submit = now_s(s);
  s->queue.push_back(q);
  s->all[q->id] = q;
  if (id) *id = q->id;
  s->cv.notify_all();
  return CIP_OK;
}

static void fill(const Request& q, cip_result* res) {
  res->state = q.state;
  res->status = q.status;
  res->iterations = q.iterations;
  res->r_rel = q.resid[0];
  res->s_rel = q.resid[1];
  res->t_submit = q.t_submit;
  res->t_admit = q.t_admit;
  res->t_done = q.t_done;
}

cip_status cip_server_poll(cip_server* s, unsigned long long id, cip_result* res) {
  if (!s || !res) return CIP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) return CIP_ERR_INVALID_ARG;
  fill(*it->second, res);
  return CIP_OK;
}

cip_status cip_server_wait(cip_server* s, unsigned long long id, cip_result* res, double timeout_s) {
  if (!s || !res) return CIP_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) return CIP_ERR_INVALID_ARG;
  auto q = it->second;
  const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
  while (q->state == RQ_QUEUED || q->state == RQ_RUNNING) {
    if (s->cv.wait_until(lk, until) == std::cv_status::timeout) {
      fill(*q, res);
      return CIP_ERR_TIMEOUT;
    }
  }
  fill(*q, res);
  return CIP_OK;
}

cip_status cip_server_cancel(cip_server* s, unsigned long long id) {
  if (!s) return CIP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) return CIP_ERR_INVALID_ARG;
  it->second->cancel = true;
  s->cv.notify_all();
  return CIP_OK;
}

cip_status cip_server_stats(cip_server* s, double* voxel_iters, int* running, int* queued, size_t* bytes_in_use,
                            int* cache_hits, int* cache_misses) {
  if (!s) return CIP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (voxel_iters) *voxel_iters = s->voxel_iters;
  if (running) *running = (int)s->running.size();
  if (queued) *queued = (int)s->queue.size();
  if (bytes_in_use) *bytes_in_use = s->used;
  if (cache_hits) *cache_hits = s->cache_hits;
  if (cache_misses) *cache_misses = s->cache_misses;
  return CIP_OK;
}

cip_status cip_server_destroy(cip_server* s) {
  if (!s) return CIP_ERR_INVALID_ARG;
  s->stop.store(true);
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto& q : s->running) {
    if (q->stream) cudaStreamSynchronize(q->stream);
    if (q->plan) cip_plan_destroy(q->plan);
    if (q->ev) cudaEventDestroy(q->ev);
    if (q->stream) cudaStreamDestroy(q->stream);
  }
  for (auto& c : s->cache) cip_plan_destroy(c.second.plan);
  cudaDeviceSynchronize();
  if (s->cache_stream) cudaStreamDestroy(s->cache_stream);
  if (s->pinned) cudaFreeHost(s->pinned);
  delete s;
  return CIP_OK;
}

}  // extern "C"
