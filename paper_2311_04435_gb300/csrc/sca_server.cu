// Serving loop: continuous batching of SCA solve requests of mixed size (L, U, Delta, T,
// n_omega) under an HBM admission budget.
//
// One worker thread owns every device object.  Each round it
//   1. admits queued requests in arrival order while a slot is free and the request's memory
//      fits the remaining budget.  Small requests (blocks that the fused kernel holds) get a
//      context and stream of their own; larger ones join the size bucket of their lattice
//      size and precision (one shared workspace of kBucketSlots block slots, created with the
//      bucket's first request and counted against the budget until its last one leaves), and
//      only their field, Adam moments and status are their own;
//   2. enqueues a batch of gated Adam iterations for every request in flight: one launch
//      sequence per small request, on its own stream, and per bucket one launch sequence for
//      all its requests (in passes of at most kBucketSlots blocks);
//   3. synchronises and retires the requests that converged (max|g| < grad_tol: the device
//      stops applying updates) or reached max_steps, releasing their slot and budget.
// A request's arithmetic does not depend on what it shares a bucket or the device with, so its
// result is the same alone and in any mix.  submit / poll / times only touch the bookkeeping
// under a mutex.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sca_internal.h"

namespace {

constexpr int32_t kRoundSteps = 8;     // Adam iterations enqueued per request per round
constexpr int kBucketSlots = 256;      // block slots of a size bucket's workspace

uint64_t bucket_bytes(int32_t L, int32_t prec, int cap) {
  const sca_params s = sca::bucket_shape(L, prec, cap);
  uint64_t b = 0;
  return sca_workspace_bytes(&s, &b) == SCA_OK ? b : ~0ull;
}

// Slots of a new bucket: kBucketSlots, or fewer (a power of two no smaller than the request's
// blocks) where the remaining budget is short; 0 if even that does not fit.
int bucket_cap(int32_t L, int32_t prec, int need, uint64_t room) {
  for (int cap = kBucketSlots; cap >= need; cap /= 2)
    if (bucket_bytes(L, prec, cap) <= room) return cap;
  return (bucket_bytes(L, prec, need) <= room) ? need : 0;
}

struct Request {
  uint64_t id = 0;
  sca_params p{};
  sca_adam a{};
  uint64_t bytes = 0;
  int state = 0;  // 0 queued, 1 running, 2 finished
  sca_status status = SCA_EPENDING;
  double t_submit = -1, t_admit = -1, t_start = -1, t_finish = -1;
  sca_ctx* ctx = nullptr;
  bool in_bucket = false;   // served through the size bucket of (L, prec)
  sca::BucketReq br;
  int32_t launched = 0;
  std::vector<double> phi;
  double omega = 0, gmax = 0;
  int32_t steps = 0;
  std::string error;  // message of the failure, if any
};

}  // namespace

struct BucketSlot {
  sca::Bucket* b = nullptr;  // null until created by the worker
  int cap = 0;
  uint64_t bytes = 0;        // its workspace, counted in `used`
  int members = 0;           // admitted requests not yet finished
};

struct sca_server {
  uint64_t budget = 0;
  int32_t slots = 0;
  uint64_t used = 0;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> queue;
  std::vector<Request*> active;  // worker-owned
  std::unordered_map<uint64_t, Request*> all;
  std::map<std::pair<int32_t, int32_t>, BucketSlot> buckets;  // (L, prec); under the mutex
  uint64_t next_id = 1;
  bool stop = false;
  std::thread worker;
  std::chrono::steady_clock::time_point t0;
  bool manual = false;   // no worker thread: sca_server_step runs each round (virtual clock)
  double vclock = 0.0;   // the virtual clock of a manual server (seconds)

  double now() const {
    if (manual) return vclock;
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  void run();
  bool round_once(bool idle_wait);
  void finish(Request* r, sca_status st);
  void run_buckets(std::vector<Request*>& active, std::vector<Request*>& still);
};

void sca_server::finish(Request* r, sca_status st) {
  if (st != SCA_OK) r->error = sca_last_error();
  if (r->ctx) {
    sca_destroy(r->ctx);
    r->ctx = nullptr;
  }
  sca::Bucket* gone = nullptr;
  if (r->in_bucket) sca::bucket_req_release(&r->br);
  {
    std::lock_guard<std::mutex> lock(mu);
    r->status = st;
    r->state = 2;
    r->t_finish = now();
    used -= r->bytes;
    if (r->in_bucket) {
      auto it = buckets.find({r->p.L, r->p.prec});
      if (it != buckets.end() && --it->second.members == 0) {  // the last one leaves
        gone = it->second.b;
        used -= it->second.bytes;
        buckets.erase(it);
      }
    }
  }
  if (gone) sca::bucket_destroy(gone);
}

// One round of every size bucket: a batch of gated steps for its requests (as many as the
// closest to its max_steps may still take), then retirement as in the single-request path:
// converged requests report the status of their last step, the others one more evaluation.
void sca_server::run_buckets(std::vector<Request*>& active, std::vector<Request*>& still) {
  std::map<std::pair<int32_t, int32_t>, std::vector<Request*>> groups;
  for (Request* r : active)
    if (r->in_bucket) groups[{r->p.L, r->p.prec}].push_back(r);
  struct Round {
    sca::Bucket* b;
    std::vector<Request*> rs;
    std::vector<sca::BucketReq*> br;
    sca_status st = SCA_OK;
  };
  std::vector<Round> rounds;
  // enqueue every bucket's batch first (each on its own stream), then collect
  for (auto& kv : groups) {
    Round rd;
    {
      std::lock_guard<std::mutex> lock(mu);
      rd.b = buckets[kv.first].b;
    }
    rd.rs = kv.second;
    int32_t n = kRoundSteps;
    for (Request* r : rd.rs) n = std::min(n, r->a.max_steps - r->launched);
    for (Request* r : rd.rs) rd.br.push_back(&r->br);
    if (n > 0) {
      rd.st = sca::bucket_run(rd.b, rd.br.data(), (int)rd.br.size(), n, true);
      if (rd.st == SCA_OK)
        for (Request* r : rd.rs) {
          if (r->t_start < 0) {
            std::lock_guard<std::mutex> lock(mu);
            r->t_start = now();
          }
          r->launched += n;
        }
    }
    rounds.push_back(std::move(rd));
  }
  for (Round& rd : rounds) {
    sca::Bucket* b = rd.b;
    std::vector<Request*>& rs = rd.rs;
    sca_status st = rd.st;
    std::vector<double> stat(8 * rs.size());
    if (st == SCA_OK) st = sca::bucket_status(b, rd.br.data(), (int)rd.br.size(), stat.data());
    if (st != SCA_OK) {
      for (Request* r : rs) finish(r, st);
      continue;
    }
    std::vector<Request*> done, evals;
    for (size_t k = 0; k < rs.size(); ++k) {
      Request* r = rs[k];
      const double* s = &stat[8 * k];
      if (((int)s[6]) & 2) {
        sca::set_error("a bounded device-side wait ran out");
        finish(r, SCA_ETIMEOUT);
        continue;
      }
      if (s[4] != 0.0) {
        sca::set_error("non-finite Omega or gradient, or a singular block");
        finish(r, SCA_ENONFINITE);
        continue;
      }
      const bool converged = s[5] < (double)r->launched;
      if (!converged && r->launched < r->a.max_steps) {
        still.push_back(r);
        continue;
      }
      r->steps = (int32_t)s[5];
      done.push_back(r);
      if (!converged) evals.push_back(r);
    }
    if (!evals.empty()) {  // Omega and max|g| at the final phi
      std::vector<sca::BucketReq*> be;
      for (Request* r : evals) be.push_back(&r->br);
      st = sca::bucket_run(b, be.data(), (int)be.size(), 1, false);
      std::vector<double> s2(8 * evals.size());
      if (st == SCA_OK) st = sca::bucket_status(b, be.data(), (int)be.size(), s2.data());
      for (size_t k = 0; k < evals.size() && st == SCA_OK; ++k)
        for (size_t i = 0; i < rs.size(); ++i)
          if (rs[i] == evals[k]) std::copy(&s2[8 * k], &s2[8 * k] + 8, &stat[8 * i]);
      if (st != SCA_OK) {
        for (Request* r : done) finish(r, st);
        continue;
      }
    }
    for (Request* r : done) {
      size_t i = 0;
      while (rs[i] != r) ++i;
      if (stat[8 * i + 4] != 0.0) {
        sca::set_error("non-finite Omega or gradient, or a singular block");
        finish(r, SCA_ENONFINITE);
        continue;
      }
      r->phi.resize((size_t)r->p.L * r->p.L);
      st = sca::bucket_get_phi(b, &r->br, r->phi.data());
      r->omega = stat[8 * i];
      r->gmax = stat[8 * i + 1];
      finish(r, st);
    }
  }
}

void sca_server::run() {
  cudaSetDevice(device);
  while (round_once(true)) {
  }
  for (Request* r : active) finish(r, SCA_ECUDA);
  active.clear();
}

// One admission pass and one round of every request in flight.  Returns false once the server
// stops (the worker then abandons what is still in flight).  idle_wait: with nothing to do,
// wait briefly for a submission (the worker thread) instead of returning at once.
bool sca_server::round_once(bool idle_wait) {
  {
    std::vector<Request*> admitted;
    {
      std::unique_lock<std::mutex> lock(mu);
      while (!queue.empty() && (int32_t)(active.size() + admitted.size()) < slots) {
        Request* r = queue.front();
        uint64_t need = r->bytes;
        int cap = 0;
        const bool bk = sca::bucketed(r->p);
        const auto key = std::make_pair(r->p.L, r->p.prec);
        if (bk && !buckets.count(key)) {  // this request creates the bucket
          if (used + need > budget) break;
          cap = bucket_cap(r->p.L, r->p.prec, 2 * r->p.n_omega, budget - used - need);
          if (cap == 0) break;
          need += bucket_bytes(r->p.L, r->p.prec, cap);
        }
        if (used + need > budget) break;
        queue.pop_front();
        used += need;
        if (bk) {
          BucketSlot& bs = buckets[key];
          if (cap) { bs.cap = cap; bs.bytes = need - r->bytes; }
          ++bs.members;
          r->in_bucket = true;
        }
        r->state = 1;
        r->t_admit = now();
        admitted.push_back(r);
      }
      if (active.empty() && admitted.empty()) {
        if (stop) return false;
        if (idle_wait) cv.wait_for(lock, std::chrono::milliseconds(20));
        return true;
      }
      if (stop) {
        for (Request* r : admitted) active.push_back(r);
        return false;
      }
    }
    for (Request* r : admitted) {
      sca_status st = SCA_OK;
      if (r->in_bucket) {
        BucketSlot* bs;
        {
          std::lock_guard<std::mutex> lock(mu);
          bs = &buckets[{r->p.L, r->p.prec}];
        }
        if (!bs->b) st = sca::bucket_create(r->p.L, r->p.prec, bs->cap, &bs->b);
        if (st == SCA_OK) st = sca::bucket_req_init(bs->b, &r->br, r->p, r->a);
      } else {
        st = sca_create(&r->p, &r->ctx);
        if (st == SCA_OK) st = sca_adam_init(r->ctx, &r->a, nullptr);
      }
      if (st != SCA_OK) {
        finish(r, st);
        continue;
      }
      active.push_back(r);
    }
    sca::NvtxRange round("sca.server_round");
    // one round: enqueue a batch for every request, then collect
    for (Request* r : active) {
      if (r->in_bucket) continue;
      const int32_t n = std::min(kRoundSteps, r->a.max_steps - r->launched);
      if (n <= 0) continue;
      if (r->t_start < 0) {
        std::lock_guard<std::mutex> lock(mu);
        r->t_start = now();
      }
      if (sca::enqueue_adam(r->ctx, n) != SCA_OK) r->launched = -1;  // flagged below
      else r->launched += n;
    }
    std::vector<Request*> still;
    run_buckets(active, still);
    for (Request* r : active) {
      if (r->in_bucket) continue;
      sca_status st = SCA_OK;
      if (r->launched < 0) st = SCA_ECUDA;
      if (st == SCA_OK) st = sca::sync_status(r->ctx, r->ctx->stream);
      if (st == SCA_OK) st = sca::check_finite(r->ctx);
      if (st != SCA_OK) {
        finish(r, st);
        continue;
      }
      const double updates = r->ctx->e.h_status[5];
      const bool converged = updates < (double)r->launched;
      const bool reached = r->launched >= r->a.max_steps;
      if (!converged && !reached) {
        still.push_back(r);
        continue;
      }
      if (!converged) st = sca::final_eval(r->ctx);  // Omega, max|g| at the final phi
      if (st == SCA_OK) {
        r->phi.resize((size_t)r->p.L * r->p.L);
        st = sca_get_phi(r->ctx, r->phi.data());
        r->omega = r->ctx->e.h_status[0];
        r->gmax = r->ctx->e.h_status[1];
        r->steps = (int32_t)updates;
      }
      finish(r, st);
    }
    active.swap(still);
  }
  return true;
}

extern "C" {

sca_status sca_server_create(uint64_t hbm_budget_bytes, int32_t max_slots, sca_server** out) {
  if (!out || max_slots < 1 || hbm_budget_bytes == 0) {
    sca::set_error("sca_server_create: need out != NULL, max_slots >= 1, budget > 0");
    return SCA_EINVAL;
  }
  *out = nullptr;
  sca_server* s = new (std::nothrow) sca_server();
  if (!s) {
    sca::set_error("host allocation failed");
    return SCA_ENOMEM;
  }
  s->budget = hbm_budget_bytes;
  s->slots = max_slots;
  s->t0 = std::chrono::steady_clock::now();
  cudaError_t err = cudaGetDevice(&s->device);
  if (err != cudaSuccess) {
    delete s;
    return sca::cuda_fail(err, "cudaGetDevice");
  }
  s->worker = std::thread([s] { s->run(); });
  *out = s;
  return SCA_OK;
}

sca_status sca_server_create_manual(uint64_t hbm_budget_bytes, int32_t max_slots,
                                    sca_server** out) {
  if (!out || max_slots < 1 || hbm_budget_bytes == 0) {
    sca::set_error("sca_server_create_manual: need out != NULL, max_slots >= 1, budget > 0");
    return SCA_EINVAL;
  }
  *out = nullptr;
  sca_server* s = new (std::nothrow) sca_server();
  if (!s) {
    sca::set_error("host allocation failed");
    return SCA_ENOMEM;
  }
  s->budget = hbm_budget_bytes;
  s->slots = max_slots;
  s->manual = true;
  cudaError_t err = cudaGetDevice(&s->device);
  if (err != cudaSuccess) {
    delete s;
    return sca::cuda_fail(err, "cudaGetDevice");
  }
  *out = s;
  return SCA_OK;
}

sca_status sca_server_step(sca_server* s, double now_s, int32_t* in_flight, int32_t* queued) {
  if (!s || !s->manual) {
    sca::set_error("sca_server_step: needs a server from sca_server_create_manual");
    return SCA_EINVAL;
  }
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (!(now_s >= s->vclock)) {
      sca::set_error("sca_server_step: the virtual clock must not run backwards");
      return SCA_EINVAL;
    }
    s->vclock = now_s;
  }
  cudaError_t err = cudaSetDevice(s->device);
  if (err != cudaSuccess) return sca::cuda_fail(err, "cudaSetDevice");
  s->round_once(false);
  std::lock_guard<std::mutex> lock(s->mu);
  if (in_flight) *in_flight = (int32_t)s->active.size();
  if (queued) *queued = (int32_t)s->queue.size();
  return SCA_OK;
}

sca_status sca_submit(sca_server* s, const sca_params* params, const sca_adam* adam,
                      uint64_t* req_id) {
  if (!s || !params || !adam || !req_id) {
    sca::set_error("sca_submit: NULL argument");
    return SCA_EINVAL;
  }
  uint64_t bytes = 0;
  sca_status st = sca_workspace_bytes(params, &bytes);
  if (st != SCA_OK) return st;
  if (!(adam->lr > 0) || !(adam->eps > 0) || adam->max_steps < 0 || !(adam->beta1 >= 0 && adam->beta1 < 1) ||
      !(adam->beta2 >= 0 && adam->beta2 < 1) || !(adam->grad_tol >= 0)) {
    sca::set_error("sca_submit: invalid Adam settings");
    return SCA_EINVAL;
  }
  uint64_t least = bytes;  // memory the request needs on an otherwise idle server
  if (sca::bucketed(*params)) {
    // its own state (phi, m, v, g and status); the bucket's workspace is shared
    bytes = sizeof(double) * (4 * (uint64_t)params->L * params->L + 8);
    least = bytes + bucket_bytes(params->L, params->prec, 2 * params->n_omega);
  }
  if (least > s->budget) {
    sca::set_error("sca_submit: the request's workspace (" + std::to_string(least) +
                   " bytes) exceeds the server's HBM budget");
    return SCA_EBUDGET;
  }
  Request* r = new (std::nothrow) Request();
  if (!r) {
    sca::set_error("host allocation failed");
    return SCA_ENOMEM;
  }
  r->p = *params;
  r->a = *adam;
  r->bytes = bytes;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    r->id = s->next_id++;
    r->t_submit = s->now();
    s->queue.push_back(r);
    s->all[r->id] = r;
  }
  s->cv.notify_one();
  *req_id = r->id;
  return SCA_OK;
}

sca_status sca_poll(sca_server* s, uint64_t req_id, double* phi_out, double* omega,
                    int32_t* steps, double* gmax) {
  if (!s) {
    sca::set_error("sca_poll: NULL server");
    return SCA_EINVAL;
  }
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->all.find(req_id);
  if (it == s->all.end()) {
    sca::set_error("sca_poll: unknown request id");
    return SCA_ENOTFOUND;
  }
  Request* r = it->second;
  if (r->state != 2) return SCA_EPENDING;
  if (r->status != SCA_OK) {
    sca::set_error("request " + std::to_string(req_id) + " failed: " + r->error);
    return r->status;
  }
  if (phi_out) std::copy(r->phi.begin(), r->phi.end(), phi_out);
  if (omega) *omega = r->omega;
  if (steps) *steps = r->steps;
  if (gmax) *gmax = r->gmax;
  return SCA_OK;
}

sca_status sca_request_times(sca_server* s, uint64_t req_id, double* submit_s, double* admit_s,
                             double* start_s, double* finish_s) {
  if (!s) {
    sca::set_error("sca_request_times: NULL server");
    return SCA_EINVAL;
  }
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->all.find(req_id);
  if (it == s->all.end()) {
    sca::set_error("sca_request_times: unknown request id");
    return SCA_ENOTFOUND;
  }
  Request* r = it->second;
  if (submit_s) *submit_s = r->t_submit;
  if (admit_s) *admit_s = r->t_admit;
  if (start_s) *start_s = r->t_start;
  if (finish_s) *finish_s = r->t_finish;
  return SCA_OK;
}

void sca_server_destroy(sca_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto& kv : s->all) {
    if (kv.second->ctx) sca_destroy(kv.second->ctx);
    if (kv.second->in_bucket) sca::bucket_req_release(&kv.second->br);
    delete kv.second;
  }
  for (auto& kv : s->buckets) sca::bucket_destroy(kv.second.b);
  for (Request* r : s->queue) (void)r;  // owned through `all`
  delete s;
}

}  // extern "C"
