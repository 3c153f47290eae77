// Serving loop: continuous batching of SCA solve requests of mixed size (L, U, Delta, T,
// n_omega) under an HBM admission budget.
//
// One worker thread owns every device object.  Each round it
//   1. admits queued requests in arrival order while a slot is free and the request's
//      workspace fits the remaining budget (each admitted request gets its own context,
//      stream and SplitMix64 start field; phi, m and v stay resident on the device),
//   2. enqueues a batch of gated Adam iterations for every request in flight, each on its
//      own stream, so the requests' kernels overlap on the device,
//   3. synchronises each request's stream in turn and retires the ones that converged
//      (max|g| < grad_tol: the device stops applying updates) or reached max_steps,
//      releasing their slot and budget for the next admission.
// A request's arithmetic depends only on its own context, so its result is the same alone
// and in any mix.  submit / poll / times only touch the bookkeeping under a mutex.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sca_internal.h"

namespace {

constexpr int32_t kRoundSteps = 8;  // Adam iterations enqueued per request per round

struct Request {
  uint64_t id = 0;
  sca_params p{};
  sca_adam a{};
  uint64_t bytes = 0;
  int state = 0;  // 0 queued, 1 running, 2 finished
  sca_status status = SCA_EPENDING;
  double t_submit = -1, t_admit = -1, t_start = -1, t_finish = -1;
  sca_ctx* ctx = nullptr;
  int32_t launched = 0;
  std::vector<double> phi;
  double omega = 0, gmax = 0;
  int32_t steps = 0;
  std::string error;  // message of the failure, if any
};

}  // namespace

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
  uint64_t next_id = 1;
  bool stop = false;
  std::thread worker;
  std::chrono::steady_clock::time_point t0;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  void run();
  void finish(Request* r, sca_status st);
};

void sca_server::finish(Request* r, sca_status st) {
  if (st != SCA_OK) r->error = sca_last_error();
  if (r->ctx) {
    sca_destroy(r->ctx);
    r->ctx = nullptr;
  }
  std::lock_guard<std::mutex> lock(mu);
  r->status = st;
  r->state = 2;
  r->t_finish = now();
  used -= r->bytes;
}

void sca_server::run() {
  cudaSetDevice(device);
  while (true) {
    std::vector<Request*> admitted;
    {
      std::unique_lock<std::mutex> lock(mu);
      while (!queue.empty() && (int32_t)(active.size() + admitted.size()) < slots &&
             used + queue.front()->bytes <= budget) {
        Request* r = queue.front();
        queue.pop_front();
        used += r->bytes;
        r->state = 1;
        r->t_admit = now();
        admitted.push_back(r);
      }
      if (active.empty() && admitted.empty()) {
        if (stop) break;
        cv.wait_for(lock, std::chrono::milliseconds(20));
        continue;
      }
      if (stop) {
        for (Request* r : admitted) active.push_back(r);
        break;
      }
    }
    for (Request* r : admitted) {
      sca_status st = sca_create(&r->p, &r->ctx);
      if (st == SCA_OK) st = sca_adam_init(r->ctx, &r->a, nullptr);
      if (st != SCA_OK) {
        finish(r, st);
        continue;
      }
      active.push_back(r);
    }
    // one round: enqueue a batch for every request, then collect
    for (Request* r : active) {
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
    for (Request* r : active) {
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
  for (Request* r : active) finish(r, SCA_ECUDA);
  active.clear();
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
  if (bytes > s->budget) {
    sca::set_error("sca_submit: the request's workspace (" + std::to_string(bytes) +
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
    delete kv.second;
  }
  for (Request* r : s->queue) (void)r;  // owned through `all`
  delete s;
}

}  // extern "C"
