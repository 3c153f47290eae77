// Size buckets: the factorisations of several solve requests with the same lattice size and
// precision share one workspace and one launch sequence.  Each pass stacks the blocks of a set
// of requests (the pivoted blocks of all of them first, then the dominant ones, each request's
// in block order), with a per-slot table of the request's field, t, Delta_eff, mu, T, n and
// sigma; one reduction CTA per request then forms its Omega, gradient and Adam update from its
// own blocks.  Every block goes through the same kernels as in a pass of its own request, and
// the sums run over the request's blocks in block order, so a request's result does not depend
// on what shares its passes.  Requests that do not fit one pass are spread over several.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <new>
#include <vector>

#include "sca_device.cuh"
#include "sca_internal.h"

namespace sca {

struct Bucket {
  sca_ctx* ctx = nullptr;  // engine for the bucket's size and precision, `cap` block slots
  int cap = 0;
  int rmax = 0;             // requests per pass at most (each has at least two blocks)
  int passes = 0, steps = 0;  // table capacity
  BlockDesc* d_bd = nullptr;  // [passes][cap]
  int* d_slots = nullptr;     // [passes][cap]
  ReqDesc* d_req = nullptr;   // [passes][steps][rmax]
  BlockDesc* h_bd = nullptr;  // pinned staging of the same
  int* h_slots = nullptr;
  ReqDesc* h_req = nullptr;
};

namespace {

int pivoted_count(const sca_params& p) {
  int n_piv = 0;
  const double thr = 4.0 * std::fabs(p.t) * (1.0 + 1e-3);
  while (n_piv < p.n_omega && (2.0 * n_piv + 1.0) * M_PI * p.T <= thr) ++n_piv;
  int np = 2 * n_piv;
  if (const char* v = std::getenv("SCA_PIVOT_ALL"))
    if (std::atoi(v) != 0) np = 2 * p.n_omega;
  return np;
}

void free_tables(Bucket* b) {
  if (b->d_bd) cudaFree(b->d_bd);
  if (b->d_slots) cudaFree(b->d_slots);
  if (b->d_req) cudaFree(b->d_req);
  if (b->h_bd) cudaFreeHost(b->h_bd);
  if (b->h_slots) cudaFreeHost(b->h_slots);
  if (b->h_req) cudaFreeHost(b->h_req);
  b->d_bd = nullptr; b->d_slots = nullptr; b->d_req = nullptr;
  b->h_bd = nullptr; b->h_slots = nullptr; b->h_req = nullptr;
  b->passes = b->steps = 0;
}

sca_status ensure_tables(Bucket* b, int passes, int steps) {
  if (passes <= b->passes && steps <= b->steps) return SCA_OK;
  cudaError_t err = cudaStreamSynchronize(b->ctx->stream);
  if (err != cudaSuccess) return cuda_fail(err, "bucket tables");
  passes = std::max(passes, b->passes);
  steps = std::max(steps, b->steps);
  free_tables(b);
  const size_t nbd = (size_t)passes * b->cap, nreq = (size_t)passes * steps * b->rmax;
  err = cudaMalloc((void**)&b->d_bd, sizeof(BlockDesc) * nbd);
  if (err == cudaSuccess) err = cudaMalloc((void**)&b->d_slots, sizeof(int) * nbd);
  if (err == cudaSuccess) err = cudaMalloc((void**)&b->d_req, sizeof(ReqDesc) * nreq);
  if (err == cudaSuccess) err = cudaMallocHost((void**)&b->h_bd, sizeof(BlockDesc) * nbd);
  if (err == cudaSuccess) err = cudaMallocHost((void**)&b->h_slots, sizeof(int) * nbd);
  if (err == cudaSuccess) err = cudaMallocHost((void**)&b->h_req, sizeof(ReqDesc) * nreq);
  if (err != cudaSuccess) {
    free_tables(b);
    return cuda_fail(err, "bucket tables");
  }
  b->passes = passes;
  b->steps = steps;
  return SCA_OK;
}

}  // namespace

sca_params bucket_shape(int32_t L, int32_t prec, int cap) {
  sca_params s{};
  s.L = L;
  s.n_omega = std::max(1, cap / 2);
  s.prec = prec;
  s.ionic = SCA_IONIC_PAPER;
  s.t = 1.0;
  s.U = 1.0;
  s.delta = 0.0;
  s.T = 1.0;
  s.mu = 0.0;
  return s;
}

bool bucketed(const sca_params& p) {
  const int N = p.L * p.L;
  return N > (p.prec == SCA_PREC_FP64 ? 64 : 144);  // smaller sizes use the fused kernel
}

sca_status bucket_create(int32_t L, int32_t prec, int cap, Bucket** out) {
  *out = nullptr;
  Bucket* b = new (std::nothrow) Bucket();
  if (!b) { set_error("host allocation failed"); return SCA_ENOMEM; }
  b->cap = cap;
  b->rmax = std::max(1, cap / 2);
  const sca_params shape = bucket_shape(L, prec, cap);
  sca_status st = sca_create(&shape, &b->ctx);
  if (st != SCA_OK) { delete b; return st; }
  *out = b;
  return SCA_OK;
}

void bucket_destroy(Bucket* b) {
  if (!b) return;
  if (b->ctx) cudaStreamSynchronize(b->ctx->stream);
  free_tables(b);
  sca_destroy(b->ctx);
  delete b;
}

cudaStream_t bucket_stream(Bucket* b) { return b->ctx->stream; }

sca_status bucket_req_init(Bucket* b, BucketReq* r, const sca_params& p, const sca_adam& a) {
  const int N = p.L * p.L;
  r->p = p;
  r->a = a;
  r->step = 0;
  r->nb = 2 * p.n_omega;
  r->npiv = pivoted_count(p);
  r->delta_eff = (p.ionic == SCA_IONIC_HALF) ? 0.5 * p.delta : p.delta;
  cudaError_t err = cudaMalloc((void**)&r->d, sizeof(double) * (4 * (size_t)N + 8));
  if (err != cudaSuccess) { r->d = nullptr; return cuda_fail(err, "request state"); }
  cudaStream_t s = b->ctx->stream;
  sca_status st = run_seed_phi(r->d, N, a.seed, s);
  if (st != SCA_OK) return st;
  err = cudaMemsetAsync(r->d + N, 0, sizeof(double) * (3 * (size_t)N + 8), s);
  if (err != cudaSuccess) return cuda_fail(err, "request state");
  return SCA_OK;
}

void bucket_req_release(BucketReq* r) {
  if (r->d) cudaFree(r->d);
  r->d = nullptr;
}

sca_status bucket_run(Bucket* b, BucketReq* const* reqs, int n, int nsteps, bool adam) {
  NvtxRange range("sca.bucket_run");
  Engine& e = b->ctx->e;
  cudaStream_t s = b->ctx->stream;
  const int N = e.N;
  if (n <= 0 || nsteps <= 0) return SCA_OK;
  // the staging buffers of the previous call are free once its copies have run
  cudaError_t err = cudaStreamSynchronize(s);
  if (err != cudaSuccess) return cuda_fail(err, "bucket run");
  // passes: requests in order while their blocks fit the slots
  std::vector<int> first, count;
  for (int i = 0, used = 0; i < n; ++i) {
    if (reqs[i]->nb > b->cap) {
      set_error("request has more blocks than its size bucket");
      return SCA_EINVAL;
    }
    if (first.empty() || used + reqs[i]->nb > b->cap || count.back() == b->rmax) {
      first.push_back(i);
      count.push_back(0);
      used = 0;
    }
    ++count.back();
    used += reqs[i]->nb;
  }
  const int P = (int)first.size();
  sca_status st = ensure_tables(b, P, nsteps);
  if (st != SCA_OK) return st;
  std::vector<int> npiv(P), ntot(P);
  for (int p = 0; p < P; ++p) {
    BlockDesc* bd = b->h_bd + (size_t)p * b->cap;
    int* slots = b->h_slots + (size_t)p * b->cap;
    // slot of each request's blocks: pivoted blocks of every request first, then the rest
    int next = 0, off = 0;
    std::vector<int> base(count[p]);
    for (int k = 0; k < count[p]; ++k) { base[k] = off; off += reqs[first[p] + k]->nb; }
    for (int pass_piv = 1; pass_piv >= 0; --pass_piv)
      for (int k = 0; k < count[p]; ++k) {
        const BucketReq* r = reqs[first[p] + k];
        const int lo = pass_piv ? 0 : r->npiv, hi = pass_piv ? r->npiv : r->nb;
        for (int blk = lo; blk < hi; ++blk) {
          BlockDesc d;
          d.phi = r->d;
          d.eps_extra = nullptr;
          d.t = r->p.t;
          d.delta_eff = r->delta_eff;
          d.mu = r->p.mu;
          d.T = r->p.T;
          d.n = blk >> 1;
          d.sg = (blk & 1) ? -1 : 1;
          bd[next] = d;
          slots[base[k] + blk] = next;
          ++next;
        }
        if (pass_piv && k == count[p] - 1) npiv[p] = next;
      }
    ntot[p] = next;
    for (int sidx = 0; sidx < nsteps; ++sidx) {
      ReqDesc* rq = b->h_req + ((size_t)p * b->steps + sidx) * b->rmax;
      for (int k = 0; k < count[p]; ++k) {
        BucketReq* r = reqs[first[p] + k];
        ReqDesc q;
        q.phi = r->d;
        q.m = r->d + N;
        q.v = r->d + 2 * (size_t)N;
        q.g = r->d + 3 * (size_t)N;
        q.status = r->d + 4 * (size_t)N;
        q.slots = b->d_slots + (size_t)p * b->cap + base[k];
        q.nblocks = r->nb;
        q.U = r->p.U;
        q.T = r->p.T;
        q.do_adam = adam ? 1 : 0;
        q.adam = adam ? adam_step_args(r->a, r->step + 1 + sidx) : AdamStep{0, 1, 0, 0, 0, 0};
        rq[k] = q;
      }
    }
    err = cudaMemcpyAsync(b->d_bd + (size_t)p * b->cap, bd, sizeof(BlockDesc) * next,
                          cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(b->d_slots + (size_t)p * b->cap, slots, sizeof(int) * next,
                            cudaMemcpyHostToDevice, s);
    if (err != cudaSuccess) return cuda_fail(err, "bucket tables upload");
  }
  err = cudaMemcpyAsync(b->d_req, b->h_req, sizeof(ReqDesc) * (size_t)P * b->steps * b->rmax,
                        cudaMemcpyHostToDevice, s);
  if (err != cudaSuccess) return cuda_fail(err, "bucket tables upload");
  const int B0 = e.B, piv0 = e.piv_blocks;
  for (int sidx = 0; sidx < nsteps && st == SCA_OK; ++sidx)
    for (int p = 0; p < P && st == SCA_OK; ++p) {
      e.B = ntot[p];
      e.piv_blocks = npiv[p];
      e.bd = b->d_bd + (size_t)p * b->cap;
      st = run_blocks(e, reqs[first[p]]->d, true, s);
      if (st == SCA_OK)
        st = run_reduce_batch(e, b->d_req + ((size_t)p * b->steps + sidx) * b->rmax, count[p], s);
    }
  e.B = B0;
  e.piv_blocks = piv0;
  e.bd = nullptr;
  if (st != SCA_OK) return st;
  if (adam)
    for (int i = 0; i < n; ++i) reqs[i]->step += nsteps;
  return SCA_OK;
}

// Synchronises the bucket's stream and copies each request's status (8 doubles) to `out`:
// [0] Omega [1] max|g| [4] non-finite [5] updates applied [6] the pass's flags word.
sca_status bucket_status(Bucket* b, BucketReq* const* reqs, int n, double* out) {
  cudaStream_t s = b->ctx->stream;
  for (int i = 0; i < n; ++i) {
    const size_t N = (size_t)reqs[i]->p.L * reqs[i]->p.L;
    cudaError_t err = cudaMemcpyAsync(out + 8 * (size_t)i, reqs[i]->d + 4 * N, 8 * sizeof(double),
                                      cudaMemcpyDeviceToHost, s);
    if (err != cudaSuccess) return cuda_fail(err, "bucket status");
  }
  cudaError_t err = cudaStreamSynchronize(s);
  if (err != cudaSuccess) return cuda_fail(err, "bucket status");
  return SCA_OK;
}

sca_status bucket_get_phi(Bucket* b, const BucketReq* r, double* out) {
  const size_t N = (size_t)r->p.L * r->p.L;
  cudaError_t err = cudaMemcpyAsync(out, r->d, N * sizeof(double), cudaMemcpyDeviceToHost,
                                    b->ctx->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(b->ctx->stream);
  if (err != cudaSuccess) return cuda_fail(err, "bucket phi read-back");
  return SCA_OK;
}

}  // namespace sca
