// C ABI of the SCA+ADAM library: parameter validation, workspace planning, contexts, the
// Adam driver and the one-shot solver.  All arithmetic runs in the kernels of sca_core.cu
// and sca_tc.cu; this file only moves data and sequences launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "sca_internal.h"

namespace sca {

std::atomic<uint64_t> g_launches{0};

namespace {
thread_local std::string t_err;

// SMs the dominant group's persistent tensor-core launches leave free while the pivoted
// group runs beside them on its own (high-priority) stream.  Above N = 2048 the pivoted chain
// (sub-panels of 4 columns at N = 4096: over 2000 launches per step) bounds the step, and more
// SMs shorten it: 64x64 workload at 121.6 / 119.0 / 113.9 / 110.6 / 112.9 / 118.7 ms per step
// with 8 / 16 / 24 / 32 / 40 / 48 SMs kept free.
constexpr int kDefaultSmReserve = 8;
constexpr int kLargeNSmReserve = 32;
// Problems with 1024 <= N <= 2048 and at least 64 dominant blocks start with an SM partition
// that keeps the dominant group's launches off this many SMs (sca_set_sm_partition changes
// it), so that the pivoted chain's kernels never wait for a dominant CTA to leave an SM.  With
// the dominant group's elimination steps merged in pairs its span shrinks, and 16 SMs for the
// pivoted chain (mode 1) balance the two spans best at 40x40 (23.2 ms against 24.3 with 8 SMs
// in mode 3 and 25.6 with 32); without merged pairs 8 SMs in mode 3 did.  At larger N the
// dominant group's work dwarfs the chain and the partition only costs.
constexpr int kDefaultPartitionSms = 8;
constexpr int kDefaultPartitionSmsPaired = 16;
}

void set_error(const std::string& msg) { t_err = msg; }

uint64_t current_context_id() {
  typedef int (*CtxGetCurrentFn)(void**);
  typedef int (*CtxGetIdFn)(void*, unsigned long long*);
  static std::atomic<CtxGetCurrentFn> get_current{nullptr};
  static std::atomic<CtxGetIdFn> get_id{nullptr};
  static std::atomic<int> tried{0};
  if (!tried.load(std::memory_order_acquire)) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current.store(reinterpret_cast<CtxGetCurrentFn>(p));
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id.store(reinterpret_cast<CtxGetIdFn>(p));
    (void)cudaGetLastError();
    tried.store(1, std::memory_order_release);
  }
  CtxGetCurrentFn gc = get_current.load();
  CtxGetIdFn gi = get_id.load();
  if (!gc || !gi) return 0;
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (gc(&ctx) != 0 || !ctx || gi(ctx, &id) != 0) return 0;
  return (uint64_t)id;
}

sca_status cuda_fail(cudaError_t e, const char* where) {
  (void)cudaGetLastError();  // a failed call also records itself as the thread's last error
  set_error(std::string("CUDA error in ") + where + ": " + cudaGetErrorString(e));
  return SCA_ECUDA;
}

static sca_status validate(const sca_params* p) {
  if (!p) { set_error("params is NULL"); return SCA_EINVAL; }
  if (p->L < 2 || p->L > 64 || (p->L & 1)) {
    set_error("L must be even with 2 <= L <= 64");
    return SCA_EINVAL;
  }
  if (p->n_omega < 1 || p->n_omega > 16384) { set_error("n_omega must be in [1, 16384]"); return SCA_EINVAL; }
  if (!(p->U > 0) || !std::isfinite(p->U)) { set_error("U must be finite and > 0"); return SCA_EINVAL; }
  if (!(p->T > 0) || !std::isfinite(p->T)) { set_error("T must be finite and > 0"); return SCA_EINVAL; }
  if (!std::isfinite(p->t) || !std::isfinite(p->delta) || !std::isfinite(p->mu)) {
    set_error("t, delta and mu must be finite");
    return SCA_EINVAL;
  }
  if (p->prec < SCA_PREC_FP64 || p->prec > SCA_PREC_BF16X3) {
    set_error("prec must be SCA_PREC_FP64, SCA_PREC_FP32, SCA_PREC_3XTF32 or SCA_PREC_BF16X3");
    return SCA_EINVAL;
  }
  if (p->ionic != SCA_IONIC_PAPER && p->ionic != SCA_IONIC_HALF) {
    set_error("ionic must be SCA_IONIC_PAPER or SCA_IONIC_HALF");
    return SCA_EINVAL;
  }
  return SCA_OK;
}

static sca_status validate_adam(const sca_adam* a) {
  if (!a) { set_error("adam is NULL"); return SCA_EINVAL; }
  if (!(a->lr > 0) || !std::isfinite(a->lr) || !(a->beta1 >= 0 && a->beta1 < 1) ||
      !(a->beta2 >= 0 && a->beta2 < 1) || !(a->eps > 0) || !(a->grad_tol >= 0) ||
      a->max_steps < 0) {
    set_error("invalid Adam settings (lr > 0, 0 <= beta < 1, eps > 0, grad_tol >= 0, max_steps >= 0)");
    return SCA_EINVAL;
  }
  return SCA_OK;
}

static size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

sca_status plan(const sca_params& p, Engine& e) {
  e.p = p;
  e.L = p.L;
  e.N = p.L * p.L;
  e.B = 2 * p.n_omega;
  e.fp64 = (p.prec == SCA_PREC_FP64);
  e.refine = !e.fp64;
  e.delta_eff = (p.ionic == SCA_IONIC_HALF) ? 0.5 * p.delta : p.delta;
  // tcgen05 path for blocks of at least 128 rows; smaller blocks use CUDA cores.
  e.tc = (p.prec == SCA_PREC_3XTF32 || p.prec == SCA_PREC_BF16X3) && e.N >= 128 &&
         tc_supported();
  e.bf16 = e.tc && p.prec == SCA_PREC_BF16X3;
  int nb = e.fp64 ? 32 : (e.tc ? 128 : 64);
  if (const char* v = std::getenv("SCA_NB")) {
    const int x = std::atoi(v);
    if (x >= 16 && x <= (e.fp64 ? 64 : 128) && (x % 16) == 0) nb = x;
  }
  e.nb = std::min(nb, e.tc ? nb : e.N);
  // Blocks with omega_n > 4|t| are strictly diagonally dominant by columns (|a_jj| >= omega_n,
  // off-diagonal column sum 4|t|); dominance survives elimination, so partial pivoting keeps
  // the diagonal and those blocks skip the pivot search.  They are b >= piv_blocks.
  int n_piv = 0;
  const double thr = 4.0 * std::fabs(p.t) * (1.0 + 1e-3);
  while (n_piv < p.n_omega && (2.0 * n_piv + 1.0) * M_PI * p.T <= thr) ++n_piv;
  e.piv_blocks = 2 * n_piv;
  if (const char* v = std::getenv("SCA_PIVOT_ALL"))
    if (std::atoi(v) != 0) e.piv_blocks = e.B;
  e.piv_planned = e.piv_blocks;
  // Width of the pivoted group's shared-memory panel: N x (nb_piv + 1) complex values
  // (rows padded by one) within 220 KB.
  const size_t cbytes = e.fp64 ? 16 : 8;
  int nbp = 1;
  while (nbp * 2 <= e.nb && (size_t)e.N * (nbp * 2 + 1) * cbytes <= 220 * 1024) nbp *= 2;
  // narrower than nb: the outer panel is factorised in sub-panels of at most 16 columns
  if (nbp < e.nb) nbp = std::min(nbp, 16);
  e.nb_piv = nbp;
  {  // a float64 panel (16 bytes per complex entry) on the float32 blocks of the mixed path
    int n64 = 1;
    while (n64 * 2 <= e.nb && (size_t)e.N * (n64 * 2 + 1) * 16 <= 220 * 1024) n64 *= 2;
    if (n64 < e.nb) n64 = std::min(n64, 16);
    e.nb_piv64 = n64;
  }
  if (const char* v = std::getenv("SCA_DIAG_TC")) e.diag_tc = std::atoi(v) != 0;
  if (const char* v = std::getenv("SCA_ALT_POLICY")) e.alt_policy = std::min(3, std::max(1, std::atoi(v)));
  e.ldm = (int)round_up((size_t)e.N, 32);
  e.chunk = e.B;
  if (const char* v = std::getenv("SCA_MAX_BLOCKS_RESIDENT")) {
    const int x = std::atoi(v);
    if (x >= 1) e.chunk = std::min(e.B, x);
  }
  const size_t S = e.fp64 ? 8 : 4;
  e.plane_stride = (size_t)e.N * e.ldm;
  e.mat_stride = 2 * e.plane_stride;
  e.fw_plane = (size_t)e.N * e.nb;
  e.fw_mat = (e.tc ? 6 : 2) * e.fw_plane;
  const size_t C = S;  // compute type of the small kernels = storage type
  // merged two-step updates of the symmetric dominant blocks (second factor pair F2, W2): on
  // the tensor-core path when at least two elimination steps remain after the first one
  e.pair = e.tc && e.nb == 128 && e.N > e.nb && e.B > e.piv_blocks;
  if (const char* v = std::getenv("SCA_PAIR"))
    if (std::atoi(v) == 0) e.pair = false;
  size_t bytes = 0;
  bytes += (size_t)e.chunk * e.mat_stride * S;           // blocks
  bytes += 2 * (size_t)e.chunk * e.fw_mat * S;            // F, W
  if (e.pair) bytes += 2 * (size_t)e.chunk * e.fw_mat * S;  // F2, W2
  bytes += (size_t)e.chunk * 2 * e.nb * e.nb * 2 * C;     // Tinv
  if (e.tc) bytes += (size_t)e.chunk * kTtPlanes * e.nb * e.nb * 4;  // -T^T split planes
  bytes += (size_t)e.chunk * e.N * 2 * sizeof(float);     // Re A_jj as double-float
  bytes += 2 * (size_t)e.chunk * e.N * sizeof(int);       // piv, perm
  bytes += (size_t)e.B * sizeof(double) * (3 + e.N);      // ld, d_z, tr, gd
  bytes += (size_t)e.N * sizeof(double) * 7 + 256;        // eps, phi, m, v, g, in, misc
  e.bytes = bytes;
  return SCA_OK;
}

template <typename T>
static sca_status dev_alloc(T** p, size_t bytes, Engine& e, const char* what) {
  cudaError_t err = cudaMalloc((void**)p, std::max<size_t>(bytes, 16));
  if (err != cudaSuccess) {
    (void)cudaGetLastError();
    release(e);
    set_error(std::string("cudaMalloc failed for ") + what + " (" + std::to_string(bytes) +
              " bytes): " + cudaGetErrorString(err));
    return SCA_ENOMEM;
  }
  return SCA_OK;
}

sca_status allocate(Engine& e) {
  const size_t S = e.fp64 ? 8 : 4;
  sca_status st;
#define SCA_ALLOC(ptr, bytes, what) \
  if ((st = dev_alloc(&(ptr), (bytes), e, what)) != SCA_OK) return st;
  SCA_ALLOC(e.M, (size_t)e.chunk * e.mat_stride * S, "blocks");
  SCA_ALLOC(e.F, (size_t)e.chunk * e.fw_mat * S, "F");
  SCA_ALLOC(e.W, (size_t)e.chunk * e.fw_mat * S, "W");
  SCA_ALLOC(e.Tinv, (size_t)e.chunk * 2 * e.nb * e.nb * 2 * S, "Tinv");
  SCA_ALLOC(e.adiag, (size_t)e.chunk * e.N * 2 * sizeof(float), "diagonal table");
  SCA_ALLOC(e.piv, (size_t)e.chunk * e.N * sizeof(int), "piv");
  SCA_ALLOC(e.perm, (size_t)e.chunk * e.N * sizeof(int), "perm");
  SCA_ALLOC(e.flags, 16, "flags");
  SCA_ALLOC(e.ld, (size_t)e.B * sizeof(double), "ld");
  SCA_ALLOC(e.d_z, (size_t)e.B * sizeof(double), "DOS shifts");
  SCA_ALLOC(e.tr, (size_t)e.B * sizeof(double), "traces");
  SCA_ALLOC(e.gd, (size_t)e.B * e.N * sizeof(double), "gd");
  SCA_ALLOC(e.d_phi, (size_t)e.N * sizeof(double), "phi");
  SCA_ALLOC(e.d_m, (size_t)e.N * sizeof(double), "m");
  SCA_ALLOC(e.d_v, (size_t)e.N * sizeof(double), "v");
  SCA_ALLOC(e.d_g, (size_t)e.N * sizeof(double), "g");
  SCA_ALLOC(e.d_status, 8 * sizeof(double), "status");
  SCA_ALLOC(e.d_omega, 8 * sizeof(double), "omega");
  cudaError_t err = cudaMallocHost((void**)&e.h_status, 8 * sizeof(double));
  if (err == cudaSuccess) err = cudaMallocHost((void**)&e.h_flags, sizeof(int));
  if (err != cudaSuccess) { release(e); return cuda_fail(err, "cudaMallocHost"); }
  *e.h_flags = 0;
  err = cudaMemset(e.flags, 0, 16);
  if (err == cudaSuccess) err = cudaMemset(e.d_status, 0, 8 * sizeof(double));
  if (err == cudaSuccess) err = cudaMemset(e.d_m, 0, (size_t)e.N * sizeof(double));
  if (err == cudaSuccess) err = cudaMemset(e.d_v, 0, (size_t)e.N * sizeof(double));
  if (err == cudaSuccess) err = cudaMemset(e.F, 0, (size_t)e.chunk * e.fw_mat * S);
  if (err == cudaSuccess) err = cudaMemset(e.W, 0, (size_t)e.chunk * e.fw_mat * S);
  if (err != cudaSuccess) { release(e); return cuda_fail(err, "cudaMemset"); }
  if (e.tc) SCA_ALLOC(e.tt, (size_t)e.chunk * kTtPlanes * e.nb * e.nb * sizeof(float), "T planes");
  if (e.pair) {
    SCA_ALLOC(e.F2, (size_t)e.chunk * e.fw_mat * S, "F2");
    SCA_ALLOC(e.W2, (size_t)e.chunk * e.fw_mat * S, "W2");
    err = cudaMemset(e.F2, 0, (size_t)e.chunk * e.fw_mat * S);
    if (err == cudaSuccess) err = cudaMemset(e.W2, 0, (size_t)e.chunk * e.fw_mat * S);
    if (err != cudaSuccess) { release(e); return cuda_fail(err, "cudaMemset"); }
  }
  if (e.tc && (st = tc_prepare(e)) != SCA_OK) { release(e); return st; }
#undef SCA_ALLOC
  if ((st = fused_prepare(e)) != SCA_OK) { release(e); return st; }
  if (e.tc && e.piv_blocks > 0) {
    // SMs kept free for the pivoted group (SCA_SM_RESERVE overrides the default)
    int r = e.N > 2048 ? kLargeNSmReserve : kDefaultSmReserve;
    if (const char* v = std::getenv("SCA_SM_RESERVE")) r = std::atoi(v);
    e.sm_reserve = std::max(0, std::min(r, tc_sms(e) / 2));
  }
  {  // the pivoted group is the latency-bound chain: its stream takes the highest priority
    int least = 0, greatest = 0;
    err = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (err == cudaSuccess) err = cudaStreamCreateWithPriority(&e.side, cudaStreamNonBlocking, greatest);
  }
  if (err == cudaSuccess) err = cudaEventCreateWithFlags(&e.ev_fork, cudaEventDisableTiming);
  if (err == cudaSuccess) err = cudaEventCreateWithFlags(&e.ev_join, cudaEventDisableTiming);
  if (err == cudaSuccess && e.tc) err = cudaStreamCreateWithFlags(&e.aux, cudaStreamNonBlocking);
  if (err == cudaSuccess && e.tc) err = cudaEventCreateWithFlags(&e.ev_aux0, cudaEventDisableTiming);
  if (err == cudaSuccess && e.tc) err = cudaEventCreateWithFlags(&e.ev_aux1, cudaEventDisableTiming);
  if (err != cudaSuccess) { release(e); return cuda_fail(err, "side stream"); }
  err = cudaEventCreateWithFlags(&e.ev_join2, cudaEventDisableTiming);
  if (err != cudaSuccess) { release(e); return cuda_fail(err, "join event"); }
  if (e.tc && e.piv_blocks > 0 && e.N >= 1024 && e.N <= 2048 && e.B - e.piv_blocks >= 64) {
    // merged pairs: one partition of 16 SMs (8 if refused); otherwise two dominant partitions
    // (mode 3), one if the driver refuses the second; ordinary streams if it refuses both
    if (e.pair) {
      if (!partition_setup(e, kDefaultPartitionSmsPaired, 1))
        (void)partition_setup(e, kDefaultPartitionSms, 1);
    } else if (!partition_setup(e, kDefaultPartitionSms, 3)) {
      (void)partition_setup(e, kDefaultPartitionSms, 1);
    }
  }
  return SCA_OK;
}

void prof_begin(Engine& e, int kind, cudaStream_t s) {
  Profiler* p = e.prof;
  if (!p || !p->on) return;
  if (p->used + 2 > p->npool) {  // grow the event pool
    const int n = std::max(64, 2 * p->npool);
    cudaEvent_t* np = (cudaEvent_t*)std::realloc(p->pool, sizeof(cudaEvent_t) * n);
    if (!np) return;
    p->pool = np;
    for (int k = p->npool; k < n; ++k) cudaEventCreate(&p->pool[k]);
    p->npool = n;
  }
  if (p->nrec + 1 > p->cap) {
    const int n = std::max(32, 2 * p->cap);
    Profiler::Rec* nr = (Profiler::Rec*)std::realloc(p->recs, sizeof(Profiler::Rec) * n);
    if (!nr) return;
    p->recs = nr;
    p->cap = n;
  }
  Profiler::Rec& r = p->recs[p->nrec++];
  r.kind = kind;
  r.a = p->pool[p->used++];
  r.b = p->pool[p->used++];
  r.s = s;
  cudaEventRecord(r.a, s);
}

int prof_span_begin(Engine& e, int kind, cudaStream_t s) {
  Profiler* p = e.prof;
  if (!p || !p->on) return -1;
  prof_begin(e, kind, s);
  return p->nrec - 1;
}

void prof_span_end(Engine& e, int rec, cudaStream_t s) {
  Profiler* p = e.prof;
  if (!p || !p->on || rec < 0 || rec >= p->nrec) return;
  cudaEventRecord(p->recs[rec].b, s);
}

void prof_end(Engine& e, int kind, cudaStream_t s) {
  Profiler* p = e.prof;
  if (!p || !p->on || p->nrec == 0) return;
  Profiler::Rec& r = p->recs[p->nrec - 1];
  if (r.kind == kind) cudaEventRecord(r.b, s);
}

// Names of the kinds in the timeline file (SCA_PROFILE_TRACE), in KernelKind order.
static const char* const kKindNames[kKinds] = {
    "assemble", "panel", "swap", "trinv", "prep", "update", "refine", "reduce", "diag",
    "update_piv", "fused", "span_pivoted", "span_dominant", "panel_update", "prep_piv",
    "update_cross"};

void prof_collect(Engine& e) {
  Profiler* p = e.prof;
  if (!p) return;
  // optional timeline: one line per launch (kind, stream index, start and duration in ms
  // from the first record of this collection), appended to the file SCA_PROFILE_TRACE names
  FILE* tf = nullptr;
  if (const char* path = std::getenv("SCA_PROFILE_TRACE"))
    if (*path && p->nrec > 0) tf = std::fopen(path, "a");
  std::vector<cudaStream_t> streams;
  if (tf) std::fprintf(tf, "# collection of %d records: kind stream start_ms dur_ms\n", p->nrec);
  for (int k = 0; k < p->nrec; ++k) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p->recs[k].a, p->recs[k].b) == cudaSuccess) {
      p->ms[p->recs[k].kind] += ms;
      p->n[p->recs[k].kind] += 1;
      float t0 = 0.f;
      if (tf && cudaEventElapsedTime(&t0, p->recs[0].a, p->recs[k].a) == cudaSuccess) {
        size_t si = 0;
        while (si < streams.size() && streams[si] != p->recs[k].s) ++si;
        if (si == streams.size()) streams.push_back(p->recs[k].s);
        std::fprintf(tf, "%s %zu %.4f %.4f\n", kKindNames[p->recs[k].kind], si, t0, ms);
      }
    }
  }
  if (tf) std::fclose(tf);
  (void)cudaGetLastError();
  p->nrec = 0;
  p->used = 0;
}

void prof_free(Engine& e) {
  Profiler* p = e.prof;
  if (!p) return;
  for (int k = 0; k < p->npool; ++k) cudaEventDestroy(p->pool[k]);
  std::free(p->pool);
  std::free(p->recs);
  delete p;
  e.prof = nullptr;
}

void release(Engine& e) {
  prof_free(e);
  tc_release(e);
  fused_release(e);
  partition_release(e);
  if (e.ev_join2) cudaEventDestroy(e.ev_join2);
  e.ev_join2 = nullptr;
  if (e.side) { cudaStreamSynchronize(e.side); cudaStreamDestroy(e.side); }
  if (e.ev_fork) cudaEventDestroy(e.ev_fork);
  if (e.ev_join) cudaEventDestroy(e.ev_join);
  if (e.aux) { cudaStreamSynchronize(e.aux); cudaStreamDestroy(e.aux); }
  if (e.ev_aux0) cudaEventDestroy(e.ev_aux0);
  if (e.ev_aux1) cudaEventDestroy(e.ev_aux1);
  e.side = e.aux = nullptr;
  e.ev_fork = e.ev_join = e.ev_aux0 = e.ev_aux1 = nullptr;
  void* ptrs[] = {e.M, e.F, e.W, e.F2, e.W2, e.Tinv, e.tt, e.adiag, e.piv, e.perm, e.flags, e.ld,
                  e.d_z, e.tr, e.gd, e.eps_extra, e.d_phi, e.d_m, e.d_v, e.d_g, e.d_status,
                  e.d_omega};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (e.h_status) cudaFreeHost(e.h_status);
  if (e.h_flags) cudaFreeHost(e.h_flags);
  e.h_flags = nullptr;
  e.M = e.F = e.W = e.F2 = e.W2 = e.Tinv = nullptr;
  e.tt = nullptr;
  e.adiag = nullptr;
  e.piv = e.perm = e.flags = nullptr;
  e.d_z = e.tr = nullptr;
  e.ld = e.gd = e.eps_extra = e.d_phi = e.d_m = e.d_v = e.d_g = e.d_status = e.d_omega = nullptr;
  e.h_status = nullptr;
}

}  // namespace sca

using namespace sca;

namespace sca {

sca_status sync_status(sca_ctx* c, cudaStream_t s) {
  cudaError_t err = cudaMemcpyAsync(c->e.h_status, c->e.d_status, 8 * sizeof(double),
                                    cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(c->e.h_flags, c->e.flags, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  if (err != cudaSuccess) return cuda_fail(err, "status read-back");
  prof_collect(c->e);
  return SCA_OK;
}

sca_status check_finite(sca_ctx* c) {
  if ((((int)c->e.h_status[6]) & 2) || (*c->e.h_flags & 2)) {
    set_error("a bounded device-side wait ran out");
    return SCA_ETIMEOUT;
  }
  if (c->e.h_status[4] != 0.0) {
    set_error("non-finite Omega or gradient, or a singular block");
    return SCA_ENONFINITE;
  }
  return SCA_OK;
}

sca_status upload_phi(sca_ctx* c, const double* phi_host) {
  if (!phi_host) { set_error("phi is NULL"); return SCA_EINVAL; }
  cudaError_t err = cudaMemcpyAsync(c->d_in, phi_host, sizeof(double) * c->e.N,
                                    cudaMemcpyHostToDevice, c->stream);
  if (err != cudaSuccess) return cuda_fail(err, "phi upload");
  return SCA_OK;
}

AdamStep adam_step_args(const sca_adam& a, int32_t step) {
  AdamStep as;
  const double bc1 = 1.0 - std::pow(a.beta1, (double)step);
  const double bc2 = 1.0 - std::pow(a.beta2, (double)step);
  as.lr_over_bc1 = a.lr / bc1;
  as.sqrt_bc2 = std::sqrt(bc2);
  as.beta1 = a.beta1;
  as.beta2 = a.beta2;
  as.eps = a.eps;
  as.grad_tol = a.grad_tol;
  return as;
}

}  // namespace sca

extern "C" {

sca_status sca_workspace_bytes(const sca_params* params, uint64_t* bytes) {
  sca_status st = validate(params);
  if (st != SCA_OK) return st;
  if (!bytes) { set_error("bytes is NULL"); return SCA_EINVAL; }
  Engine e;
  plan(*params, e);
  *bytes = e.bytes;
  return SCA_OK;
}

sca_status sca_create(const sca_params* params, sca_ctx** out) {
  sca_status st = validate(params);
  if (st != SCA_OK) return st;
  if (!out) { set_error("out is NULL"); return SCA_EINVAL; }
  *out = nullptr;
  sca_ctx* c = new (std::nothrow) sca_ctx();
  if (!c) { set_error("host allocation failed"); return SCA_ENOMEM; }
  plan(*params, c->e);
  if ((st = allocate(c->e)) != SCA_OK) { delete c; return st; }
  cudaError_t err = cudaMalloc((void**)&c->d_in, sizeof(double) * c->e.N);
  if (err != cudaSuccess) { release(c->e); delete c; return cuda_fail(err, "cudaMalloc phi"); }
  err = cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking);
  c->stream = c->own;
  if (err != cudaSuccess) {
    cudaFree(c->d_in);
    release(c->e);
    delete c;
    return cuda_fail(err, "cudaStreamCreate");
  }
  *out = c;
  return SCA_OK;
}

void sca_destroy(sca_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->own) cudaStreamDestroy(c->own);
  if (c->d_in) cudaFree(c->d_in);
  if (c->d_prop) cudaFree(c->d_prop);
  if (c->d_metro) cudaFree(c->d_metro);
  if (c->d_mtrace) cudaFree(c->d_mtrace);
  release(c->e);
  delete c;
}

sca_status sca_set_site_energy(sca_ctx* c, const double* eps_extra_host) {
  if (!c) { set_error("ctx is NULL"); return SCA_EINVAL; }
  if (!eps_extra_host) {
    if (c->e.eps_extra) { cudaStreamSynchronize(c->stream); cudaFree(c->e.eps_extra); }
    c->e.eps_extra = nullptr;
    return SCA_OK;
  }
  cudaError_t err = cudaSuccess;
  if (!c->e.eps_extra) err = cudaMalloc((void**)&c->e.eps_extra, sizeof(double) * c->e.N);
  if (err == cudaSuccess)
    err = cudaMemcpy(c->e.eps_extra, eps_extra_host, sizeof(double) * c->e.N, cudaMemcpyHostToDevice);
  if (err != cudaSuccess) return cuda_fail(err, "site energy upload");
  return SCA_OK;
}

sca_status sca_forward_dev(sca_ctx* c, const double* d_phi, double* d_omega, void* stream) {
  if (!c || !d_phi || !d_omega) { set_error("NULL argument"); return SCA_EINVAL; }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  c->kept = false;
  sca_status st = run_blocks(c->e, d_phi, true, s, /*refine_stage=*/false);
  if (st != SCA_OK) return st;
  if ((st = run_reduce(c->e, d_phi, d_omega, nullptr, nullptr, s)) != SCA_OK) return st;
  c->kept = (c->e.chunk == c->e.B);
  c->kept_phi = d_phi;
  return SCA_OK;
}

sca_status sca_backward_dev(sca_ctx* c, const double* d_phi, double* d_grad, void* stream) {
  if (!c || !d_phi || !d_grad) { set_error("NULL argument"); return SCA_EINVAL; }
  if (!c->kept || d_phi != c->kept_phi) {
    set_error("sca_backward_dev needs the resident inverses of a preceding sca_forward_dev "
              "with the same d_phi");
    return SCA_ENOSTATE;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  c->kept = false;
  sca_status st = run_refine_resident(c->e, d_phi, s);
  if (st != SCA_OK) return st;
  return run_reduce(c->e, d_phi, c->e.d_omega, d_grad, nullptr, s);
}

sca_status sca_potential_dev(sca_ctx* c, const double* d_phi, double* d_omega, void* stream) {
  if (!c || !d_phi || !d_omega) { set_error("NULL argument"); return SCA_EINVAL; }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  c->kept = false;
  sca_status st = run_blocks(c->e, d_phi, false, s);
  if (st != SCA_OK) return st;
  return run_reduce(c->e, d_phi, d_omega, nullptr, nullptr, s);
}

sca_status sca_grad_dev(sca_ctx* c, const double* d_phi, double* d_omega, double* d_grad,
                        void* stream) {
  if (!c || !d_phi || !d_omega || !d_grad) { set_error("NULL argument"); return SCA_EINVAL; }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  c->kept = false;
  sca_status st = run_blocks(c->e, d_phi, true, s);
  if (st != SCA_OK) return st;
  return run_reduce(c->e, d_phi, d_omega, d_grad, nullptr, s);
}

sca_status sca_potential(sca_ctx* c, const double* phi_host, double* omega) {
  NvtxRange range("sca_potential");
  if (!c || !omega) { set_error("NULL argument"); return SCA_EINVAL; }
  sca_status st = upload_phi(c, phi_host);
  if (st != SCA_OK) return st;
  if ((st = sca_potential_dev(c, c->d_in, c->e.d_omega, c->stream)) != SCA_OK) return st;
  if ((st = sync_status(c, c->stream)) != SCA_OK) return st;
  *omega = c->e.h_status[0];
  return check_finite(c);
}

sca_status sca_grad(sca_ctx* c, const double* phi_host, double* omega, double* grad) {
  NvtxRange range("sca_grad");
  if (!c || !omega || !grad) { set_error("NULL argument"); return SCA_EINVAL; }
  sca_status st = upload_phi(c, phi_host);
  if (st != SCA_OK) return st;
  if ((st = sca_grad_dev(c, c->d_in, c->e.d_omega, c->e.d_g, c->stream)) != SCA_OK) return st;
  cudaError_t err = cudaMemcpyAsync(grad, c->e.d_g, sizeof(double) * c->e.N,
                                    cudaMemcpyDeviceToHost, c->stream);
  if (err != cudaSuccess) return cuda_fail(err, "grad read-back");
  if ((st = sync_status(c, c->stream)) != SCA_OK) return st;
  *omega = c->e.h_status[0];
  return check_finite(c);
}

sca_status sca_blocks(sca_ctx* c, const double* phi_host, double* ld, double* gdiag) {
  if (!c || !ld) { set_error("NULL argument"); return SCA_EINVAL; }
  sca_status st = upload_phi(c, phi_host);
  if (st != SCA_OK) return st;
  const bool g = gdiag != nullptr;
  c->kept = false;
  if ((st = run_blocks(c->e, c->d_in, g, c->stream)) != SCA_OK) return st;
  if ((st = run_reduce(c->e, c->d_in, c->e.d_omega, g ? c->e.d_g : nullptr, nullptr,
                       c->stream)) != SCA_OK)
    return st;
  cudaError_t err = cudaMemcpyAsync(ld, c->e.ld, sizeof(double) * c->e.B, cudaMemcpyDeviceToHost,
                                    c->stream);
  if (err == cudaSuccess && g)
    err = cudaMemcpyAsync(gdiag, c->e.gd, sizeof(double) * c->e.B * c->e.N,
                          cudaMemcpyDeviceToHost, c->stream);
  if (err != cudaSuccess) return cuda_fail(err, "block read-back");
  if ((st = sync_status(c, c->stream)) != SCA_OK) return st;
  return check_finite(c);
}

sca_status sca_dos(sca_ctx* c, const double* phi_host, const double* w_host, int32_t n_w,
                   double eta, double* rho_out) {
  NvtxRange range("sca_dos");
  if (!c || !w_host || !rho_out || n_w < 1 || !(eta > 0.0) || !std::isfinite(eta)) {
    set_error("sca_dos: need ctx, w and rho_out, n_w >= 1 and a finite eta > 0");
    return SCA_EINVAL;
  }
  for (int32_t k = 0; k < n_w; ++k)
    if (!std::isfinite(w_host[k])) {
      set_error("sca_dos: non-finite frequency");
      return SCA_EINVAL;
    }
  sca_status st = upload_phi(c, phi_host);
  if (st != SCA_OK) return st;
  Engine& e = c->e;
  c->kept = false;
  const int half = e.B / 2;
  std::vector<double> hz((size_t)e.B), htr((size_t)e.B);
  // Every resolvent has Im z = eta: columns are strictly diagonally dominant (and the
  // elimination pivot-free) only when eta > 4|t|.
  const int saved = e.piv_blocks;
  const double thr = 4.0 * std::fabs(e.p.t) * (1.0 + 1e-3);
  e.piv_blocks = (e.nopiv || eta > thr) ? 0 : e.B;
  e.dos_mode = true;
  for (int32_t k0 = 0; k0 < n_w && st == SCA_OK; k0 += half) {
    const int cnt = std::min<int>(half, n_w - k0);
    for (int n = 0; n < half; ++n) {  // a short last batch repeats its last frequency
      hz[2 * n] = w_host[k0 + std::min(n, cnt - 1)] + e.p.mu;
      hz[2 * n + 1] = eta;
    }
    cudaError_t err = cudaMemcpyAsync(e.d_z, hz.data(), sizeof(double) * e.B,
                                      cudaMemcpyHostToDevice, c->stream);
    if (err != cudaSuccess) { st = cuda_fail(err, "DOS shifts upload"); break; }
    if ((st = run_blocks(e, c->d_in, true, c->stream, false)) != SCA_OK) break;
    err = cudaMemcpyAsync(htr.data(), e.tr, sizeof(double) * e.B, cudaMemcpyDeviceToHost,
                          c->stream);
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(e.h_flags, e.flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(c->stream);
    if (err != cudaSuccess) { st = cuda_fail(err, "DOS read-back"); break; }
    prof_collect(e);
    if (*e.h_flags != 0) {
      set_error("sca_dos: a singular resolvent or a non-finite pivot");
      st = SCA_ENONFINITE;
      break;
    }
    for (int n = 0; n < cnt; ++n) {
      rho_out[k0 + n] = -htr[2 * n] / (M_PI * e.N);
      rho_out[n_w + k0 + n] = -htr[2 * n + 1] / (M_PI * e.N);
    }
  }
  e.dos_mode = false;
  e.piv_blocks = saved;
  return st;
}

sca_status sca_debug_assemble(sca_ctx* c, const double* phi_host, int32_t b0, int32_t count,
                              double* out) {
  if (!c || !out) { set_error("NULL argument"); return SCA_EINVAL; }
  if (b0 < 0 || count < 1 || b0 + count > c->e.B || count > c->e.chunk) {
    set_error("block range out of bounds");
    return SCA_EINVAL;
  }
  sca_status st = upload_phi(c, phi_host);
  if (st != SCA_OK) return st;
  c->kept = false;
  if ((st = run_assemble_only(c->e, c->d_in, b0, count, c->stream)) != SCA_OK) return st;
  const int N = c->e.N;
  const size_t S = c->e.fp64 ? 8 : 4;
  const size_t bytes = (size_t)count * c->e.mat_stride * S;
  char* h = (char*)std::malloc(bytes);
  if (!h) { set_error("host allocation failed"); return SCA_ENOMEM; }
  cudaError_t err = cudaMemcpyAsync(h, c->e.M, bytes, cudaMemcpyDeviceToHost, c->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(c->stream);
  if (err != cudaSuccess) { std::free(h); return cuda_fail(err, "assemble read-back"); }
  for (int m = 0; m < count; ++m)
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) {
        const size_t o = (size_t)m * c->e.mat_stride + (size_t)i * c->e.ldm + j;
        const size_t q = o + c->e.plane_stride;
        double vr, vi;
        if (c->e.fp64) { vr = ((double*)h)[o]; vi = ((double*)h)[q]; }
        else { vr = ((float*)h)[o]; vi = ((float*)h)[q]; }
        out[2 * (((size_t)m * N + i) * N + j)] = vr;
        out[2 * (((size_t)m * N + i) * N + j) + 1] = vi;
      }
  std::free(h);
  return SCA_OK;
}

sca_status sca_adam_init(sca_ctx* c, const sca_adam* adam, const double* phi0_host) {
  if (!c) { set_error("ctx is NULL"); return SCA_EINVAL; }
  sca_status st = validate_adam(adam);
  if (st != SCA_OK) return st;
  cudaError_t err;
  if (phi0_host) {
    err = cudaMemcpyAsync(c->e.d_phi, phi0_host, sizeof(double) * c->e.N, cudaMemcpyHostToDevice,
                          c->stream);
    if (err != cudaSuccess) return cuda_fail(err, "phi0 upload");
  } else if ((st = run_seed_phi(c->e.d_phi, c->e.N, adam->seed, c->stream)) != SCA_OK) {
    return st;
  }
  err = cudaMemsetAsync(c->e.d_m, 0, sizeof(double) * c->e.N, c->stream);
  if (err == cudaSuccess) err = cudaMemsetAsync(c->e.d_v, 0, sizeof(double) * c->e.N, c->stream);
  if (err == cudaSuccess) err = cudaMemsetAsync(c->e.d_status, 0, 8 * sizeof(double), c->stream);
  if (err == cudaSuccess) err = cudaMemsetAsync(c->e.flags, 0, 16, c->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(c->stream);
  if (err != cudaSuccess) return cuda_fail(err, "adam init");
  c->adam = *adam;
  c->adam_ready = true;
  c->step = 0;
  return SCA_OK;
}

}  // extern "C"

namespace sca {
// Enqueues `n` Adam iterations (gradient + gated update) without synchronising.
sca_status enqueue_adam(sca_ctx* c, int32_t n) {
  c->kept = false;
  if (fused_eligible(c->e)) {  // small blocks: up to kMaxFusedSteps iterations per launch
    while (n > 0) {
      const int32_t k = std::min<int32_t>(n, kMaxFusedSteps);
      AdamStep st[kMaxFusedSteps];
      for (int32_t j = 0; j < k; ++j) st[j] = adam_step_args(c->adam, c->step + 1 + j);
      sca_status r = run_fused_adam(c->e, k, st, true, c->stream);
      if (r != SCA_OK) return r;
      c->step += k;
      n -= k;
    }
    return SCA_OK;
  }
  for (int32_t k = 0; k < n; ++k) {
    const AdamStep as = adam_step_args(c->adam, c->step + 1);
    sca_status st = run_blocks(c->e, c->e.d_phi, true, c->stream);
    if (st != SCA_OK) return st;
    if ((st = run_reduce(c->e, c->e.d_phi, c->e.d_omega, nullptr, &as, c->stream)) != SCA_OK)
      return st;
    c->step += 1;
  }
  return SCA_OK;
}

// Gated Adam on the context's resident state until max|g| < grad_tol or max_steps updates.
// The device gates each update on max|g| >= grad_tol and counts the updates it applied
// (status[5]); once converged phi no longer moves, so batches may overshoot safely.  On return
// h_status holds Omega and max|g| at the final phi and *applied the updates of this call.
sca_status run_adam_gated(sca_ctx* c, int32_t max_steps, int32_t* applied) {
  sca_status st = sync_status(c, c->stream);
  if (st != SCA_OK) return st;
  const double base = c->e.h_status[5];
  const int32_t batch = 16;
  int32_t launched = 0;
  bool converged = false;
  while (launched < max_steps && !converged) {
    const int32_t n = std::min(batch, max_steps - launched);
    if ((st = enqueue_adam(c, n)) != SCA_OK) return st;
    launched += n;
    if ((st = sync_status(c, c->stream)) != SCA_OK) return st;
    if ((st = check_finite(c)) != SCA_OK) return st;
    converged = c->e.h_status[5] - base < (double)launched;
  }
  const double done = c->e.h_status[5] - base;
  if (!converged) {  // Omega and max|g| at the final phi
    if ((st = run_blocks(c->e, c->e.d_phi, true, c->stream)) != SCA_OK) return st;
    if ((st = run_reduce(c->e, c->e.d_phi, c->e.d_omega, c->e.d_g, nullptr, c->stream)) != SCA_OK)
      return st;
    if ((st = sync_status(c, c->stream)) != SCA_OK) return st;
    if ((st = check_finite(c)) != SCA_OK) return st;
  }
  *applied = (int32_t)done;
  return SCA_OK;
}

// Omega and max|g| at the current phi (no update), synchronised into h_status.
sca_status final_eval(sca_ctx* c) {
  sca_status st = run_blocks(c->e, c->e.d_phi, true, c->stream);
  if (st != SCA_OK) return st;
  if ((st = run_reduce(c->e, c->e.d_phi, c->e.d_omega, c->e.d_g, nullptr, c->stream)) != SCA_OK)
    return st;
  if ((st = sync_status(c, c->stream)) != SCA_OK) return st;
  return check_finite(c);
}
}  // namespace sca

extern "C" {

sca_status sca_adam_step(sca_ctx* c, int32_t nsteps, double* omega, double* gmax) {
  NvtxRange range("sca_adam_step");
  if (!c) { set_error("ctx is NULL"); return SCA_EINVAL; }
  if (!c->adam_ready) { set_error("sca_adam_init has not been called"); return SCA_ENOSTATE; }
  if (nsteps < 1) { set_error("nsteps must be >= 1"); return SCA_EINVAL; }
  // Plain Adam: no convergence gate for explicit steps.
  const double tol = c->adam.grad_tol;
  c->adam.grad_tol = 0.0;
  sca_status st = enqueue_adam(c, nsteps);
  c->adam.grad_tol = tol;
  if (st != SCA_OK) return st;
  if ((st = sync_status(c, c->stream)) != SCA_OK) return st;
  if (omega) *omega = c->e.h_status[0];
  if (gmax) *gmax = c->e.h_status[1];
  return check_finite(c);
}

sca_status sca_get_phi(sca_ctx* c, double* phi_out) {
  if (!c || !phi_out) { set_error("NULL argument"); return SCA_EINVAL; }
  cudaError_t err = cudaMemcpyAsync(phi_out, c->e.d_phi, sizeof(double) * c->e.N,
                                    cudaMemcpyDeviceToHost, c->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(c->stream);
  if (err != cudaSuccess) return cuda_fail(err, "phi read-back");
  return SCA_OK;
}

sca_status sca_get_state(sca_ctx* c, double* phi, double* m, double* v, int32_t* step) {
  if (!c) { set_error("ctx is NULL"); return SCA_EINVAL; }
  const size_t nb = sizeof(double) * c->e.N;
  cudaError_t err = cudaSuccess;
  if (phi) err = cudaMemcpyAsync(phi, c->e.d_phi, nb, cudaMemcpyDeviceToHost, c->stream);
  if (err == cudaSuccess && m) err = cudaMemcpyAsync(m, c->e.d_m, nb, cudaMemcpyDeviceToHost, c->stream);
  if (err == cudaSuccess && v) err = cudaMemcpyAsync(v, c->e.d_v, nb, cudaMemcpyDeviceToHost, c->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(c->stream);
  if (err != cudaSuccess) return cuda_fail(err, "state read-back");
  if (step) *step = c->step;
  return SCA_OK;
}

sca_status sca_set_state(sca_ctx* c, const sca_adam* adam, const double* phi, const double* m,
                         const double* v, int32_t step) {
  if (!c || !phi || !m || !v) { set_error("NULL argument"); return SCA_EINVAL; }
  sca_status st = validate_adam(adam);
  if (st != SCA_OK) return st;
  if (step < 0) { set_error("step must be >= 0"); return SCA_EINVAL; }
  const size_t nb = sizeof(double) * c->e.N;
  cudaError_t err = cudaMemcpyAsync(c->e.d_phi, phi, nb, cudaMemcpyHostToDevice, c->stream);
  if (err == cudaSuccess) err = cudaMemcpyAsync(c->e.d_m, m, nb, cudaMemcpyHostToDevice, c->stream);
  if (err == cudaSuccess) err = cudaMemcpyAsync(c->e.d_v, v, nb, cudaMemcpyHostToDevice, c->stream);
  if (err == cudaSuccess) err = cudaMemsetAsync(c->e.d_status, 0, 8 * sizeof(double), c->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(c->stream);
  if (err != cudaSuccess) return cuda_fail(err, "state upload");
  c->adam = *adam;
  c->adam_ready = true;
  c->step = step;
  return SCA_OK;
}

sca_status sca_solve(const sca_params* params, const sca_adam* adam, const double* phi0_host,
                     double* phi_out, double* omega, int32_t* steps, double* gmax) {
  NvtxRange range("sca_solve");
  sca_status st = validate_adam(adam);
  if (st != SCA_OK) return st;
  sca_ctx* c = nullptr;
  if ((st = sca_create(params, &c)) != SCA_OK) return st;
  if ((st = sca_adam_init(c, adam, phi0_host)) != SCA_OK) { sca_destroy(c); return st; }
  int32_t applied = 0;
  if ((st = run_adam_gated(c, adam->max_steps, &applied)) != SCA_OK) { sca_destroy(c); return st; }
  if (omega) *omega = c->e.h_status[0];
  if (gmax) *gmax = c->e.h_status[1];
  if (steps) *steps = applied;
  if (phi_out) st = sca_get_phi(c, phi_out);
  sca_destroy(c);
  return st;
}

sca_status sca_adam_run(sca_ctx* c, int32_t max_steps, int32_t* steps, double* omega,
                        double* gmax) {
  NvtxRange range("sca_adam_run");
  if (!c) { set_error("ctx is NULL"); return SCA_EINVAL; }
  if (!c->adam_ready) { set_error("sca_adam_init has not been called"); return SCA_ENOSTATE; }
  if (max_steps < 0) { set_error("max_steps must be >= 0"); return SCA_EINVAL; }
  int32_t applied = 0;
  sca_status st = run_adam_gated(c, max_steps, &applied);
  if (st != SCA_OK) return st;
  if (steps) *steps = applied;
  if (omega) *omega = c->e.h_status[0];
  if (gmax) *gmax = c->e.h_status[1];
  return SCA_OK;
}

sca_status sca_set_stream(sca_ctx* c, void* stream) {
  if (!c) { set_error("ctx is NULL"); return SCA_EINVAL; }
  cudaError_t err = cudaStreamSynchronize(c->stream);
  if (err != cudaSuccess) return cuda_fail(err, "stream switch");
  c->stream = stream ? static_cast<cudaStream_t>(stream) : c->own;
  return SCA_OK;
}

sca_status sca_set_wait_limit(sca_ctx* c, int64_t cycles) {
  if (!c || cycles < 0) { set_error("bad context or wait limit"); return SCA_EINVAL; }
  c->e.wait_cycles = cycles ? (long long)cycles : 4000000000ll;
  return SCA_OK;
}

sca_status sca_set_pivoting(sca_ctx* c, int32_t mode) {
  if (!c || (mode != SCA_PIVOT_PARTIAL && mode != SCA_PIVOT_NONE)) {
    set_error("bad context or pivoting mode");
    return SCA_EINVAL;
  }
  c->e.piv_blocks = (mode == SCA_PIVOT_NONE) ? 0 : c->e.piv_planned;
  c->e.nopiv = (mode == SCA_PIVOT_NONE);
  return SCA_OK;
}

sca_status sca_set_panel_precision(sca_ctx* c, int32_t prec) {
  if (!c || (prec != SCA_PREC_FP64 && prec != SCA_PREC_FP32) ||
      (c->e.fp64 && prec != SCA_PREC_FP64)) {
    set_error("bad context or panel precision (SCA_PREC_FP32 or SCA_PREC_FP64; float64 blocks "
              "take only SCA_PREC_FP64)");
    return SCA_EINVAL;
  }
  c->e.panel_fp64 = !c->e.fp64 && prec == SCA_PREC_FP64;
  return SCA_OK;
}

sca_status sca_set_sm_partition(sca_ctx* c, int32_t pivoted_sms, int32_t mode) {
  if (!c || pivoted_sms < 0 ||
      (pivoted_sms > 0 && mode != SCA_PARTITION_DOMINANT && mode != SCA_PARTITION_BOTH &&
       mode != SCA_PARTITION_ALTERNATE)) {
    set_error("bad context, SM count or partition mode");
    return SCA_EINVAL;
  }
  cudaError_t err = cudaStreamSynchronize(c->stream);
  if (err != cudaSuccess) return cuda_fail(err, "partition change");
  partition_release(c->e);
  if (pivoted_sms == 0) return SCA_OK;
  if (!c->e.tc) {
    set_error("SM partitions need the tensor-core path (3xTF32 or BF16x3)");
    return SCA_EINVAL;
  }
  if (!partition_setup(c->e, pivoted_sms, mode)) {
    set_error("green-context SM partition unavailable or refused");
    return SCA_ECUDA;
  }
  return SCA_OK;
}

sca_status sca_sm_partition(sca_ctx* c, int32_t* pivoted_sms, int32_t* dominant_sms) {
  if (!c) { set_error("ctx is NULL"); return SCA_EINVAL; }
  if (pivoted_sms) *pivoted_sms = c->e.dom ? c->e.part_sms[0] : 0;
  if (dominant_sms) *dominant_sms = c->e.dom ? c->e.part_sms[1] : 0;
  return SCA_OK;
}

sca_status sca_profile_enable(sca_ctx* c, int32_t enable) {
  if (!c) { set_error("ctx is NULL"); return SCA_EINVAL; }
  if (!c->e.prof) {
    c->e.prof = new (std::nothrow) Profiler();
    if (!c->e.prof) { set_error("host allocation failed"); return SCA_ENOMEM; }
  }
  cudaStreamSynchronize(c->stream);
  prof_collect(c->e);
  c->e.prof->on = enable != 0;
  for (int k = 0; k < kKinds; ++k) { c->e.prof->ms[k] = 0.0; c->e.prof->n[k] = 0; }
  return SCA_OK;
}

sca_status sca_profile_read(sca_ctx* c, int32_t kind, double* total_ms, uint64_t* launches) {
  if (!c || kind < 0 || kind >= kKinds) { set_error("bad context or kernel kind"); return SCA_EINVAL; }
  cudaError_t err = cudaStreamSynchronize(c->stream);
  if (err != cudaSuccess) return cuda_fail(err, "profile read");
  prof_collect(c->e);
  if (total_ms) *total_ms = c->e.prof ? c->e.prof->ms[kind] : 0.0;
  if (launches) *launches = c->e.prof ? c->e.prof->n[kind] : 0;
  return SCA_OK;
}

double sca_flops_per_grad(const sca_params* p) {
  if (!p) return 0.0;
  const double N = (double)p->L * p->L;
  return 8.0 * N * N * N * 2.0 * p->n_omega;
}

int32_t sca_pivoted_blocks(const sca_params* p) {
  if (validate(p) != SCA_OK) return -1;
  Engine e;
  plan(*p, e);
  return e.piv_blocks;
}

const char* sca_last_error(void) { return t_err.c_str(); }

const char* sca_version(void) { return "sca-gb300 0.1 (sm_103a)"; }

uint64_t sca_kernel_launches(void) { return g_launches.load(); }

}  // extern "C"
