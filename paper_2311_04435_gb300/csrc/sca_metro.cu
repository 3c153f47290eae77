// Metropolis sampling of the static-field weight exp(-Omega(phi)/T) of the SCA partition
// function (Sec. II: Z is an integral over phi_1 .. phi_N with weight exp(-beta V); Omega here
// is V).  The chain lives on the device: every step proposes phi' = phi + delta g with g
// standard normal, evaluates Omega(phi') with the LU-only elimination (the log-determinants
// of all blocks), and accepts or rejects in one single-CTA kernel, so a batch of steps needs
// no host round trip.
//
// Random numbers are counter-based, so a chain is reproducible from (seed, step):
//   U(s, k)  = top 53 bits of output k of the SplitMix64 stream started at s, times 2^-53;
//   g_i      = sqrt(-2 ln(1 - U(seed, 2(tN + i)))) cos(2 pi U(seed, 2(tN + i) + 1))
//              (the Box-Muller transform) at global step t;
//   accepted iff U(seed + 1, t) < exp(-(Omega(phi') - Omega(phi)) / T).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "sca_device.cuh"
#include "sca_internal.h"

namespace sca {
namespace {

__device__ __forceinline__ double u01(unsigned long long seed, unsigned long long k) {
  unsigned long long z = seed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return (double)(z >> 11) * 0x1.0p-53;
}

__global__ void k_metro_propose(const double* __restrict__ phi, double* __restrict__ prop, int N,
                                unsigned long long seed, long long step, double delta) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const unsigned long long k = 2ull * ((unsigned long long)step * (unsigned long long)N + i);
  const double u1 = u01(seed, k), u2 = u01(seed, k + 1ull);
  const double g = sqrt(-2.0 * log(1.0 - u1)) * cos(2.0 * kPi * u2);
  prop[i] = phi[i] + delta * g;
}

// Omega(prop) = sum prop^2 / U - 2T sum_b ld_b (fixed-order reductions, as in the gradient's
// reduction); then the Metropolis decision.  init: take prop as the chain's state
// unconditionally (the start field).  metro: [0] Omega of the state, [1] accepted steps,
// [2] Omega of the last proposal, [3] rejected non-finite proposals.  trace (optional):
// Omega of the state after this step and the accept flag (1.0 / 0.0).
constexpr int MT = 1024;
__global__ void __launch_bounds__(MT)
    k_metro_accept(int N, int B, const double* __restrict__ ld, const double* __restrict__ prop,
                   double* __restrict__ phi, double* __restrict__ metro, const int* flags,
                   double U, double T, unsigned long long seed, long long step, int init,
                   double* trace) {
  __shared__ double s_q[MT];
  __shared__ int s_acc;
  const int tid = threadIdx.x;
  double q = 0.0;
  for (int i = tid; i < N; i += MT) q += prop[i] * prop[i];
  s_q[tid] = q;
  __syncthreads();
  for (int h = MT / 2; h > 0; h >>= 1) {
    if (tid < h) s_q[tid] += s_q[tid + h];
    __syncthreads();
  }
  if (tid == 0) {
    double sld = 0.0;
    for (int b = 0; b < B; ++b) sld += ld[b];
    const double om2 = s_q[0] / U - 2.0 * T * sld;
    const bool finite = isfinite(om2) && !(flags && *flags);
    int acc;
    if (init) {
      acc = finite ? 1 : 0;
    } else {
      const double u = u01(seed + 1ull, (unsigned long long)step);
      acc = (finite && u < exp(-(om2 - metro[0]) / T)) ? 1 : 0;
    }
    if (!finite) metro[3] += 1.0;
    metro[2] = om2;
    if (acc) metro[0] = om2;
    if (acc && !init) metro[1] += 1.0;
    if (trace) {
      trace[0] = metro[0];
      trace[1] = acc ? 1.0 : 0.0;
    }
    s_acc = acc;
  }
  __syncthreads();
  if (s_acc && prop != phi)
    for (int i = tid; i < N; i += MT) phi[i] = prop[i];
}

#define SCA_LAUNCH_CHECK(where)                                   \
  do {                                                            \
    g_launches.fetch_add(1, std::memory_order_relaxed);           \
    cudaError_t err__ = cudaGetLastError();                       \
    if (err__ != cudaSuccess) return cuda_fail(err__, where);     \
  } while (0)

sca_status ensure_buffers(sca_ctx* c, int32_t trace_steps) {
  cudaError_t err = cudaSuccess;
  if (!c->d_prop) err = cudaMalloc((void**)&c->d_prop, sizeof(double) * c->e.N);
  if (err == cudaSuccess && !c->d_metro) err = cudaMalloc((void**)&c->d_metro, 4 * sizeof(double));
  if (err == cudaSuccess && trace_steps > c->mtrace_cap) {
    if (c->d_mtrace) {
      cudaStreamSynchronize(c->stream);
      cudaFree(c->d_mtrace);
      c->d_mtrace = nullptr;
      c->mtrace_cap = 0;
    }
    err = cudaMalloc((void**)&c->d_mtrace, sizeof(double) * 2 * (size_t)trace_steps);
    if (err == cudaSuccess) c->mtrace_cap = trace_steps;
  }
  if (err != cudaSuccess) return cuda_fail(err, "Metropolis buffers");
  return SCA_OK;
}

// One step on the context's stream: propose, eliminate (log-determinants only), decide.
sca_status enqueue_metro_step(sca_ctx* c, int init, double* trace) {
  Engine& e = c->e;
  const int N = e.N;
  const double* src = e.d_phi;
  if (!init) {
    k_metro_propose<<<(N + 255) / 256, 256, 0, c->stream>>>(e.d_phi, c->d_prop, N,
                                                           (unsigned long long)c->m_seed,
                                                           (long long)c->m_step, c->m_delta);
    SCA_LAUNCH_CHECK("Metropolis proposal");
    src = c->d_prop;
  }
  sca_status st = run_blocks(e, src, false, c->stream);
  if (st != SCA_OK) return st;
  k_metro_accept<<<1, MT, 0, c->stream>>>(N, e.B, e.ld, src, e.d_phi, c->d_metro, e.flags,
                                          e.p.U, e.p.T, (unsigned long long)c->m_seed,
                                          (long long)c->m_step, init, trace);
  SCA_LAUNCH_CHECK("Metropolis decision");
  if (!init) ++c->m_step;
  return SCA_OK;
}

}  // namespace
}  // namespace sca

using namespace sca;

extern "C" {

sca_status sca_metropolis_init(sca_ctx* c, const double* phi0_host, double delta, uint64_t seed) {
  if (!c || !(delta >= 0.0) || !std::isfinite(delta)) {
    set_error("sca_metropolis_init: need ctx and a finite delta >= 0");
    return SCA_EINVAL;
  }
  sca_status st = ensure_buffers(c, 0);
  if (st != SCA_OK) return st;
  cudaError_t err;
  if (phi0_host) {
    err = cudaMemcpyAsync(c->e.d_phi, phi0_host, sizeof(double) * c->e.N, cudaMemcpyHostToDevice,
                          c->stream);
    if (err != cudaSuccess) return cuda_fail(err, "phi0 upload");
  } else if ((st = run_seed_phi(c->e.d_phi, c->e.N, seed, c->stream)) != SCA_OK) {
    return st;
  }
  err = cudaMemsetAsync(c->d_metro, 0, 4 * sizeof(double), c->stream);
  if (err != cudaSuccess) return cuda_fail(err, "Metropolis state");
  c->kept = false;
  c->m_delta = delta;
  c->m_seed = seed;
  c->m_step = 0;
  if ((st = enqueue_metro_step(c, 1, nullptr)) != SCA_OK) return st;
  double h[4];
  err = cudaMemcpyAsync(h, c->d_metro, sizeof(h), cudaMemcpyDeviceToHost, c->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(c->stream);
  if (err != cudaSuccess) return cuda_fail(err, "Metropolis init");
  if (h[3] != 0.0) {
    set_error("sca_metropolis_init: non-finite Omega at the start field");
    return SCA_ENONFINITE;
  }
  c->metro_ready = true;
  return SCA_OK;
}

sca_status sca_metropolis_step(sca_ctx* c, int32_t n_steps, double* omega_trace,
                               uint8_t* accepted, double* omega, int64_t* accepted_total) {
  if (!c || n_steps < 0) {
    set_error("sca_metropolis_step: need ctx and n_steps >= 0");
    return SCA_EINVAL;
  }
  if (!c->metro_ready) {
    set_error("sca_metropolis_step before sca_metropolis_init");
    return SCA_ENOSTATE;
  }
  const bool want_trace = omega_trace || accepted;
  sca_status st = ensure_buffers(c, want_trace ? n_steps : 0);
  if (st != SCA_OK) return st;
  c->kept = false;
  for (int32_t s = 0; s < n_steps; ++s)
    if ((st = enqueue_metro_step(c, 0, want_trace ? c->d_mtrace + 2 * (size_t)s : nullptr)) !=
        SCA_OK)
      return st;
  double h[4];
  std::vector<double> tr(want_trace ? 2 * (size_t)n_steps : 0);
  cudaError_t err = cudaMemcpyAsync(h, c->d_metro, sizeof(h), cudaMemcpyDeviceToHost, c->stream);
  if (err == cudaSuccess && want_trace && n_steps > 0)
    err = cudaMemcpyAsync(tr.data(), c->d_mtrace, sizeof(double) * tr.size(),
                          cudaMemcpyDeviceToHost, c->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(c->stream);
  if (err != cudaSuccess) return cuda_fail(err, "Metropolis read-back");
  prof_collect(c->e);
  for (int32_t s = 0; s < n_steps && want_trace; ++s) {
    if (omega_trace) omega_trace[s] = tr[2 * (size_t)s];
    if (accepted) accepted[s] = tr[2 * (size_t)s + 1] != 0.0 ? 1 : 0;
  }
  if (omega) *omega = h[0];
  if (accepted_total) *accepted_total = (int64_t)h[1];
  if (h[3] != 0.0) {
    set_error("sca_metropolis_step: a proposal gave a non-finite Omega (rejected)");
    return SCA_ENONFINITE;
  }
  return SCA_OK;
}

}  // extern "C"
