// Fused persistent Adam kernel for small blocks (N = L^2 up to 144 in float32, 64 in float64):
// one cooperative launch runs up to kMaxFusedSteps Adam iterations of the whole batch.
//
// Per iteration every CTA takes blocks b = blockIdx.x, blockIdx.x + gridDim.x, ... and, with
// the block in shared memory,
//   assembles A_b = (i w_n + mu) I - H_sigma(phi) (Eq. 1, Eq. 2),
//   inverts it by Gauss-Jordan with partial pivoting (row of largest |z|^2, first on ties),
//   ln|det A_b| = sum ln|pivot| (float64), G_ii from the inverse (float32 blocks: one
//   refinement step 2 x_i - x^T A x in double-float arithmetic, as in the blocked path),
// then all CTAs meet at a grid barrier; CTA 0 reduces Omega and the gradient in a fixed order
// and applies the gated Adam update; a second barrier publishes phi.  Grid barriers spin on a
// global generation counter with a clock64 limit: a time-out sets bit 2 of the flags word
// (SCA_ETIMEOUT on the host) and every CTA leaves.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>

#include "sca_device.cuh"
#include "sca_internal.h"

namespace sca {
namespace {

constexpr int FT = 512;                            // threads per CTA

struct FusedArgs {
  int L, N, B, ksteps, do_adam;
  double t, delta_eff, mu, T, U;
  const double* eps_extra;
  double *phi, *m, *v, *g, *gd, *ld, *status;
  unsigned* bar;  // [0] arrivals, [1] generation
  int* flags;
  long long wait_cycles;
  double beta1, beta2, eps, grad_tol;
  double step[kMaxFusedSteps], sbc2[kMaxFusedSteps];
};

// Grid-wide barrier over all CTAs of a cooperative launch, bounded.
__device__ bool grid_sync(const FusedArgs& a) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = a.bar + 1;
    const unsigned g0 = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(a.bar, 1u) + 1u;
    int ok = 1;
    if (arrived == gridDim.x) {
      a.bar[0] = 0;
      __threadfence();
      atomicAdd(a.bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*gen == g0) {
        if (*(volatile int*)a.flags & 2) { ok = 0; break; }
        if (clock64() - t0 > a.wait_cycles) {
          atomicOr(a.flags, 2);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <typename S>
__device__ void solve_block(const FusedArgs& a, int b, unsigned char* smem) {
  const int N = a.N, L = a.L;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = FT / 32;
  const int n = b >> 1, sg = (b & 1) ? -1 : 1;
  const double w = (2.0 * n + 1.0) * kPi * a.T;
  cpx<S>* Mb = reinterpret_cast<cpx<S>*>(smem);                 // N x N
  cpx<S>* prow = Mb + N * N;                                     // N
  cpx<S>* pcol = prow + N;                                       // N
  double* piv2 = reinterpret_cast<double*>(pcol + N);            // N
  int* perm = reinterpret_cast<int*>(piv2 + N);                  // N
  cpx<S>* rows = reinterpret_cast<cpx<S>*>(perm + ((N + 3) & ~3));  // nwarps x N
  __shared__ double red_v[FT / 32];
  __shared__ int red_i[FT / 32];
  __shared__ int s_p;
  // ---- assemble
  for (int e = tid; e < N * N; e += FT) Mb[e] = {(S)0, (S)0};
  __syncthreads();
  for (int i = tid; i < N; i += FT) {
    const int x = i / L, y = i - x * L;
    const int nb4[4] = {((x + 1) % L) * L + y, ((x + L - 1) % L) * L + y, x * L + (y + 1) % L,
                        x * L + (y + L - 1) % L};
    for (int k = 0; k < 4; ++k) Mb[i * N + nb4[k]].re += (S)a.t;  // bonds accumulate (L = 2)
    const double s = ((x + y) & 1) ? -1.0 : 1.0;
    const double h = -s * a.delta_eff + (a.eps_extra ? a.eps_extra[i] : 0.0) - sg * a.phi[i];
    Mb[i * N + i] = {(S)(a.mu - h), (S)w};
    perm[i] = i;
  }
  __syncthreads();
  // ---- Gauss-Jordan with partial pivoting, in place: leaves R = (P A)^{-1}
  for (int c = 0; c < N; ++c) {
    double best = -1.0;
    int bi = N;
    for (int r = c + tid; r < N; r += FT) {
      const cpx<S> z = Mb[r * N + c];
      const double v = (double)z.re * z.re + (double)z.im * z.im;
      if (v > best) { best = v; bi = r; }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const double ov = __shfl_down_sync(0xffffffffu, best, off);
      const int oi = __shfl_down_sync(0xffffffffu, bi, off);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { red_v[warp] = best; red_i[warp] = bi; }
    __syncthreads();
    if (warp == 0) {
      best = (lane < nwarps) ? red_v[lane] : -1.0;
      bi = (lane < nwarps) ? red_i[lane] : N;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
      }
      if (lane == 0) s_p = (bi < N) ? bi : c;
    }
    __syncthreads();
    const int p = s_p;
    if (p != c) {
      for (int j = tid; j < N; j += FT) {
        const cpx<S> t = Mb[c * N + j];
        Mb[c * N + j] = Mb[p * N + j];
        Mb[p * N + j] = t;
      }
      if (tid == 0) {
        const int t = perm[c];
        perm[c] = perm[p];
        perm[p] = t;
      }
    }
    __syncthreads();
    const cpx<S> d = Mb[c * N + c];
    const S m2 = d.re * d.re + d.im * d.im;
    const cpx<S> dinv = (m2 > (S)0) ? cpx<S>{d.re / m2, -d.im / m2} : cpx<S>{(S)0, (S)0};
    if (tid == 0) piv2[c] = (double)d.re * d.re + (double)d.im * d.im;
    for (int j = tid; j < N; j += FT) {
      prow[j] = (j == c) ? dinv : cmul(Mb[c * N + j], dinv);
      pcol[j] = Mb[j * N + c];
    }
    __syncthreads();
    for (int r = warp; r < N; r += nwarps)
      for (int j = lane; j < N; j += 32) {
        cpx<S>& x = Mb[r * N + j];
        if (r == c) {
          x = prow[j];
        } else if (j == c) {
          const cpx<S> q = cmul(pcol[r], dinv);
          x = {-q.re, -q.im};
        } else {
          const cpx<S> l = pcol[r], u = prow[j];
          x.re -= l.re * u.re - l.im * u.im;
          x.im -= l.re * u.im + l.im * u.re;
        }
      }
    __syncthreads();
  }
  {
    const double s = logdet_sum<FT>(piv2, N, a.flags);
    if (tid == 0) a.ld[b] = s;
  }
  // ---- diag(G): X[i, perm[r]] = R[i, r]; float32 blocks get one refinement step
  cpx<S>* x = rows + (size_t)warp * N;
  const dsf w2 = ds_of(2.0 * w), t2 = ds_of(2.0 * a.t);
  for (int i = warp; i < N; i += nwarps) {
    for (int r = lane; r < N; r += 32) x[perm[r]] = Mb[i * N + r];
    __syncwarp();
    double gii;
    if (sizeof(S) == 8) {
      gii = (double)x[i].re;
    } else {
      dsf acc = {0.f, 0.f};
      for (int j = lane; j < N; j += 32) {
        const int xx = j / L, yy = j - xx * L;
        const int jx = (xx + 1 == L) ? yy : j + L;
        const int jy = (yy + 1 == L) ? j + 1 - L : j + 1;
        const double s = ((xx + yy) & 1) ? -1.0 : 1.0;
        const double h = -s * a.delta_eff + (a.eps_extra ? a.eps_extra[j] : 0.0) - sg * a.phi[j];
        const dsf ajj = ds_of(a.mu - h);
        const float ar = (float)x[j].re, bq = (float)x[j].im;
        const float ax = (float)x[jx].re, bx = (float)x[jx].im;
        const float ay = (float)x[jy].re, by = (float)x[jy].im;
        const dsf q = ds_sub(two_prod(ar, ar), two_prod(bq, bq));
        const dsf ab = two_prod(ar, bq);
        const dsf u = ds_add(ds_sub(two_prod(ar, ax), two_prod(bq, bx)),
                             ds_sub(two_prod(ar, ay), two_prod(bq, by)));
        acc = ds_add(acc, ds_add(ds_sub(ds_mul(ajj, q), ds_mul(w2, ab)), ds_mul(t2, u)));
      }
      double qs = (double)acc.h + (double)acc.l;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) qs += __shfl_xor_sync(0xffffffffu, qs, off);
      gii = 2.0 * (double)x[i].re - qs;
    }
    if (lane == 0) a.gd[(size_t)b * N + i] = sg * gii;
    __syncwarp();
  }
  __syncthreads();
}

// CTA 0: Omega, gradient and the gated Adam update (same arithmetic as the blocked path).
__device__ void reduce_adam(const FusedArgs& a, int it) {
  __shared__ double s_q[FT], s_gm[FT], s_st[FT], s_ab[FT];
  __shared__ int s_bad;
  __shared__ double s_om;
  const int tid = threadIdx.x, N = a.N, L = a.L;
  if (tid == 0) s_bad = 0;
  double q = 0.0, gm = 0.0, st = 0.0, ab = 0.0;
  bool bad = false;
  for (int i = tid; i < N; i += FT) {
    const double ph = a.phi[i];
    const int x = i / L, y = i - x * L;
    q += ph * ph;
    st += ((x + y) & 1) ? -ph : ph;
    ab += fabs(ph);
    double acc = 0.0;
    for (int b = 0; b < a.B; ++b) acc += a.gd[(size_t)b * N + i];
    const double g = 2.0 * ph / a.U - 2.0 * a.T * acc;
    if (!isfinite(g)) bad = true;
    gm = fmax(gm, fabs(g));
    a.g[i] = g;
  }
  s_q[tid] = q; s_gm[tid] = gm; s_st[tid] = st; s_ab[tid] = ab;
  __syncthreads();
  if (bad) atomicOr(&s_bad, 1);
  for (int h = FT / 2; h > 0; h >>= 1) {
    if (tid < h) {
      s_q[tid] += s_q[tid + h];
      s_gm[tid] = fmax(s_gm[tid], s_gm[tid + h]);
      s_st[tid] += s_st[tid + h];
      s_ab[tid] += s_ab[tid + h];
    }
    __syncthreads();
  }
  if (tid == 0) {
    double sld = 0.0;
    for (int b = 0; b < a.B; ++b) sld += a.ld[b];
    s_om = s_q[0] / a.U - 2.0 * a.T * sld;
  }
  __syncthreads();
  const double om = s_om;
  const bool nonfinite = s_bad || !isfinite(om) || (*(volatile int*)a.flags & 1);
  const bool update = a.do_adam && !nonfinite && !(s_gm[0] < a.grad_tol);
  if (update)
    for (int i = tid; i < N; i += FT) {
      const double g = a.g[i];
      const double mi = a.beta1 * a.m[i] + (1.0 - a.beta1) * g;
      const double vi = a.beta2 * a.v[i] + (1.0 - a.beta2) * g * g;
      a.m[i] = mi;
      a.v[i] = vi;
      const double denom = sqrt(vi) / a.sbc2[it] + a.eps;
      a.phi[i] = a.phi[i] - a.step[it] * mi / denom;
    }
  if (tid == 0) {
    a.status[0] = om;
    a.status[1] = s_gm[0];
    a.status[2] = fabs(s_st[0] / N);
    a.status[3] = s_ab[0] / N;
    a.status[4] = nonfinite ? 1.0 : 0.0;
    if (update) a.status[5] += 1.0;
    a.status[6] = (double)*(volatile int*)a.flags;
  }
}

template <typename S>
__global__ void __launch_bounds__(FT) k_fused(FusedArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for (int it = 0; it < a.ksteps; ++it) {
    for (int b = blockIdx.x; b < a.B; b += gridDim.x) solve_block<S>(a, b, smem_raw);
    if (!grid_sync(a)) return;
    if (blockIdx.x == 0) reduce_adam(a, it);
    if (!grid_sync(a)) return;
  }
}

size_t fused_smem(int N, bool fp64) {
  const size_t c = fp64 ? 16 : 8;
  return c * ((size_t)N * N + 2 * N) + 8 * (size_t)N + 4 * (size_t)((N + 3) & ~3) +
         c * (size_t)(FT / 32) * N;
}

}  // namespace

bool fused_eligible(const Engine& e) {
  if (const char* v = std::getenv("SCA_FUSED"))
    if (std::atoi(v) == 0) return false;
  if (e.fused_grid <= 0) return false;
  return true;
}

sca_status fused_prepare(Engine& e) {
  e.fused_grid = 0;
  const int nmax = e.fp64 ? 64 : 144;
  if (e.N > nmax) return SCA_OK;
  const size_t sm = fused_smem(e.N, e.fp64);
  cudaError_t err;
  auto kern = e.fp64 ? (void*)k_fused<double> : (void*)k_fused<float>;
  int dev = 0, sms = 0, per = 0;
  if ((err = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(err, "fused set-up");
  if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return cuda_fail(err, "fused set-up");
  // The limit is a property of the kernel shared by every context on a device: set it once per
  // CUDA context to the largest size any eligible problem needs; occupancy below uses this
  // context's size.
  static ContextOnce limit_set[2];
  if (!limit_set[e.fp64 ? 1 : 0].done()) {
    const size_t smax = fused_smem(nmax, e.fp64);
    if ((err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax)) !=
        cudaSuccess) {
      (void)cudaGetLastError();
      return SCA_OK;  // not eligible
    }
    limit_set[e.fp64 ? 1 : 0].mark();
  }
  if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, FT, sm)) != cudaSuccess ||
      per < 1) {
    (void)cudaGetLastError();
    return SCA_OK;
  }
  e.fused_grid = std::min(e.B, per * sms);
  e.fused_smem = sm;
  if ((err = cudaMalloc((void**)&e.fused_bar, 2 * sizeof(unsigned))) != cudaSuccess)
    return cuda_fail(err, "fused barrier");
  if ((err = cudaMemset(e.fused_bar, 0, 2 * sizeof(unsigned))) != cudaSuccess)
    return cuda_fail(err, "fused barrier");
  return SCA_OK;
}

void fused_release(Engine& e) {
  if (e.fused_bar) cudaFree(e.fused_bar);
  e.fused_bar = nullptr;
  e.fused_grid = 0;
}

sca_status run_fused_adam(Engine& e, int nsteps, const AdamStep* steps, bool do_adam,
                          cudaStream_t s) {
  if (nsteps < 1 || nsteps > kMaxFusedSteps) {
    set_error("fused kernel: 1..16 steps per launch");
    return SCA_EINVAL;
  }
  FusedArgs a;
  a.L = e.L;
  a.N = e.N;
  a.B = e.B;
  a.ksteps = nsteps;
  a.do_adam = do_adam ? 1 : 0;
  a.t = e.p.t;
  a.delta_eff = e.delta_eff;
  a.mu = e.p.mu;
  a.T = e.p.T;
  a.U = e.p.U;
  a.eps_extra = e.eps_extra;
  a.phi = e.d_phi;
  a.m = e.d_m;
  a.v = e.d_v;
  a.g = e.d_g;
  a.gd = e.gd;
  a.ld = e.ld;
  a.status = e.d_status;
  a.bar = e.fused_bar;
  a.flags = e.flags;
  a.wait_cycles = e.wait_cycles;
  a.beta1 = steps ? steps[0].beta1 : 0.0;
  a.beta2 = steps ? steps[0].beta2 : 0.0;
  a.eps = steps ? steps[0].eps : 0.0;
  a.grad_tol = steps ? steps[0].grad_tol : 0.0;
  for (int k = 0; k < kMaxFusedSteps; ++k) {
    a.step[k] = (steps && k < nsteps) ? steps[k].lr_over_bc1 : 0.0;
    a.sbc2[k] = (steps && k < nsteps) ? steps[k].sqrt_bc2 : 1.0;
  }
  cudaError_t err = cudaMemsetAsync(e.flags, 0, sizeof(int), s);
  if (err == cudaSuccess) err = cudaMemsetAsync(e.fused_bar, 0, 2 * sizeof(unsigned), s);
  if (err != cudaSuccess) return cuda_fail(err, "fused reset");
  void* args[] = {&a};
  auto kern = e.fp64 ? (void*)k_fused<double> : (void*)k_fused<float>;
  prof_begin(e, kFused, s);
  err = cudaLaunchCooperativeKernel(kern, dim3(e.fused_grid), dim3(FT), args, e.fused_smem, s);
  prof_end(e, kFused, s);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (err != cudaSuccess) return cuda_fail(err, "fused launch");
  return SCA_OK;
}

}  // namespace sca
