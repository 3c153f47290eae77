// Device helpers shared by the CUDA translation units of the SCA library.
#pragma once

#include <cuda_runtime.h>

namespace sca {

constexpr double kPi = 3.14159265358979323846;

template <typename C>
struct cpx {
  C re, im;
};

template <typename C>
__device__ __forceinline__ cpx<C> cmul(cpx<C> a, cpx<C> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}

// Physics of one block slot when several requests share a pass (size-bucket batching):
// block (n, sg) of a request with its own field, site energies, t, Delta_eff, mu and T.
struct BlockDesc {
  const double* phi;
  const double* eps_extra;
  double t, delta_eff, mu, T;
  int n, sg;
};

struct Lattice {
  int L, N;
  double t, delta_eff, mu, T;
  const double* phi;
  const double* eps_extra;
  const double* zshift;  // null: z_n = mu + i omega_n; else z_n = zshift[2n] + i zshift[2n+1]
  const BlockDesc* bd;   // null: slot b is block (b >> 1, sigma = b & 1 ? -1 : +1) of one set
};

// The lattice of slot b and its frequency index n and spin sg.
__device__ __forceinline__ Lattice block_lattice(const Lattice& la, int b, int& n, int& sg) {
  if (!la.bd) {
    n = b >> 1;
    sg = (b & 1) ? -1 : 1;
    return la;
  }
  const BlockDesc d = la.bd[b];
  Lattice l = la;
  l.t = d.t; l.delta_eff = d.delta_eff; l.mu = d.mu; l.T = d.T;
  l.phi = d.phi; l.eps_extra = d.eps_extra;
  n = d.n;
  sg = d.sg;
  return l;
}

__device__ __forceinline__ double site_energy(const Lattice& la, int i, int sg) {
  const int x = i / la.L, y = i - x * la.L;
  const double s = ((x + y) & 1) ? -1.0 : 1.0;
  return -s * la.delta_eff + (la.eps_extra ? la.eps_extra[i] : 0.0) - sg * la.phi[i];
}


struct dsf {
  float h, l;
};
__device__ __forceinline__ dsf two_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ dsf two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dsf fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ dsf ds_add(dsf x, dsf y) {
  const dsf s = two_sum(x.h, y.h);
  return fast_two_sum(s.h, s.l + x.l + y.l);
}
__device__ __forceinline__ dsf ds_sub(dsf x, dsf y) { return ds_add(x, {-y.h, -y.l}); }
__device__ __forceinline__ dsf ds_mul(dsf x, dsf y) {
  const dsf p = two_prod(x.h, y.h);
  return fast_two_sum(p.h, p.l + (x.h * y.l + x.l * y.h));
}
__device__ __forceinline__ dsf ds_of(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}


// sum_k 0.5 ln(mag2[k]) over k < n: logs in parallel, then a pairwise reduction in a fixed
// order (deterministic); every thread gets the sum.  Flags non-positive / non-finite moduli.
template <int NT>
__device__ double logdet_sum(double* mag2, int n, int* flags) {
  for (int k = threadIdx.x; k < n; k += NT) {
    const double m = mag2[k];
    const bool ok = (m > 0.0) && isfinite(m);
    if (!ok) atomicOr(flags, 1);
    mag2[k] = 0.5 * log(ok ? m : 1.0);
  }
  __syncthreads();
  // pairwise sums in a fixed order (float64 adds are a slow pipe here: a serial chain of n
  // of them by one thread would cost more than the logs)
  int w = 1;
  while (w < n) w <<= 1;
  for (int h = w >> 1; h > 0; h >>= 1) {
    for (int k = threadIdx.x; k < h; k += NT)
      if (k + h < n) mag2[k] += mag2[k + h];
    __syncthreads();
  }
  const double total = n > 0 ? mag2[0] : 0.0;
  __syncthreads();  // every thread has read the sum before the caller reuses the buffer
  return total;
}


}  // namespace sca
