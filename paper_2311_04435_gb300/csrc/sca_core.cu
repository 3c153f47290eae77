// Blocked Gauss-Jordan / LU engine for the SCA blocks A_{n,sigma} = (i w_n + mu) I - H_sigma(phi)
// (arXiv 2311.04435, Eq. 1 and Eq. 2), CUDA-core kernels for sm_103a.
//
// One Omega/gradient evaluation runs, for every resident block, N/nb steps of
//   panel  : pivoted LU of the m x nb column panel (partial pivoting, |z|^2 argmax by warp
//            shuffles), ln|u_kk| accumulated in float64
//   swap   : the panel's row interchanges applied to the other columns
//   trinv  : inv(L11), inv(U11) of the nb x nb pivot block
//   prep   : the rank-nb factors F (N x nb) and W^T (N x nb)
//   update : M <- mask(M) - F W  (CUDA cores here; tcgen05 3xTF32 in sca_tc.cu)
// With the Gauss-Jordan factors (gradient) the sweep leaves R = (P A)^{-1} in place, so
// X = A^{-1} has X[i, perm[r]] = R[i, r]; with the LU factors (potential only) the update is
// restricted to the trailing block.  Then
//   refine : G_ii = 2 X_ii - (X A X^T)_ii with the exact sparse A in float64 (reduced
//            precisions) or G_ii = X_ii (float64), stored as sigma Re G_ii
//   reduce : Omega = sum phi^2/U - 2T sum_b ld_b, g_i = 2 phi_i/U - 2T sum_b sigma Re G_b,ii,
//            in a fixed order, fused with the Adam update.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>

#include "sca_internal.h"

namespace sca {

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr size_t kRefineSmem = 208 * 1024;

template <typename C>
struct cpx {
  C re, im;
};

template <typename C>
__device__ __forceinline__ cpx<C> cmul(cpx<C> a, cpx<C> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}

struct Lattice {
  int L, N;
  double t, delta_eff, mu, T;
  const double* phi;
  const double* eps_extra;
};

__device__ __forceinline__ double site_energy(const Lattice& la, int i, int sg) {
  const int x = i / la.L, y = i - x * la.L;
  const double s = ((x + y) & 1) ? -1.0 : 1.0;
  return -s * la.delta_eff + (la.eps_extra ? la.eps_extra[i] : 0.0) - sg * la.phi[i];
}

// ------------------------------------------------------------------ assemble
// A_b = (i w_n + mu) I - H_sigma(phi), b = 2n + s (Eq. 1 hopping +t off-diagonal per bond,
// accumulated; diagonal mu - h_i + i w_n with h_i = eps_i - sigma phi_i).
template <typename S>
__global__ void k_assemble(S* M, int ldm, size_t mat_stride, size_t plane_stride, int b0,
                           Lattice la, double* ld, int* perm) {
  const int mat = blockIdx.y, b = b0 + mat, n = b >> 1, sg = (b & 1) ? -1 : 1;
  const int N = la.N, L = la.L;
  const double w = (2.0 * n + 1.0) * kPi * la.T;
  S* re = M + mat * mat_stride;
  S* im = re + plane_stride;
  for (int i = blockIdx.x; i < N; i += gridDim.x) {
    const int x = i / L, y = i - x * L;
    const int jxp = ((x + 1) % L) * L + y, jxm = ((x + L - 1) % L) * L + y;
    const int jyp = x * L + (y + 1) % L, jym = x * L + (y + L - 1) % L;
    const double h = site_energy(la, i, sg);
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
      double v = 0.0, q = 0.0;
      if (j == jxp) v += la.t;
      if (j == jxm) v += la.t;
      if (j == jyp) v += la.t;
      if (j == jym) v += la.t;
      if (j == i) { v = la.mu - h; q = w; }
      re[(size_t)i * ldm + j] = (S)v;
      im[(size_t)i * ldm + j] = (S)q;
    }
  }
  if (blockIdx.x == 0) {
    for (int r = threadIdx.x; r < N; r += blockDim.x) perm[(size_t)mat * N + r] = r;
    if (threadIdx.x == 0) ld[b] = 0.0;
  }
}

// --------------------------------------------------------------------- panel
// Pivoted LU of the column panel rows [k0, N) x cols [k0, k0+kb) of each block, in place.
// One CTA per block.  Pivot: row of largest |z|^2 (first index on ties), found with warp
// shuffles then across warps.  ld[b] += sum ln|u_kk| in float64.
template <typename S, typename C, int NT>
__global__ void __launch_bounds__(NT) k_panel(S* M, int N, int ldm, size_t mat_stride,
                                              size_t plane_stride, int k0, int kb, int b0,
                                              double* ld, int* piv, int* perm, int* flags) {
  const int mat = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  S* re = M + mat * mat_stride;
  S* im = re + plane_stride;
  __shared__ C prow_re[256], prow_im[256];
  __shared__ double red_v[NT / 32];
  __shared__ int red_i[NT / 32];
  __shared__ int s_p;
  double ldacc = 0.0;
  for (int c = 0; c < kb; ++c) {
    const int col = k0 + c;
    double best = -1.0;
    int bi = N;
    for (int r = col + tid; r < N; r += NT) {
      const double a = (double)re[(size_t)r * ldm + col], q = (double)im[(size_t)r * ldm + col];
      const double v = a * a + q * q;
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
      best = (lane < NT / 32) ? red_v[lane] : -1.0;
      bi = (lane < NT / 32) ? red_i[lane] : N;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
      }
      if (lane == 0) s_p = (bi < N) ? bi : col;
    }
    __syncthreads();
    const int p = s_p;
    if (p != col)
      for (int j = tid; j < kb; j += NT) {
        const size_t a = (size_t)col * ldm + k0 + j, q = (size_t)p * ldm + k0 + j;
        const S tr = re[a], ti = im[a];
        re[a] = re[q]; im[a] = im[q];
        re[q] = tr; im[q] = ti;
      }
    if (tid == 0) {
      piv[(size_t)mat * N + col] = p;
      if (p != col) {
        int* pm = perm + (size_t)mat * N;
        const int tmp = pm[col];
        pm[col] = pm[p];
        pm[p] = tmp;
      }
    }
    __syncthreads();
    for (int j = c + tid; j < kb; j += NT) {
      prow_re[j] = (C)re[(size_t)col * ldm + k0 + j];
      prow_im[j] = (C)im[(size_t)col * ldm + k0 + j];
    }
    __syncthreads();
    const double dre = (double)prow_re[c], dim = (double)prow_im[c];
    const double mag2 = dre * dre + dim * dim;
    const bool ok = (mag2 > 0.0) && isfinite(mag2);
    if (tid == 0) {
      if (!ok) atomicOr(flags, 1);
      ldacc += 0.5 * log(ok ? mag2 : 1.0);
    }
    const C ire = ok ? (C)(dre / mag2) : (C)0, iim = ok ? (C)(-dim / mag2) : (C)0;
    for (int r = col + 1 + tid; r < N; r += NT) {
      S* rr = re + (size_t)r * ldm + k0;
      S* ri = im + (size_t)r * ldm + k0;
      const C are = (C)rr[c], aim = (C)ri[c];
      const C lre = are * ire - aim * iim, lim = are * iim + aim * ire;
      rr[c] = (S)lre;
      ri[c] = (S)lim;
      for (int j = c + 1; j < kb; ++j) {
        const C ur = prow_re[j], ui = prow_im[j];
        rr[j] = (S)((C)rr[j] - (lre * ur - lim * ui));
        ri[j] = (S)((C)ri[j] - (lre * ui + lim * ur));
      }
    }
    __syncthreads();
  }
  if (tid == 0) ld[b0 + mat] += ldacc;
}

// ---------------------------------------------------------------------- swap
// Applies the panel's interchanges, in order, to the columns outside the panel
// (columns >= jstart only).
template <typename S>
__global__ void k_swap(S* M, int N, int ldm, size_t mat_stride, size_t plane_stride, int k0,
                       int kb, int jstart, const int* piv) {
  const int mat = blockIdx.y;
  __shared__ int sp[256];
  for (int c = threadIdx.x; c < kb; c += blockDim.x) sp[c] = piv[(size_t)mat * N + k0 + c];
  __syncthreads();
  const int j = jstart + blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N || (j >= k0 && j < k0 + kb)) return;
  S* re = M + mat * mat_stride;
  S* im = re + plane_stride;
  for (int c = 0; c < kb; ++c) {
    const int p = sp[c];
    if (p != k0 + c) {
      const size_t a = (size_t)(k0 + c) * ldm + j, q = (size_t)p * ldm + j;
      const S tr = re[a], ti = im[a];
      re[a] = re[q]; im[a] = im[q];
      re[q] = tr; im[q] = ti;
    }
  }
}

// --------------------------------------------------------------------- trinv
// inv(L11) (unit lower) and inv(U11) (upper) of the kb x kb pivot block, zero padded to
// nb x nb.  Tinv layout per block: [0] = inv(L11), [1] = inv(U11), row-major nb x nb cpx<C>.
template <typename S, typename C>
__global__ void k_trinv(const S* M, int ldm, size_t mat_stride, size_t plane_stride, int k0,
                        int kb, int nb, cpx<C>* Tinv) {
  extern __shared__ unsigned char smem_raw[];
  cpx<C>* blk = reinterpret_cast<cpx<C>*>(smem_raw);  // kb x kb
  cpx<C>* Y = blk + kb * kb;                           // nb x nb
  const int mat = blockIdx.x, tid = threadIdx.x;
  const S* re = M + mat * mat_stride;
  const S* im = re + plane_stride;
  for (int e = tid; e < kb * kb; e += blockDim.x) {
    const int r = e / kb, c = e - r * kb;
    blk[e] = {(C)re[(size_t)(k0 + r) * ldm + k0 + c], (C)im[(size_t)(k0 + r) * ldm + k0 + c]};
  }
  for (int e = tid; e < nb * nb; e += blockDim.x) Y[e] = {(C)0, (C)0};
  __syncthreads();
  cpx<C>* TL = Tinv + (size_t)mat * 2 * nb * nb;
  cpx<C>* TU = TL + nb * nb;
  const int j = tid;
  if (j < kb) {  // column j of inv(L11): forward substitution with unit diagonal
    Y[j * nb + j] = {(C)1, (C)0};
    for (int r = j + 1; r < kb; ++r) {
      cpx<C> s = {(C)0, (C)0};
      for (int c = j; c < r; ++c) {
        const cpx<C> t = cmul(blk[r * kb + c], Y[c * nb + j]);
        s.re += t.re; s.im += t.im;
      }
      Y[r * nb + j] = {-s.re, -s.im};
    }
  }
  __syncthreads();
  for (int e = tid; e < nb * nb; e += blockDim.x) TL[e] = Y[e];
  __syncthreads();
  for (int e = tid; e < nb * nb; e += blockDim.x) Y[e] = {(C)0, (C)0};
  __syncthreads();
  if (j < kb) {  // column j of inv(U11): back substitution
    {
      const cpx<C> d = blk[j * kb + j];
      const C m2 = d.re * d.re + d.im * d.im;
      Y[j * nb + j] = {d.re / m2, -d.im / m2};
    }
    for (int r = j - 1; r >= 0; --r) {
      cpx<C> s = {(C)0, (C)0};
      for (int c = r + 1; c <= j; ++c) {
        const cpx<C> t = cmul(blk[r * kb + c], Y[c * nb + j]);
        s.re += t.re; s.im += t.im;
      }
      const cpx<C> d = blk[r * kb + r];
      const C m2 = d.re * d.re + d.im * d.im;
      const cpx<C> id = {d.re / m2, -d.im / m2};
      const cpx<C> q = cmul(s, id);
      Y[r * nb + j] = {-q.re, -q.im};
    }
  }
  __syncthreads();
  for (int e = tid; e < nb * nb; e += blockDim.x) TU[e] = Y[e];
}

// ---------------------------------------------------------------------- prep
// Rank-nb factors of one elimination step, written K-contiguous (N x nb, planar):
//   Gauss-Jordan: F = [ M[i<k0, K] inv(U11) ; -inv(U11) ; M[i>=k0+kb, K] (= L21) ],
//                 W^T[j] = (inv(L11) M[K, j])^T for j outside K, inv(L11)[:, j-k0] for j in K;
//   LU:           F = L21 rows only, W^T[j] for j >= k0+kb only.
// Then M' = mask(M) - F W (mask zeroes row block K and column block K for Gauss-Jordan).
// With `split`, planes are {re_hi, im_hi, re_lo, im_lo}: hi = value with the low 13
// mantissa bits cleared (exact TF32), lo = value - hi.
// W additionally carries -im (hi, lo) in planes 4 and 5 for the tensor-core complex product.
template <typename S>
__device__ __forceinline__ void store_fw(S* base, size_t plane, size_t off, double vre, double vim,
                                         bool split, bool neg) {
  if (!split) {
    base[off] = (S)vre;
    base[plane + off] = (S)vim;
  } else {
    const float fr = (float)vre, fi = (float)vim;
    const float hr = __uint_as_float(__float_as_uint(fr) & 0xffffe000u);
    const float hi = __uint_as_float(__float_as_uint(fi) & 0xffffe000u);
    float* b = reinterpret_cast<float*>(base);
    b[off] = hr;
    b[plane + off] = hi;
    b[2 * plane + off] = fr - hr;
    b[3 * plane + off] = fi - hi;
    if (neg) {
      b[4 * plane + off] = -hi;
      b[5 * plane + off] = -(fi - hi);
    }
  }
}

template <typename S, typename C, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
    k_prep(const S* M, int N, int ldm, size_t mat_stride, size_t plane_stride, int k0, int kb,
           int nb, const cpx<C>* Tinv, S* F, S* W, size_t fw_plane, size_t fw_mat, int gj,
           int split) {
  extern __shared__ unsigned char smem_raw[];
  cpx<C>* T = reinterpret_cast<cpx<C>*>(smem_raw);  // nb x nb
  const int mat = blockIdx.y, which = blockIdx.z;   // 0: F rows, 1: W rows
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const S* re = M + mat * mat_stride;
  const S* im = re + plane_stride;
  const cpx<C>* TL = Tinv + (size_t)mat * 2 * nb * nb;
  const cpx<C>* TU = TL + nb * nb;
  // F uses inv(U11) as stored ([c'][c]); W uses inv(L11) transposed ([c'][c] = invL[c][c']).
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    if (which == 0) {
      T[e] = TU[e];
    } else {
      const int cp = e / nb, c = e - cp * nb;
      T[e] = TL[c * nb + cp];
    }
  }
  __syncthreads();
  S* out = (which == 0 ? F : W) + (size_t)mat * fw_mat;
  const int row = blockIdx.x * WARPS + warp;
  if (row >= N) return;
  const int kend = k0 + kb;
  const size_t obase = (size_t)row * nb;
  if (!gj && row < kend) return;  // LU: only trailing rows / columns are used
  for (int c = lane; c < nb; c += 32) {
    double vre = 0.0, vim = 0.0;
    if (c < kb) {
      if (which == 0) {
        if (row < k0) {
          cpx<C> s = {(C)0, (C)0};
          for (int cp = 0; cp < kb; ++cp) {
            const cpx<C> x = {(C)re[(size_t)row * ldm + k0 + cp], (C)im[(size_t)row * ldm + k0 + cp]};
            const cpx<C> t = cmul(x, T[cp * nb + c]);
            s.re += t.re; s.im += t.im;
          }
          vre = (double)s.re; vim = (double)s.im;
        } else if (row < kend) {
          const cpx<C> t = T[(row - k0) * nb + c];
          vre = -(double)t.re; vim = -(double)t.im;
        } else {
          vre = (double)re[(size_t)row * ldm + k0 + c];
          vim = (double)im[(size_t)row * ldm + k0 + c];
        }
      } else {
        if (row >= k0 && row < kend) {
          const cpx<C> t = T[(row - k0) * nb + c];  // invL[c][row-k0]
          vre = (double)t.re; vim = (double)t.im;
        } else {
          cpx<C> s = {(C)0, (C)0};
          for (int cp = 0; cp < kb; ++cp) {
            const cpx<C> x = {(C)re[(size_t)(k0 + cp) * ldm + row], (C)im[(size_t)(k0 + cp) * ldm + row]};
            const cpx<C> t = cmul(T[cp * nb + c], x);
            s.re += t.re; s.im += t.im;
          }
          vre = (double)s.re; vim = (double)s.im;
        }
      }
    }
    store_fw(out, fw_plane, obase + c, vre, vim, split != 0, which == 1);
  }
}

// ------------------------------------------------------------- update (SIMT)
// M[i, j] <- mask(i, j) * M[i, j] - sum_c F[i, c] W[j, c]  for i >= r0, j >= c0.
// 64 x 64 output tile per CTA, 256 threads, 4 x 4 complex accumulators per thread.
template <typename S>
__global__ void __launch_bounds__(256)
    k_update_simt(S* M, int N, int ldm, size_t mat_stride, size_t plane_stride, const S* F,
                  const S* W, int nb, size_t fw_plane, size_t fw_mat, int r0, int c0, int k0,
                  int kb, int gj) {
  constexpr int BM = 64, BN = 64, KC = 16;
  __shared__ S Fs[2][KC][BM + 1];
  __shared__ S Ws[2][KC][BN + 1];
  const int mat = blockIdx.z;
  const int i0 = r0 + blockIdx.y * BM, j0 = c0 + blockIdx.x * BN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const S* Fm = F + (size_t)mat * fw_mat;
  const S* Wm = W + (size_t)mat * fw_mat;
  S acc_re[4][4], acc_im[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) { acc_re[a][b] = 0; acc_im[a][b] = 0; }
  for (int kc = 0; kc < nb; kc += KC) {
    for (int e = threadIdx.x; e < BM * KC; e += 256) {
      const int r = e / KC, k = e - r * KC;
      const int gi = i0 + r, gj2 = j0 + r;
      const bool kin = (kc + k) < nb;
      Fs[0][k][r] = (gi < N && kin) ? Fm[(size_t)gi * nb + kc + k] : (S)0;
      Fs[1][k][r] = (gi < N && kin) ? Fm[fw_plane + (size_t)gi * nb + kc + k] : (S)0;
      Ws[0][k][r] = (gj2 < N && kin) ? Wm[(size_t)gj2 * nb + kc + k] : (S)0;
      Ws[1][k][r] = (gj2 < N && kin) ? Wm[fw_plane + (size_t)gj2 * nb + kc + k] : (S)0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      S fr[4], fi[4], wr[4], wi[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) { fr[a] = Fs[0][k][ty + 16 * a]; fi[a] = Fs[1][k][ty + 16 * a]; }
#pragma unroll
      for (int b = 0; b < 4; ++b) { wr[b] = Ws[0][k][tx + 16 * b]; wi[b] = Ws[1][k][tx + 16 * b]; }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          acc_re[a][b] = fma(fr[a], wr[b], acc_re[a][b]);
          acc_re[a][b] = fma(-fi[a], wi[b], acc_re[a][b]);
          acc_im[a][b] = fma(fr[a], wi[b], acc_im[a][b]);
          acc_im[a][b] = fma(fi[a], wr[b], acc_im[a][b]);
        }
    }
    __syncthreads();
  }
  S* re = M + mat * mat_stride;
  S* im = re + plane_stride;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = i0 + ty + 16 * a;
    if (i >= N) continue;
    const bool rowk = gj && i >= k0 && i < k0 + kb;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int j = j0 + tx + 16 * b;
      if (j >= N) continue;
      const bool keep = !(rowk || (gj && j >= k0 && j < k0 + kb));
      const size_t o = (size_t)i * ldm + j;
      const S mr = keep ? re[o] : (S)0, mi = keep ? im[o] : (S)0;
      re[o] = mr - acc_re[a][b];
      im[o] = mi - acc_im[a][b];
    }
  }
}

// -------------------------------------------------------------------- refine
// Per block and row i: x = row i of X = A^{-1} (X[i, perm[r]] = R[i, r]), then
//   G_ii = 2 x_i - sum_j x_j (A x)_j   (refine; (A x)_j from the 5-point stencil in float64)
//   G_ii = x_i                          (no refinement)
// and gd[b*N + i] = sigma_b Re G_ii.  Refinement: one warp per row, the row scattered into
// natural order in shared memory.  Without refinement: one thread per row reads R[i, pinv[i]].
template <typename S>
__global__ void k_refine(const S* M, int ldm, size_t mat_stride, size_t plane_stride, int b0,
                         Lattice la, const int* perm, double* gd, int refine) {
  extern __shared__ unsigned char smem_raw[];
  const int N = la.N, L = la.L;
  const int mat = blockIdx.y, b = b0 + mat, n = b >> 1, sg = (b & 1) ? -1 : 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  int* sperm = reinterpret_cast<int*>(smem_raw);
  const S* re = M + mat * mat_stride;
  const S* im = re + plane_stride;
  if (!refine) {  // sperm holds the inverse permutation
    for (int r = threadIdx.x; r < N; r += blockDim.x) sperm[perm[(size_t)mat * N + r]] = r;
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
      gd[(size_t)b * N + i] = sg * (double)re[(size_t)i * ldm + sperm[i]];
    return;
  }
  cpx<S>* rows = reinterpret_cast<cpx<S>*>(smem_raw + ((N * sizeof(int) + 15) / 16) * 16);
  cpx<S>* x = rows + (size_t)warp * N;
  for (int r = threadIdx.x; r < N; r += blockDim.x) sperm[r] = perm[(size_t)mat * N + r];
  __syncthreads();
  const double w = (2.0 * n + 1.0) * kPi * la.T;
  for (int i = blockIdx.x * nwarps + warp; i < N; i += gridDim.x * nwarps) {
    for (int r = lane; r < N; r += 32)
      x[sperm[r]] = {re[(size_t)i * ldm + r], im[(size_t)i * ldm + r]};
    __syncwarp();
    double ar = 0.0, ai = 0.0;
    for (int j = lane; j < N; j += 32) {
      const int xx = j / L, yy = j - xx * L;
      const int jxp = ((xx + 1) % L) * L + yy, jxm = ((xx + L - 1) % L) * L + yy;
      const int jyp = xx * L + (yy + 1) % L, jym = xx * L + (yy + L - 1) % L;
      const double dr = la.mu - site_energy(la, j, sg), di = w;  // A_jj
      const double xjr = (double)x[j].re, xji = (double)x[j].im;
      double yr = dr * xjr - di * xji, yi = dr * xji + di * xjr;  // (A x)_j
      yr += la.t * ((double)x[jxp].re + (double)x[jxm].re + (double)x[jyp].re + (double)x[jym].re);
      yi += la.t * ((double)x[jxp].im + (double)x[jxm].im + (double)x[jyp].im + (double)x[jym].im);
      ar += xjr * yr - xji * yi;
      ai += xjr * yi + xji * yr;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      ar += __shfl_xor_sync(0xffffffffu, ar, off);
      ai += __shfl_xor_sync(0xffffffffu, ai, off);
    }
    if (lane == 0) gd[(size_t)b * N + i] = sg * (2.0 * (double)x[i].re - ar);
    __syncwarp();
  }
}

// -------------------------------------------------------------- reduce/Adam
// Omega = sum_i phi_i^2/U - 2T sum_b ld_b ; g_i = 2 phi_i/U - 2T sum_b gd[b, i] (b ascending);
// then, if Adam is on and max|g| >= grad_tol, the update of phi in PyTorch's order
// (m, v, denom = sqrt(v)/sqrt(bc2) + eps, phi -= (lr/bc1) m / denom).  One CTA, fixed-order
// tree reductions, so the result does not depend on what else runs on the device.
// status: [0] Omega [1] max|g| [2] |mean s_i phi_i| [3] mean |phi_i| [4] nonfinite flag
// (all at the phi the gradient was taken at) [5] number of updates applied (accumulates).
constexpr int RT = 1024;
__global__ void __launch_bounds__(RT)
    k_reduce(int N, int L, int B, const double* ld, const double* gd, const double* phi,
             double* phi_out, double* m, double* v, double* g_out, double* omega_out,
             double* status, const int* flags, double U, double T, int want_grad, int do_adam,
             double step, double sbc2, double beta1, double beta2, double eps, double grad_tol) {
  __shared__ double s_q[RT], s_gm[RT], s_st[RT], s_ab[RT];
  __shared__ int s_bad;
  const int tid = threadIdx.x;
  if (tid == 0) s_bad = 0;
  double q = 0.0, gm = 0.0, st = 0.0, ab = 0.0;
  bool bad = false;
  for (int i = tid; i < N; i += RT) {
    const double ph = phi[i];
    const int x = i / L, y = i - x * L;
    q += ph * ph;
    st += ((x + y) & 1) ? -ph : ph;
    ab += fabs(ph);
    if (want_grad) {
      double acc = 0.0;
      for (int b = 0; b < B; ++b) acc += gd[(size_t)b * N + i];
      const double g = 2.0 * ph / U - 2.0 * T * acc;
      if (!isfinite(g)) bad = true;
      gm = fmax(gm, fabs(g));
      g_out[i] = g;
    }
  }
  s_q[tid] = q; s_gm[tid] = gm; s_st[tid] = st; s_ab[tid] = ab;
  __syncthreads();
  if (bad) atomicOr(&s_bad, 1);
  for (int h = RT / 2; h > 0; h >>= 1) {
    if (tid < h) {
      s_q[tid] += s_q[tid + h];
      s_gm[tid] = fmax(s_gm[tid], s_gm[tid + h]);
      s_st[tid] += s_st[tid + h];
      s_ab[tid] += s_ab[tid + h];
    }
    __syncthreads();
  }
  __shared__ double s_om;
  if (tid == 0) {
    double sld = 0.0;
    for (int b = 0; b < B; ++b) sld += ld[b];
    s_om = s_q[0] / U - 2.0 * T * sld;
  }
  __syncthreads();
  const double om = s_om;
  const bool nonfinite = s_bad || !isfinite(om) || (flags && *flags);
  const bool update = do_adam && want_grad && !nonfinite && !(s_gm[0] < grad_tol);
  if (update)
    for (int i = tid; i < N; i += RT) {
      const double g = g_out[i];
      const double mi = beta1 * m[i] + (1.0 - beta1) * g;
      const double vi = beta2 * v[i] + (1.0 - beta2) * g * g;
      m[i] = mi;
      v[i] = vi;
      const double denom = sqrt(vi) / sbc2 + eps;
      phi_out[i] = phi[i] - step * mi / denom;
    }
  if (tid == 0) {
    if (omega_out) *omega_out = om;
    status[0] = om;
    status[1] = s_gm[0];
    status[2] = fabs(s_st[0] / N);
    status[3] = s_ab[0] / N;
    status[4] = nonfinite ? 1.0 : 0.0;
    if (update) status[5] += 1.0;
    status[6] = flags ? (double)*flags : 0.0;
  }
}

__global__ void k_seed_phi(double* phi, int N, unsigned long long seed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  unsigned long long z = seed + (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  phi[i] = (double)(z >> 11) * 0x1.0p-53 - 0.5;
}

Lattice make_lattice(const Engine& e, const double* d_phi) {
  Lattice la;
  la.L = e.L; la.N = e.N; la.t = e.p.t; la.delta_eff = e.delta_eff; la.mu = e.p.mu; la.T = e.p.T;
  la.phi = d_phi; la.eps_extra = e.eps_extra;
  return la;
}

#define SCA_LAUNCH_CHECK(where)                                   \
  do {                                                            \
    g_launches.fetch_add(1, std::memory_order_relaxed);           \
    cudaError_t err__ = cudaGetLastError();                       \
    if (err__ != cudaSuccess) return cuda_fail(err__, where);     \
  } while (0)

template <typename S>
sca_status launch_refine(Engine& e, const Lattice& la, int b0, int cnt, cudaStream_t s) {
  const int N = e.N;
  S* M = static_cast<S*>(e.M);
  const size_t perm_bytes = ((N * sizeof(int) + 15) / 16) * 16;
  prof_begin(e, kRefine, s);
  if (e.refine) {
    const size_t row_bytes = (size_t)N * sizeof(cpx<S>);
    const int warps = (int)std::max<size_t>(1, std::min<size_t>(4, (kRefineSmem - perm_bytes) / row_bytes));
    const int gx = std::max(1, std::min((N + warps - 1) / warps, 64));
    k_refine<S><<<dim3(gx, cnt), warps * 32, perm_bytes + warps * row_bytes, s>>>(
        M, e.ldm, e.mat_stride, e.plane_stride, b0, la, e.perm, e.gd, 1);
  } else {
    const int gx = std::max(1, std::min((N + 255) / 256, 16));
    k_refine<S><<<dim3(gx, cnt), 256, perm_bytes, s>>>(M, e.ldm, e.mat_stride, e.plane_stride,
                                                       b0, la, e.perm, e.gd, 0);
  }
  prof_end(e, kRefine, s);
  SCA_LAUNCH_CHECK("refine");
  return SCA_OK;
}

template <typename S, typename C>
sca_status run_blocks_t(Engine& e, const double* d_phi, bool want_grad, bool refine_stage,
                        cudaStream_t s) {
  const Lattice la = make_lattice(e, d_phi);
  const int N = e.N, nb = e.nb;
  S* M = static_cast<S*>(e.M);
  S* F = static_cast<S*>(e.F);
  S* W = static_cast<S*>(e.W);
  cpx<C>* Tinv = static_cast<cpx<C>*>(e.Tinv);
  cudaError_t err = cudaMemsetAsync(e.flags, 0, sizeof(int), s);
  if (err != cudaSuccess) return cuda_fail(err, "flags reset");
  for (int b0 = 0; b0 < e.B; b0 += e.chunk) {
    const int cnt = std::min(e.chunk, e.B - b0);
    prof_begin(e, kAssemble, s);
    k_assemble<S><<<dim3(N, cnt), 256, 0, s>>>(M, e.ldm, e.mat_stride, e.plane_stride, b0, la,
                                               e.ld, e.perm);
    prof_end(e, kAssemble, s);
    SCA_LAUNCH_CHECK("assemble");
    for (int k0 = 0; k0 < N; k0 += nb) {
      const int kb = std::min(nb, N - k0);
      const int kend = k0 + kb;
      prof_begin(e, kPanel, s);
      k_panel<S, C, 256><<<cnt, 256, 0, s>>>(M, N, e.ldm, e.mat_stride, e.plane_stride, k0, kb,
                                             b0, e.ld, e.piv, e.perm, e.flags);
      prof_end(e, kPanel, s);
      SCA_LAUNCH_CHECK("panel");
      if (!want_grad && kend == N) break;  // LU: nothing trails the last panel
      const int jstart = want_grad ? 0 : kend;
      {
        const int ncols = N - jstart;
        prof_begin(e, kSwap, s);
        k_swap<S><<<dim3((ncols + 255) / 256, cnt), 256, 0, s>>>(M, N, e.ldm, e.mat_stride,
                                                                   e.plane_stride, k0, kb,
                                                                   jstart, e.piv);
        prof_end(e, kSwap, s);
        SCA_LAUNCH_CHECK("swap");
      }
      {
        const size_t sm = sizeof(cpx<C>) * ((size_t)kb * kb + (size_t)nb * nb);
        prof_begin(e, kTrinv, s);
        k_trinv<S, C><<<cnt, nb, sm, s>>>(M, e.ldm, e.mat_stride, e.plane_stride, k0, kb, nb,
                                          Tinv);
        prof_end(e, kTrinv, s);
        SCA_LAUNCH_CHECK("trinv");
      }
      {
        constexpr int WARPS = 8;
        const size_t sm = sizeof(cpx<C>) * (size_t)nb * nb;
        prof_begin(e, kPrep, s);
        k_prep<S, C, WARPS><<<dim3((N + WARPS - 1) / WARPS, cnt, 2), WARPS * 32, sm, s>>>(
            M, N, e.ldm, e.mat_stride, e.plane_stride, k0, kb, nb, Tinv, F, W, e.fw_plane,
            e.fw_mat, want_grad ? 1 : 0, e.tc ? 1 : 0);
        prof_end(e, kPrep, s);
        SCA_LAUNCH_CHECK("prep");
      }
      const int r0 = want_grad ? 0 : kend, c0 = want_grad ? 0 : kend;
      prof_begin(e, kUpdate, s);
      if (e.tc) {
        sca_status st = tc_update(e, cnt, k0, kb, r0, c0, want_grad, s);
        if (st != SCA_OK) return st;
      } else {
        dim3 grid((N - c0 + 63) / 64, (N - r0 + 63) / 64, cnt);
        k_update_simt<S><<<grid, 256, 0, s>>>(M, N, e.ldm, e.mat_stride, e.plane_stride, F, W, nb,
                                              e.fw_plane, e.fw_mat, r0, c0, k0, kb,
                                              want_grad ? 1 : 0);
        SCA_LAUNCH_CHECK("update");
      }
      prof_end(e, kUpdate, s);
    }
    if (want_grad && refine_stage) {
      sca_status st = launch_refine<S>(e, la, b0, cnt, s);
      if (st != SCA_OK) return st;
    }
  }
  return SCA_OK;
}

template <typename S, typename C>
sca_status set_smem_limits() {
  static bool done = false;
  if (done) return SCA_OK;
  cudaError_t err;
  err = cudaFuncSetAttribute(k_trinv<S, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (err != cudaSuccess) return cuda_fail(err, "smem trinv");
  err = cudaFuncSetAttribute(k_prep<S, C, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (err != cudaSuccess) return cuda_fail(err, "smem prep");
  err = cudaFuncSetAttribute(k_refine<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRefineSmem);
  if (err != cudaSuccess) return cuda_fail(err, "smem refine");
  done = true;
  return SCA_OK;
}

}  // namespace

sca_status run_blocks(Engine& e, const double* d_phi, bool want_grad, cudaStream_t s,
                      bool refine_stage) {
  sca_status st;
  if (e.fp64) {
    if ((st = set_smem_limits<double, double>()) != SCA_OK) return st;
    return run_blocks_t<double, double>(e, d_phi, want_grad, refine_stage, s);
  }
  if ((st = set_smem_limits<float, float>()) != SCA_OK) return st;
  return run_blocks_t<float, float>(e, d_phi, want_grad, refine_stage, s);
}

sca_status run_refine_resident(Engine& e, const double* d_phi, cudaStream_t s) {
  if (e.chunk != e.B) {
    set_error("the inverses of all blocks are not resident (chunked workspace)");
    return SCA_ENOSTATE;
  }
  const Lattice la = make_lattice(e, d_phi);
  if (e.fp64) return launch_refine<double>(e, la, 0, e.B, s);
  return launch_refine<float>(e, la, 0, e.B, s);
}

sca_status run_assemble_only(Engine& e, const double* d_phi, int b0, int count, cudaStream_t s) {
  const Lattice la = make_lattice(e, d_phi);
  if (e.fp64)
    k_assemble<double><<<dim3(e.N, count), 256, 0, s>>>(static_cast<double*>(e.M), e.ldm,
                                                         e.mat_stride, e.plane_stride, b0, la,
                                                         e.ld, e.perm);
  else
    k_assemble<float><<<dim3(e.N, count), 256, 0, s>>>(static_cast<float*>(e.M), e.ldm,
                                                        e.mat_stride, e.plane_stride, b0, la,
                                                        e.ld, e.perm);
  SCA_LAUNCH_CHECK("assemble");
  return SCA_OK;
}

sca_status run_reduce(Engine& e, const double* d_phi, double* d_omega, double* d_grad,
                      const AdamStep* adam, cudaStream_t s) {
  const bool want_grad = (d_grad != nullptr) || (adam != nullptr);
  double* g = d_grad ? d_grad : e.d_g;
  prof_begin(e, kReduce, s);
  k_reduce<<<1, RT, 0, s>>>(e.N, e.L, e.B, e.ld, e.gd, d_phi, adam ? e.d_phi : nullptr, e.d_m,
                            e.d_v, g, d_omega, e.d_status, e.flags, e.p.U, e.p.T,
                            want_grad ? 1 : 0, adam ? 1 : 0, adam ? adam->lr_over_bc1 : 0.0,
                            adam ? adam->sqrt_bc2 : 1.0, adam ? adam->beta1 : 0.0,
                            adam ? adam->beta2 : 0.0, adam ? adam->eps : 0.0,
                            adam ? adam->grad_tol : 0.0);
  prof_end(e, kReduce, s);
  SCA_LAUNCH_CHECK("reduce");
  return SCA_OK;
}

sca_status run_seed_phi(double* d_phi, int N, uint64_t seed, cudaStream_t s) {
  k_seed_phi<<<(N + 255) / 256, 256, 0, s>>>(d_phi, N, (unsigned long long)seed);
  SCA_LAUNCH_CHECK("seed_phi");
  return SCA_OK;
}

}  // namespace sca
