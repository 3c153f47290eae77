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
#include <cstdlib>
#include <cstring>

#include <cuda_bf16.h>

#include "sca_internal.h"
#include "sca_device.cuh"

namespace sca {

namespace {

constexpr size_t kRefineSmem = 208 * 1024;

// ------------------------------------------------------------------ assemble
// A_b = (i w_n + mu) I - H_sigma(phi), b = 2n + s (Eq. 1 hopping: +t off-diagonal per bond,
// accumulated; diagonal mu - h_i + i w_n with h_i = eps_i - sigma phi_i).  The blocks are
// zero-filled with cudaMemsetAsync first; this kernel writes the stencil entries of each
// row, one thread per row.
template <typename S>
__global__ void k_assemble(S* M, int ldm, size_t mat_stride, size_t plane_stride, int b0,
                           Lattice la0, double* ld, int* perm) {
  const int mat = blockIdx.y, b = b0 + mat;
  int n, sg;
  const Lattice la = block_lattice(la0, b, n, sg);
  const int N = la.N, L = la.L;
  const double w = la.zshift ? la.zshift[2 * n + 1] : (2.0 * n + 1.0) * kPi * la.T;
  const double zr = la.zshift ? la.zshift[2 * n] : la.mu;
  S* re = M + mat * mat_stride;
  S* im = re + plane_stride;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) {
    const int x = i / L, y = i - x * L;
    const int jxp = ((x + 1) % L) * L + y, jxm = ((x + L - 1) % L) * L + y;
    const int jyp = x * L + (y + 1) % L, jym = x * L + (y + L - 1) % L;
    const size_t row = (size_t)i * ldm;
    // bonds accumulate: for L = 2 the +x and -x neighbours are the same site
    re[row + jxp] += (S)la.t;
    re[row + jxm] += (S)la.t;
    re[row + jyp] += (S)la.t;
    re[row + jym] += (S)la.t;
    re[row + i] = (S)(zr - site_energy(la, i, sg));
    im[row + i] = (S)w;
    perm[(size_t)mat * N + i] = i;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) ld[b] = 0.0;
}

// Zero fill and assembly in one pass, one warp per row (16-byte zero stores): blocks
// [0, full_blocks) get whole rows; the later ones (symmetric dominant blocks, lower tiles
// only) get the columns up to the end of the row's diagonal tile of width `tile`: their
// strictly upper tiles are never read (the refinement reads the lower triangle; only the
// whole-row comparison path has k_mirror fill them first).
template <typename S>
__global__ void __launch_bounds__(256)
    k_assemble_rows(S* M, int ldm, size_t mat_stride, size_t plane_stride, int b0, Lattice la0,
                    double* ld, int* perm, int full_blocks, int tile) {
  const int mat = blockIdx.y, b = b0 + mat;
  int n, sg;
  const Lattice la = block_lattice(la0, b, n, sg);
  const int N = la.N, L = la.L;
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i < N) {
    const int end = mat < full_blocks ? N : min(N, (i / tile + 1) * tile);
    S* rr = M + mat * mat_stride + (size_t)i * ldm;
    S* ri = rr + plane_stride;
    constexpr int V = 16 / (int)sizeof(S);  // N and the tile width are multiples of V
    for (int c = lane * V; c < end; c += 32 * V) {
      *reinterpret_cast<uint4*>(rr + c) = make_uint4(0u, 0u, 0u, 0u);
      *reinterpret_cast<uint4*>(ri + c) = make_uint4(0u, 0u, 0u, 0u);
    }
    __syncwarp();
    if (lane == 0) {
      const double w = la.zshift ? la.zshift[2 * n + 1] : (2.0 * n + 1.0) * kPi * la.T;
      const double zr = la.zshift ? la.zshift[2 * n] : la.mu;
      const int x = i / L, y = i - x * L;
      const int nbr[4] = {((x + 1) % L) * L + y, ((x + L - 1) % L) * L + y, x * L + (y + 1) % L,
                          x * L + (y + L - 1) % L};
      // bonds accumulate: for L = 2 the +x and -x neighbours are the same site
      for (int k = 0; k < 4; ++k)
        if (nbr[k] < end) rr[nbr[k]] += (S)la.t;
      rr[i] = (S)(zr - site_energy(la, i, sg));
      ri[i] = (S)w;
      perm[(size_t)mat * N + i] = i;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) ld[b] = 0.0;
}

// --------------------------------------------------------- panel-local update
// Two-level blocking of the pivoted group: an outer panel of width kbo is factorised by
// shared-memory sub-panels of width kbi; after each sub-panel [s0, s0+kbi) the rest of the outer
// panel (columns [s0+kbi, c_end)) is brought up to date as in a right-looking LU:
//   U12 = inv(L11) A12  (rows [s0, s0+kbi), k_swap_trsm)   then   A22 -= L21 U12  (rows >= s0+kbi).
// k_gemm_panel: A22[r][c] -= sum_k L21[r][k] U12[k][c] for rows r >= s0+kbi (kGemmPanelRows
// per CTA), columns [s0+kbi, c_end), K = kbi <= 16; L21 and U12 staged in shared memory.
constexpr int kGemmPanelRows = 32;
template <typename S, typename C>
__global__ void __launch_bounds__(256)
    k_gemm_panel(S* M, int N, int ldm, size_t mat_stride, size_t plane_stride, int s0, int kbi,
                 int c_end) {
  // columns of the outer panel: nb = 32 on the float64 path, up to 128 with float32 storage
  // (also when the panel computes in float64)
  constexpr int NCMAX = sizeof(S) == 8 ? 64 : 128;
  constexpr int RSTEP = 256 / NCMAX;               // rows covered by one pass of the CTA
  constexpr int MA = kGemmPanelRows / RSTEP;       // A22 entries per thread
  constexpr int MU = 16 / RSTEP;                   // U12 entries per thread
  constexpr int ML = kGemmPanelRows * 16 / 256;    // L21 entries per thread
  __shared__ cpx<C> Us[16][NCMAX];
  __shared__ cpx<C> Ls[kGemmPanelRows][17];
  const int mat = blockIdx.y;
  const int c0 = s0 + kbi, nc = c_end - c0;
  const int r0 = c0 + blockIdx.x * kGemmPanelRows;
  S* re = M + mat * mat_stride;
  S* im = re + plane_stride;
  // a thread owns one column c and every RSTEP-th row; all its global loads are issued before
  // any is used, so a CTA waits one memory round trip instead of one per entry
  const int c = threadIdx.x % NCMAX, rl = threadIdx.x / NCMAX;
  const bool cin = c < nc;
  cpx<C> uv[MU], lv[ML], av[MA];
#pragma unroll
  for (int t = 0; t < MU; ++t) {
    const int k = rl + RSTEP * t;
    if (cin && k < kbi) {
      const size_t o = (size_t)(s0 + k) * ldm + c0 + c;
      uv[t] = {(C)re[o], (C)im[o]};
    }
  }
#pragma unroll
  for (int t = 0; t < ML; ++t) {
    const int e = threadIdx.x + 256 * t;
    const int gr = r0 + (e >> 4), k = e & 15;
    lv[t] = (gr < N && k < kbi)
                ? cpx<C>{(C)re[(size_t)gr * ldm + s0 + k], (C)im[(size_t)gr * ldm + s0 + k]}
                : cpx<C>{(C)0, (C)0};
  }
#pragma unroll
  for (int t = 0; t < MA; ++t) {
    const int gr = r0 + rl + RSTEP * t;
    if (cin && gr < N) {
      const size_t o = (size_t)gr * ldm + c0 + c;
      av[t] = {(C)re[o], (C)im[o]};
    }
  }
#pragma unroll
  for (int t = 0; t < MU; ++t) {
    const int k = rl + RSTEP * t;
    if (cin && k < kbi) Us[k][c] = uv[t];
  }
#pragma unroll
  for (int t = 0; t < ML; ++t) {
    const int e = threadIdx.x + 256 * t;
    Ls[e >> 4][e & 15] = lv[t];
  }
  __syncthreads();
  if (!cin) return;
#pragma unroll
  for (int t = 0; t < MA; ++t) {
    const int r = rl + RSTEP * t, gr = r0 + r;
    if (gr >= N) continue;
    cpx<C> a = av[t];
    for (int k = 0; k < kbi; ++k) {
      const cpx<C> l = Ls[r][k], u = Us[k][c];
      a.re -= l.re * u.re - l.im * u.im;
      a.im -= l.re * u.im + l.im * u.re;
    }
    const size_t o = (size_t)gr * ldm + c0 + c;
    re[o] = (S)a.re;
    im[o] = (S)a.im;
  }
}

// ------------------------------------------------------------ swap + trsm
// The interchanges (s0 + c, sp[c]), c = 0 .. kbi - 1 (kbi <= 16; sp absolute rows) composed into
// one list of row moves over the at most 2 kbi rows they touch: row dst[t] takes the old
// content of row src[t].  One thread.
__device__ int compose_moves(const int* sp, int kbi, int s0, int* mv_dst, int* mv_src) {
  constexpr int TMAX = 16;
  int row[2 * TMAX], from[2 * TMAX], ns = kbi;
  for (int x = 0; x < kbi; ++x) row[x] = s0 + x, from[x] = x;
  for (int cc = 0; cc < kbi; ++cc) {
    const int p = sp[cc];
    if (p == s0 + cc) continue;
    int q = p - s0;
    if (q >= kbi) {
      q = kbi;
      while (q < ns && row[q] != p) ++q;
      if (q == ns) row[ns] = p, from[ns] = ns, ++ns;
    }
    const int t = from[cc];
    from[cc] = from[q];
    from[q] = t;
  }
  int nmv = 0;
  for (int x = 0; x < ns; ++x)
    if (from[x] != x) mv_dst[nmv] = row[x], mv_src[nmv] = row[from[x]], ++nmv;
  return nmv;
}

// Column j outside the sub-panel [s0, s0 + kbi) (kbi <= 16): the composed row moves (every load
// before any store: one memory round trip) and, where trsm is set (the outer panel's columns
// still to be factored), the forward substitution U12 = inv(L11) A12 with the unit-lower L11
// (Ls, row stride lst), in place.
template <typename S, typename C>
__device__ __forceinline__ void swap_trsm_column(S* re, S* im, int ldm, int j, int nmv,
                                                 const int* mv_dst, const int* mv_src,
                                                 const cpx<C>* Ls, int lst, int kbi, int s0,
                                                 bool trsm) {
  constexpr int TMAX = 16;
  S vr[2 * TMAX], vi[2 * TMAX];
#pragma unroll
  for (int t = 0; t < 2 * TMAX; ++t)
    if (t < nmv) {
      const size_t q = (size_t)mv_src[t] * ldm + j;
      vr[t] = re[q];
      vi[t] = im[q];
    }
#pragma unroll
  for (int t = 0; t < 2 * TMAX; ++t)
    if (t < nmv) {
      const size_t a = (size_t)mv_dst[t] * ldm + j;
      re[a] = vr[t];
      im[a] = vi[t];
    }
  if (!trsm) return;
  cpx<C> u[TMAX];
#pragma unroll
  for (int r = 0; r < TMAX; ++r)
    if (r < kbi) {
      const size_t o = (size_t)(s0 + r) * ldm + j;
      u[r] = {(C)re[o], (C)im[o]};
    }
#pragma unroll
  for (int r = 0; r < TMAX; ++r) {
    if (r >= kbi) break;
    cpx<C> acc = u[r];
#pragma unroll
    for (int k = 0; k < TMAX; ++k) {
      if (k >= r) break;
      const cpx<C> t = cmul(Ls[r * lst + k], u[k]);
      acc.re -= t.re;
      acc.im -= t.im;
    }
    u[r] = acc;
    const size_t o = (size_t)(s0 + r) * ldm + j;
    re[o] = (S)acc.re;
    im[o] = (S)acc.im;
  }
}

// Column j of the outer panel outside the sub-panel [s0, s0 + kbi) (kbi <= 16), in one memory
// round trip: row s0 + r takes the old content of row srow[r], row far_dst[t] (below the
// sub-panel) that of far_src[t]; every load before any store.  Where trsm is set the
// sub-panel's rows are then solved, U12 = inv(L11) A12 with the unit-lower L11 (Ls, row stride
// lst), before they are stored.  Entry for entry the same result as swap_trsm_column.
template <typename S, typename C>
__device__ __forceinline__ void panel_column_tail(S* re, S* im, int ldm, int j, int kbi, int s0,
                                                  const int* srow, int nfar, const int* far_dst,
                                                  const int* far_src, const cpx<C>* Ls, int lst,
                                                  bool trsm) {
  constexpr int TMAX = 16;
  cpx<C> u[TMAX];
  S fr[TMAX], fi[TMAX];
#pragma unroll
  for (int r = 0; r < TMAX; ++r)
    if (r < kbi) {
      const size_t q = (size_t)srow[r] * ldm + j;
      u[r] = {(C)re[q], (C)im[q]};
    }
#pragma unroll
  for (int t = 0; t < TMAX; ++t)
    if (t < nfar) {
      const size_t q = (size_t)far_src[t] * ldm + j;
      fr[t] = re[q];
      fi[t] = im[q];
    }
#pragma unroll
  for (int t = 0; t < TMAX; ++t)
    if (t < nfar) {
      const size_t a = (size_t)far_dst[t] * ldm + j;
      re[a] = fr[t];
      im[a] = fi[t];
    }
  if (!trsm) {
#pragma unroll
    for (int r = 0; r < TMAX; ++r)
      if (r < kbi && srow[r] != s0 + r) {
        const size_t o = (size_t)(s0 + r) * ldm + j;
        re[o] = (S)u[r].re;
        im[o] = (S)u[r].im;
      }
    return;
  }
#pragma unroll
  for (int r = 0; r < TMAX; ++r) {
    if (r >= kbi) break;
    cpx<C> acc = u[r];
#pragma unroll
    for (int k = 0; k < TMAX; ++k) {
      if (k >= r) break;
      const cpx<C> t = cmul(Ls[r * lst + k], u[k]);
      acc.re -= t.re;
      acc.im -= t.im;
    }
    u[r] = acc;
    const size_t o = (size_t)(s0 + r) * ldm + j;
    re[o] = (S)acc.re;
    im[o] = (S)acc.im;
  }
}

// After a pivoted sub-panel [s0, s0+kbi): each thread takes one column j >= jstart outside the
// sub-panel, applies the sub-panel's interchanges to it in order and, for the columns of the
// outer panel still to be factored ([s0+kbi, c_end)), the forward substitution with the
// unit-lower L11 of the sub-panel (U12 = inv(L11) A12), in place.  A sub-panel as wide as its
// outer panel (up to 128 columns) leaves no such columns; narrower ones are at most 16 wide.
template <typename S, typename C>
__global__ void __launch_bounds__(128)
    k_swap_trsm(S* M, int N, int ldm, size_t mat_stride, size_t plane_stride, int s0, int kbi,
                int jstart, int c_end, const int* piv) {
  constexpr int KMAX = 128;  // widest sub-panel
  constexpr int TMAX = 16;   // widest sub-panel that leaves outer-panel columns behind
  __shared__ cpx<C> Ls[TMAX][TMAX + 1];
  __shared__ int sp[KMAX];
  __shared__ int mv_dst[2 * TMAX], mv_src[2 * TMAX], s_nmv;
  const int mat = blockIdx.y;
  S* re = M + mat * mat_stride;
  S* im = re + plane_stride;
  const bool tr = c_end > s0 + kbi && kbi <= TMAX;  // the host never asks otherwise
  if (tr)
    for (int e = threadIdx.x; e < kbi * kbi; e += blockDim.x) {
      const int r = e / kbi, cc = e - r * kbi;
      const size_t o = (size_t)(s0 + r) * ldm + s0 + cc;
      Ls[r][cc] = {(C)re[o], (C)im[o]};
    }
  for (int t = threadIdx.x; t < kbi && t < KMAX; t += blockDim.x)
    sp[t] = piv[(size_t)mat * N + s0 + t];
  __syncthreads();
  if (threadIdx.x == 0) s_nmv = kbi <= TMAX ? compose_moves(sp, kbi, s0, mv_dst, mv_src) : -1;
  __syncthreads();
  const int j = jstart + blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N || (j >= s0 && j < s0 + kbi)) return;
  const int nmv = s_nmv;
  if (nmv >= 0) {
    swap_trsm_column<S, C>(re, im, ldm, j, nmv, mv_dst, mv_src, &Ls[0][0], TMAX + 1, kbi, s0,
                           tr && j >= s0 + kbi && j < c_end);
    return;
  }
  // a sub-panel as wide as its outer panel: the interchanges in order, nothing left to solve
  for (int cc = 0; cc < kbi && cc < KMAX; ++cc) {
    const int p = sp[cc];
    if (p != s0 + cc) {
      const size_t a = (size_t)(s0 + cc) * ldm + j, q = (size_t)p * ldm + j;
      const S xr = re[a], xi = im[a];
      re[a] = re[q]; im[a] = im[q];
      re[q] = xr; im[q] = xi;
    }
  }
}

// The interchanges of a whole outer panel [k0, k0 + kb) (piv: its columns' pivot rows, in
// order) on the columns outside it, [jstart, k0) and [k0 + kb, N).  Each CTA composes them
// into one list of at most 2 kb row moves (row dst takes the old content of row src), then
// moves strips of kSwapStrip columns: every source entry of the strip into shared memory,
// then every destination.  grid (CTAs per block, blocks); dynamic shared memory
// swap_outer_smem(N - k0, kb, sizeof(S)).
constexpr int kSwapStrip = 32;
constexpr int kSwapCtas = 4;  // CTAs per block (each composes the moves once)
__host__ __device__ constexpr size_t swap_outer_smem(int m, int kb, int es) {
  return ((sizeof(int) * ((size_t)m + 5 * (size_t)kb) + 15) / 16) * 16 +
         (size_t)es * 2 * 2 * kb * kSwapStrip;
}
template <typename S>
__global__ void __launch_bounds__(256)
    k_swap_outer(S* M, int N, int ldm, size_t mat_stride, size_t plane_stride, int k0, int kb,
                 int jstart, const int* piv) {
  extern __shared__ unsigned char smem_raw[];
  const int m = N - k0, kend = k0 + kb, tid = threadIdx.x;
  int* cur = reinterpret_cast<int*>(smem_raw);  // content of position k0 + x: old row k0 + cur[x]
  int* mv_dst = cur + m;
  int* mv_src = mv_dst + 2 * kb;
  int* sp = mv_src + 2 * kb;
  S* bre = reinterpret_cast<S*>(smem_raw + ((sizeof(int) * ((size_t)m + 5 * kb) + 15) / 16) * 16);
  S* bim = bre + 2 * kb * kSwapStrip;
  __shared__ int s_nmv;
  const int mat = blockIdx.y;
  S* re = M + mat * mat_stride;
  S* im = re + plane_stride;
  for (int x = tid; x < m; x += blockDim.x) cur[x] = x;
  for (int c = tid; c < kb; c += blockDim.x) sp[c] = piv[(size_t)mat * N + k0 + c] - k0;
  if (tid == 0) s_nmv = 0;
  __syncthreads();
  if (tid == 0)
    for (int c = 0; c < kb; ++c) {
      const int p = sp[c];
      if (p <= c || p >= m) continue;  // no interchange (a pivot row is never above its column)
      const int t = cur[c];
      cur[c] = cur[p];
      cur[p] = t;
    }
  __syncthreads();
  for (int x = tid; x < m; x += blockDim.x)
    if (cur[x] != x) {
      const int t = atomicAdd(&s_nmv, 1);
      if (t < 2 * kb) mv_dst[t] = k0 + x, mv_src[t] = k0 + cur[x];
    }
  __syncthreads();
  const int nmv = s_nmv;  // at most 2 kb: the interchanges touch no other rows
  if (nmv == 0 || nmv > 2 * kb) return;
  const int nl = k0 - jstart, nco = nl + (N - kend);
  const int tot = nmv * kSwapStrip;
  constexpr int U = 8;
  for (int v0 = blockIdx.x * kSwapStrip; v0 < nco; v0 += gridDim.x * kSwapStrip) {
    for (int e0 = tid; e0 < tot; e0 += 256 * U) {
      S vr[U] = {}, vi[U] = {};
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + 256 * u, v = v0 + (e & (kSwapStrip - 1));
        if (e < tot && v < nco) {
          const int j = v < nl ? jstart + v : kend + (v - nl);
          const size_t q = (size_t)mv_src[e / kSwapStrip] * ldm + j;
          vr[u] = re[q];
          vi[u] = im[q];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + 256 * u;
        if (e < tot) bre[e] = vr[u], bim[e] = vi[u];
      }
    }
    __syncthreads();
    for (int e = tid; e < tot; e += 256) {
      const int v = v0 + (e & (kSwapStrip - 1));
      if (v < nco) {
        const int j = v < nl ? jstart + v : kend + (v - nl);
        const size_t a = (size_t)mv_dst[e / kSwapStrip] * ldm + j;
        re[a] = bre[e];
        im[a] = bim[e];
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------ panel (SMEM)
// Pivoted LU of the column panel rows [k0, N) x cols [k0, k0+kb) of each block, one CTA per
// block, the m x kb panel (m = N - k0) held in shared memory for the whole column loop.
// Pivot: row of largest |z|^2 in the compute type (first index on ties), found with warp
// shuffles then across warps.  ld[b] += sum ln|u_kk| in float64; piv / perm record the
// interchanges.
template <typename S, typename C, int NT>
__global__ void __launch_bounds__(NT) k_panel_smem(S* M, int N, int ldm, size_t mat_stride,
                                                   size_t plane_stride, int k0, int kb, int b0,
                                                   double* ld, int* piv, int* perm, int* flags,
                                                   int swap_from, int c_end) {
  extern __shared__ unsigned char smem_raw[];
  cpx<C>* P = reinterpret_cast<cpx<C>*>(smem_raw);  // m x (kb+1), row-major, padded
  const int ps = kb + 1;  // odd row stride: conflict-free column access
  __shared__ C red_v[NT / 32];
  __shared__ int red_i[NT / 32];
  __shared__ double piv2[256];
  // sub-panels <= 16: the source row of each row of the sub-panel, and the moves to rows below it
  __shared__ int s_srow[16], s_fdst[16], s_fsrc[16], s_nfar;
  const int mat = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m = N - k0;
  // after the panel: the pivot row (panel-relative) of each column, then the perm entries
  // the interchanges touch (positions and values, 2 kb each)
  int* s_sw = reinterpret_cast<int*>(P + (size_t)m * ps);
  int* s_pos = s_sw + kb;
  int* s_val = s_pos + 2 * kb;
  S* re = M + mat * mat_stride;
  S* im = re + plane_stride;
  if (sizeof(S) == 4 && kb == 16 && k0 % 4 == 0 && ldm % 4 == 0) {
    // 16 columns: float4 loads of 4 consecutive entries of one plane, LB of them in flight
    // per thread; the row, plane and column of unit e by shifts (8 units per row)
    constexpr int LB = 8;
    const int tot = m * 8;
    for (int e0 = tid; e0 < tot; e0 += NT * LB) {
      float4 v[LB];
#pragma unroll
      for (int u = 0; u < LB; ++u) {
        const int e = e0 + NT * u;
        if (e < tot) {
          const int r = e >> 3, pl = (e >> 2) & 1, c4 = (e & 3) * 4;
          const S* src = (pl == 0 ? re : im) + (size_t)(k0 + r) * ldm + k0 + c4;
          v[u] = *reinterpret_cast<const float4*>(src);
        }
      }
#pragma unroll
      for (int u = 0; u < LB; ++u) {
        const int e = e0 + NT * u;
        if (e < tot) {
          const int r = e >> 3, pl = (e >> 2) & 1, c4 = (e & 3) * 4;
          C* dst = reinterpret_cast<C*>(P + r * ps + c4) + pl;  // .re or .im of 4 entries
          dst[0] = (C)v[u].x;
          dst[2] = (C)v[u].y;
          dst[4] = (C)v[u].z;
          dst[6] = (C)v[u].w;
        }
      }
    }
  } else if (sizeof(S) == 4 && kb % 4 == 0 && k0 % 4 == 0 && ldm % 4 == 0) {
    // float4 loads of 4 consecutive entries of one plane, LB of them in flight per thread
    constexpr int LB = 8;
    const int q4 = kb / 4, per_row = 2 * q4, tot = m * per_row;
    for (int e0 = tid; e0 < tot; e0 += NT * LB) {
      float4 v[LB];
#pragma unroll
      for (int u = 0; u < LB; ++u) {
        const int e = e0 + NT * u;
        if (e < tot) {
          const int r = e / per_row, x = e - r * per_row;
          const int pl = x / q4, c4 = (x - pl * q4) * 4;
          const S* src = (pl == 0 ? re : im) + (size_t)(k0 + r) * ldm + k0 + c4;
          v[u] = *reinterpret_cast<const float4*>(src);
        }
      }
#pragma unroll
      for (int u = 0; u < LB; ++u) {
        const int e = e0 + NT * u;
        if (e < tot) {
          const int r = e / per_row, x = e - r * per_row;
          const int pl = x / q4, c4 = (x - pl * q4) * 4;
          C* dst = reinterpret_cast<C*>(P + r * ps + c4) + pl;  // .re or .im of 4 entries
          dst[0] = (C)v[u].x;
          dst[2] = (C)v[u].y;
          dst[4] = (C)v[u].z;
          dst[6] = (C)v[u].w;
        }
      }
    }
  } else {
    for (int e = tid; e < m * kb; e += NT) {
      const int r = e / kb, c = e - r * kb;
      const size_t o = (size_t)(k0 + r) * ldm + k0 + c;
      P[r * ps + c] = {(C)re[o], (C)im[o]};
    }
  }
  __syncthreads();
  // argmax of |z|^2 over rows >= c of column c: thread-local candidates, then warp shuffles,
  // then every warp reduces the per-warp winners itself (no broadcast barrier)
  auto pick = [&](C best, int bi, int c) -> int {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const C ov = __shfl_down_sync(0xffffffffu, best, off);
      const int oi = __shfl_down_sync(0xffffffffu, bi, off);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { red_v[warp] = best; red_i[warp] = bi; }
    __syncthreads();
    best = (lane < NT / 32) ? red_v[lane] : (C)-1;
    bi = (lane < NT / 32) ? red_i[lane] : m;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const C ov = __shfl_xor_sync(0xffffffffu, best, off);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    return bi < m ? bi : c;
  };
  C best = (C)-1;
  int bi = m;
  for (int r = tid; r < m; r += NT) {
    const cpx<C> z = P[r * ps];
    const C v = z.re * z.re + z.im * z.im;
    if (v > best) { best = v; bi = r; }
  }
  int p = pick(best, bi, 0);
  for (int c = 0; c < kb; ++c) {
    // red_v / red_i are read by every warp above; the next writes come after a barrier
    if (p != c)
      for (int j = tid; j < kb; j += NT) {
        const cpx<C> t = P[c * ps + j];
        P[c * ps + j] = P[p * ps + j];
        P[p * ps + j] = t;
      }
    if (tid == 0) {
      piv[(size_t)mat * N + k0 + c] = k0 + p;
      s_sw[c] = p;
    }
    __syncthreads();
    const cpx<C> d = P[c * ps + c];
    const C m2 = d.re * d.re + d.im * d.im;
    const cpx<C> inv = (m2 > (C)0) ? cpx<C>{d.re / m2, -d.im / m2} : cpx<C>{(C)0, (C)0};
    if (tid == 0) piv2[c] = (double)d.re * d.re + (double)d.im * d.im;
    // eliminate below the pivot; the new column c+1 feeds the next pivot search
    best = (C)-1;
    bi = m;
    // two rows per pass (r and r + NT): each entry of the pivot row is read once for both
    for (int r = c + 1 + tid; r < m; r += 2 * NT) {
      const int r2 = r + NT;
      const bool two = r2 < m;
      cpx<C>* row = P + r * ps;
      cpx<C>* row2 = P + (two ? r2 : r) * ps;
      const cpx<C> l = cmul(row[c], inv);
      const cpx<C> l2 = cmul(row2[c], inv);
      row[c] = l;
      if (two) row2[c] = l2;
      for (int j = c + 1; j < kb; ++j) {
        const cpx<C> u = P[c * ps + j];
        row[j].re -= l.re * u.re - l.im * u.im;
        row[j].im -= l.re * u.im + l.im * u.re;
        if (two) {
          row2[j].re -= l2.re * u.re - l2.im * u.im;
          row2[j].im -= l2.re * u.im + l2.im * u.re;
        }
      }
      if (c + 1 < kb) {
        const cpx<C> z = row[c + 1];
        const C v = z.re * z.re + z.im * z.im;
        if (v > best) { best = v; bi = r; }
        if (two) {
          const cpx<C> z2 = row2[c + 1];
          const C v2 = z2.re * z2.re + z2.im * z2.im;
          if (v2 > best) { best = v2; bi = r2; }
        }
      }
    }
    if (c + 1 < kb) {
      p = pick(best, bi, c + 1);
    } else {
      __syncthreads();
    }
  }
  if (kb <= 16) {
    // a warp per row: lanes 0-15 the real parts, 16-31 the imaginary parts of its columns
    const int c = lane & 15;
    S* dstp = lane < 16 ? re : im;
    if (c < kb)
      for (int r = warp; r < m; r += NT / 32) {
        const cpx<C> z = P[r * ps + c];
        dstp[(size_t)(k0 + r) * ldm + k0 + c] = (S)(lane < 16 ? z.re : z.im);
      }
  } else {
    for (int e = tid; e < m * kb; e += NT) {
      const int r = e / kb, c = e - r * kb;
      const size_t o = (size_t)(k0 + r) * ldm + k0 + c;
      re[o] = (S)P[r * ps + c].re;
      im[o] = (S)P[r * ps + c].im;
    }
  }
  // The row permutation of the kb interchanges (c, s_sw[c]), c in order, over the at most 2 kb
  // positions they touch.  Slot c < kb is position c; slot kb + c is position s_sw[c] >= kb if
  // c is the first column with that pivot row (s_pos[kb + c] = kb + that first column; -1 for
  // pivot rows < kb).  s_val[t] ends as the slot whose old content slot t takes.
  {
    int* pm = perm + (size_t)mat * N + k0;
    if (tid < 2 * kb) {
      int q = tid;
      if (tid >= kb) {
        const int p = s_sw[tid - kb];
        q = -1;
        if (p >= kb) {
          int f = 0;
          while (s_sw[f] != p) ++f;  // ends at tid - kb at the latest
          q = kb + f;
        }
      }
      s_pos[tid] = q;
      s_val[tid] = tid;
    }
    __syncthreads();
    if (tid == 0)
      for (int c = 0; c < kb; ++c) {
        const int p = s_sw[c];
        if (p == c) continue;
        const int b = p < kb ? p : s_pos[kb + c];
        const int t = s_val[c];
        s_val[c] = s_val[b];
        s_val[b] = t;
      }
    __syncthreads();
    // slot tid: in use, its position, the position its content comes from
    const bool used = tid < kb || (tid < 2 * kb && s_pos[tid] == tid);
    int pos = 0, from = 0;
    if (used) {
      const int st = s_val[tid];
      pos = tid < kb ? tid : s_sw[tid - kb];
      from = st < kb ? st : s_sw[st - kb];
    }
    const bool moved = used && from != pos;
    const int old = moved ? pm[from] : 0;
    // for the fused tail (kb <= 16: every slot in warp 0): the source rows of the sub-panel's
    // rows and the moves to rows below it, in slot order
    if (warp == 0 && kb <= 16) {
      if (lane < kb) s_srow[lane] = k0 + from;
      const unsigned mask = __ballot_sync(0xffffffffu, moved && lane >= kb);
      if (moved && lane >= kb) {
        const int x = __popc(mask & ((1u << lane) - 1u));
        s_fdst[x] = k0 + pos;
        s_fsrc[x] = k0 + from;
      }
      if (lane == 0) s_nfar = __popc(mask);
    }
    __syncthreads();
    if (moved) pm[pos] = old;
  }
  {
    const double s = logdet_sum<NT>(piv2, kb, flags);
    if (tid == 0) ld[b0 + mat] += s;
  }
  // swap_from >= 0 (sub-panels of at most 16 columns): the sub-panel's interchanges on the
  // columns [swap_from, c_end) outside it (the rest of its outer panel) and U12 for the columns
  // [k0 + kb, c_end), with L11 still in the shared panel.  The columns outside the outer panel
  // take all of its interchanges at once afterwards (k_swap_outer).
  if (swap_from >= 0 && kb <= 16) {
    const int nfar = s_nfar;
    for (int j = swap_from + tid; j < c_end; j += NT) {
      if (j >= k0 && j < k0 + kb) continue;
      panel_column_tail<S, C>(re, im, ldm, j, kb, k0, s_srow, nfar, s_fdst, s_fsrc, P, ps,
                              j >= k0 + kb);
    }
  }
}

// ------------------------------------------------------- dominant pivot block
// T = inv(M_KK) for a pivot block that needs no interchanges (a strictly column-diagonally
// dominant block keeps its diagonal under partial pivoting, and the complex-symmetric
// elimination takes none) by in-place Gauss-Jordan, the block held in registers: thread (r0, j) owns
// column j, rows r0, r0 + RS, ... (RS = NT / kb row groups); each of the kb sweeps exchanges
// only the pivot row and column through shared memory.  ld[b] += sum ln|pivot| (the pivots of
// the LU).  Writes T to Tinv slot 0 (nb x nb, zero padded) and, if TT != null, the split planes
// of W_T[j][k] = -T[k][j] for the tensor-core product F = M[:, K] T
// (planes re_hi, im_hi, re_lo, im_lo; kb x kb per block, K-contiguous).
template <typename S, typename C, int NT>
__global__ void __launch_bounds__(NT) k_diag_gj(const S* M, int ldm, size_t mat_stride,
                                                size_t plane_stride, int k0, int kb, int nb,
                                                int b0, double* ld, cpx<C>* Tinv, float* TT,
                                                int tt_bf16, int* flags) {
  // The block is padded to KB x KB with the identity (pivots 1: no effect on ln|det|; the
  // padded inverse is diag(T, I)), so the thread -> (row, column) map is compile-time:
  // column j = tid % KB, rows r = tid / KB + q * RS.  The owners of row / column c + 1
  // publish them into the other half of a double buffer right after their own update of
  // sweep c, so each sweep needs a single barrier.
  constexpr int KB = sizeof(C) == 8 ? 64 : 128;
  constexpr int RS = NT / KB;
  constexpr int MAXR = (KB + RS - 1) / RS;
  __shared__ cpx<C> prow[2][KB], pcol[2][KB];
  __shared__ double piv2[KB];
  const int mat = blockIdx.x, tid = threadIdx.x;
  const int j = tid % KB, rg = tid / KB;
  const S* re = M + mat * mat_stride;
  const S* im = re + plane_stride;
  cpx<C> a[MAXR];
#pragma unroll
  for (int q = 0; q < MAXR; ++q) {
    const int r = rg + q * RS;
    if (r < kb && j < kb) {
      const size_t o = (size_t)(k0 + r) * ldm + k0 + j;
      a[q] = {(C)re[o], (C)im[o]};
    } else {
      a[q] = {(C)(r == j ? 1 : 0), (C)0};
    }
  }
  // publish row / column 0
#pragma unroll
  for (int q = 0; q < MAXR; ++q) {
    const int r = rg + q * RS;
    if (r == 0) prow[0][j] = a[q];
    if (j == 0 && r < KB) pcol[0][r] = a[q];
  }
  __syncthreads();
  for (int c = 0; c < KB; ++c) {
    const int cb = c & 1, nbuf = cb ^ 1;
    const cpx<C> d = pcol[cb][c];
    const C m2 = d.re * d.re + d.im * d.im;
    const cpx<C> dinv = (m2 > (C)0) ? cpx<C>{d.re / m2, -d.im / m2} : cpx<C>{(C)0, (C)0};
    if (tid == 0) piv2[c] = (double)d.re * d.re + (double)d.im * d.im;
    // u_j = prow_j / d (j != c), u_c = 1/d; new = (r == c) ? u_j : (j == c ? 0 : a) - pcol_r u_j
    const bool jc = (j == c);
    const cpx<C> u = jc ? dinv : cmul(prow[cb][j], dinv);
#pragma unroll
    for (int q = 0; q < MAXR; ++q) {
      const int r = rg + q * RS;
      if (r >= KB) continue;
      const cpx<C> l = pcol[cb][r];
      cpx<C> v = jc ? cpx<C>{(C)0, (C)0} : a[q];
      v.re -= l.re * u.re - l.im * u.im;
      v.im -= l.re * u.im + l.im * u.re;
      a[q] = (r == c) ? u : v;
      // publish the next pivot row / column from the freshly updated values
      if (r == c + 1) prow[nbuf][j] = a[q];
      if (j == c + 1) pcol[nbuf][r] = a[q];
    }
    __syncthreads();
  }
  {
    const double s = logdet_sum<NT>(piv2, kb, flags);  // padded pivots are 1
    if (tid == 0) ld[b0 + mat] += s;
  }
  cpx<C>* T = Tinv + (size_t)mat * 2 * nb * nb;
  const size_t P = (size_t)nb * nb;  // one plane of W_T (nb x nb, K-contiguous)
  float* tt = TT ? TT + (size_t)mat * kTtPlanes * P : nullptr;
#pragma unroll
  for (int q = 0; q < MAXR; ++q) {
    const int r = rg + q * RS;
    if (r >= nb || j >= nb) continue;
    const bool in = r < kb && j < kb;
    const cpx<C> v = in ? a[q] : cpx<C>{(C)0, (C)0};
    T[(size_t)r * nb + j] = v;
    if (tt && tt_bf16) {  // W_T[j][r] = -T[r][j], split into bf16 planes
      const size_t o = (size_t)j * nb + r;
      const float fr = -(float)v.re, fi = -(float)v.im;
      const __nv_bfloat16 hr = __float2bfloat16_rn(fr), hi = __float2bfloat16_rn(fi);
      const __nv_bfloat16 lr = __float2bfloat16_rn(fr - __bfloat162float(hr));
      const __nv_bfloat16 li = __float2bfloat16_rn(fi - __bfloat162float(hi));
      reinterpret_cast<__nv_bfloat16*>(tt)[o] = hr;
      reinterpret_cast<__nv_bfloat16*>(tt + P)[o] = hi;
      reinterpret_cast<__nv_bfloat16*>(tt + 2 * P)[o] = lr;
      reinterpret_cast<__nv_bfloat16*>(tt + 3 * P)[o] = li;
    } else if (tt) {  // W_T[j][r] = -T[r][j], split for TF32
      float* o = tt + (size_t)j * nb + r;
      const float fr = -(float)v.re, fi = -(float)v.im;
      const float hr = __uint_as_float(__float_as_uint(fr) & 0xffffe000u);
      const float hi = __uint_as_float(__float_as_uint(fi) & 0xffffe000u);
      o[0] = hr; o[P] = hi; o[2 * P] = fr - hr; o[3 * P] = fi - hi;
    }
  }
}

// Blocked form of k_diag_gj for float32 (same outputs).  The tableau stays in registers
// (thread (rg, j) owns column j, rows rg + RS q) and is swept in 8 panels of 16 pivots.  Per
// panel P: M[:, P] and W = M[P, :] (identity in the columns of P) go to shared memory; one
// warp inverts the 16 x 16 pivot block M_PP by Gauss-Jordan (its pivots are those of the LU,
// so ln|det| is the same); all threads form F = M[:, P] inv(M_PP) (rows of P: -inv(M_PP));
// then each thread applies the rank-16 update M <- mask(M) - F W to the entries it owns
// (mask: zero in the rows and the columns of P).  Four barriers per panel instead of one per
// pivot, and the update is 32 FMAs per 8 broadcast loads.
template <int NT>
__global__ void __launch_bounds__(NT) k_diag_gjb(const float* M, int ldm, size_t mat_stride,
                                                 size_t plane_stride, int k0, int kb, int nb,
                                                 int b0, double* ld, cpx<float>* Tinv,
                                                 float* TT, int tt_bf16, int* flags) {
  constexpr int KB = 128, PW = 16;
  constexpr int RS = NT / KB;
  constexpr int MAXR = (KB + RS - 1) / RS;
  __shared__ cpx<float> Ms[KB][PW + 1];  // M[:, P], then F in place
  __shared__ cpx<float> Ws[PW][KB];      // W = M[P, :]
  __shared__ cpx<float> Tp[PW][PW + 1];  // inv(M_PP)
  __shared__ double piv2[KB];
  __shared__ cpx<float> pivd[KB];  // the pivots; |pivot|^2 in float64 after the sweep
  const int mat = blockIdx.x, tid = threadIdx.x;
  const int j = tid % KB, rg = tid / KB;
  const float* re = M + mat * mat_stride;
  const float* im = re + plane_stride;
  cpx<float> a[MAXR];
#pragma unroll
  for (int q = 0; q < MAXR; ++q) {
    const int r = rg + q * RS;
    if (r < kb && j < kb) {
      const size_t o = (size_t)(k0 + r) * ldm + k0 + j;
      a[q] = {re[o], im[o]};
    } else {
      a[q] = {(r == j) ? 1.f : 0.f, 0.f};
    }
  }
  for (int p0 = 0; p0 < KB; p0 += PW) {
    const bool jP = (unsigned)(j - p0) < (unsigned)PW;
    // (a) the panel's columns and rows
#pragma unroll
    for (int q = 0; q < MAXR; ++q) {
      const int r = rg + q * RS;
      if (q == MAXR - 1 && r >= KB) break;
      if (jP) Ms[r][j - p0] = a[q];
      if ((unsigned)(r - p0) < (unsigned)PW)
        Ws[r - p0][j] = jP ? cpx<float>{(j == r) ? 1.f : 0.f, 0.f} : a[q];
    }
    __syncthreads();
    // (b) one warp: inv(M_PP) by Gauss-Jordan in registers; lane owns column lane % 16 of
    // rows lane / 16 + 2 m, and the pivot row, column and entry of each step come by shuffle
    if (tid < 32) {
      const int cl = tid & 15, r0 = tid >> 4;
      cpx<float> v[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) v[m] = Ms[p0 + r0 + 2 * m][cl];
#pragma unroll
      for (int cc = 0; cc < PW; ++cc) {
        const int own = (cc & 1) * 16;  // lanes holding row cc, in slot cc / 2
        cpx<float> d, pr, pc[8];
        d.re = __shfl_sync(0xffffffffu, v[cc >> 1].re, own + cc);
        d.im = __shfl_sync(0xffffffffu, v[cc >> 1].im, own + cc);
        pr.re = __shfl_sync(0xffffffffu, v[cc >> 1].re, own + cl);  // pivot row, my column
        pr.im = __shfl_sync(0xffffffffu, v[cc >> 1].im, own + cl);
#pragma unroll
        for (int m = 0; m < 8; ++m) {  // pivot column, my rows
          pc[m].re = __shfl_sync(0xffffffffu, v[m].re, r0 * 16 + cc);
          pc[m].im = __shfl_sync(0xffffffffu, v[m].im, r0 * 16 + cc);
        }
        const float m2 = d.re * d.re + d.im * d.im;
        const float rm = (m2 > 0.f) ? 1.f / m2 : 0.f;
        const cpx<float> dinv = {d.re * rm, -d.im * rm};
        if (tid == 0) pivd[p0 + cc] = d;
        const cpx<float> u = cmul(pr, dinv);
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const int r = r0 + 2 * m;
          if (r == cc) {
            v[m] = (cl == cc) ? dinv : cmul(v[m], dinv);
          } else if (cl == cc) {
            const cpx<float> q2 = cmul(pc[m], dinv);
            v[m] = {-q2.re, -q2.im};
          } else {
            v[m] = {v[m].re - (pc[m].re * u.re - pc[m].im * u.im),
                    v[m].im - (pc[m].re * u.im + pc[m].im * u.re)};
          }
        }
      }
#pragma unroll
      for (int m = 0; m < 8; ++m) Tp[r0 + 2 * m][cl] = v[m];
    }
    __syncthreads();
    // (c) F = M[:, P] inv(M_PP) (rows of P: -inv(M_PP)), in place of M[:, P]: four threads
    // per row, 4 columns each, all reads before the barrier
    {
      constexpr int FC = 4;
      const bool act = tid < (PW / FC) * KB;
      const int r = tid / (PW / FC), kh = (tid % (PW / FC)) * FC;
      cpx<float> f[FC];
      if (act) {
        if ((unsigned)(r - p0) < (unsigned)PW) {
#pragma unroll
          for (int k = 0; k < FC; ++k) {
            const cpx<float> t = Tp[r - p0][kh + k];
            f[k] = {-t.re, -t.im};
          }
        } else {
#pragma unroll
          for (int k = 0; k < FC; ++k) f[k] = {0.f, 0.f};
#pragma unroll
          for (int m = 0; m < PW; ++m) {
            const cpx<float> x = Ms[r][m];
#pragma unroll
            for (int k = 0; k < FC; ++k) {
              const cpx<float> t = Tp[m][kh + k];
              f[k].re += x.re * t.re - x.im * t.im;
              f[k].im += x.re * t.im + x.im * t.re;
            }
          }
        }
      }
      __syncthreads();
      if (act) {
#pragma unroll
        for (int k = 0; k < FC; ++k) Ms[r][kh + k] = f[k];
      }
    }
    __syncthreads();
    // (d) M <- mask(M) - F W on the owned entries
#pragma unroll
    for (int q = 0; q < MAXR; ++q) {
      const int r = rg + q * RS;
      if (jP || (unsigned)(r - p0) < (unsigned)PW) a[q] = {0.f, 0.f};
    }
#pragma unroll 2
    for (int k = 0; k < PW; ++k) {
      const cpx<float> w = Ws[k][j];
#pragma unroll
      for (int q = 0; q < MAXR; ++q) {  // independent chains: the loads run ahead
        const int r = rg + q * RS;
        if (q == MAXR - 1 && r >= KB) break;
        const cpx<float> f = Ms[r][k];
        a[q].re -= f.re * w.re - f.im * w.im;
        a[q].im -= f.re * w.im + f.im * w.re;
      }
    }
    __syncthreads();
  }
  {
    for (int k = tid; k < kb; k += NT)
      piv2[k] = (double)pivd[k].re * pivd[k].re + (double)pivd[k].im * pivd[k].im;
    __syncthreads();
    const double s = logdet_sum<NT>(piv2, kb, flags);  // padded pivots are 1
    if (tid == 0) ld[b0 + mat] += s;
  }
  cpx<float>* T = Tinv + (size_t)mat * 2 * nb * nb;
#pragma unroll
  for (int q = 0; q < MAXR; ++q) {
    const int r = rg + q * RS;
    if (r >= nb || j >= nb) continue;
    T[(size_t)r * nb + j] = (r < kb && j < kb) ? a[q] : cpx<float>{0.f, 0.f};
  }
  if (!TT) return;
  // W_T[j][r] = -T[r][j] in split planes, 16 rows j at a time through shared memory (the
  // owners of columns j deposit them, then every thread writes 4 consecutive r of one row)
  const size_t P = (size_t)nb * nb;
  float* tt = TT + (size_t)mat * kTtPlanes * P;
  cpx<float>(*S)[KB] = Ws;  // [16][KB]
  for (int jc0 = 0; jc0 < nb; jc0 += PW) {
    if ((unsigned)(j - jc0) < (unsigned)PW) {
#pragma unroll
      for (int q = 0; q < MAXR; ++q) {
        const int r = rg + q * RS;
        if (q == MAXR - 1 && r >= KB) break;
        S[j - jc0][r] = (r < kb && j < kb) ? a[q] : cpx<float>{0.f, 0.f};
      }
    }
    __syncthreads();
    for (int e = tid; e < PW * (KB / 4); e += NT) {
      const int jj = e / (KB / 4), r4 = (e - jj * (KB / 4)) * 4;
      const int jr = jc0 + jj;
      if (jr >= nb || r4 >= nb) continue;
      float fr[4], fi[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) { fr[t] = -S[jj][r4 + t].re; fi[t] = -S[jj][r4 + t].im; }
      const size_t o = (size_t)jr * nb + r4;
      if (tt_bf16) {
        __nv_bfloat16 h[4][4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          h[0][t] = __float2bfloat16_rn(fr[t]);
          h[1][t] = __float2bfloat16_rn(fi[t]);
          h[2][t] = __float2bfloat16_rn(fr[t] - __bfloat162float(h[0][t]));
          h[3][t] = __float2bfloat16_rn(fi[t] - __bfloat162float(h[1][t]));
        }
#pragma unroll
        for (int pl = 0; pl < 4; ++pl)
          *reinterpret_cast<uint2*>(reinterpret_cast<__nv_bfloat16*>(tt + pl * P) + o) =
              *reinterpret_cast<const uint2*>(h[pl]);
      } else {
        float4 v[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const float hr = __uint_as_float(__float_as_uint(fr[t]) & 0xffffe000u);
          const float hi = __uint_as_float(__float_as_uint(fi[t]) & 0xffffe000u);
          (&v[0].x)[t] = hr; (&v[1].x)[t] = hi; (&v[2].x)[t] = fr[t] - hr;
          (&v[3].x)[t] = fi[t] - hi;
        }
#pragma unroll
        for (int pl = 0; pl < 4; ++pl) *reinterpret_cast<float4*>(tt + pl * P + o) = v[pl];
      }
    }
    __syncthreads();
  }
}

// Split copy of the pivot columns for the tensor-core product F = M[:, K] T:
// Fs[i][k] = split(M[i][k0 + k]) (planes re_hi, im_hi, re_lo, im_lo; N x nb, zero for k >= kb).
template <typename S>
__global__ void k_split_cols(const S* M, int N, int ldm, size_t mat_stride, size_t plane_stride,
                             int k0, int kb, int nb, float* Fs, size_t fs_plane, size_t fs_mat,
                             int r_begin) {
  const int mat = blockIdx.y;
  const size_t e = (size_t)r_begin * nb + (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)N * nb) return;
  const int i = (int)(e / nb), k = (int)(e - (size_t)i * nb);
  const S* re = M + mat * mat_stride;
  const S* im = re + plane_stride;
  float fr = 0.f, fi = 0.f;
  if (k < kb) {
    fr = (float)re[(size_t)i * ldm + k0 + k];
    fi = (float)im[(size_t)i * ldm + k0 + k];
  }
  const float hr = __uint_as_float(__float_as_uint(fr) & 0xffffe000u);
  const float hi = __uint_as_float(__float_as_uint(fi) & 0xffffe000u);
  float* o = Fs + (size_t)mat * fs_mat + e;
  o[0] = hr; o[fs_plane] = hi; o[2 * fs_plane] = fr - hr; o[3 * fs_plane] = fi - hi;
}

// Symmetric dominant blocks.  A_{n,sigma} is complex symmetric and the dominant blocks are
// never pivoted, so after sweeping the index set S the tableau satisfies
// M_ij = eps_ij M_ji with eps_ij = -1 when exactly one of i, j is in S, +1 otherwise.  The
// tensor-core update then computes only the tiles on or below the diagonal; reads that would
// touch an upper tile are redirected to the transposed lower entry with that sign.

// Completes the fully swept (symmetric) inverse: M[i][j] = M[j][i] for i < j, 32x32 tiles
// through shared memory.  Only for the whole-row refinement (SCA_REFINE_LOWER=0); by default
// diag(G) is refined from the lower triangle.
template <typename S>
__global__ void k_mirror(S* M, int N, int ldm, size_t mat_stride, size_t plane_stride) {
  __shared__ S tr[32][33], ti[32][33];
  const int mat = blockIdx.y;
  // destination tile (bi, bj), bi <= bj, from the linear index t = bj (bj + 1) / 2 + bi
  const int t = blockIdx.x;
  int bj = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
  while ((bj + 1) * (bj + 2) / 2 <= t) ++bj;
  while (bj * (bj + 1) / 2 > t) --bj;
  const int bi = t - bj * (bj + 1) / 2;
  S* re = M + mat * mat_stride;
  S* im = re + plane_stride;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < 32; r += 8) {  // source: tile (bj, bi), rows bj*32 + r
    const int gr = bj * 32 + r, gc = bi * 32 + tx;
    if (gr < N && gc < N) {
      tr[r][tx] = re[(size_t)gr * ldm + gc];
      ti[r][tx] = im[(size_t)gr * ldm + gc];
    }
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int gi = bi * 32 + r, gj = bj * 32 + tx;
    if (gi < N && gj < N && gi < gj) {
      re[(size_t)gi * ldm + gj] = tr[tx][r];
      im[(size_t)gi * ldm + gj] = ti[tx][r];
    }
  }
}

// F planes for the update from the tensor-core product Fp = M[:, K] T (planar re, im; N x nb):
// rows outside K take Fp, rows in K (Gauss-Jordan) take -T, columns >= kb are zero.
template <typename C>
__global__ void k_split_f(const float* Fp, size_t fp_plane, size_t fp_mat, const cpx<C>* Tinv,
                          int N, int k0, int kb, int nb, int r_begin, int gj, float* F,
                          size_t fw_plane, size_t fw_mat) {
  const int mat = blockIdx.y;
  const size_t e = (size_t)r_begin * nb + (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)N * nb) return;
  const int i = (int)(e / nb), c = (int)(e - (size_t)i * nb);
  float vr = 0.f, vi = 0.f;
  if (c < kb) {
    if (gj && i >= k0 && i < k0 + kb) {
      const cpx<C> t = Tinv[(size_t)mat * 2 * nb * nb + (size_t)(i - k0) * nb + c];
      vr = -(float)t.re; vi = -(float)t.im;
    } else {
      vr = Fp[(size_t)mat * fp_mat + e];
      vi = Fp[(size_t)mat * fp_mat + fp_plane + e];
    }
  }
  const float hr = __uint_as_float(__float_as_uint(vr) & 0xffffe000u);
  const float hi = __uint_as_float(__float_as_uint(vi) & 0xffffe000u);
  float* o = F + (size_t)mat * fw_mat + e;
  o[0] = hr; o[fw_plane] = hi; o[2 * fw_plane] = vr - hr; o[3 * fw_plane] = vi - hi;
}

// ---------------------------------------------------------------------- prep
// Rank-nb factors of one elimination step, written K-contiguous (N x nb, planar):
//   F[i]   = M[i, K] T              (rows outside K; T = inv(M_KK))
//   F[i]   = M[i, K] inv(L11)       (rows below K after the pivoted panel: M[i, K] = L21)
//   F[i]   = -T[i - k0]             (rows in K, Gauss-Jordan)
//   W^T[j] = M[K, j]                (columns outside K)
//   W^T[j] = e_{j - k0}             (columns in K, Gauss-Jordan)
// so that M' = mask(M) - F W is one Gauss-Jordan sweep over K (mask zeroes row and column
// block K) or, restricted to rows and columns past K, the LU Schur complement.
// With `split`, planes are {re_hi, im_hi, re_lo, im_lo} (hi = value with the low 13 mantissa
// bits cleared, exact in TF32; lo = value - hi), for F and W alike.
template <typename S>
__device__ __forceinline__ void store_fw(S* base, size_t plane, size_t off, double vre, double vim,
                                         int split) {
  if (!split) {
    base[off] = (S)vre;
    base[plane + off] = (S)vim;
  } else if (split == 2) {
    // bf16 planes (BF16x3): hi = RN_bf16(v), lo = RN_bf16(v - hi); a plane starts where the
    // float32 plane would, element `off` at 2 bytes
    const float fr = (float)vre, fi = (float)vim;
    const __nv_bfloat16 hr = __float2bfloat16_rn(fr), hi = __float2bfloat16_rn(fi);
    const __nv_bfloat16 lr = __float2bfloat16_rn(fr - __bfloat162float(hr));
    const __nv_bfloat16 li = __float2bfloat16_rn(fi - __bfloat162float(hi));
    float* b = reinterpret_cast<float*>(base);
    reinterpret_cast<__nv_bfloat16*>(b)[off] = hr;
    reinterpret_cast<__nv_bfloat16*>(b + plane)[off] = hi;
    reinterpret_cast<__nv_bfloat16*>(b + 2 * plane)[off] = lr;
    reinterpret_cast<__nv_bfloat16*>(b + 3 * plane)[off] = li;
  } else {
    const float fr = (float)vre, fi = (float)vim;
    const float hr = __uint_as_float(__float_as_uint(fr) & 0xffffe000u);
    const float hi = __uint_as_float(__float_as_uint(fi) & 0xffffe000u);
    float* b = reinterpret_cast<float*>(base);
    b[off] = hr;
    b[plane + off] = hi;
    b[2 * plane + off] = fr - hr;
    b[3 * plane + off] = fi - hi;
  }
}

// F: 64 rows x nb columns per CTA, 256 threads, 4 x (nb/16) complex outputs per thread.
template <typename S, typename C>
__global__ void __launch_bounds__(256)
    k_prep_f(const S* M, int N, int ldm, size_t mat_stride, size_t plane_stride, int k0, int kb,
             int nb, const cpx<C>* Tinv, S* F, size_t fw_plane, size_t fw_mat, int r_begin, int gj,
             int pivoted, int split) {
  constexpr int BR = 64;
  constexpr int KC = sizeof(C) == 8 ? 8 : 16;
  constexpr int NBMAX = sizeof(C) == 8 ? 64 : 128;
  constexpr int MAXC = NBMAX / 16;
  __shared__ C As[2][KC][BR + 1];
  __shared__ cpx<C> Xs[2][KC][NBMAX];  // [0]: T chunk, [1]: inv(L11) chunk (pivoted)
  const int mat = blockIdx.y;
  const int i0 = r_begin + blockIdx.x * BR;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const S* re = M + mat * mat_stride;
  const S* im = re + plane_stride;
  const cpx<C>* T = Tinv + (size_t)mat * 2 * nb * nb;
  const cpx<C>* Li = T + (size_t)nb * nb;
  const int kend = k0 + kb;
  const int ncg = (nb + 15) / 16;  // column groups per thread
  C ar[4][MAXC], ai[4][MAXC];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int q = 0; q < MAXC; ++q) { ar[a][q] = 0; ai[a][q] = 0; }
  bool useL[4];  // pivoted rows below K: F_i = L_iK inv(L11)
#pragma unroll
  for (int a = 0; a < 4; ++a) useL[a] = pivoted && (i0 + ty + 16 * a) >= kend;
  for (int kc = 0; kc < kb; kc += KC) {
    for (int e = threadIdx.x; e < BR * KC; e += 256) {
      const int r = e / KC, k = e - r * KC;
      const int gi = i0 + r;
      const bool in = gi < N && (kc + k) < kb;
      As[0][k][r] = in ? (C)re[(size_t)gi * ldm + k0 + kc + k] : (C)0;
      As[1][k][r] = in ? (C)im[(size_t)gi * ldm + k0 + kc + k] : (C)0;
    }
    for (int e = threadIdx.x; e < KC * nb; e += 256) {
      const int k = e / nb, c = e - k * nb;
      const bool in = (kc + k) < kb;
      Xs[0][k][c] = in ? T[(size_t)(kc + k) * nb + c] : cpx<C>{(C)0, (C)0};
      Xs[1][k][c] = (in && pivoted) ? Li[(size_t)(kc + k) * nb + c] : cpx<C>{(C)0, (C)0};
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < KC; ++k) {
      C fr[4], fi[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) { fr[a] = As[0][k][ty + 16 * a]; fi[a] = As[1][k][ty + 16 * a]; }
#pragma unroll
      for (int q = 0; q < MAXC; ++q) {
        if (q < ncg) {
          const cpx<C> xt = Xs[0][k][tx + 16 * q];
          const cpx<C> xl = Xs[1][k][tx + 16 * q];
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const cpx<C> xv = useL[a] ? xl : xt;
            ar[a][q] = fma(fr[a], xv.re, ar[a][q]);
            ar[a][q] = fma(-fi[a], xv.im, ar[a][q]);
            ai[a][q] = fma(fr[a], xv.im, ai[a][q]);
            ai[a][q] = fma(fi[a], xv.re, ai[a][q]);
          }
        }
      }
    }
    __syncthreads();
  }
  S* out = F + (size_t)mat * fw_mat;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = i0 + ty + 16 * a;
    if (i >= N) continue;
    const bool ink = gj && i >= k0 && i < kend;
#pragma unroll
    for (int q = 0; q < MAXC; ++q) {
      if (q >= ncg) continue;
      const int c = tx + 16 * q;
      if (c >= nb) continue;
      double vr, vi;
      if (c >= kb) {
        vr = 0.0; vi = 0.0;
      } else if (ink) {
        const cpx<C> t = T[(size_t)(i - k0) * nb + c];
        vr = -(double)t.re; vi = -(double)t.im;
      } else {
        vr = (double)ar[a][q]; vi = (double)ai[a][q];
      }
      store_fw(out, fw_plane, (size_t)i * nb + c, vr, vi, split);
    }
  }
}

// B operands of the tensor-core prep product F = M[:, K] X as bf16 split planes of -X^T
// (re_hi, im_hi, re_lo, im_lo; element [j][r] = -X[r][j]): X = T in the first half of each of
// the block's float-plane slots, X = inv(L) in the second half.  The rows of T and inv(L) just
// written to global memory are read back through the shared-memory buffer Sm ([nb][nb + 1]).
template <typename C, int NT>
__device__ void tinv_split_planes(const cpx<C>* outT, const cpx<C>* outL, cpx<C>* Sm, float* TT,
                                  int nb, int mat) {
  const int tid = threadIdx.x;
  const size_t P = (size_t)nb * nb;
  float* tt = TT + (size_t)mat * kTtPlanes * P;
  for (int part = 0; part < 2; ++part) {
    const cpx<C>* src = part == 0 ? outT : outL;
    for (int e = tid; e < nb * nb; e += NT) {
      const int r = e / nb, j = e - r * nb;
      Sm[(size_t)r * (nb + 1) + j] = src[e];
    }
    __syncthreads();
    __nv_bfloat16* dst = reinterpret_cast<__nv_bfloat16*>(tt + (part == 0 ? 0 : P / 2));
    for (int e = tid; e < nb * (nb / 4); e += NT) {
      const int jr = e / (nb / 4), r4 = (e - jr * (nb / 4)) * 4;
      __nv_bfloat16 h[4][4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const cpx<C> v = Sm[(size_t)(r4 + t) * (nb + 1) + jr];
        const float fr = -(float)v.re, fi = -(float)v.im;
        h[0][t] = __float2bfloat16_rn(fr);
        h[1][t] = __float2bfloat16_rn(fi);
        h[2][t] = __float2bfloat16_rn(fr - __bfloat162float(h[0][t]));
        h[3][t] = __float2bfloat16_rn(fi - __bfloat162float(h[1][t]));
      }
      const size_t o = (size_t)jr * nb + r4;
#pragma unroll
      for (int pl = 0; pl < 4; ++pl)
        *reinterpret_cast<uint2*>(dst + 2 * pl * P + o) = *reinterpret_cast<const uint2*>(h[pl]);
    }
    __syncthreads();
  }
}

// Inverses of the pivoted group's pivot block from the packed LU of the outer panel (the
// interchanges already moved the pivot rows into K, so M_KK = L_KK U_KK):
//   Tinv slot 0: T = inv(M_KK) = inv(U_KK) inv(L_KK)        slot 1: inv(L_KK)
// row by row, as solves from the right of unit rows e_r: row r of T is e_r inv(U) inv(L)
// (forward with U from column r on, then backward with the unit-lower L), row r of inv(L)
// is e_r inv(L) (backward from column r down).  One CTA per block: the packed kb x kb LU and
// the reciprocals 1/u_jj sit in shared memory, and each warp solves whole rows with the row
// held in registers (lane l keeps columns l, l + 32, ...; the pivot entry of a step comes by
// shuffle), so a step needs no barrier.  Warp w of W takes the pairs (row r of T, row r of
// inv(L)) for r = w, w + W, ..., whose lengths add up to 2 kb steps.
template <typename S, typename C, int NT, bool FULL>
__global__ void __launch_bounds__(NT)
    k_tinv_warp(const S* M, int ldm, size_t mat_stride, size_t plane_stride, int k0, int kb,
                int nb, cpx<C>* Tinv, float* TT) {
  constexpr int NBMAX = sizeof(C) == 8 ? 64 : 128;
  constexpr int KQ = NBMAX / 32;  // columns per lane
  extern __shared__ unsigned char smem_raw[];
  cpx<C>* LU = reinterpret_cast<cpx<C>*>(smem_raw);  // kb x kb
  cpx<C>* dinv = LU + (size_t)kb * kb;               // kb
  const int mat = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const S* re = M + mat * mat_stride + (size_t)k0 * ldm + k0;  // the packed pivot block
  const S* im = re + plane_stride;
  for (int e = tid; e < kb * kb; e += blockDim.x) {
    const int a = e / kb, b = e - a * kb;
    const size_t o = (size_t)a * ldm + b;
    LU[e] = {(C)re[o], (C)im[o]};
  }
  __syncthreads();
  for (int k = tid; k < kb; k += blockDim.x) {
    const cpx<C> d = LU[k * kb + k];
    const C m2 = d.re * d.re + d.im * d.im;
    dinv[k] = {d.re / m2, -d.im / m2};
  }
  __syncthreads();
  cpx<C>* outT = Tinv + (size_t)mat * 2 * nb * nb;
  cpx<C>* outL = outT + (size_t)nb * nb;
  for (int r = warp; r < nb; r += NT / 32) {
#pragma unroll 1
    for (int part = 0; part < 2; ++part) {  // 0: row r of T, 1: row r of inv(L)
      C xr[KQ], xi[KQ];
#pragma unroll
      for (int q = 0; q < KQ; ++q) {
        xr[q] = (C)((q * 32 + lane == r) ? 1 : 0);
        xi[q] = (C)0;
      }
      if (r < kb) {
        if (part == 0) {  // x <- x inv(U): x_j /= u_jj, then x_k -= x_j u_jk (k > j)
#pragma unroll
          for (int q = 0; q < KQ; ++q) {
            for (int jj = 0; jj < 32; ++jj) {
              const int j = q * 32 + jj;
              if (j < r || j >= kb) continue;
              const C yr0 = __shfl_sync(0xffffffffu, xr[q], jj);
              const C yi0 = __shfl_sync(0xffffffffu, xi[q], jj);
              const cpx<C> d = dinv[j];
              const C yr = yr0 * d.re - yi0 * d.im, yi = yr0 * d.im + yi0 * d.re;
              if (lane == jj) { xr[q] = yr; xi[q] = yi; }
              const cpx<C>* u = LU + (size_t)j * kb;
#pragma unroll
              for (int q2 = q; q2 < KQ; ++q2) {  // k > j holds past chunk q
                const int k = q2 * 32 + lane;
                if ((q2 > q || lane > jj) && (FULL || k < kb)) {
                  const cpx<C> uv = u[k];
                  xr[q2] -= yr * uv.re - yi * uv.im;
                  xi[q2] -= yr * uv.im + yi * uv.re;
                }
              }
            }
          }
        }
        // x <- x inv(L): for j descending, x_k -= x_j l_jk (k < j); a unit row e_r of
        // inv(L) has x_j = 0 above r
        const int jtop = part == 0 ? kb - 1 : r;
#pragma unroll
        for (int q = KQ - 1; q >= 0; --q) {
          for (int jj = 31; jj >= 0; --jj) {
            const int j = q * 32 + jj;
            if (j > jtop || j < 1) continue;
            const C yr = __shfl_sync(0xffffffffu, xr[q], jj);
            const C yi = __shfl_sync(0xffffffffu, xi[q], jj);
            const cpx<C>* l = LU + (size_t)j * kb;
#pragma unroll
            for (int q2 = 0; q2 <= q; ++q2) {  // k < j holds before chunk q
              const int k = q2 * 32 + lane;
              if (q2 < q || lane < jj) {
                const cpx<C> lv = l[k];
                xr[q2] -= yr * lv.re - yi * lv.im;
                xi[q2] -= yr * lv.im + yi * lv.re;
              }
            }
          }
        }
      }
      cpx<C>* out = (part == 0 ? outT : outL) + (size_t)r * nb;
#pragma unroll
      for (int q = 0; q < KQ; ++q) {
        const int k = q * 32 + lane;
        if (k < nb) out[k] = (r < kb && k < kb) ? cpx<C>{xr[q], xi[q]} : cpx<C>{(C)0, (C)0};
      }
    }
  }
  if (!TT) return;
  __syncthreads();  // every row of T and inv(L) is written; the LU is no longer needed
  tinv_split_planes<C, NT>(outT, outL, LU, TT, nb, mat);
}

// The outputs of k_tinv_warp (float) by blocked triangular inversion, kb a multiple of 16:
//   1. the 16 x 16 diagonal blocks of L (unit lower) and of U (upper) inverted in place, one
//      warp per block and one lane per column (L's strictly lower part and U's upper part of a
//      diagonal block are disjoint, so the two warps of a block never touch each other's data);
//   2. X = inv(L) block row by block row downwards: Y = L[i, <i] X[<i, <i] into a buffer, then
//      X[i, <i] = -inv(L_ii) Y in place;
//   3. inv(U) block row by block row upwards the same way;
//   4. T = inv(U) inv(L), written with inv(L).
// Products run on 4 x 4 complex register tiles (4 + 4 operand loads per 16 complex FMAs).  In
// the block-row products each tile belongs to a group of 8 lanes that split its k-range and add
// their partial tiles by shuffles in a fixed order, so the result does not depend on timing.
constexpr int kTinvB = 16;

__device__ __forceinline__ void tile_fma(cpx<float> (&acc)[4][4], const cpx<float> (&a)[4],
                                         const cpx<float> (&b)[4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      acc[i][j].re = fmaf(a[i].re, b[j].re, fmaf(-a[i].im, b[j].im, acc[i][j].re));
      acc[i][j].im = fmaf(a[i].re, b[j].im, fmaf(a[i].im, b[j].re, acc[i][j].im));
    }
}

__device__ __forceinline__ void tile_zero(cpx<float> (&acc)[4][4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = {0.f, 0.f};
}

// sum of the tiles of the 8 lanes of a group (lanes 8g .. 8g + 7), every lane of the warp
__device__ __forceinline__ void tile_group_sum(cpx<float> (&acc)[4][4]) {
#pragma unroll
  for (int off = 1; off < 8; off <<= 1)
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        acc[i][j].re += __shfl_xor_sync(0xffffffffu, acc[i][j].re, off);
        acc[i][j].im += __shfl_xor_sync(0xffffffffu, acc[i][j].im, off);
      }
}

template <typename S, int NT>
__global__ void __launch_bounds__(NT)
    k_tinv_blocked(const S* M, int ldm, size_t mat_stride, size_t plane_stride, int k0, int kb,
                   int nb, cpx<float>* Tinv, float* TT) {
  using C = float;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // row stride kb + 2: tile columns stay 16-byte aligned and consecutive rows start 4 banks
  // apart, so the column reads of 8 consecutive rows (the block-row products) do not conflict
  const int ls = kb + 2;
  cpx<C>* A = reinterpret_cast<cpx<C>*>(smem_raw);          // kb x ls: LU, then the inverses
  cpx<C>* Y = A + (size_t)kb * ls;                          // kTinvB x kb block-row products
  const int mat = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int grp = tid >> 3, sub = tid & 7;                  // groups of 8 lanes
  const int nbk = kb / kTinvB;
  const cpx<C> one = {(C)1, (C)0}, zero = {(C)0, (C)0};
  const S* re = M + mat * mat_stride + (size_t)k0 * ldm + k0;  // the packed pivot block
  const S* im = re + plane_stride;
  for (int e = tid; e < kb * kb; e += NT) {
    const int a = e / kb, b = e - a * kb;
    A[(size_t)a * ls + b] = {(C)re[(size_t)a * ldm + b], (C)im[(size_t)a * ldm + b]};
  }
  __syncthreads();
  // 1. diagonal blocks: lane l computes column l of the block's inverse, then writes it
  for (int task = warp; task < 2 * nbk; task += NT / 32) {
    if (lane < kTinvB) {
      const int d0 = (task >> 1) * kTinvB, l = lane;
      cpx<C>* D = A + (size_t)d0 * ls + d0;
      cpx<C> x[kTinvB];
      if ((task & 1) == 0) {  // unit lower: forward substitution
#pragma unroll
        for (int r = 0; r < kTinvB; ++r) {
          cpx<C> v = (r == l) ? one : zero;
#pragma unroll
          for (int k = 0; k < r; ++k) {
            const cpx<C> t = cmul(D[r * ls + k], x[k]);
            v.re -= t.re;
            v.im -= t.im;
          }
          x[r] = v;
        }
        __syncwarp(0xffffu);
#pragma unroll
        for (int r = 0; r < kTinvB; ++r)
          if (r > l) D[r * ls + l] = x[r];
      } else {  // upper: back substitution with the diagonal
#pragma unroll
        for (int r = kTinvB - 1; r >= 0; --r) {
          cpx<C> v = (r == l) ? one : zero;
#pragma unroll
          for (int k = r + 1; k < kTinvB; ++k) {
            const cpx<C> t = cmul(D[r * ls + k], x[k]);
            v.re -= t.re;
            v.im -= t.im;
          }
          const cpx<C> u = D[r * ls + r];
          const C m2 = u.re * u.re + u.im * u.im;
          x[r] = cmul(v, cpx<C>{u.re / m2, -u.im / m2});
        }
        __syncwarp(0xffffu);
#pragma unroll
        for (int r = 0; r < kTinvB; ++r)
          if (r <= l) D[r * ls + l] = x[r];
      }
    }
  }
  __syncthreads();
  // 2. inv(L) downwards.  X[k][c] = 1 (k == c), A[k][c] (k > c), 0 (k < c)
  for (int bi = 1; bi < nbk; ++bi) {
    const int r0 = bi * kTinvB, tcs = r0 / 4, ntile = 4 * tcs;
    // (a) Y = L[r0 .., 0 .. r0) X[0 .. r0, 0 .. r0): tile (4 rows R, 4 columns C0), k >= C0
    for (int t0 = 0; t0 < ntile; t0 += NT / 8) {
      const int t = t0 + grp;
      const bool act = t < ntile;
      const int R = act ? 4 * (t / tcs) : 0, C0 = act ? 4 * (t % tcs) : 0;
      cpx<C> acc[4][4];
      tile_zero(acc);
      if (act)
        for (int k = C0 + sub; k < r0; k += 8) {
          cpx<C> a[4], x[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) a[i] = A[(size_t)(r0 + R + i) * ls + k];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int c = C0 + j;
            x[j] = k > c ? A[(size_t)k * ls + c] : (k == c ? one : zero);
          }
          tile_fma(acc, a, x);
        }
      tile_group_sum(acc);
      if (act && sub == 0)
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) Y[(R + i) * kb + C0 + j] = acc[i][j];
    }
    __syncthreads();
    // (b) X[r0 + r][c] = -(Y[r][c] + sum_{m < r} inv(L_ii)[r][m] Y[m][c]), a tile per thread
    for (int t = tid; t < ntile; t += NT) {
      const int R = 4 * (t / tcs), C0 = 4 * (t % tcs);
      cpx<C> acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = Y[(R + i) * kb + C0 + j];
#pragma unroll 4
      for (int m = 0; m < R + 3; ++m) {
        cpx<C> a[4], y[4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
          a[i] = m < R + i ? A[(size_t)(r0 + R + i) * ls + r0 + m] : zero;
#pragma unroll
        for (int j = 0; j < 4; ++j) y[j] = Y[m * kb + C0 + j];
        tile_fma(acc, a, y);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          A[(size_t)(r0 + R + i) * ls + C0 + j] = {-acc[i][j].re, -acc[i][j].im};
    }
    __syncthreads();
  }
  // 3. inv(U) upwards.  XU[k][c] = A[k][c] (k <= c), 0 (k > c)
  for (int bi = nbk - 2; bi >= 0; --bi) {
    const int r0 = bi * kTinvB, c0 = r0 + kTinvB, tcs = (kb - c0) / 4, ntile = 4 * tcs;
    // (a) Y[r][cc] = sum_{k = c0}^{c} U[r0 + r][k] XU[k][c], c = c0 + cc
    for (int t0 = 0; t0 < ntile; t0 += NT / 8) {
      const int t = t0 + grp;
      const bool act = t < ntile;
      const int R = act ? 4 * (t / tcs) : 0, C0 = act ? 4 * (t % tcs) : 0;
      cpx<C> acc[4][4];
      tile_zero(acc);
      if (act)
        for (int k = c0 + sub; k <= c0 + C0 + 3; k += 8) {
          cpx<C> a[4], x[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) a[i] = A[(size_t)(r0 + R + i) * ls + k];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int c = c0 + C0 + j;
            x[j] = k <= c ? A[(size_t)k * ls + c] : zero;
          }
          tile_fma(acc, a, x);
        }
      tile_group_sum(acc);
      if (act && sub == 0)
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) Y[(R + i) * kb + C0 + j] = acc[i][j];
    }
    __syncthreads();
    // (b) X[r0 + r][c] = -sum_{m >= r} inv(U_ii)[r][m] Y[m][cc], a tile per thread
    for (int t = tid; t < ntile; t += NT) {
      const int R = 4 * (t / tcs), C0 = 4 * (t % tcs);
      cpx<C> acc[4][4];
      tile_zero(acc);
#pragma unroll 4
      for (int m = R; m < kTinvB; ++m) {
        cpx<C> a[4], y[4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
          a[i] = m >= R + i ? A[(size_t)(r0 + R + i) * ls + r0 + m] : zero;
#pragma unroll
        for (int j = 0; j < 4; ++j) y[j] = Y[m * kb + C0 + j];
        tile_fma(acc, a, y);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          A[(size_t)(r0 + R + i) * ls + c0 + C0 + j] = {-acc[i][j].re, -acc[i][j].im};
    }
    __syncthreads();
  }
  // 4. T[r][c] = sum_{k >= max(r, c)} XU[r][k] XL[k][c]: warp = tile row, lane = tile column
  cpx<C>* outT = Tinv + (size_t)mat * 2 * nb * nb;
  cpx<C>* outL = outT + (size_t)nb * nb;
  for (int tr = warp; tr < nb / 4; tr += NT / 32) {
    const int R0 = 4 * tr;
    for (int tcl = lane; tcl < nb / 4; tcl += 32) {
      const int C0 = 4 * tcl;
      cpx<C> acc[4][4];
      tile_zero(acc);
      if (R0 < kb && C0 < kb)
        for (int k = R0; k < kb; ++k) {
          cpx<C> u[4], x[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) u[i] = k >= R0 + i ? A[(size_t)(R0 + i) * ls + k] : zero;
          const float4 x01 = *reinterpret_cast<const float4*>(A + (size_t)k * ls + C0);
          const float4 x23 = *reinterpret_cast<const float4*>(A + (size_t)k * ls + C0 + 2);
          const cpx<C> xs[4] = {{x01.x, x01.y}, {x01.z, x01.w}, {x23.x, x23.y}, {x23.z, x23.w}};
#pragma unroll
          for (int j = 0; j < 4; ++j) x[j] = k > C0 + j ? xs[j] : (k == C0 + j ? one : zero);
          tile_fma(acc, u, x);
        }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int r = R0 + i, c = C0 + j;
          const bool in = r < kb && c < kb;
          outT[(size_t)r * nb + c] = in ? acc[i][j] : zero;
          outL[(size_t)r * nb + c] =
              (in && r >= c) ? (r == c ? one : A[(size_t)r * ls + c]) : zero;
        }
    }
  }
  if (!TT) return;
  __syncthreads();  // every row of T and inv(L) is written; the LU copy is no longer needed
  tinv_split_planes<C, NT>(outT, outL, A, TT, nb, mat);
}

// A operand of the pivoted group's tensor-core prep product: the columns K of rows
// [r_begin, N) as bf16 split planes (re_hi, im_hi, re_lo, im_lo; columns past kb zero) in the
// block's W planes, which k_prep_w rewrites afterwards.  4 columns per thread.
template <typename S>
__global__ void __launch_bounds__(256)
    k_split_a(const S* M, int N, int ldm, size_t mat_stride, size_t plane_stride, int k0, int kb,
              int nb, float* W, size_t fw_plane, size_t fw_mat, int r_begin) {
  const int mat = blockIdx.y;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int q4 = nb / 4;
  const int i = r_begin + (int)(e / q4), c4 = (int)(e % q4) * 4;
  if (i >= N) return;
  const S* re = M + mat * mat_stride + (size_t)i * ldm + k0;
  const S* im = re + plane_stride;
  __nv_bfloat16 h[4][4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int c = c4 + t;
    const float fr = c < kb ? (float)re[c] : 0.f, fi = c < kb ? (float)im[c] : 0.f;
    h[0][t] = __float2bfloat16_rn(fr);
    h[1][t] = __float2bfloat16_rn(fi);
    h[2][t] = __float2bfloat16_rn(fr - __bfloat162float(h[0][t]));
    h[3][t] = __float2bfloat16_rn(fi - __bfloat162float(h[1][t]));
  }
  float* w = W + mat * fw_mat;
  const size_t o = (size_t)i * nb + c4;
#pragma unroll
  for (int pl = 0; pl < 4; ++pl)
    *reinterpret_cast<uint2*>(reinterpret_cast<__nv_bfloat16*>(w + pl * fw_plane) + o) =
        *reinterpret_cast<const uint2*>(h[pl]);
}

// Eight consecutive entries of the F/W planes starting at element o (8-aligned): re/im planes
// of S (split 0; only the first n entries), TF32-split float planes (1) or bf16-split planes
// (2), {re_hi, im_hi, re_lo, im_lo} for both splits (row length a multiple of 8 there).
template <typename S>
__device__ __forceinline__ void store_fw8(S* base, size_t plane, size_t o, const float* vr,
                                          const float* vi, const S* dr, const S* di, int split,
                                          int n) {
  if (split == 2) {
    __nv_bfloat16 h[4][8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      h[0][e] = __float2bfloat16_rn(vr[e]);
      h[1][e] = __float2bfloat16_rn(vi[e]);
      h[2][e] = __float2bfloat16_rn(vr[e] - __bfloat162float(h[0][e]));
      h[3][e] = __float2bfloat16_rn(vi[e] - __bfloat162float(h[1][e]));
    }
    float* b = reinterpret_cast<float*>(base);
#pragma unroll
    for (int pl = 0; pl < 4; ++pl)
      *reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(b + pl * plane) + o) =
          *reinterpret_cast<const uint4*>(h[pl]);
  } else if (split == 1) {
    float f[4][8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const float hr = __uint_as_float(__float_as_uint(vr[e]) & 0xffffe000u);
      const float hi = __uint_as_float(__float_as_uint(vi[e]) & 0xffffe000u);
      f[0][e] = hr; f[1][e] = hi; f[2][e] = vr[e] - hr; f[3][e] = vi[e] - hi;
    }
    float* b = reinterpret_cast<float*>(base);
#pragma unroll
    for (int pl = 0; pl < 4; ++pl) {
      float4* d = reinterpret_cast<float4*>(b + pl * plane + o);
      d[0] = make_float4(f[pl][0], f[pl][1], f[pl][2], f[pl][3]);
      d[1] = make_float4(f[pl][4], f[pl][5], f[pl][6], f[pl][7]);
    }
  } else {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      if (e < n) {
        base[o + e] = dr[e];
        base[plane + o + e] = di[e];
      }
    }
  }
}

// W^T: 64 columns j x nb per CTA.  Columns past K of a symmetric block come from the column
// strip M[j][K] (the upper entries M[K][j] are the transposed lower ones, both unswept) and
// are copied row by row; the others come from the row strip M[K][j] and are transposed
// through shared memory.  Each thread converts and writes 8 consecutive entries of a W^T row.
template <typename S>
__global__ void __launch_bounds__(256)
    k_prep_w(const S* M, int N, int ldm, size_t mat_stride, size_t plane_stride, int k0, int kb,
             int nb, S* W, size_t fw_plane, size_t fw_mat, int c_begin, int gj, int split,
             int sym) {
  extern __shared__ unsigned char smem_raw[];
  const int ts = nb + 4;                    // shared row stride (16-byte aligned rows)
  S* tr = reinterpret_cast<S*>(smem_raw);   // [64][ts]
  S* ti = tr + (size_t)64 * ts;
  const int mat = blockIdx.y;
  const int j0 = c_begin + blockIdx.x * 64;
  const S* re = M + mat * mat_stride;
  const S* im = re + plane_stride;
  const bool direct = sym && j0 >= k0 + kb;
  if (!direct) {
    // the row strip's loads go out eight at a time before their shared-memory stores
    constexpr int LU = 8;
    for (int e0 = threadIdx.x; e0 < nb * 64; e0 += 256 * LU) {
      S xr[LU], xi[LU];
#pragma unroll
      for (int u = 0; u < LU; ++u) {
        const int e = e0 + 256 * u;
        const int c = e >> 6, j = j0 + (e & 63);
        const bool in = e < nb * 64 && c < kb && j < N;
        xr[u] = in ? re[(size_t)(k0 + c) * ldm + j] : (S)0;
        xi[u] = in ? im[(size_t)(k0 + c) * ldm + j] : (S)0;
      }
#pragma unroll
      for (int u = 0; u < LU; ++u) {
        const int e = e0 + 256 * u;
        if (e < nb * 64) {
          tr[(e & 63) * ts + (e >> 6)] = xr[u];
          ti[(e & 63) * ts + (e >> 6)] = xi[u];
        }
      }
    }
    __syncthreads();
  }
  S* out = W + (size_t)mat * fw_mat;
  const int g8 = (nb + 7) / 8;  // the split planes have nb = 128; plain ones may be narrower
  // IT groups of 8 entries per thread: every load of the IT groups is issued before the first
  // conversion and store
  constexpr int IT = sizeof(S) == 4 ? 4 : 2;
  for (int e0 = threadIdx.x; e0 < 64 * g8; e0 += 256 * IT) {
    S dr[IT][8], di[IT][8];
#pragma unroll
    for (int u = 0; u < IT; ++u) {
      const int e = e0 + 256 * u;
      const int jj = e / g8, c8 = (e - jj * g8) * 8;
      const int j = j0 + jj;
      if (e >= 64 * g8 || j >= N) continue;
      if (gj && j >= k0 && j < k0 + kb) {
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          dr[u][t] = (c8 + t == j - k0) ? (S)1 : (S)0;
          di[u][t] = (S)0;
        }
      } else if (direct) {
        const S* rr = re + (size_t)j * ldm + k0 + c8;
        const S* ri = im + (size_t)j * ldm + k0 + c8;
        if (sizeof(S) == 4 && c8 + 8 <= kb &&
            ((reinterpret_cast<uintptr_t>(rr) | reinterpret_cast<uintptr_t>(ri)) & 15) == 0) {
          const float4* vr4 = reinterpret_cast<const float4*>(rr);
          const float4* vi4 = reinterpret_cast<const float4*>(ri);
          const float4 a0 = vr4[0], a1 = vr4[1], b0 = vi4[0], b1 = vi4[1];
          const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
          const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            dr[u][t] = (S)av[t];
            di[u][t] = (S)bv[t];
          }
        } else {
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            const bool in = c8 + t < kb;
            dr[u][t] = in ? rr[t] : (S)0;
            di[u][t] = in ? ri[t] : (S)0;
          }
        }
      } else {
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const bool in = c8 + t < nb;
          dr[u][t] = in ? tr[jj * ts + c8 + t] : (S)0;
          di[u][t] = in ? ti[jj * ts + c8 + t] : (S)0;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < IT; ++u) {
      const int e = e0 + 256 * u;
      const int jj = e / g8, c8 = (e - jj * g8) * 8;
      const int j = j0 + jj;
      if (e >= 64 * g8 || j >= N) continue;
      float vr[8], vi[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) { vr[t] = (float)dr[u][t]; vi[t] = (float)di[u][t]; }
      store_fw8(out, fw_plane, (size_t)j * nb + c8, vr, vi, dr[u], di[u], split, nb - c8);
    }
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
// Adjoint diag(G).  Per block and row i: x = row i of X = A^{-1} (X[i, perm[r]] = R[i, r]),
//   G_ii = 2 x_i - (x^T A x)    (refine: one Newton step on the inverse, diagonal only)
//   G_ii = x_i                  (no refinement)
// and gd[b*N + i] = sigma_b Re G_ii.  With A the 5-point stencil (A_jj = a_j + i w_n,
// A_jk = t per bond) the quadratic form is a sum over sites and bonds:
//   Re(x^T A x) = sum_j [a_j (Re x_j^2) - w_n Im x_j^2 + 2t Re(x_j (x_{j+x} + x_{j+y}))].
// The residual it cancels against is ~1e-6 of its size, so it is evaluated to about 2^-44
// relative: products of the stored float32 values are split exactly with FMA (TwoProduct)
// and summed in double-float (TwoSum) arithmetic on the FP32 pipes, except for 32-site chunks
// far from site i, whose terms are bounded as in k_refine_direct and summed in float32; the
// float64 result is formed once per row.  One warp per row, the row scattered into natural order in shared
// memory, a_j cached per CTA as a double-float pair.
template <typename S>
__global__ void k_refine(const S* M, int ldm, size_t mat_stride, size_t plane_stride, int b0,
                         Lattice la0, const int* perm, double* gd, int refine) {
  extern __shared__ unsigned char smem_raw[];
  const int N = la0.N, L = la0.L;
  const int mat = blockIdx.y, b = b0 + mat;
  int n, sg;
  const Lattice la = block_lattice(la0, b, n, sg);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  int* sperm = reinterpret_cast<int*>(smem_raw);
  const S* re = M + mat * mat_stride;
  const S* im = re + plane_stride;
  if (!refine || sizeof(S) != 4) {  // sperm holds the inverse permutation
    for (int r = threadIdx.x; r < N; r += blockDim.x) sperm[perm[(size_t)mat * N + r]] = r;
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
      gd[(size_t)b * N + i] = sg * (double)re[(size_t)i * ldm + sperm[i]];
    return;
  }
  const size_t perm_bytes = ((N * sizeof(int) + 15) / 16) * 16;
  dsf* adiag = reinterpret_cast<dsf*>(smem_raw + perm_bytes);  // N: Re A_jj as double-float
  cpx<S>* rows = reinterpret_cast<cpx<S>*>(smem_raw + perm_bytes + (size_t)N * sizeof(dsf));
  cpx<S>* x = rows + (size_t)warp * N;
  for (int r = threadIdx.x; r < N; r += blockDim.x) {
    sperm[r] = perm[(size_t)mat * N + r];
    adiag[r] = ds_of(la.mu - site_energy(la, r, sg));
  }
  __syncthreads();
  const double w = (2.0 * n + 1.0) * kPi * la.T;
  const dsf w2 = ds_of(2.0 * w), t2 = ds_of(2.0 * la.t);
  const float w2f = w2.h, t2f = t2.h, w2a = fabsf(w2.h), t2a = fabsf(t2.h);
  const float small = 0x1.0p-18f / (float)N;  // the float32 bound of k_refine_direct
  const int dxs = 32 / L, dys = 32 % L;  // advance of (x, y) when j grows by 32
  for (int i = blockIdx.x * nwarps + warp; i < N; i += gridDim.x * nwarps) {
    for (int r = lane; r < N; r += 32)
      x[sperm[r]] = {re[(size_t)i * ldm + r], im[(size_t)i * ldm + r]};
    __syncwarp();
    dsf acc = {0.f, 0.f};
    float accf = 0.f;
    int xx = lane / L, yy = lane - (lane / L) * L;
    for (int j0 = 0; j0 < N; j0 += 32) {  // warp-uniform trip count
      const int j = j0 + lane;
      const bool in = j < N;
      const int jx = (xx + 1 == L) ? yy : j + L;
      const int jy = (yy + 1 == L) ? j + 1 - L : j + 1;
      const float a = in ? (float)x[j].re : 0.f, bq = in ? (float)x[j].im : 0.f;
      const float ax = in ? (float)x[jx].re : 0.f, bx = in ? (float)x[jx].im : 0.f;
      const float ay = in ? (float)x[jy].re : 0.f, by = in ? (float)x[jy].im : 0.f;
      const dsf ad = in ? adiag[j] : dsf{0.f, 0.f};
      yy += dys;
      xx += dxs;
      if (yy >= L) { yy -= L; xx += 1; }
      const float aa = fabsf(a), ba = fabsf(bq);
      const float sj = fabsf(ad.h) * (aa * aa + ba * ba) + w2a * (aa * ba) +
                       t2a * (aa * (fabsf(ax) + fabsf(ay)) + ba * (fabsf(bx) + fabsf(by)));
      if (__any_sync(0xffffffffu, !(sj <= small))) {
        const dsf q = ds_sub(two_prod(a, a), two_prod(bq, bq));   // Re x_j^2
        const dsf ab = two_prod(a, bq);                            // Im x_j^2 / 2
        const dsf u = ds_add(ds_sub(two_prod(a, ax), two_prod(bq, bx)),
                             ds_sub(two_prod(a, ay), two_prod(bq, by)));
        const dsf e = ds_add(ds_sub(ds_mul(ad, q), ds_mul(w2, ab)), ds_mul(t2, u));
        acc = ds_add(acc, e);
      } else {
        accf += ad.h * (a * a - bq * bq) - w2f * (a * bq) + t2f * (a * (ax + ay) - bq * (bx + by));
      }
    }
    acc = ds_add(acc, dsf{accf, 0.f});
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const dsf o = {__shfl_xor_sync(0xffffffffu, acc.h, off),
                     __shfl_xor_sync(0xffffffffu, acc.l, off)};
      acc = ds_add(acc, o);
    }
    if (lane == 0) {
      const double qsum = (double)acc.h + (double)acc.l;
      gd[(size_t)b * N + i] = sg * (2.0 * (double)x[i].re - qsum);
    }
    __syncwarp();
  }
}

// The same refinement for unpivoted blocks (X = R, no permutation): each warp reads its row
// straight from the inverse, the bond partners x_{j+L} and x_{j+1} come through L1, and only
// the double-float a_j sit in shared memory.  The double-float arithmetic costs ~140 FP32
// operations per site, so the kernel is ALU-bound; away from site i, where the inverse has
// decayed, it is not needed: a warp whose 32 sites all have term magnitudes
//   s_j = |a_j| |x_j|^2 + 2 w_n |Re x_j Im x_j| + 2|t| (|Re x_j| (|Re x_{j+x}| + |Re x_{j+y}|)
//         + |Im x_j| (|Im x_{j+x}| + |Im x_{j+y}|))
// below 2^-18 / N sums them in plain float32 into a second accumulator.  Each such term is
// then off by less than ~2^-21 s_j, so all of them together by less than 2^-39 (absolute) in
// G_ii; the sites near i keep the double-float arithmetic of k_refine.
constexpr int kRefineRowsPerCta = 64;
constexpr int kRefineUnroll = 4;

// Re A_jj = mu - eps_j of each block as a double-float pair, once per block (FP64 is a slow
// pipe here; the refinement's CTAs then stage the table instead of recomputing it).
__global__ void __launch_bounds__(256)
    k_adiag(Lattice la0, int b0, dsf* __restrict__ out) {
  const int N = la0.N;
  const int mat = blockIdx.y, b = b0 + mat;
  int n, sg;
  const Lattice la = block_lattice(la0, b, n, sg);
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < N) out[(size_t)mat * N + r] = ds_of(la.mu - site_energy(la, r, sg));
}

__global__ void __launch_bounds__(256, 4)
    k_refine_direct(const float* __restrict__ M, int ldm, size_t mat_stride, size_t plane_stride,
                    int b0, Lattice la0, const dsf* __restrict__ adiag_g, double* __restrict__ gd) {
  extern __shared__ unsigned char smem_raw[];
  dsf* adiag = reinterpret_cast<dsf*>(smem_raw);
  const int N = la0.N, L = la0.L;
  const int mat = blockIdx.y, b = b0 + mat;
  int n, sg;
  const Lattice la = block_lattice(la0, b, n, sg);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int r = threadIdx.x; r < N; r += blockDim.x) adiag[r] = adiag_g[(size_t)mat * N + r];
  __syncthreads();
  const float* re0 = M + mat * mat_stride;
  const float* im0 = re0 + plane_stride;
  const double w = (2.0 * n + 1.0) * kPi * la.T;
  const dsf w2 = ds_of(2.0 * w), t2 = ds_of(2.0 * la.t);
  const float w2f = w2.h, t2f = t2.h, w2a = fabsf(w2.h), t2a = fabsf(t2.h);
  const float small = 0x1.0p-18f / (float)N;
  const int dxs = 32 / L, dys = 32 % L;
  const int i_end = min(N, (int)(blockIdx.x + 1) * kRefineRowsPerCta);
  for (int i = blockIdx.x * kRefineRowsPerCta + warp; i < i_end; i += 8) {
    const float* re = re0 + (size_t)i * ldm;
    const float* im = im0 + (size_t)i * ldm;
    dsf acc = {0.f, 0.f};
    float accf = 0.f;
    int xx = lane / L, yy = lane - (lane / L) * L;
    // kRefineUnroll chunks of 32 sites per round: all their loads are issued before any of
    // them is used, so a warp keeps several row segments in flight
    for (int j0 = 0; j0 < N; j0 += 32 * kRefineUnroll) {  // warp-uniform trip count
      float a[kRefineUnroll], bq[kRefineUnroll], ax[kRefineUnroll], bx[kRefineUnroll];
      float ay[kRefineUnroll], by[kRefineUnroll];
#pragma unroll
      for (int u = 0; u < kRefineUnroll; ++u) {
        const int j = j0 + 32 * u + lane;
        const bool in = j < N;
        const int jx = (xx + 1 == L) ? yy : j + L;
        const int jy = (yy + 1 == L) ? j + 1 - L : j + 1;
        a[u] = in ? re[j] : 0.f;
        bq[u] = in ? im[j] : 0.f;
        ax[u] = in ? re[jx] : 0.f;
        bx[u] = in ? im[jx] : 0.f;
        ay[u] = in ? re[jy] : 0.f;
        by[u] = in ? im[jy] : 0.f;
        yy += dys;
        xx += dxs;
        if (yy >= L) { yy -= L; xx += 1; }
      }
#pragma unroll
      for (int u = 0; u < kRefineUnroll; ++u) {
        const int j = j0 + 32 * u + lane;
        const dsf ad = j < N ? adiag[j] : dsf{0.f, 0.f};
        const float aa = fabsf(a[u]), ba = fabsf(bq[u]);
        const float sj = fabsf(ad.h) * (aa * aa + ba * ba) + w2a * (aa * ba) +
                         t2a * (aa * (fabsf(ax[u]) + fabsf(ay[u])) +
                                ba * (fabsf(bx[u]) + fabsf(by[u])));
        if (__any_sync(0xffffffffu, !(sj <= small))) {
          const dsf q = ds_sub(two_prod(a[u], a[u]), two_prod(bq[u], bq[u]));
          const dsf ab = two_prod(a[u], bq[u]);
          const dsf uu = ds_add(ds_sub(two_prod(a[u], ax[u]), two_prod(bq[u], bx[u])),
                                ds_sub(two_prod(a[u], ay[u]), two_prod(bq[u], by[u])));
          const dsf e = ds_add(ds_sub(ds_mul(ad, q), ds_mul(w2, ab)), ds_mul(t2, uu));
          acc = ds_add(acc, e);
        } else {
          accf += ad.h * (a[u] * a[u] - bq[u] * bq[u]) - w2f * (a[u] * bq[u]) +
                  t2f * (a[u] * (ax[u] + ay[u]) - bq[u] * (bx[u] + by[u]));
        }
      }
    }
    // the warp's sum in double-float too; float64 only for the one result of the row
    acc = ds_add(acc, dsf{accf, 0.f});
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const dsf o = {__shfl_xor_sync(0xffffffffu, acc.h, off),
                     __shfl_xor_sync(0xffffffffu, acc.l, off)};
      acc = ds_add(acc, o);
    }
    if (lane == 0) {
      const double qsum = (double)acc.h + (double)acc.l;
      gd[(size_t)b * N + i] = sg * (2.0 * (double)re[i] - qsum);
    }
  }
}

// ---------------------------------------------- refinement from the lower triangle
// The symmetric dominant blocks leave X = A^{-1} in the tiles on or below the diagonal only.
// The quadratic form of row i, q_i = Re(x^T A x) with x_j = X_ij, is a sum over sites j of
//   e_j = a_j Re x_j^2 - 2 w Re x_j Im x_j + 2t Re(x_j (x_{j+x} + x_{j+y}))
// (a_j = Re A_jj, bonds to the +x and +y neighbours), which splits exactly into
//   row part     : the site terms of j <= i and the bonds with both ends <= i (x_j = X[i][j]),
//   column part  : the site terms of j > i and the bonds with both ends > i (x_j = X[j][i]),
//   boundary     : the bonds with one end on each side: (i, i+1), (j, j+L) for i-L < j <= i, and
//                  the periodic wraps (j, j+1-L) for i < j < i+L with y_j = L-1, (j, j+L-N) for
//                  j >= N-L with j+L-N <= i (at most 2L+2 bonds, in double-float),
// so every value comes from the lower triangle and no mirror pass is needed.  k_refine_lower_rows
// sums the row part and the boundary (one warp per row) into a double-float partial;
// k_refine_lower_cols streams each 64-column strip down its rows for the column part, adds the
// partial in a fixed order and writes G_ii.
//
// Both kernels take two adjacent entries per lane (8-byte loads; L and N are even, so a pair
// never straddles a lattice row in the row kernel and the +x partners form a pair too) and
// vote per group of 64 entries on m = the largest |Re|, |Im| among the entries and their bond
// partners.  Every term satisfies |e_j| <= C m^2 with C = 2 max|a_j| + 2w + 4|2t|, so a group
// with m^2 <= small / C (small = 2^-18 / N, the bound of k_refine_direct) is summed in float32
// within the same 2^-39 total error; any other group takes the double-float path.  There the
// exact products (two_prod) go into three compensated sums (the terms a_j Re x_j^2, the Re x Im x
// products and the bond products; each a float32 sum and the float32 sum of the rounding errors
// of its additions), scaled by -2w and 2t once per row.
constexpr int kLowerRowsPerCta = 64;
constexpr int kLowerUnroll = 2;  // 64-entry groups per round of loads

// compensated float32 sum of exact products: s the running sum, e the rounding errors of its
// additions plus the products' low parts
struct csum {
  float s, e;
};
__device__ __forceinline__ void csum_add(csum& c, dsf p) {
  const dsf t = two_sum(c.s, p.h);
  c.s = t.h;
  c.e += t.l + p.l;
}
__device__ __forceinline__ dsf csum_val(csum c) { return fast_two_sum(c.s, c.e); }

// the double-float terms of one site: a_j Re x^2 into s1, Re x Im x into s2, the two bond
// products Re(x x_x) + Re(x x_y) into s3
__device__ __forceinline__ void site_terms_ds(float a, float b, float ax, float bx, float ay,
                                              float by, dsf ad, csum& s1, csum& s2, csum& s3) {
  csum_add(s1, ds_mul(ad, ds_sub(two_prod(a, a), two_prod(b, b))));
  csum_add(s2, two_prod(a, b));
  csum_add(s3, two_prod(a, ax));
  csum_add(s3, two_prod(-b, bx));
  csum_add(s3, two_prod(a, ay));
  csum_add(s3, two_prod(-b, by));
}

// the same terms in float32 (f1: a_j Re x^2, f2: Re x Im x, f3: bond products)
__device__ __forceinline__ void site_terms_f(float a, float b, float ax, float bx, float ay,
                                             float by, float adh, float& f1, float& f2,
                                             float& f3) {
  f1 = fmaf(adh, fmaf(a, a, -b * b), f1);
  f2 = fmaf(a, b, f2);
  f3 = fmaf(a, ax + ay, f3);
  f3 = fmaf(-b, bx + by, f3);
}

// one lane's total: S1 - 2w S2 + 2t S3 plus the float32 parts
__device__ __forceinline__ dsf lane_total(csum s1, csum s2, csum s3, float f1, float f2,
                                          float f3, dsf w2, dsf t2) {
  dsf r = ds_sub(csum_val(s1), ds_mul(w2, csum_val(s2)));
  r = ds_add(r, ds_mul(t2, csum_val(s3)));
  return ds_add(r, two_sum(f1, fmaf(-w2.h, f2, t2.h * f3)));
}

// stage the block's Re A_jj table in shared memory and return m^2's threshold small / C
__device__ __forceinline__ float stage_adiag(const dsf* __restrict__ adiag_g, dsf* adiag, int N,
                                             float w2a, float t2a, float* red) {
  float amax = 0.f;
  for (int r = threadIdx.x; r < N; r += blockDim.x) {
    const dsf v = adiag_g[r];
    adiag[r] = v;
    amax = fmaxf(amax, fabsf(v.h));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = amax;
  __syncthreads();
  amax = 0.f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) amax = fmaxf(amax, red[w]);
  // C rounded up by a relative 2^-20 (|a_j| carries its low part, w and t their roundings)
  const float C = (2.f * amax + w2a + 4.f * t2a) * (1.f + 0x1.0p-20f);
  return (0x1.0p-18f / (float)N) / C;
}

// Row part and boundary bonds, one warp per row i.  Round r covers the sites j0 .. j0 + 127 as
// two groups of 64, lane l taking the pair (p, p + 1), p = j0 + 64 u + 2 l: y_p is even, so p + 1
// is p's +y partner (no wrap) and p's +x partner jx is even with jx + 1 the +x partner of p + 1;
// only p + 1's +y partner (p + 2, or p + 2 - L on a wrap) is loaded on its own.  Masks are
// applied only in the rounds that reach past site i - L.
__global__ void __launch_bounds__(256, 4)
    k_refine_lower_rows(const float* __restrict__ M, int ldm, size_t mat_stride,
                        size_t plane_stride, int b0, Lattice la0,
                        const dsf* __restrict__ adiag_g, double* __restrict__ gd) {
  extern __shared__ unsigned char smem_raw[];
  dsf* adiag = reinterpret_cast<dsf*>(smem_raw);
  __shared__ float red[8];
  const int N = la0.N, L = la0.L;
  const int mat = blockIdx.y, b = b0 + mat;
  int n, sg;
  const Lattice la = block_lattice(la0, b, n, sg);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float* re0 = M + mat * mat_stride;
  const float* im0 = re0 + plane_stride;
  const double w = (2.0 * n + 1.0) * kPi * la.T;
  const dsf w2 = ds_of(2.0 * w), t2 = ds_of(2.0 * la.t);
  const float thr2 = stage_adiag(adiag_g + (size_t)mat * N, adiag, N, fabsf(w2.h), fabsf(t2.h), red);
  const int dx64 = 64 / L, dy64 = 64 % L;
  const int i_end = min(N, (int)(blockIdx.x + 1) * kLowerRowsPerCta);
  for (int i = blockIdx.x * kLowerRowsPerCta + warp; i < i_end; i += 8) {
    const float* re = re0 + (size_t)i * ldm;  // row i: X[i][j] for j <= i
    const float* im = im0 + (size_t)i * ldm;
    csum s1 = {0.f, 0.f}, s2 = {0.f, 0.f}, s3 = {0.f, 0.f};
    float f1 = 0.f, f2 = 0.f, f3 = 0.f;
    int xx = (2 * lane) / L, yy = (2 * lane) - ((2 * lane) / L) * L;
    for (int j0 = 0; j0 <= i; j0 += 64 * kLowerUnroll) {  // warp-uniform trip count
      const bool full = j0 + 64 * kLowerUnroll + L <= i;  // every entry and partner <= i
      float2 a[kLowerUnroll], bq[kLowerUnroll], ax[kLowerUnroll], bx[kLowerUnroll];
      float ay[kLowerUnroll], by[kLowerUnroll];
#pragma unroll
      for (int u = 0; u < kLowerUnroll; ++u) {
        const int p = j0 + 64 * u + 2 * lane;
        const int jx = (xx + 1 == L) ? yy : p + L;
        const int jy = (yy + 2 == L) ? p + 2 - L : p + 2;
        if (full) {
          a[u] = *reinterpret_cast<const float2*>(re + p);
          bq[u] = *reinterpret_cast<const float2*>(im + p);
          ax[u] = *reinterpret_cast<const float2*>(re + jx);
          bx[u] = *reinterpret_cast<const float2*>(im + jx);
          ay[u] = re[jy];
          by[u] = im[jy];
        } else {
          const bool in0 = p <= i, in1 = p + 1 <= i;
          const bool inx0 = in0 && jx <= i, inx1 = in1 && jx + 1 <= i, iny1 = in1 && jy <= i;
          const float2 z = make_float2(0.f, 0.f);
          a[u] = in0 ? *reinterpret_cast<const float2*>(re + p) : z;
          bq[u] = in0 ? *reinterpret_cast<const float2*>(im + p) : z;
          ax[u] = inx0 ? *reinterpret_cast<const float2*>(re + jx) : z;
          bx[u] = inx0 ? *reinterpret_cast<const float2*>(im + jx) : z;
          ay[u] = iny1 ? re[jy] : 0.f;
          by[u] = iny1 ? im[jy] : 0.f;
          if (!in1) { a[u].y = 0.f; bq[u].y = 0.f; }
          if (!inx1) { ax[u].y = 0.f; bx[u].y = 0.f; }
        }
        yy += dy64;
        xx += dx64;
        if (yy >= L) { yy -= L; xx += 1; }
      }
#pragma unroll
      for (int u = 0; u < kLowerUnroll; ++u) {
        const int pc = min(j0 + 64 * u + 2 * lane, N - 2);  // masked lanes read a valid entry
        const dsf ad0 = adiag[pc], ad1 = adiag[pc + 1];
        const float m = fmaxf(fmaxf(fmaxf(fabsf(a[u].x), fabsf(a[u].y)),
                                    fmaxf(fabsf(bq[u].x), fabsf(bq[u].y))),
                              fmaxf(fmaxf(fmaxf(fabsf(ax[u].x), fabsf(ax[u].y)),
                                          fmaxf(fabsf(bx[u].x), fabsf(bx[u].y))),
                                    fmaxf(fabsf(ay[u]), fabsf(by[u]))));
        if (__any_sync(0xffffffffu, !(m * m <= thr2))) {
          site_terms_ds(a[u].x, bq[u].x, ax[u].x, bx[u].x, a[u].y, bq[u].y, ad0, s1, s2, s3);
          site_terms_ds(a[u].y, bq[u].y, ax[u].y, bx[u].y, ay[u], by[u], ad1, s1, s2, s3);
        } else {
          site_terms_f(a[u].x, bq[u].x, ax[u].x, bx[u].x, a[u].y, bq[u].y, ad0.h, f1, f2, f3);
          site_terms_f(a[u].y, bq[u].y, ax[u].y, bx[u].y, ay[u], by[u], ad1.h, f1, f2, f3);
        }
      }
    }
    // boundary bonds into the bond sum: candidate t of 3L (t < L: (i-t, i-t+L); t == L:
    // (i, i+1); L < t < 2L: (j, j+1-L) with j = i + t - L; t >= 2L: (j, j+L-N) with
    // j = N - 3L + t, i.e. N - L <= j < N); the end <= i from row i, the other from column i
    for (int t = lane; t < 3 * L; t += 32) {
      int jr = -1, kc = -1;
      if (t < L) {
        const int j = i - t;
        if (j >= 0 && j / L != L - 1 && j + L > i) { jr = j; kc = j + L; }
      } else if (t == L) {
        if (i % L != L - 1 && i + 1 < N) { jr = i; kc = i + 1; }
      } else if (t < 2 * L) {
        const int j = i + t - L;
        if (j < N && j % L == L - 1 && j + 1 - L <= i) { jr = j + 1 - L; kc = j; }
      } else {
        const int j = N - 3 * L + t;
        if (j > i && j + L - N <= i) { jr = j + L - N; kc = j; }
      }
      if (jr >= 0) {
        const float ra = re[jr], rb = im[jr];
        const float ca = re0[(size_t)kc * ldm + i], cb = im0[(size_t)kc * ldm + i];
        csum_add(s3, two_prod(ra, ca));
        csum_add(s3, two_prod(-rb, cb));
      }
    }
    dsf tl = lane_total(s1, s2, s3, f1, f2, f3, w2, t2);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const dsf o = {__shfl_xor_sync(0xffffffffu, tl.h, off),
                     __shfl_xor_sync(0xffffffffu, tl.l, off)};
      tl = ds_add(tl, o);
    }
    if (lane == 0) gd[(size_t)b * N + i] = (double)tl.h + (double)tl.l;
  }
}

// Column part of the refinement and the combine.  A CTA takes the 64 columns [i0, i0 + 64) of
// one block (lane = the column pair c, c + 1 with c = i0 + 2 lane) and its 8 warps take the
// rows below i0 in turn (warp w the rows i0 + 1 + w + 8k); row j contributes, for each column
// c < j, the site term of x_j = X[j][c] and its bonds to the partners x_{j+x}, x_{j+y} that lie
// past c (X[j+x][c], X[j+y][c]).  The CTA sweeps down its strip together, so the partner rows,
// at most L rows ahead, are still in L1 when their own warp reaches them: 256-byte row segments
// of the lower triangle, each read once from DRAM.  The 8 warp partials are added to the
// row part in warp order, so the result does not depend on scheduling.  The row part arrives in
// gd as the float64 value of a double-float pair and is split back into one.
constexpr int kColUnroll = 2;

__global__ void __launch_bounds__(256, 3)
    k_refine_lower_cols(const float* __restrict__ M, int ldm, size_t mat_stride,
                        size_t plane_stride, int b0, Lattice la0,
                        const dsf* __restrict__ adiag_g, double* __restrict__ gd) {
  extern __shared__ unsigned char smem_raw[];
  dsf* adiag = reinterpret_cast<dsf*>(smem_raw);
  __shared__ float red[8];
  __shared__ dsf part[8][64];
  const int N = la0.N, L = la0.L;
  const int mat = blockIdx.y, b = b0 + mat;
  int n, sg;
  const Lattice la = block_lattice(la0, b, n, sg);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i0 = blockIdx.x * 64, c = i0 + 2 * lane;
  const float* re0 = M + mat * mat_stride;
  const float* im0 = re0 + plane_stride;
  const double w = (2.0 * n + 1.0) * kPi * la.T;
  const dsf w2 = ds_of(2.0 * w), t2 = ds_of(2.0 * la.t);
  const float thr2 = stage_adiag(adiag_g + (size_t)mat * N, adiag, N, fabsf(w2.h), fabsf(t2.h), red);
  const int cc = min(c, N - 2);  // lanes past N read a valid column pair and are masked
  // rows i0 + 1 + warp + 8k below the strip
  const int jb = i0 + 1 + warp;
  const int dx8 = 8 / L, dy8 = 8 % L;
  csum s1[2] = {}, s2[2] = {}, s3[2] = {};
  float f1[2] = {0.f, 0.f}, f2[2] = {0.f, 0.f}, f3[2] = {0.f, 0.f};
  int xj = jb / L, yj = jb - (jb / L) * L;
  for (int j0 = jb; j0 < N; j0 += 8 * kColUnroll) {  // warp-uniform trip count
    float2 a[kColUnroll], bq[kColUnroll], ax[kColUnroll], bx[kColUnroll];
    float2 ay[kColUnroll], by[kColUnroll];
#pragma unroll
    for (int u = 0; u < kColUnroll; ++u) {
      const int j = j0 + 8 * u;
      const int jx = (xj + 1 == L) ? yj : j + L;
      const int jy = (yj + 1 == L) ? j + 1 - L : j + 1;
      const bool row = j < N;
      const bool in0 = row && j > c, in1 = row && j > c + 1;
      const bool inx0 = in0 && jx > c, inx1 = in1 && jx > c + 1;
      const bool iny0 = in0 && jy > c, iny1 = in1 && jy > c + 1;
      const float2 z = make_float2(0.f, 0.f);
      a[u] = in0 ? *reinterpret_cast<const float2*>(re0 + (size_t)j * ldm + cc) : z;
      bq[u] = in0 ? *reinterpret_cast<const float2*>(im0 + (size_t)j * ldm + cc) : z;
      ax[u] = inx0 ? *reinterpret_cast<const float2*>(re0 + (size_t)jx * ldm + cc) : z;
      bx[u] = inx0 ? *reinterpret_cast<const float2*>(im0 + (size_t)jx * ldm + cc) : z;
      ay[u] = iny0 ? *reinterpret_cast<const float2*>(re0 + (size_t)jy * ldm + cc) : z;
      by[u] = iny0 ? *reinterpret_cast<const float2*>(im0 + (size_t)jy * ldm + cc) : z;
      if (!in1) { a[u].y = 0.f; bq[u].y = 0.f; }
      if (!inx1) { ax[u].y = 0.f; bx[u].y = 0.f; }
      if (!iny1) { ay[u].y = 0.f; by[u].y = 0.f; }
      yj += dy8;
      xj += dx8;
      if (yj >= L) { yj -= L; ++xj; }
    }
#pragma unroll
    for (int u = 0; u < kColUnroll; ++u) {
      const dsf ad = adiag[min(j0 + 8 * u, N - 1)];
      const float m = fmaxf(fmaxf(fmaxf(fmaxf(fabsf(a[u].x), fabsf(a[u].y)),
                                        fmaxf(fabsf(bq[u].x), fabsf(bq[u].y))),
                                  fmaxf(fmaxf(fabsf(ax[u].x), fabsf(ax[u].y)),
                                        fmaxf(fabsf(bx[u].x), fabsf(bx[u].y)))),
                            fmaxf(fmaxf(fabsf(ay[u].x), fabsf(ay[u].y)),
                                  fmaxf(fabsf(by[u].x), fabsf(by[u].y))));
      if (__any_sync(0xffffffffu, !(m * m <= thr2))) {
        site_terms_ds(a[u].x, bq[u].x, ax[u].x, bx[u].x, ay[u].x, by[u].x, ad, s1[0], s2[0], s3[0]);
        site_terms_ds(a[u].y, bq[u].y, ax[u].y, bx[u].y, ay[u].y, by[u].y, ad, s1[1], s2[1], s3[1]);
      } else {
        site_terms_f(a[u].x, bq[u].x, ax[u].x, bx[u].x, ay[u].x, by[u].x, ad.h, f1[0], f2[0], f3[0]);
        site_terms_f(a[u].y, bq[u].y, ax[u].y, bx[u].y, ay[u].y, by[u].y, ad.h, f1[1], f2[1], f3[1]);
      }
    }
  }
  part[warp][2 * lane] = lane_total(s1[0], s2[0], s3[0], f1[0], f2[0], f3[0], w2, t2);
  part[warp][2 * lane + 1] = lane_total(s1[1], s2[1], s3[1], f1[1], f2[1], f3[1], w2, t2);
  __syncthreads();
  const int ic = i0 + (int)threadIdx.x;
  if (threadIdx.x < 64 && ic < N) {
    const double r = gd[(size_t)b * N + ic];
    const float rh = (float)r;
    dsf tot = {rh, (float)(r - (double)rh)};
#pragma unroll
    for (int k = 0; k < 8; ++k) tot = ds_add(tot, part[k][threadIdx.x]);
    const double qsum = (double)tot.h + (double)tot.l;
    gd[(size_t)b * N + ic] = sg * (2.0 * (double)re0[(size_t)ic * ldm + ic] - qsum);
  }
}


// Im Tr G per block for the density of states: X_ii = R[i, sperm[i]] (sperm the inverse of
// the column permutation of the pivoted elimination), summed in float64 in a fixed order.
template <typename S>
__global__ void __launch_bounds__(256)
    k_trace(const S* M, int ldm, size_t mat_stride, size_t plane_stride, int N, const int* perm,
            int b0, double* tr) {
  extern __shared__ int sperm_dyn[];
  __shared__ double part[256];
  const int mat = blockIdx.x;
  const S* im = M + mat * mat_stride + plane_stride;
  for (int r = threadIdx.x; r < N; r += 256) sperm_dyn[perm[(size_t)mat * N + r]] = r;
  __syncthreads();
  double s = 0.0;
  for (int i = threadIdx.x; i < N; i += 256) s += (double)im[(size_t)i * ldm + sperm_dyn[i]];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) part[threadIdx.x] += part[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) tr[b0 + mat] = part[0];
}

// -------------------------------------------------------------- reduce/Adam
// Omega = sum_i phi_i^2/U - 2T sum_b ld_b ; g_i = 2 phi_i/U - 2T sum_b gd[b, i] (b ascending);
// then, if Adam is on and max|g| >= grad_tol, the update of phi in PyTorch's order
// (m, v, denom = sqrt(v)/sqrt(bc2) + eps, phi -= (lr/bc1) m / denom).  One CTA, fixed-order
// tree reductions, so the result does not depend on what else runs on the device.
// status: [0] Omega [1] max|g| [2] |mean s_i phi_i| [3] mean |phi_i| [4] nonfinite flag
// (all at the phi the gradient was taken at) [5] number of updates applied (accumulates).
// slots (optional): the workspace slot of each of the B blocks, in block order.
constexpr int RT = 1024;
// g_i = 2 phi_i / U - 2T sum_b gd[slot(b), i], b ascending, one thread per site: the B-term
// sums are float64 chains (a slow pipe on this GPU), so they are spread over N / 128 CTAs
// instead of the single reduction CTA.  slots (optional): the workspace slot of each block.
__device__ __forceinline__ void grad_sites(int N, int B, const int* slots, const double* gd,
                                           const double* phi, double U, double T, double* g_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double acc = 0.0;
  for (int b = 0; b < B; ++b) acc += gd[(size_t)(slots ? slots[b] : b) * N + i];
  g_out[i] = 2.0 * phi[i] / U - 2.0 * T * acc;
}

__global__ void __launch_bounds__(128)
    k_grad_sites(int N, int B, const double* gd, const double* phi, double U, double T,
                 double* g_out) {
  grad_sites(N, B, nullptr, gd, phi, U, T, g_out);
}

__global__ void __launch_bounds__(128)
    k_grad_sites_batch(int N, const ReqDesc* rq, const double* gd) {
  const ReqDesc r = rq[blockIdx.y];
  grad_sites(N, r.nblocks, r.slots, gd, r.phi, r.U, r.T, r.g);
}

__device__ __forceinline__ void reduce_body(
    int N, int L, int B, const int* slots, const double* ld, const double* gd,
    const double* phi, double* phi_out, double* m, double* v, double* g_out, double* omega_out,
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
    if (want_grad) {  // g_i from k_grad_sites
      const double g = g_out[i];
      if (!isfinite(g)) bad = true;
      gm = fmax(gm, fabs(g));
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
    for (int b = 0; b < B; ++b) sld += ld[slots ? slots[b] : b];
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

__global__ void __launch_bounds__(RT)
    k_reduce(int N, int L, int B, const double* ld, const double* gd, const double* phi,
             double* phi_out, double* m, double* v, double* g_out, double* omega_out,
             double* status, const int* flags, double U, double T, int want_grad, int do_adam,
             double step, double sbc2, double beta1, double beta2, double eps, double grad_tol) {
  reduce_body(N, L, B, nullptr, ld, gd, phi, phi_out, m, v, g_out, omega_out, status, flags, U,
              T, want_grad, do_adam, step, sbc2, beta1, beta2, eps, grad_tol);
}

// One CTA per request of a shared pass: its Omega, gradient and gated Adam update from its
// own blocks (slots in block order), exactly as a pass of its own would compute them.
__global__ void __launch_bounds__(RT) k_reduce_batch(int N, int L, const ReqDesc* rq,
                                                     const double* ld, const double* gd,
                                                     const int* flags) {
  const ReqDesc r = rq[blockIdx.x];
  reduce_body(N, L, r.nblocks, r.slots, ld, gd, r.phi, r.phi, r.m, r.v, r.g, nullptr, r.status,
              flags, r.U, r.T, 1, r.do_adam, r.adam.lr_over_bc1, r.adam.sqrt_bc2, r.adam.beta1,
              r.adam.beta2, r.adam.eps, r.adam.grad_tol);
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
  la.zshift = e.dos_mode ? e.d_z : nullptr;
  la.bd = e.bd;
  return la;
}

#define SCA_LAUNCH_CHECK(where)                                   \
  do {                                                            \
    g_launches.fetch_add(1, std::memory_order_relaxed);           \
    cudaError_t err__ = cudaGetLastError();                       \
    if (err__ != cudaSuccess) return cuda_fail(err__, where);     \
  } while (0)

// The dominant blocks on the tensor cores are inverted in their lower tiles only.  With the
// float32 refinement on, diag(G) is read from those tiles (k_refine_lower_rows/_cols) and the
// upper tiles are never filled; otherwise k_mirror copies the lower triangle up and the row
// kernels read whole rows.
// The pivoted sub-panel's interchanges and U12 inside the panel launch; k_swap_trsm as a
// separate launch where SCA_FUSED_SWAP=0 (the comparison path of its test).
bool fused_panel_swap() {
  if (const char* v = std::getenv("SCA_FUSED_SWAP"))
    if (std::atoi(v) == 0) return false;
  return true;
}

bool pivoted_first() {
  const char* v = std::getenv("SCA_PIVOTED_FIRST");
  return v && std::atoi(v) != 0;
}

// The pivoted group's pivot-block inverse by blocked triangular inversion (k_tinv_blocked); the
// row-solve kernel k_tinv_warp where SCA_TINV_BLOCKED=0 (the comparison path of its test).
bool blocked_tinv() {
  if (const char* v = std::getenv("SCA_TINV_BLOCKED"))
    if (std::atoi(v) == 0) return false;
  return true;
}

bool lower_refine(const Engine& e) {
  if (!e.refine || e.fp64 || !e.tc || e.tt == nullptr) return false;
  if (const char* v = std::getenv("SCA_SYM"))
    if (std::atoi(v) == 0) return false;
  if (const char* v = std::getenv("SCA_REFINE_LOWER"))
    if (std::atoi(v) == 0) return false;
  return true;
}

// diag(G) of the workspace slots m0 .. m0+cnt-1 (global blocks b0 + m0 ..): pivoted blocks
// through the permutation (k_refine), unpivoted ones by the direct kernel or, for blocks held
// as a lower triangle, by the row and column parts.
template <typename S>
sca_status launch_refine(Engine& e, const Lattice& la, int b0, int m0, int cnt, cudaStream_t s) {
  if (cnt <= 0) return SCA_OK;
  const int N = e.N;
  S* M = static_cast<S*>(e.M) + (size_t)m0 * e.mat_stride;
  const int* perm = e.perm + (size_t)m0 * N;
  const int bg = b0 + m0;
  const size_t perm_bytes = ((N * sizeof(int) + 15) / 16) * 16;
  prof_begin(e, kRefine, s);
  if (e.refine && sizeof(S) == 4) {
    const int np = std::max(0, std::min(cnt, e.piv_blocks - bg));
    if (np > 0) {
      const size_t fixed = perm_bytes + (size_t)N * 2 * sizeof(float);
      const size_t row_bytes = (size_t)N * sizeof(cpx<S>);
      const int warps = (int)std::max<size_t>(1, std::min<size_t>(8, (kRefineSmem - fixed) / row_bytes));
      const int gx = std::max(1, std::min((N + warps - 1) / warps, 32));
      k_refine<S><<<dim3(gx, np), warps * 32, fixed + warps * row_bytes, s>>>(
          M, e.ldm, e.mat_stride, e.plane_stride, bg, la, perm, e.gd, 1);
      SCA_LAUNCH_CHECK("refine");
    }
    if (cnt > np) {
      if (!e.adiag) {
        set_error("refinement without a diagonal table in the workspace");
        return SCA_ENOSTATE;
      }
      const int gx = (N + kRefineRowsPerCta - 1) / kRefineRowsPerCta;
      dsf* tab = reinterpret_cast<dsf*>(e.adiag) + (size_t)(m0 + np) * N;
      k_adiag<<<dim3((N + 255) / 256, cnt - np), 256, 0, s>>>(la, bg + np, tab);
      SCA_LAUNCH_CHECK("diagonal table");
      const float* Md = reinterpret_cast<const float*>(M) + (size_t)np * e.mat_stride;
      if (lower_refine(e)) {
        const int gr = (N + kLowerRowsPerCta - 1) / kLowerRowsPerCta;
        k_refine_lower_rows<<<dim3(gr, cnt - np), 256, (size_t)N * sizeof(dsf), s>>>(
            Md, e.ldm, e.mat_stride, e.plane_stride, bg + np, la, tab, e.gd);
        SCA_LAUNCH_CHECK("refine rows");
        k_refine_lower_cols<<<dim3((N + 63) / 64, cnt - np), 256, (size_t)N * sizeof(dsf), s>>>(
            Md, e.ldm, e.mat_stride, e.plane_stride, bg + np, la, tab, e.gd);
        SCA_LAUNCH_CHECK("refine columns");
      } else {
        k_refine_direct<<<dim3(gx, cnt - np), 256, (size_t)N * sizeof(dsf), s>>>(
            Md, e.ldm, e.mat_stride, e.plane_stride, bg + np, la, tab, e.gd);
        SCA_LAUNCH_CHECK("refine direct");
      }
    }
  } else {
    const int gx = std::max(1, std::min((N + 255) / 256, 16));
    k_refine<S><<<dim3(gx, cnt), 256, perm_bytes, s>>>(M, e.ldm, e.mat_stride, e.plane_stride,
                                                       bg, la, perm, e.gd, 0);
    SCA_LAUNCH_CHECK("refine");
  }
  prof_end(e, kRefine, s);
  return SCA_OK;
}

// Pivoted outer panel [k0, k0 + kb) of the slots in M .. (cnt blocks) by shared-memory sub-panels
// of width nb_sub, in compute type CP: each sub-panel's pivoted LU, its interchanges on the
// other columns with U12 for the rest of the outer panel, then A22 -= L21 U12 there.
template <typename S, typename CP>
sca_status piv_subpanels(Engine& e, S* M, int b0, int cnt, int k0, int kb, int nb_sub, int* piv,
                         int* perm, bool want_grad, cudaStream_t s) {
  const int N = e.N, kend = k0 + kb;
  const int nbi = std::min(nb_sub, kb);
  const int jstart = want_grad ? 0 : k0;
  // sub-panels of at most 16 columns apply their interchanges to the rest of the outer panel
  // and solve U12 there in the same launch; the columns outside the outer panel take all of
  // its interchanges in one k_swap_outer launch at the end (fused).  Otherwise (a sub-panel as
  // wide as its outer panel) k_swap_trsm applies them to every other column.
  const bool fused = nbi <= 16 && fused_panel_swap();
  for (int s0 = k0; s0 < kend; s0 += nbi) {
    const int kbi = std::min(nbi, kend - s0);
    const size_t sm = sizeof(cpx<CP>) * (size_t)(N - s0) * (kbi + 1) + 5 * sizeof(int) * kbi;
    const bool lu_done = !want_grad && s0 + kbi == N;  // LU only: nothing trails the last one
    if (s0 + kbi < kend && kbi > 16) {
      set_error("pivoted sub-panel wider than 16 inside an outer panel");
      return SCA_EINVAL;
    }
    prof_begin(e, kPanel, s);
    k_panel_smem<S, CP, 512><<<cnt, 512, sm, s>>>(M, N, e.ldm, e.mat_stride, e.plane_stride, s0,
                                                   kbi, b0, e.ld, piv, perm, e.flags,
                                                   fused && !lu_done ? k0 : -1, kend);
    prof_end(e, kPanel, s);
    SCA_LAUNCH_CHECK("panel");
    if (lu_done) break;
    if (!fused) {
      const int ncols = N - jstart;
      prof_begin(e, kSwap, s);
      k_swap_trsm<S, CP><<<dim3((ncols + 127) / 128, cnt), 128, 0, s>>>(
          M, N, e.ldm, e.mat_stride, e.plane_stride, s0, kbi, jstart, kend, piv);
      prof_end(e, kSwap, s);
      SCA_LAUNCH_CHECK("swap");
    }
    if (s0 + kbi < kend) {  // bring the rest of the outer panel up to date
      prof_begin(e, kPanelUpd, s);
      const int gx = (N - s0 - kbi + kGemmPanelRows - 1) / kGemmPanelRows;
      k_gemm_panel<S, CP><<<dim3(gx, cnt), 256, 0, s>>>(M, N, e.ldm, e.mat_stride,
                                                         e.plane_stride, s0, kbi, kend);
      prof_end(e, kPanelUpd, s);
      SCA_LAUNCH_CHECK("panel update");
    }
  }
  const int nco = (k0 - jstart) + (N - kend);  // columns outside the outer panel
  if (fused && nco > 0) {
    const size_t smo = swap_outer_smem(N - k0, kb, sizeof(S));
    const int gx = std::min((nco + kSwapStrip - 1) / kSwapStrip, kSwapCtas);
    prof_begin(e, kSwap, s);
    k_swap_outer<S><<<dim3(gx, cnt), 256, smo, s>>>(M, N, e.ldm, e.mat_stride, e.plane_stride,
                                                     k0, kb, jstart, piv);
    prof_end(e, kSwap, s);
    SCA_LAUNCH_CHECK("outer swap");
  }
  return SCA_OK;
}

// One group of blocks (workspace slots m0 .. m0+cnt-1, global indices b0 ..) through all
// elimination steps.  pivoted: partial pivoting with the shared-memory panel of width nb;
// otherwise the blocks are diagonally dominant and only the pivot block is factorised.
template <typename S, typename C>
sca_status run_group(Engine& e, int b0, int m0, int cnt, bool pivoted, int nb, bool tcg,
                     bool want_grad, cudaStream_t s) {
  const int N = e.N;
  S* M = static_cast<S*>(e.M) + (size_t)m0 * e.mat_stride;
  S* F = static_cast<S*>(e.F) + (size_t)m0 * e.fw_mat;
  S* W = static_cast<S*>(e.W) + (size_t)m0 * e.fw_mat;
  cpx<C>* Tinv = static_cast<cpx<C>*>(e.Tinv) + (size_t)m0 * 2 * e.nb * e.nb;
  int* piv = e.piv + (size_t)m0 * N;
  int* perm = e.perm + (size_t)m0 * N;
  const size_t fw_plane = (size_t)N * nb;
  const int split = tcg ? (e.bf16 ? 2 : 1) : 0;
  // the pivoted group's prep product on the tensor cores (BF16x3 with the -T^T planes)
  const bool piv_tc_prep =
      pivoted && tcg && e.bf16 && e.tt != nullptr && nb == e.nb && sizeof(C) == 4;
  // dominant blocks on the tensor cores: symmetric updates (lower tiles only)
  bool sym = tcg && !pivoted && e.tt != nullptr;
  if (const char* v = std::getenv("SCA_SYM"))
    if (std::atoi(v) == 0) sym = false;
  // inverses of symmetric dominant blocks: elimination steps merged in pairs
  const bool pair_ok = sym && want_grad && e.pair && e.F2 && e.W2 && e.tmap && nb == e.nb &&
                       sizeof(S) == 4;
  // SM partition mode 3: some of the dominant group's launches run on the second partition
  // (more SMs left to the pivoted group), by step and phase (alt_policy); each switch of
  // stream is ordered by an event
  const bool alt = !pivoted && e.alt_on && e.dom_alt && e.aux_alt && e.ev_alt;
  const cudaStream_t s_home = s, aux_home = e.aux;
  const int cap_home = e.tc_cap;
  auto switch_to = [&](bool second) -> cudaError_t {
    const cudaStream_t next = second ? e.dom_alt : s_home;
    e.aux = second ? e.aux_alt : aux_home;
    e.tc_cap = second ? e.alt_sms : cap_home;
    if (next == s) return cudaSuccess;
    cudaError_t err = cudaEventRecord(e.ev_alt, s);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(next, e.ev_alt, 0);
    s = next;
    return err;
  };
  for (int k0 = 0; k0 < N; k0 += nb) {
    const int kb = std::min(nb, N - k0);
    const int kend = k0 + kb;
    const bool odd = ((k0 / nb) & 1) != 0;
    // policy 1: odd steps on the second partition; 2 (default): every step's pivot-block
    // inverse and prep products there, the updates (HBM-bound, they want every SM) on the
    // first; 3: both (odd steps whole, even steps' prep there).  40x40: all three within
    // 0.1 ms of each other, 0.5 ms faster than mode 1; 1 and 3 cost the update 0.02 of HBM.
    const bool pre2 = alt && (e.alt_policy == 1 ? odd : true);
    const bool upd2 = alt && (e.alt_policy == 2 ? false : odd);
    if (alt) {
      const cudaError_t err = switch_to(pre2);
      if (err != cudaSuccess) return cuda_fail(err, "partition switch");
    }
    if (pair_ok && kend < N) {
      // Two Gauss-Jordan steps K1 = [k0, kend), K2 = [kend, kend + kb2) in one pass over the
      // lower triangle: K1's factors update only K2's cross (its row and column strips), K2's
      // pivot block and factors follow from that, and one K = 2 nb update does the rest.
      const int k2 = kend, kb2 = std::min(nb, N - k2);
      S* W2 = static_cast<S*>(e.W2) + (size_t)m0 * e.fw_mat;
      const size_t smw = 2 * sizeof(S) * (size_t)64 * (nb + 4);
      for (int step = 0; step < 2; ++step) {
        const int ka = step == 0 ? k0 : k2, kba = step == 0 ? kb : kb2;
        S* Wout = step == 0 ? W : W2;
        cudaStream_t sw = e.aux ? e.aux : s;
        if (e.aux) {
          cudaError_t err = cudaEventRecord(e.ev_aux0, s);
          if (err == cudaSuccess) err = cudaStreamWaitEvent(e.aux, e.ev_aux0, 0);
          if (err != cudaSuccess) return cuda_fail(err, "aux fork");
        }
        prof_begin(e, kPrep, sw);
        k_prep_w<S><<<dim3((N + 63) / 64, cnt), 256, smw, sw>>>(
            M, N, e.ldm, e.mat_stride, e.plane_stride, ka, kba, nb, Wout, fw_plane, e.fw_mat, 0,
            1, split, 1);
        prof_end(e, kPrep, sw);
        SCA_LAUNCH_CHECK("prep w");
        if (e.aux) {
          cudaError_t err = cudaEventRecord(e.ev_aux1, e.aux);
          if (err != cudaSuccess) return cuda_fail(err, "aux join");
        }
        prof_begin(e, kDiag, s);
        {
          float* TT = e.tt + (size_t)m0 * kTtPlanes * e.nb * e.nb;
          sca_status st;
          if constexpr (sizeof(C) == 4) {
            if (e.tmap && e.diag_tc) {
              st = tc_diag(M, e.ldm, e.mat_stride, e.plane_stride, cnt, ka, kba, nb, b0, e.ld,
                           Tinv, TT, e.bf16 ? 1 : 0, e.flags, s);
              if (st != SCA_OK) return st;
            } else {
              k_diag_gjb<512><<<cnt, 512, 0, s>>>(M, e.ldm, e.mat_stride, e.plane_stride, ka, kba,
                                                  nb, b0, e.ld, Tinv, TT, e.bf16 ? 1 : 0, e.flags);
            }
          } else {
            (void)TT;
            (void)st;
            set_error("merged two-step update needs float32 blocks");
            return SCA_EINVAL;
          }
        }
        prof_end(e, kDiag, s);
        SCA_LAUNCH_CHECK("diag");
        if (e.aux) {
          cudaError_t err = cudaStreamWaitEvent(s, e.ev_aux1, 0);
          if (err != cudaSuccess) return cuda_fail(err, "aux join");
        }
        prof_begin(e, kPrep, s);
        sca_status st = tc_prep_split(e, m0, cnt, 0, ka, kba, true, s, step == 1);
        if (st != SCA_OK) return st;
        prof_end(e, kPrep, s);
        if (alt) {
          const cudaError_t err = switch_to(upd2);
          if (err != cudaSuccess) return cuda_fail(err, "partition switch");
        }
        const int kind = step == 0 ? kUpdateCross : kUpdate;
        prof_begin(e, kind, s);
        st = tc_update_pair(e, m0, cnt, k0, kb, k2, kb2, step == 0 ? 1 : 2, s);
        if (st != SCA_OK) return st;
        prof_end(e, kind, s);
        if (alt && step == 0) {
          const cudaError_t err = switch_to(pre2);
          if (err != cudaSuccess) return cuda_fail(err, "partition switch");
        }
      }
      k0 += nb;  // the loop adds the first step's width
      continue;
    }
    if (pivoted) {
      // outer panel [k0, kend) factorised by shared-memory sub-panels; float64 arithmetic in
      // them when the context asks for it (sca_set_panel_precision), else the compute type
      sca_status st;
      if (e.panel_fp64 && sizeof(C) == 4)
        st = piv_subpanels<S, double>(e, M, b0, cnt, k0, kb, e.nb_piv64, piv, perm, want_grad, s);
      else
        st = piv_subpanels<S, C>(e, M, b0, cnt, k0, kb, e.nb_piv, piv, perm, want_grad, s);
      if (st != SCA_OK) return st;
      if (!want_grad && kend == N) break;
    }
    const bool last_lu = !want_grad && kend == N;  // LU: nothing trails the last pivot block
    bool w_aux = false;
    if (sym && !last_lu && e.aux) {
      // the W^T planes do not depend on the pivot-block inverse: build them on the auxiliary
      // stream while the inverse runs (both are short; side by side or in sequence they take
      // the same time, and the stream keeps them independent of each other)
      cudaError_t err = cudaEventRecord(e.ev_aux0, s);
      if (err == cudaSuccess) err = cudaStreamWaitEvent(e.aux, e.ev_aux0, 0);
      if (err != cudaSuccess) return cuda_fail(err, "aux fork");
      const int cw = want_grad ? 0 : kend;
      const size_t smw = 2 * sizeof(S) * (size_t)64 * (nb + 4);
      prof_begin(e, kPrep, e.aux);
      k_prep_w<S><<<dim3((N - cw + 63) / 64, cnt), 256, smw, e.aux>>>(
          M, N, e.ldm, e.mat_stride, e.plane_stride, k0, kb, nb, W, fw_plane, e.fw_mat, cw,
          want_grad ? 1 : 0, split, 1);
      prof_end(e, kPrep, e.aux);
      SCA_LAUNCH_CHECK("prep w");
      if ((err = cudaEventRecord(e.ev_aux1, e.aux)) != cudaSuccess) return cuda_fail(err, "aux join");
      w_aux = true;
    }
    if (pivoted) {
      // T and inv(L_KK) of the factored pivot block, for F = M[:, K] T (inv(L_KK) below K)
      prof_begin(e, kTrinv, s);
      const size_t smt = sizeof(cpx<C>) * std::max((size_t)kb * kb + kb, (size_t)nb * (nb + 1));
      constexpr int NT = sizeof(C) == 8 ? 512 : 1024;
      constexpr int NBMAX = sizeof(C) == 8 ? 64 : 128;
      float* TT = piv_tc_prep ? e.tt + (size_t)m0 * kTtPlanes * e.nb * e.nb : nullptr;
      bool blocked = false;
      if constexpr (sizeof(C) == 4) {
        if (kb % kTinvB == 0 && nb % kTinvB == 0 && kb <= nb && blocked_tinv()) {
          const size_t smb = sizeof(cpx<C>) * std::max((size_t)kb * (kb + 2) + (size_t)kTinvB * kb,
                                                       (size_t)nb * (nb + 1));
          k_tinv_blocked<S, 512><<<cnt, 512, smb, s>>>(M, e.ldm, e.mat_stride, e.plane_stride, k0,
                                                       kb, nb, Tinv, TT);
          blocked = true;
        }
      }
      if (!blocked) {
        if (kb == NBMAX)
          k_tinv_warp<S, C, NT, true><<<cnt, NT, smt, s>>>(M, e.ldm, e.mat_stride,
                                                            e.plane_stride, k0, kb, nb, Tinv, TT);
        else
          k_tinv_warp<S, C, NT, false><<<cnt, NT, smt, s>>>(M, e.ldm, e.mat_stride,
                                                             e.plane_stride, k0, kb, nb, Tinv, TT);
      }
      prof_end(e, kTrinv, s);
      SCA_LAUNCH_CHECK("pivot-block inverse");
    } else {
      prof_begin(e, kDiag, s);
      float* TT = (tcg && e.tt) ? e.tt + (size_t)m0 * kTtPlanes * e.nb * e.nb : nullptr;
      if constexpr (sizeof(C) == 4) {
        if (tcg && e.tmap && nb == 128 && e.diag_tc) {
          sca_status st = tc_diag(M, e.ldm, e.mat_stride, e.plane_stride, cnt, k0, kb, nb, b0,
                                  e.ld, Tinv, TT, e.bf16 ? 1 : 0, e.flags, s);
          if (st != SCA_OK) return st;
        } else {
          k_diag_gjb<512><<<cnt, 512, 0, s>>>(M, e.ldm, e.mat_stride, e.plane_stride, k0, kb,
                                              nb, b0, e.ld, Tinv, TT, e.bf16 ? 1 : 0, e.flags);
        }
      } else {
        k_diag_gj<S, C, 768><<<cnt, 768, 0, s>>>(M, e.ldm, e.mat_stride, e.plane_stride, k0,
                                                  kb, nb, b0, e.ld, Tinv, TT, e.bf16 ? 1 : 0,
                                                  e.flags);
      }
      prof_end(e, kDiag, s);
      SCA_LAUNCH_CHECK("diag");
    }
    if (last_lu) break;
    const int r0 = want_grad ? 0 : kend, c0 = want_grad ? 0 : kend;
    if (sym) {
      // W^T planes first: they are also the A operand of the prep product, since the swept
      // rows of M[:, K] are -W^T and the unswept ones +W^T (the sign rule above)
      if (w_aux) {
        cudaError_t err = cudaStreamWaitEvent(s, e.ev_aux1, 0);
        if (err != cudaSuccess) return cuda_fail(err, "aux join");
      } else {
        const size_t sm = 2 * sizeof(S) * (size_t)64 * (nb + 4);
        prof_begin(e, kPrep, s);
        k_prep_w<S><<<dim3((N - c0 + 63) / 64, cnt), 256, sm, s>>>(
            M, N, e.ldm, e.mat_stride, e.plane_stride, k0, kb, nb, W, fw_plane, e.fw_mat, c0,
            want_grad ? 1 : 0, split, 1);
        prof_end(e, kPrep, s);
        SCA_LAUNCH_CHECK("prep w");
      }
      prof_begin(e, kPrep, s);
      sca_status st = tc_prep_split(e, m0, cnt, r0, k0, kb, want_grad, s);
      if (st != SCA_OK) return st;
      prof_end(e, kPrep, s);
    } else {
      prof_begin(e, pivoted ? kPrepPiv : kPrep, s);
      if (tcg && !pivoted && nb == e.nb && e.tt && !e.bf16) {
        // F = M[:, K] T on the tensor cores (scratch: the W planes, rewritten below)
        const int rs = r0;
        const size_t tot = (size_t)(N - rs) * nb;
        k_split_cols<S><<<dim3((unsigned)((tot + 255) / 256), cnt), 256, 0, s>>>(
            M, N, e.ldm, e.mat_stride, e.plane_stride, k0, kb, nb, reinterpret_cast<float*>(W),
            fw_plane, e.fw_mat, rs);
        SCA_LAUNCH_CHECK("split cols");
        sca_status st = tc_prep(e, m0, cnt, r0, s);
        if (st != SCA_OK) return st;
        const size_t rem = (size_t)(N - r0) * nb;
        k_split_f<C><<<dim3((unsigned)((rem + 255) / 256), cnt), 256, 0, s>>>(
            reinterpret_cast<const float*>(W) + 4 * fw_plane, fw_plane, e.fw_mat, Tinv, N, k0, kb,
            nb, r0, want_grad ? 1 : 0, reinterpret_cast<float*>(F), fw_plane, e.fw_mat);
        SCA_LAUNCH_CHECK("split f");
      } else if (piv_tc_prep) {
        // F = M[:, K] T (rows above K; rows of K: -T) and L21 inv(L11) (rows below K) on the
        // tensor cores: A = split pivot columns in the W planes, B = the planes k_tinv_warp wrote
        const size_t tot = (size_t)(N - r0) * (nb / 4);
        k_split_a<S><<<dim3((unsigned)((tot + 255) / 256), cnt), 256, 0, s>>>(
            M, N, e.ldm, e.mat_stride, e.plane_stride, k0, kb, nb, reinterpret_cast<float*>(W),
            fw_plane, e.fw_mat, r0);
        SCA_LAUNCH_CHECK("split a");
        sca_status st = tc_prep_piv(e, m0, cnt, r0, k0, kb, want_grad, s);
        if (st != SCA_OK) return st;
      } else {
        k_prep_f<S, C><<<dim3((N - r0 + 63) / 64, cnt), 256, 0, s>>>(
            M, N, e.ldm, e.mat_stride, e.plane_stride, k0, kb, nb, Tinv, F, fw_plane, e.fw_mat,
            r0, want_grad ? 1 : 0, pivoted ? 1 : 0, split);
      }
      const size_t sm = 2 * sizeof(S) * (size_t)64 * (nb + 4);
      k_prep_w<S><<<dim3((N - c0 + 63) / 64, cnt), 256, sm, s>>>(
          M, N, e.ldm, e.mat_stride, e.plane_stride, k0, kb, nb, W, fw_plane, e.fw_mat, c0,
          want_grad ? 1 : 0, split, 0);
      prof_end(e, pivoted ? kPrepPiv : kPrep, s);
      SCA_LAUNCH_CHECK("prep");
    }
    if (alt) {
      const cudaError_t err = switch_to(upd2);
      if (err != cudaSuccess) return cuda_fail(err, "partition switch");
    }
    const int ukind = pivoted ? kUpdatePiv : kUpdate;
    prof_begin(e, ukind, s);
    if (tcg) {
      sca_status st = tc_update(e, m0, cnt, k0, kb, r0, c0, want_grad, s, nb, sym);
      if (st != SCA_OK) return st;
    } else {
      dim3 grid((N - c0 + 63) / 64, (N - r0 + 63) / 64, cnt);
      k_update_simt<S><<<grid, 256, 0, s>>>(M, N, e.ldm, e.mat_stride, e.plane_stride, F, W, nb,
                                            fw_plane, e.fw_mat, r0, c0, k0, kb, want_grad ? 1 : 0);
      SCA_LAUNCH_CHECK("update");
    }
    prof_end(e, ukind, s);
  }
  if (alt) {
    const cudaError_t err = switch_to(false);
    if (err != cudaSuccess) return cuda_fail(err, "partition switch");
  }
  if (sym && want_grad && !lower_refine(e)) {  // symmetric inverse: fill the upper tiles
    const int nt = (N + 31) / 32;
    prof_begin(e, kPrep, s);
    k_mirror<S><<<dim3(nt * (nt + 1) / 2, cnt), 256, 0, s>>>(M, N, e.ldm, e.mat_stride,
                                                             e.plane_stride);
    prof_end(e, kPrep, s);
    SCA_LAUNCH_CHECK("mirror");
  }
  return SCA_OK;
}

template <typename S, typename C>
sca_status run_blocks_t(Engine& e, const double* d_phi, bool want_grad, bool refine_stage,
                        cudaStream_t s) {
  const Lattice la = make_lattice(e, d_phi);
  const int N = e.N;
  S* M = static_cast<S*>(e.M);
  cudaError_t err = cudaMemsetAsync(e.flags, 0, sizeof(int), s);
  if (err != cudaSuccess) return cuda_fail(err, "flags reset");
  // dominant blocks on the tensor cores are eliminated symmetrically (lower tiles only)
  bool sym_dom = e.tc && e.tt != nullptr && e.nb % 4 == 0;
  if (const char* v = std::getenv("SCA_SYM"))
    if (std::atoi(v) == 0) sym_dom = false;
  for (int b0 = 0; b0 < e.B; b0 += e.chunk) {
    const int cnt = std::min(e.chunk, e.B - b0);
    const int npiv = std::max(0, std::min(cnt, e.piv_blocks - b0));
    prof_begin(e, kAssemble, s);
    k_assemble_rows<S><<<dim3((N + 7) / 8, cnt), 256, 0, s>>>(
        M, e.ldm, e.mat_stride, e.plane_stride, b0, la, e.ld, e.perm, sym_dom ? npiv : cnt, e.nb);
    prof_end(e, kAssemble, s);
    SCA_LAUNCH_CHECK("assemble");
    if (e.tc) {
      sca_status st0 = tc_reset_counters(e, s);
      if (st0 != SCA_OK) return st0;
    }
    // blocks [0, piv_blocks) need pivoting (lowest frequencies), the rest are dominant
    const int np = std::max(0, std::min(cnt, e.piv_blocks - b0));
    const int nd = cnt - np;
    const bool fork = np > 0 && nd > 0 && e.side != nullptr;
    // with SM partitions the dominant group runs on its partition's stream (and W-plane
    // stream), the pivoted group on the SMs left over
    const bool parted = fork && e.dom != nullptr;
    cudaStream_t sp = s, sd = s;
    cudaStream_t aux_saved = e.aux;
    if (fork) {
      sp = e.part_side ? e.part_side : e.side;
      if ((err = cudaEventRecord(e.ev_fork, s)) != cudaSuccess) return cuda_fail(err, "fork");
      if ((err = cudaStreamWaitEvent(sp, e.ev_fork, 0)) != cudaSuccess) return cuda_fail(err, "fork");
      if (parted) {
        sd = e.dom;
        if ((err = cudaStreamWaitEvent(sd, e.ev_fork, 0)) != cudaSuccess) return cuda_fail(err, "fork");
      }
    }
    sca_status st = SCA_OK;
    // While both groups run, the dominant group's persistent tensor-core launches leave
    // sm_reserve SMs to the pivoted group's kernels (with partitions: each group's
    // tensor-core launches take one CTA per SM of its partition).
    auto pivoted_group = [&]() -> sca_status {
      e.tc_cap = parted && e.part_side ? e.part_sms[0] : 0;
      const int span_p = np > 0 ? prof_span_begin(e, kSpanPiv, sp) : -1;
      sca_status r = SCA_OK;
      if (np > 0) {
        NvtxRange range("sca.pivoted_group");
        r = run_group<S, C>(e, b0, 0, np, true, e.nb, e.tc, want_grad, sp);
      }
      e.tc_cap = 0;
      if (r == SCA_OK) prof_span_end(e, span_p, sp);
      return r;
    };
    auto dominant_group = [&]() -> sca_status {
      if (parted) {
        e.tc_cap = e.part_sms[1];
        if (e.aux) e.aux = e.part_aux;
        e.alt_on = e.dom_alt != nullptr;
      } else if (fork && e.sm_reserve > 0 && e.tmap) {
        e.tc_cap = tc_sms(e) - e.sm_reserve;
      }
      const int span_d = nd > 0 ? prof_span_begin(e, kSpanDom, sd) : -1;
      sca_status r = SCA_OK;
      if (nd > 0) {
        NvtxRange range("sca.dominant_group");
        r = run_group<S, C>(e, b0 + np, np, nd, false, e.nb, e.tc, want_grad, sd);
      }
      e.tc_cap = 0;
      e.aux = aux_saved;
      e.alt_on = false;
      if (r == SCA_OK) prof_span_end(e, span_d, sd);
      return r;
    };
    // The dominant group is enqueued first: its few long launches then start at once, while
    // the pivoted group's many short ones are still being enqueued (the host stays ahead of
    // that chain on the device).  Enqueued the other way round, a long pivoted chain (2000+
    // launches at N = 4096) fills the launch queue, the host blocks, and the dominant group
    // starts only when the chain has drained far enough.  SCA_PIVOTED_FIRST=1 restores that
    // order without partitions (the comparison of the two orders).
    if (parted || !pivoted_first()) {
      if ((st = dominant_group()) != SCA_OK || (st = pivoted_group()) != SCA_OK) return st;
    } else {
      if ((st = pivoted_group()) != SCA_OK || (st = dominant_group()) != SCA_OK) return st;
    }
    if (fork) {
      if (want_grad && refine_stage && !e.dos_mode) {  // each group refines its own blocks
        if ((st = launch_refine<S>(e, la, b0, 0, np, sp)) != SCA_OK) return st;
        if ((st = launch_refine<S>(e, la, b0, np, nd, sd)) != SCA_OK) return st;
      }
      if ((err = cudaEventRecord(e.ev_join, sp)) != cudaSuccess) return cuda_fail(err, "join");
      if ((err = cudaStreamWaitEvent(s, e.ev_join, 0)) != cudaSuccess) return cuda_fail(err, "join");
      if (parted) {
        if ((err = cudaEventRecord(e.ev_join2, sd)) != cudaSuccess) return cuda_fail(err, "join");
        if ((err = cudaStreamWaitEvent(s, e.ev_join2, 0)) != cudaSuccess) return cuda_fail(err, "join");
      }
    }
    if (want_grad && e.dos_mode) {
      prof_begin(e, kRefine, s);
      k_trace<S><<<cnt, 256, (size_t)N * sizeof(int), s>>>(M, e.ldm, e.mat_stride, e.plane_stride,
                                                           N, e.perm, b0, e.tr);
      prof_end(e, kRefine, s);
      SCA_LAUNCH_CHECK("trace");
    } else if (want_grad && refine_stage && !fork) {
      sca_status st2 = launch_refine<S>(e, la, b0, 0, cnt, s);
      if (st2 != SCA_OK) return st2;
    }
  }
  return SCA_OK;
}

// Dynamic shared-memory limit of a kernel: the device's opt-in maximum per block minus the
// kernel's static shared memory.
template <typename K>
cudaError_t allow_max_smem(K* kernel) {
  int dev = 0, optin = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err == cudaSuccess) err = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  if (err == cudaSuccess) err = cudaFuncGetAttributes(&fa, kernel);
  if (err == cudaSuccess)
    err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               optin - (int)fa.sharedSizeBytes);
  return err;
}

template <typename S, typename C>
sca_status set_smem_limits() {
  static ContextOnce once;
  if (once.done()) return SCA_OK;
  cudaError_t err;
  if ((err = allow_max_smem(k_panel_smem<S, C, 512>)) != cudaSuccess) return cuda_fail(err, "smem panel");
  if constexpr (sizeof(S) == 4)  // the float64 panel of the mixed path
    if ((err = allow_max_smem(k_panel_smem<S, double, 512>)) != cudaSuccess)
      return cuda_fail(err, "smem panel fp64");
  if ((err = allow_max_smem(k_prep_w<S>)) != cudaSuccess) return cuda_fail(err, "smem prep");
  if ((err = allow_max_smem(k_tinv_warp<S, C, sizeof(C) == 8 ? 512 : 1024, true>)) != cudaSuccess ||
      (err = allow_max_smem(k_tinv_warp<S, C, sizeof(C) == 8 ? 512 : 1024, false>)) != cudaSuccess)
    return cuda_fail(err, "smem tinv");
  if constexpr (sizeof(C) == 4)
    if ((err = allow_max_smem(k_tinv_blocked<S, 512>)) != cudaSuccess)
      return cuda_fail(err, "smem tinv blocked");
  if ((err = allow_max_smem(k_refine<S>)) != cudaSuccess) return cuda_fail(err, "smem refine");
  if ((err = allow_max_smem(k_swap_outer<S>)) != cudaSuccess) return cuda_fail(err, "smem swap");
  once.mark();
  return SCA_OK;
}

}  // namespace

sca_status run_blocks(Engine& e, const double* d_phi, bool want_grad, cudaStream_t s,
                      bool refine_stage) {
  NvtxRange range(want_grad ? "sca.blocks(inverse)" : "sca.blocks(log-det)");
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
  if (e.fp64) return launch_refine<double>(e, la, 0, 0, e.B, s);
  return launch_refine<float>(e, la, 0, 0, e.B, s);
}

sca_status run_assemble_only(Engine& e, const double* d_phi, int b0, int count, cudaStream_t s) {
  const Lattice la = make_lattice(e, d_phi);
  const size_t S = e.fp64 ? 8 : 4;
  cudaError_t err = cudaMemsetAsync(e.M, 0, (size_t)count * e.mat_stride * S, s);
  if (err != cudaSuccess) return cuda_fail(err, "assemble zero fill");
  if (e.fp64)
    k_assemble<double><<<dim3((e.N + 127) / 128, count), 128, 0, s>>>(
        static_cast<double*>(e.M), e.ldm, e.mat_stride, e.plane_stride, b0, la, e.ld, e.perm);
  else
    k_assemble<float><<<dim3((e.N + 127) / 128, count), 128, 0, s>>>(
        static_cast<float*>(e.M), e.ldm, e.mat_stride, e.plane_stride, b0, la, e.ld, e.perm);
  SCA_LAUNCH_CHECK("assemble");
  return SCA_OK;
}

sca_status run_reduce(Engine& e, const double* d_phi, double* d_omega, double* d_grad,
                      const AdamStep* adam, cudaStream_t s) {
  const bool want_grad = (d_grad != nullptr) || (adam != nullptr);
  double* g = d_grad ? d_grad : e.d_g;
  prof_begin(e, kReduce, s);
  if (want_grad) {
    k_grad_sites<<<(e.N + 127) / 128, 128, 0, s>>>(e.N, e.B, e.gd, d_phi, e.p.U, e.p.T, g);
    SCA_LAUNCH_CHECK("gradient sums");
  }
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

sca_status run_reduce_batch(Engine& e, const ReqDesc* rq, int nreq, cudaStream_t s) {
  prof_begin(e, kReduce, s);
  k_grad_sites_batch<<<dim3((e.N + 127) / 128, nreq), 128, 0, s>>>(e.N, rq, e.gd);
  SCA_LAUNCH_CHECK("gradient sums");
  k_reduce_batch<<<nreq, RT, 0, s>>>(e.N, e.L, rq, e.ld, e.gd, e.flags);
  prof_end(e, kReduce, s);
  SCA_LAUNCH_CHECK("reduce batch");
  return SCA_OK;
}

sca_status run_seed_phi(double* d_phi, int N, uint64_t seed, cudaStream_t s) {
  k_seed_phi<<<(N + 255) / 256, 256, 0, s>>>(d_phi, N, (unsigned long long)seed);
  SCA_LAUNCH_CHECK("seed_phi");
  return SCA_OK;
}

}  // namespace sca
