/*
 * sca_oracle.c -- plain, slow FP64 CPU oracle for the SCA+ADAM potential.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * execute this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code with the CUDA path.
 *
 * What it computes (paper: Park & Lee, "Hubbard model on semiclassical
 * approximation in combination with an optimizer based on GPU technology",
 * arXiv 2311.04435):
 *
 *   Lattice and Hamiltonian (Eq. 1, "IHH"): L x L periodic square lattice,
 *   site i = x*L + y, sublattice sign s_i = (-1)^(x+y) (A <=> s = +1).
 *   Nearest-neighbour hopping -t on every bond i -> i+x, i -> i+y (bonds are
 *   accumulated, so L = 2 gives -2t), ionic site energy eps_i = -s_i * Delta
 *   (Eq. 1 puts -Delta on A and +Delta on B; IONIC_HALF uses Delta/2).
 *
 *   Static auxiliary field (Sec. II, HS line and Eq. 2 "Eq2"): the spin-z
 *   coupling enters H_sigma(phi) = K + diag(eps_i - sigma*phi_i) with
 *   sigma = +1 (up), -1 (down); normalisation reading: the quadratic term is
 *   sum_i phi_i^2 / U (the HS line with phi -> 2 phi), whose saddle point is
 *   the Hartree-Fock gap phi_i = U m_i / 2.
 *
 *   Matsubara grid (Eq. 2 and the Fig. 1 caption): omega_n = (2n+1) pi T,
 *   n = 0 .. n_omega-1; the negative-n half is the complex conjugate, so
 *       Omega(phi) = sum_i phi_i^2/U - 2T sum_{n>=0} sum_sigma ln|det A_{n,sigma}|,
 *       A_{n,sigma} = (i omega_n + mu) I - H_sigma(phi).
 *   The -beta inside the determinant of Eq. 2 only adds a phi-independent
 *   constant and is dropped.
 *
 *   Gradient (derivative of Eq. 2): d ln det A / d phi_i = sigma * G_ii with
 *   G = A^{-1}, so
 *       dOmega/dphi_i = 2 phi_i / U - 2T sum_{n,sigma} sigma Re G_{n sigma, ii}.
 *
 *   Optimiser (Sec. II, "ADAM optimizer based on the PyTorch library";
 *   Kingma & Ba 2014): Adam with bias correction, no weight decay, in the
 *   arithmetic order of the PyTorch reference implementation.
 *
 *   Seeded initial field: phi0_i = u_i - 1/2 with u_i the top 53 bits of
 *   splitmix64 (Steele, Lea & Flood, OOPSLA 2014; Vigna's public-domain
 *   splitmix64.c) applied to state seed + (i+1) * 0x9E3779B97F4A7C15.
 *
 * Each determinant and each inverse diagonal is the plain definition: dense
 * complex LU with partial pivoting (row of largest |z|^2, first on ties),
 * ln|det| = sum_k ln|u_kk|, and G = A^{-1} column by column from the factors.
 * A second, independent route diagonalises the real symmetric H_sigma with
 * cyclic Jacobi rotations and sums over eigenvalues.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex zc;

typedef struct {
  int32_t L, n_omega, prec, ionic;
  double t, U, delta, T, mu;
} orc_params;

typedef struct {
  double lr, beta1, beta2, eps, grad_tol;
  int32_t max_steps;
  uint64_t seed;
} orc_adam;

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ---------------------------------------------------------------- Eq. 1 -- */

/* Dense real symmetric H_sigma(phi) (row-major N x N).  eps_extra (N values or
 * NULL) adds an arbitrary per-site energy (disordered model of Sec. IV). */
void orc_hamiltonian(const orc_params* p, const double* eps_extra, const double* phi,
                     int sigma, double* H) {
  const int L = p->L, N = L * L;
  const double d = (p->ionic == 1) ? 0.5 * p->delta : p->delta;
  memset(H, 0, sizeof(double) * (size_t)N * N);
  for (int x = 0; x < L; ++x)
    for (int y = 0; y < L; ++y) {
      const int i = x * L + y;
      const int jx = ((x + 1) % L) * L + y;
      const int jy = x * L + (y + 1) % L;
      H[(size_t)i * N + jx] += -p->t;
      H[(size_t)jx * N + i] += -p->t;
      H[(size_t)i * N + jy] += -p->t;
      H[(size_t)jy * N + i] += -p->t;
      const double s = ((x + y) & 1) ? -1.0 : 1.0;
      H[(size_t)i * N + i] += -s * d + (eps_extra ? eps_extra[i] : 0.0) - sigma * phi[i];
    }
}

/* Matsubara frequency omega_n = (2n+1) pi T. */
double orc_omega_n(const orc_params* p, int n) { return (2.0 * n + 1.0) * M_PI * p->T; }

/* ------------------------------------------------ dense LU and inverse -- */

static double abs2(zc z) { return creal(z) * creal(z) + cimag(z) * cimag(z); }

static zc zdiv(zc a, zc b) {
  const double den = abs2(b);
  return a * conj(b) / den;
}

/* In-place complex LU with partial pivoting, P A = L U (L unit lower).
 * piv[k] = row swapped with row k at step k.  Returns 0, or -1 if singular.
 * *ld = sum_k ln|u_kk|. */
int orc_zgetrf(int N, zc* A, int* piv, double* ld) {
  double acc = 0.0;
  for (int k = 0; k < N; ++k) {
    int p = k;
    double best = abs2(A[(size_t)k * N + k]);
    for (int r = k + 1; r < N; ++r) {
      const double v = abs2(A[(size_t)r * N + k]);
      if (v > best) { best = v; p = r; }
    }
    piv[k] = p;
    if (best == 0.0) return -1;
    if (p != k)
      for (int j = 0; j < N; ++j) {
        const zc tmp = A[(size_t)k * N + j];
        A[(size_t)k * N + j] = A[(size_t)p * N + j];
        A[(size_t)p * N + j] = tmp;
      }
    const zc d = A[(size_t)k * N + k];
    acc += 0.5 * log(abs2(d));
    for (int r = k + 1; r < N; ++r) {
      const zc l = zdiv(A[(size_t)r * N + k], d);
      A[(size_t)r * N + k] = l;
      if (l != 0.0)
        for (int j = k + 1; j < N; ++j) A[(size_t)r * N + j] -= l * A[(size_t)k * N + j];
    }
  }
  *ld = acc;
  return 0;
}

/* Column j of A^{-1} from the factors: b = P e_j, L y = b, U x = y. */
static void lu_solve_unit(int N, const zc* F, const int* piv, int j, zc* x) {
  for (int r = 0; r < N; ++r) x[r] = 0.0;
  x[j] = 1.0;
  for (int k = 0; k < N; ++k)
    if (piv[k] != k) { const zc tmp = x[k]; x[k] = x[piv[k]]; x[piv[k]] = tmp; }
  for (int r = 0; r < N; ++r) {
    zc s = x[r];
    for (int c = 0; c < r; ++c) s -= F[(size_t)r * N + c] * x[c];
    x[r] = s;
  }
  for (int r = N - 1; r >= 0; --r) {
    zc s = x[r];
    for (int c = r + 1; c < N; ++c) s -= F[(size_t)r * N + c] * x[c];
    x[r] = zdiv(s, F[(size_t)r * N + r]);
  }
}

/* A_{n,sigma} = (i omega_n + mu) I - H_sigma, dense complex. */
static void build_A(const orc_params* p, const double* H, int n, zc* A) {
  const int N = p->L * p->L;
  const zc z = p->mu + I * orc_omega_n(p, n);
  for (size_t k = 0; k < (size_t)N * N; ++k) A[k] = -H[k];
  for (int i = 0; i < N; ++i) A[(size_t)i * N + i] += z;
}

/* One (n, sigma) block: ln|det A| and, if diag != NULL, Re and Im of G_ii.
 * If full != NULL it receives all of G = A^{-1} (row-major, interleaved re/im). */
int orc_block(const orc_params* p, const double* eps_extra, const double* phi, int n,
              int sigma, double* ld, double* diag_re, double* diag_im, double* full) {
  const int N = p->L * p->L;
  double* H = (double*)malloc(sizeof(double) * (size_t)N * N);
  zc* A = (zc*)malloc(sizeof(zc) * (size_t)N * N);
  int* piv = (int*)malloc(sizeof(int) * N);
  zc* x = (zc*)malloc(sizeof(zc) * N);
  orc_hamiltonian(p, eps_extra, phi, sigma, H);
  build_A(p, H, n, A);
  int rc = orc_zgetrf(N, A, piv, ld);
  if (rc == 0 && (diag_re || full)) {
    for (int j = 0; j < N; ++j) {
      lu_solve_unit(N, A, piv, j, x);
      if (diag_re) diag_re[j] = creal(x[j]);
      if (diag_im) diag_im[j] = cimag(x[j]);
      if (full)
        for (int r = 0; r < N; ++r) {
          full[2 * ((size_t)r * N + j)] = creal(x[r]);
          full[2 * ((size_t)r * N + j) + 1] = cimag(x[r]);
        }
    }
  }
  free(H); free(A); free(piv); free(x);
  return rc;
}

/* Matrix index of block (n, sigma): b = 2n + s, s = 0 (sigma=+1), 1 (sigma=-1). */
static int sigma_of(int s) { return s == 0 ? +1 : -1; }

/* Omega and dOmega/dphi over all (n, sigma) blocks, by the LU route.
 * ld_out (2*n_omega) and gdiag_out (2*n_omega*N, holding sigma*Re G_ii) are
 * optional per-block outputs.  The sums run in the fixed order b = 0, 1, ... */
int orc_omega_grad(const orc_params* p, const double* eps_extra, const double* phi,
                   double* omega, double* grad, double* ld_out, double* gdiag_out) {
  const int N = p->L * p->L, B = 2 * p->n_omega;
  double* ld = (double*)calloc(B, sizeof(double));
  double* gd = grad ? (double*)calloc((size_t)B * N, sizeof(double)) : NULL;
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
  for (int b = 0; b < B; ++b) {
    const int n = b / 2, sg = sigma_of(b % 2);
    double* dre = gd ? gd + (size_t)b * N : NULL;
    if (orc_block(p, eps_extra, phi, n, sg, &ld[b], dre, NULL, NULL) != 0) bad = 1;
    if (dre)
      for (int i = 0; i < N; ++i) dre[i] *= sg;
  }
  double q = 0.0, s = 0.0;
  for (int i = 0; i < N; ++i) q += phi[i] * phi[i];
  for (int b = 0; b < B; ++b) s += ld[b];
  if (omega) *omega = q / p->U - 2.0 * p->T * s;
  if (grad)
    for (int i = 0; i < N; ++i) {
      double acc = 0.0;
      for (int b = 0; b < B; ++b) acc += gd[(size_t)b * N + i];
      grad[i] = 2.0 * phi[i] / p->U - 2.0 * p->T * acc;
    }
  if (ld_out) memcpy(ld_out, ld, sizeof(double) * B);
  if (gdiag_out && gd) memcpy(gdiag_out, gd, sizeof(double) * (size_t)B * N);
  free(ld); free(gd);
  return bad ? -1 : 0;
}

/* Same per-block quantities for a chosen list of blocks (for sampled checks
 * at sizes where the whole batch is too slow). */
int orc_blocks_sample(const orc_params* p, const double* eps_extra, const double* phi,
                      int count, const int* blocks, double* ld_out, double* gdiag_out) {
  const int N = p->L * p->L;
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
  for (int c = 0; c < count; ++c) {
    const int b = blocks[c], n = b / 2, sg = sigma_of(b % 2);
    double* dre = gdiag_out ? gdiag_out + (size_t)c * N : NULL;
    if (orc_block(p, eps_extra, phi, n, sg, &ld_out[c], dre, NULL, NULL) != 0) bad = 1;
    if (dre)
      for (int i = 0; i < N; ++i) dre[i] *= sg;
  }
  return bad ? -1 : 0;
}

/* ------------------------------------------- eigenvalue route (Jacobi) -- */

/* Cyclic Jacobi diagonalisation of a real symmetric N x N matrix (row-major,
 * destroyed).  evec columns are eigenvectors: H = V diag(e) V^T. */
int orc_jacobi(int N, double* A, double* e, double* V) {
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) V[(size_t)i * N + j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) {
        const double a = A[(size_t)i * N + j] * A[(size_t)i * N + j];
        tot += a;
        if (i != j) off += a;
      }
    if (off <= 1e-30 * (tot > 0 ? tot : 1.0)) break;
    for (int pq = 0; pq < N; ++pq)
      for (int q = pq + 1; q < N; ++q) {
        const int pp = pq;
        const double apq = A[(size_t)pp * N + q];
        if (apq == 0.0) continue;
        const double app = A[(size_t)pp * N + pp], aqq = A[(size_t)q * N + q];
        const double theta = (aqq - app) / (2.0 * apq);
        const double tt = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(tt * tt + 1.0), s = tt * c;
        for (int k = 0; k < N; ++k) { /* columns pp, q */
          const double akp = A[(size_t)k * N + pp], akq = A[(size_t)k * N + q];
          A[(size_t)k * N + pp] = c * akp - s * akq;
          A[(size_t)k * N + q] = s * akp + c * akq;
        }
        for (int k = 0; k < N; ++k) { /* rows pp, q */
          const double apk = A[(size_t)pp * N + k], aqk = A[(size_t)q * N + k];
          A[(size_t)pp * N + k] = c * apk - s * aqk;
          A[(size_t)q * N + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < N; ++k) {
          const double vkp = V[(size_t)k * N + pp], vkq = V[(size_t)k * N + q];
          V[(size_t)k * N + pp] = c * vkp - s * vkq;
          V[(size_t)k * N + q] = s * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < N; ++i) e[i] = A[(size_t)i * N + i];
  return 0;
}

/* Omega and gradient from the spectrum of H_sigma: for each eigenpair (e_a, V_.a)
 *   ln|det A_n| = sum_a 1/2 ln(omega_n^2 + (mu - e_a)^2),
 *   Re G_ii     = sum_a V_ia^2 (mu - e_a) / (omega_n^2 + (mu - e_a)^2). */
int orc_omega_grad_eig(const orc_params* p, const double* eps_extra, const double* phi,
                       double* omega, double* grad, double* ld_out, double* gdiag_out) {
  const int N = p->L * p->L, B = 2 * p->n_omega;
  double* H = (double*)malloc(sizeof(double) * (size_t)N * N);
  double* V = (double*)malloc(sizeof(double) * (size_t)N * N);
  double* e = (double*)malloc(sizeof(double) * N);
  double* ld = (double*)calloc(B, sizeof(double));
  double* gd = (double*)calloc((size_t)B * N, sizeof(double));
  for (int s = 0; s < 2; ++s) {
    const int sg = sigma_of(s);
    orc_hamiltonian(p, eps_extra, phi, sg, H);
    orc_jacobi(N, H, e, V);
    for (int n = 0; n < p->n_omega; ++n) {
      const double w = orc_omega_n(p, n);
      const int b = 2 * n + s;
      double acc = 0.0;
      for (int a = 0; a < N; ++a) acc += 0.5 * log(w * w + (p->mu - e[a]) * (p->mu - e[a]));
      ld[b] = acc;
      for (int i = 0; i < N; ++i) {
        double g = 0.0;
        for (int a = 0; a < N; ++a) {
          const double xi = p->mu - e[a];
          g += V[(size_t)i * N + a] * V[(size_t)i * N + a] * xi / (w * w + xi * xi);
        }
        gd[(size_t)b * N + i] = sg * g;
      }
    }
  }
  double q = 0.0, sum = 0.0;
  for (int i = 0; i < N; ++i) q += phi[i] * phi[i];
  for (int b = 0; b < B; ++b) sum += ld[b];
  if (omega) *omega = q / p->U - 2.0 * p->T * sum;
  if (grad)
    for (int i = 0; i < N; ++i) {
      double acc = 0.0;
      for (int b = 0; b < B; ++b) acc += gd[(size_t)b * N + i];
      grad[i] = 2.0 * phi[i] / p->U - 2.0 * p->T * acc;
    }
  if (ld_out) memcpy(ld_out, ld, sizeof(double) * B);
  if (gdiag_out) memcpy(gdiag_out, gd, sizeof(double) * (size_t)B * N);
  free(H); free(V); free(e); free(ld); free(gd);
  return 0;
}

/* ------------------------------------------------ density of states ----- */

/* Density of states of spin sigma at the field phi (Sec. II, the equation after Eq. 2, with
 * H_SCA = H_sigma(phi)):
 *     rho_sigma(w) = -(1/(pi N)) Im Tr [(w + i eta + mu) I - H_sigma]^{-1},
 * the trace normalised per site (the paper prints the resolvent without naming the trace;
 * the per-site normalisation makes rho integrate to 1 over w).  LU route: each resolvent is
 * the dense complex LU with partial pivoting and the inverse column by column, as in
 * orc_block.  rho_out[k] for the count frequencies w[k], OpenMP over k. */
int orc_dos(const orc_params* p, const double* eps_extra, const double* phi, int sigma,
            int count, const double* w, double eta, double* rho_out) {
  const int N = p->L * p->L;
  double* H = (double*)malloc(sizeof(double) * (size_t)N * N);
  orc_hamiltonian(p, eps_extra, phi, sigma, H);
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
  for (int k = 0; k < count; ++k) {
    zc* A = (zc*)malloc(sizeof(zc) * (size_t)N * N);
    int* piv = (int*)malloc(sizeof(int) * N);
    zc* x = (zc*)malloc(sizeof(zc) * N);
    const zc z = w[k] + p->mu + I * eta;
    for (size_t q = 0; q < (size_t)N * N; ++q) A[q] = -H[q];
    for (int i = 0; i < N; ++i) A[(size_t)i * N + i] += z;
    double ld = 0.0;
    if (orc_zgetrf(N, A, piv, &ld) != 0) {
      bad = 1;
    } else {
      double tr = 0.0;
      for (int j = 0; j < N; ++j) {
        lu_solve_unit(N, A, piv, j, x);
        tr += cimag(x[j]);
      }
      rho_out[k] = -tr / (M_PI * N);
    }
    free(A); free(piv); free(x);
  }
  free(H);
  return bad ? -1 : 0;
}

/* The same density of states by the eigenvalue route: H_sigma = V diag(e) V^T (Jacobi), so
 * Tr [z - H]^{-1} = sum_a 1 / (z - e_a) and
 *     rho_sigma(w) = (1/(pi N)) sum_a eta / ((w + mu - e_a)^2 + eta^2),
 * a sum of Lorentzians of unit weight. */
int orc_dos_eig(const orc_params* p, const double* eps_extra, const double* phi, int sigma,
                int count, const double* w, double eta, double* rho_out) {
  const int N = p->L * p->L;
  double* H = (double*)malloc(sizeof(double) * (size_t)N * N);
  double* V = (double*)malloc(sizeof(double) * (size_t)N * N);
  double* e = (double*)malloc(sizeof(double) * N);
  orc_hamiltonian(p, eps_extra, phi, sigma, H);
  orc_jacobi(N, H, e, V);
  for (int k = 0; k < count; ++k) {
    double acc = 0.0;
    for (int a = 0; a < N; ++a) {
      const double d = w[k] + p->mu - e[a];
      acc += eta / (d * d + eta * eta);
    }
    rho_out[k] = acc / (M_PI * N);
  }
  free(H); free(V); free(e);
  return 0;
}

/* ------------------------------------------------------ seeded phi0 ------ */

static uint64_t splitmix64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* k-th output (k = 0, 1, ...) of the splitmix64 stream started at `seed`. */
uint64_t orc_splitmix64(uint64_t seed, uint64_t k) {
  return splitmix64_mix(seed + (k + 1) * 0x9E3779B97F4A7C15ULL);
}

/* phi0_i = (top 53 bits of the i-th output) * 2^-53 - 1/2, in [-0.5, 0.5). */
void orc_seed_phi(uint64_t seed, int N, double* phi) {
  for (int i = 0; i < N; ++i)
    phi[i] = (double)(orc_splitmix64(seed, (uint64_t)i) >> 11) * 0x1.0p-53 - 0.5;
}

/* -------------------------------------------------------------- Adam ----- */

/* ------------------------------------------------- Metropolis sampling -- */

/* Uniform in [0, 1): the top 53 bits of output k of the splitmix64 stream `seed`. */
static double u01(uint64_t seed, uint64_t k) {
  return (double)(orc_splitmix64(seed, k) >> 11) * 0x1.0p-53;
}

/* Standard normal number j of step s: the Box-Muller transform (Box & Muller 1958) of the
 * uniforms U(seed, 2(sN + j)) and U(seed, 2(sN + j) + 1). */
double orc_metro_normal(uint64_t seed, int64_t s, int N, int j) {
  const uint64_t k = 2ull * ((uint64_t)s * (uint64_t)N + (uint64_t)j);
  const double u1 = u01(seed, k), u2 = u01(seed, k + 1);
  return sqrt(-2.0 * log(1.0 - u1)) * cos(2.0 * M_PI * u2);
}

/* Metropolis sampling of the static-field weight exp(-V(phi)/T) of the SCA partition function
 * (Sec. II, the integral over phi_1 .. phi_N with weight exp(-beta V)), V = Omega as defined
 * above.  Step s (global index step0 + s of the chain):
 *     phi'_i = phi_i + delta g_i,       g_i = orc_metro_normal(seed, s, N, i),
 *     accepted iff U(seed + 1, s) < exp(-(Omega(phi') - Omega(phi)) / T).
 * Omega by the LU route.  phi is updated in place; omega_trace[s] = Omega of the chain's state
 * after step s and accepted[s] in {0, 1} (both optional). */
int orc_metropolis(const orc_params* p, const double* eps_extra, double* phi, int n_steps,
                   double delta, uint64_t seed, int64_t step0, double* omega_trace,
                   int* accepted) {
  const int N = p->L * p->L;
  double* prop = (double*)malloc(sizeof(double) * N);
  double om = 0.0;
  if (orc_omega_grad(p, eps_extra, phi, &om, NULL, NULL, NULL) != 0) { free(prop); return -1; }
  for (int s = 0; s < n_steps; ++s) {
    const int64_t gs = step0 + s;
    for (int i = 0; i < N; ++i) prop[i] = phi[i] + delta * orc_metro_normal(seed, gs, N, i);
    double om2 = 0.0;
    if (orc_omega_grad(p, eps_extra, prop, &om2, NULL, NULL, NULL) != 0) { free(prop); return -1; }
    const int acc = u01(seed + 1, (uint64_t)gs) < exp(-(om2 - om) / p->T);
    if (acc) {
      memcpy(phi, prop, sizeof(double) * N);
      om = om2;
    }
    if (omega_trace) omega_trace[s] = om;
    if (accepted) accepted[s] = acc;
  }
  free(prop);
  return 0;
}

/* Runs Adam on Omega from phi (in/out).  Each iteration evaluates the
 * gradient at the current phi; if max|g| < grad_tol it stops, else it takes
 * one Adam step.  Histories (max_steps entries, optional) hold Omega and
 * max|g| at the phi each gradient was taken at.  Returns the number of Adam
 * updates applied in *steps. */
int orc_adam_run(const orc_params* p, const double* eps_extra, const orc_adam* a, double* phi,
                 double* omega_hist, double* gmax_hist, int32_t* steps, double* omega_last,
                 double* gmax_last) {
  const int N = p->L * p->L;
  double* m = (double*)calloc(N, sizeof(double));
  double* v = (double*)calloc(N, sizeof(double));
  double* g = (double*)malloc(sizeof(double) * N);
  int k = 0, rc = 0;
  double om = 0.0, gm = 0.0;
  for (;;) {
    if (orc_omega_grad(p, eps_extra, phi, &om, g, NULL, NULL) != 0) { rc = -1; break; }
    gm = 0.0;
    for (int i = 0; i < N; ++i) gm = fmax(gm, fabs(g[i]));
    if (k < a->max_steps) {
      if (omega_hist) omega_hist[k] = om;
      if (gmax_hist) gmax_hist[k] = gm;
    }
    if (gm < a->grad_tol || k >= a->max_steps) break;
    ++k;
    const double bc1 = 1.0 - pow(a->beta1, k), bc2 = 1.0 - pow(a->beta2, k);
    const double step = a->lr / bc1, sbc2 = sqrt(bc2);
    for (int i = 0; i < N; ++i) {
      m[i] = a->beta1 * m[i] + (1.0 - a->beta1) * g[i];
      v[i] = a->beta2 * v[i] + (1.0 - a->beta2) * g[i] * g[i];
      const double denom = sqrt(v[i]) / sbc2 + a->eps;
      phi[i] -= step * m[i] / denom;
    }
  }
  if (steps) *steps = k;
  if (omega_last) *omega_last = om;
  if (gmax_last) *gmax_last = gm;
  free(m); free(v); free(g);
  return rc;
}
