/*
 * sca.h -- C ABI of the GB300 (sm_103a) SCA+ADAM library.
 *
 * The library evaluates, differentiates and minimises the semiclassical (SCA)
 * potential of the 2D ionic Hubbard model of Park & Lee, arXiv 2311.04435:
 *
 *   Omega(phi) = sum_i phi_i^2 / U  -  2T sum_{n=0}^{n_omega-1} sum_{sigma=+-1}
 *                ln |det A_{n,sigma}(phi)|,
 *   A_{n,sigma} = (i omega_n + mu) I - H_sigma(phi),  omega_n = (2n+1) pi T,
 *   H_sigma(phi) = K + diag(eps_i - sigma phi_i),
 *
 * on an L x L periodic square lattice (site i = x*L + y, sublattice sign
 * s_i = (-1)^(x+y), A <=> s = +1), K the nearest-neighbour hopping -t with
 * bonds accumulated (L = 2 gives -2t), eps_i = -s_i Delta (Eq. 1: -Delta on A,
 * +Delta on B) or -s_i Delta/2 with SCA_IONIC_HALF.  (Paper: Eq. 1 for the
 * Hamiltonian, Sec. II HS line and Eq. 2 for the potential; the factor 2 and
 * n >= 0 pair each omega_n with -omega_n, whose determinant is the complex
 * conjugate; the -beta inside the determinant of Eq. 2 is a constant and is
 * dropped; phi is normalised so that the stationary point is the Hartree-Fock
 * gap phi_i = U m_i / 2.)
 *
 * Gradient: dOmega/dphi_i = 2 phi_i / U - 2T sum_{n,sigma} sigma Re G_{n sigma, ii},
 * G = A^{-1}.  Minimisation: Adam (Sec. II: "ADAM optimizer based on the
 * PyTorch library"; Kingma & Ba 2014) with bias correction and PyTorch's
 * arithmetic order.
 *
 * Conventions for every call:
 *  - Every function returns an sca_status; none aborts.  On failure,
 *    sca_last_error() returns a message for the calling thread.
 *  - The caller owns every pointer it passes; the library copies host arrays
 *    in and out before returning.  The context owns all device workspace.
 *  - "host" arrays are ordinary CPU memory; "_dev" arrays are device pointers
 *    (cudaMalloc / torch CUDA tensors) on the context's device.
 *  - Arrays of N = L*L sites are float64 in site order i = x*L + y.
 *  - A context is not thread-safe; use one per thread.  A server is safe for
 *    concurrent sca_submit / sca_poll from several threads.
 *  - Blocks are numbered b = 2n + s with s = 0 for sigma = +1 (up) and s = 1
 *    for sigma = -1 (down).
 */
#ifndef SCA_GB300_H
#define SCA_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sca_ctx sca_ctx;
typedef struct sca_server sca_server;

typedef enum {
  SCA_OK = 0,
  SCA_EINVAL = 1,      /* invalid argument (parameters, sizes, NULL pointers) */
  SCA_ENOMEM = 2,      /* device or host allocation failed */
  SCA_EBUDGET = 3,     /* request does not fit the server's HBM budget */
  SCA_ECUDA = 4,       /* a CUDA runtime call failed (message has the CUDA error) */
  SCA_ETIMEOUT = 5,    /* a bounded device-side wait ran out */
  SCA_EPENDING = 6,    /* request not finished yet (sca_poll) */
  SCA_ENONFINITE = 7,  /* Omega or the gradient became NaN/Inf, or a block was singular */
  SCA_ENOTFOUND = 8,   /* unknown request id */
  SCA_ENOSTATE = 9     /* call order: e.g. sca_adam_step before sca_adam_init */
} sca_status;

/* Arithmetic of the dense contractions.  FP64: everything in float64.
 * FP32: blocks stored as complex64, CUDA-core float32 contractions.
 * 3XTF32: complex64 blocks, contractions on tcgen05 tensor cores in split
 * TF32 (hi*hi + hi*lo + lo*hi, hi = the value with 13 low mantissa bits cleared) with
 * float32 accumulation.
 * BF16X3: complex64 blocks, the same contractions with bf16 halves (hi = RN_bf16(v),
 * lo = RN_bf16(v - hi): about 17 significant bits) on kind::f16 at twice the TF32 rate.
 * For the three reduced-precision modes ln|u_kk| is accumulated in float64
 * and every diagonal G_ii gets one float64 refinement step
 * (G_ii <- 2 X_ii - (X A X^T)_ii with the sparse A).  Blocks below 128 x 128 take the FP32
 * path in both split modes. */
typedef enum {
  SCA_PREC_FP64 = 0,
  SCA_PREC_FP32 = 1,
  SCA_PREC_3XTF32 = 2,
  SCA_PREC_BF16X3 = 3
} sca_prec;

typedef enum {
  SCA_IONIC_PAPER = 0, /* eps_i = -s_i * Delta (Eq. 1) */
  SCA_IONIC_HALF = 1   /* eps_i = -s_i * Delta / 2 */
} sca_ionic;

/* Physical parameters.  L even, 2 <= L <= 64; 1 <= n_omega <= 16384; U > 0; T > 0;
 * t, Delta, mu finite. */
typedef struct {
  int32_t L, n_omega, prec, ionic;
  double t, U, delta, T, mu;
} sca_params;

/* Adam settings.  lr > 0, 0 <= beta1, beta2 < 1, eps > 0.  grad_tol and
 * max_steps are used by sca_solve and the server (stop when max|g| < grad_tol
 * or after max_steps updates).  seed selects the SplitMix64 start field
 * phi0_i = top53(splitmix64(seed, i)) * 2^-53 - 1/2 when no phi0 is given. */
typedef struct {
  double lr, beta1, beta2, eps, grad_tol;
  int32_t max_steps;
  uint64_t seed;
} sca_adam;

/* ----------------------------------------------------------- contexts ---- */

/* Creates a context for one parameter set on the current CUDA device and
 * allocates its device workspace (all 2*n_omega blocks resident unless the
 * environment variable SCA_MAX_BLOCKS_RESIDENT caps the chunk size).
 * Errors: SCA_EINVAL (bad parameters, out != NULL required), SCA_ENOMEM,
 * SCA_ECUDA. */
sca_status sca_create(const sca_params* params, sca_ctx** out);

/* Frees the context and its workspace.  NULL is ignored. */
void sca_destroy(sca_ctx* ctx);

/* Bytes of device memory a context with these parameters allocates. */
sca_status sca_workspace_bytes(const sca_params* params, uint64_t* bytes);

/* Adds a per-site energy eps_extra[i] (N host doubles) to H_sigma, e.g. the
 * random on-site potential of the disordered model (Sec. IV).  NULL clears
 * it.  Errors: SCA_EINVAL, SCA_ECUDA. */
sca_status sca_set_site_energy(sca_ctx* ctx, const double* eps_extra_host);

/* Omega(phi) for a host field phi (N doubles).  Runs the blocked pivoted LU
 * of every block (Eq. 2; no inverse).  Errors: SCA_EINVAL, SCA_ENONFINITE,
 * SCA_ECUDA. */
sca_status sca_potential(sca_ctx* ctx, const double* phi_host, double* omega);

/* Omega(phi) and its gradient (grad: N host doubles).  Runs the blocked
 * Gauss-Jordan inversion of every block, whose pivots are those of the LU
 * (same ln|det|) and whose result is G = A^{-1}.  Errors as sca_potential. */
sca_status sca_grad(sca_ctx* ctx, const double* phi_host, double* omega, double* grad);

/* Device-pointer variants.  d_phi: N doubles; d_omega: 1 double; d_grad: N
 * doubles; stream: a cudaStream_t (NULL = legacy default stream).  They
 * enqueue the work on `stream` and return without synchronising; Omega is
 * written by a kernel.  A non-finite result is not reported here (check the
 * outputs); launch errors return SCA_ECUDA. */
sca_status sca_potential_dev(sca_ctx* ctx, const double* d_phi, double* d_omega, void* stream);
sca_status sca_grad_dev(sca_ctx* ctx, const double* d_phi, double* d_omega, double* d_grad,
                        void* stream);

/* Autograd split (device pointers, asynchronous on `stream`).
 * sca_forward_dev: Omega(phi) through the blocked Gauss-Jordan inversion of every block; the
 * inverses stay resident in the context's workspace.
 * sca_backward_dev: the adjoint stage from those resident inverses: the diagonal of
 * G = A^{-1} (refined in float64 for the reduced precisions) reduced into
 * d_grad = dOmega/dphi.  It must follow a sca_forward_dev with the same d_phi contents and no
 * other call on the context in between; it returns SCA_ENOSTATE otherwise, or when the
 * workspace is chunked (not every block resident). */
sca_status sca_forward_dev(sca_ctx* ctx, const double* d_phi, double* d_omega, void* stream);
sca_status sca_backward_dev(sca_ctx* ctx, const double* d_phi, double* d_grad, void* stream);

/* Per-block diagnostics for testing each step of the path (host outputs):
 * ld[b] = ln|det A_b| (2*n_omega doubles) and, if gdiag != NULL,
 * gdiag[b*N + i] = sigma_b * Re G_{b,ii} (refined as for sca_grad). */
sca_status sca_blocks(sca_ctx* ctx, const double* phi_host, double* ld, double* gdiag);

/* Writes the assembled blocks A_b (before factorisation) for b in
 * [b0, b0+count) as interleaved complex128, row-major N x N each, into host
 * memory out (count*N*N*2 doubles).  For testing the assembly step. */
sca_status sca_debug_assemble(sca_ctx* ctx, const double* phi_host, int32_t b0, int32_t count,
                              double* out);

/* -------------------------------------------------------------- Adam ---- */

/* Starts an Adam run: phi <- phi0 (N host doubles) or the SplitMix64 field
 * of adam->seed when phi0 == NULL; moments m = v = 0; step counter 0.  phi,
 * m and v stay resident on the device.  Errors: SCA_EINVAL, SCA_ECUDA. */
sca_status sca_adam_init(sca_ctx* ctx, const sca_adam* adam, const double* phi0_host);

/* Applies nsteps >= 1 Adam updates.  Each update evaluates Omega and the
 * gradient at the current phi, then moves phi.  *omega and *gmax (may be
 * NULL) receive Omega and max|g| at the phi of the last update's gradient.
 * Errors: SCA_ENOSTATE (no sca_adam_init), SCA_ENONFINITE, SCA_ECUDA. */
sca_status sca_adam_step(sca_ctx* ctx, int32_t nsteps, double* omega, double* gmax);

/* Runs Adam on the context's resident state with the convergence gate of sca_solve: each
 * update is applied only while max|g| >= grad_tol (the settings of sca_adam_init or
 * sca_set_state), and the call returns once an evaluation finds max|g| < grad_tol or after
 * max_steps >= 0 updates.  *steps receives the updates this call applied; *omega and *gmax
 * receive Omega and max|g| at the final phi (any may be NULL).  Unlike sca_solve it keeps the
 * context's site energies (sca_set_site_energy), pivoting mode and stream.  Errors:
 * SCA_EINVAL, SCA_ENOSTATE (no sca_adam_init), SCA_ENONFINITE, SCA_ETIMEOUT, SCA_ECUDA. */
sca_status sca_adam_run(sca_ctx* ctx, int32_t max_steps, int32_t* steps, double* omega,
                        double* gmax);

/* Copies the current phi (N doubles) to host memory. */
sca_status sca_get_phi(sca_ctx* ctx, double* phi_out);

/* Copies phi, m, v (N doubles each, any may be NULL) and the step count. */
sca_status sca_get_state(sca_ctx* ctx, double* phi, double* m, double* v, int32_t* step);

/* Restores phi, m, v and the step count (checkpoint resume).  The run then
 * continues bit-identically to one that was never interrupted. */
sca_status sca_set_state(sca_ctx* ctx, const sca_adam* adam, const double* phi, const double* m,
                         const double* v, int32_t step);

/* One-shot minimisation: creates a context, runs Adam from phi0 (NULL =
 * seeded) until max|g| < adam->grad_tol or adam->max_steps updates, and
 * returns the final phi (N doubles, may be NULL), Omega and max|g| at the
 * final phi and the number of updates applied. */
sca_status sca_solve(const sca_params* params, const sca_adam* adam, const double* phi0_host,
                     double* phi_out, double* omega, int32_t* steps, double* gmax);

/* ------------------------------------------------------------ serving ---- */

/* Creates a serving loop on the current device with an HBM admission budget
 * (bytes of device memory that admitted requests may hold at once) and at most
 * max_slots requests in flight.  A host thread admits queued requests in
 * arrival order as slots and budget free up and advances all admitted
 * requests together, a few gated Adam updates per round, so new requests join
 * while others run (continuous batching).  Requests whose blocks exceed the
 * fused kernel's size (N > 144; FP64: N > 64) are batched by size bucket: those
 * with the same L and precision share one workspace of up to 256 block slots
 * (counted against the budget while the bucket has requests) and one launch
 * sequence per step.  A request's result is the same bit for bit as with
 * sca_solve.  Errors: SCA_EINVAL, SCA_ENOMEM, SCA_ECUDA. */
sca_status sca_server_create(uint64_t hbm_budget_bytes, int32_t max_slots, sca_server** out);

/* Queues a solve request (parameters and Adam settings are copied; phi0 is
 * the seeded field of adam->seed).  *req_id receives its id.  Errors:
 * SCA_EINVAL, SCA_EBUDGET (the request alone, with a bucket just large enough
 * for its blocks where it is bucketed, exceeds the budget). */
sca_status sca_submit(sca_server* srv, const sca_params* params, const sca_adam* adam,
                      uint64_t* req_id);

/* Result of a request: SCA_EPENDING while queued or running; SCA_OK with phi
 * (N doubles, may be NULL), Omega, updates applied and max|g| once done; the
 * request's own error status if it failed; SCA_ENOTFOUND for unknown ids.
 * A finished request stays pollable until the server is destroyed. */
sca_status sca_poll(sca_server* srv, uint64_t req_id, double* phi_out, double* omega,
                    int32_t* steps, double* gmax);

/* Per-request timing in seconds since server creation: arrival (submit),
 * admission, first update, completion (negative while not reached). */
sca_status sca_request_times(sca_server* srv, uint64_t req_id, double* submit_s, double* admit_s,
                             double* start_s, double* finish_s);

/* Stops the loop (in-flight requests are abandoned) and frees everything. */
void sca_server_destroy(sca_server* srv);

/* A server without a worker thread, for replaying an arrival trace deterministically: the
 * caller drives it with sca_server_step, and its clock is virtual (the times of
 * sca_request_times are the now_s values of the steps, and a submission is stamped with the
 * clock of the last step).  Admission, batching and retirement are those of the threaded
 * server, so a replay of the same submissions and steps gives the same admission order,
 * in-flight counts, update counts, times and results, bit for bit.  Errors as
 * sca_server_create. */
sca_status sca_server_create_manual(uint64_t hbm_budget_bytes, int32_t max_slots,
                                    sca_server** out);

/* One round of a manual server at virtual time now_s (non-decreasing): admission of queued
 * requests, one batch of gated Adam updates for every request in flight, retirement of the
 * finished ones.  *in_flight and *queued (may be NULL) receive the requests running and
 * waiting after the round.  Runs on the calling thread and returns when the round is done.
 * Errors: SCA_EINVAL (not a manual server, clock running backwards). */
sca_status sca_server_step(sca_server* srv, double now_s, int32_t* in_flight, int32_t* queued);

/* ------------------------------------------------------ allocation-free ---- */

/* Omega and dOmega/dphi like sca_grad_dev, without allocating any memory.  (The paper has
 * no counterpart: this entry point exists for callers that cannot let a library allocate,
 * e.g. a process whose device memory is reserved up front by its own pool allocator, or a
 * steady-state loop that must not call cudaMalloc/cudaFree because they can synchronise
 * the device.)
 *  - params: as for sca_create, with prec SCA_PREC_FP64 or SCA_PREC_FP32 (CUDA-core
 *    contractions); d_phi: N device doubles (input); d_omega: 1 device double and d_grad:
 *    N device doubles (outputs, written by kernels); stream: cudaStream_t or NULL.
 *  - Workspace: one file-scope device array of 64 MiB that every GPU which loads the
 *    library holds until the process exits.  The blocks are processed in chunks that fit
 *    it; a problem whose single block (plus the per-block log-dets and diagonals) does not
 *    fit is rejected with SCA_EINVAL and a message, before anything is enqueued.
 *  - Every call looks up the array's device address on the calling thread's current device
 *    (a host-side query that allocates and enqueues nothing; the address follows the device's
 *    context, which cudaDeviceReset re-creates).  The first call in a process on a device also
 *    loads the library's device code there: make that first call before any stream capture.
 *  - Every call on a device shares the one array and leaves its contents behind; the call
 *    clears what must start at zero.  Calls that overlap on the GPU (other streams or
 *    threads) race on the array and give wrong results: serialise them.
 *  - Makes no cudaMalloc, cudaFree or other allocating call.  Returns without
 *    synchronising; launch errors return SCA_ECUDA. */
sca_status sca_grad_noalloc_dev(const sca_params* params, const double* d_phi, double* d_omega,
                                double* d_grad, void* stream);

/* ------------------------------------------------------------ streams ---- */

/* Makes every later call on this context enqueue on `stream` (a cudaStream_t; NULL
 * restores the context's own stream).  The host-buffer calls still synchronise that
 * stream before returning. */
sca_status sca_set_stream(sca_ctx* ctx, void* stream);

/* Bound of every device-side spin wait issued for this context (grid barriers of the fused
 * small-block kernel), in SM clock cycles; 0 restores the default (4e9, about 2 s).  A wait
 * that runs out makes the call return SCA_ETIMEOUT; the context stays usable. */
sca_status sca_set_wait_limit(sca_ctx* ctx, int64_t cycles);

/* Density of states of both spins at the field phi (Sec. II, the equation after Eq. 2, with
 * H_SCA = H_sigma(phi) and the trace taken per site):
 *     rho_sigma(w) = -(1/(pi N)) Im Tr [(w + i eta + mu) I - H_sigma(phi)]^{-1}.
 * phi_host: N doubles (host); w_host: n_w real frequencies (host, finite); eta > 0: the
 * broadening.  rho_out (host, 2 n_w doubles): spin up (sigma = +1) at [0, n_w), spin down at
 * [n_w, 2 n_w).  The resolvents go through the same batched elimination as the gradient, in
 * batches of n_omega frequencies (the context's block slots), with partial pivoting unless
 * eta > 4|t| or the context is set to SCA_PIVOT_NONE; the mixed precisions take Im G_ii from
 * the float32 inverse without refinement.  Invalidates the inverses kept for
 * sca_backward_dev.  SCA_EINVAL for bad arguments, SCA_ENONFINITE for a singular resolvent. */
sca_status sca_dos(sca_ctx* ctx, const double* phi_host, const double* w_host, int32_t n_w,
                   double eta, double* rho_out);

/* Metropolis sampling of the static-field weight exp(-Omega(phi)/T) of the SCA partition
 * function (Sec. II: Z is an integral over phi_1 .. phi_N with weight exp(-beta V), V = Omega).
 * The chain's state is the context's resident field (the one sca_get_phi returns; Adam's
 * moments are left alone).  Step t (t = 0, 1, ... counted from sca_metropolis_init):
 *     phi'_i = phi_i + delta g_i,  g_i = sqrt(-2 ln(1 - U(seed, 2(tN+i)))) cos(2 pi U(seed, 2(tN+i)+1)),
 *     accepted iff U(seed + 1, t) < exp(-(Omega(phi') - Omega(phi)) / T),
 * with U(s, k) the top 53 bits of output k of the SplitMix64 stream started at s, times 2^-53.
 * Omega(phi') comes from the LU-only elimination in the context's precision; steps run on the
 * device without host round trips.
 * sca_metropolis_init: phi0_host (N doubles, host) or NULL for the seeded start field;
 *   delta >= 0 finite; evaluates Omega(phi0).  SCA_EINVAL for bad arguments.
 * sca_metropolis_step: n_steps >= 0 further steps; optional host outputs omega_trace (n_steps
 *   doubles: Omega of the state after each step) and accepted (n_steps bytes, 0/1); omega: Omega
 *   of the final state; accepted_total: accepted steps since init.  SCA_ENOSTATE before init;
 *   SCA_ENONFINITE if a proposal gave a non-finite Omega (it was rejected).
 * The paper has no device-side sampler; it names the integral the field is drawn from. */
sca_status sca_metropolis_init(sca_ctx* ctx, const double* phi0_host, double delta, uint64_t seed);
sca_status sca_metropolis_step(sca_ctx* ctx, int32_t n_steps, double* omega_trace,
                               uint8_t* accepted, double* omega, int64_t* accepted_total);

/* Pivoting of the batched elimination of the A_{n,sigma} (Sec. II, Eq. 2).
 *   SCA_PIVOT_PARTIAL (default): partial pivoting for the blocks whose column diagonal
 *     dominance is not guaranteed (omega_n <= 4|t|); the remaining blocks provably keep their
 *     diagonal pivots and skip the search.
 *   SCA_PIVOT_NONE: every block is eliminated without interchanges, as a complex-symmetric
 *     (LDL^T-type) elimination that updates one triangle on the tensor-core path.  The paper
 *     has no such variant.  -i A_{n,sigma} has Hermitian part omega_n I > 0, so every leading
 *     principal minor is nonzero and the elimination exists; its growth has no a-priori bound
 *     and rises as omega_n falls (the largest growth met in tests is below 10, down to
 *     T = 0.02).  The fused small-block path (N <= 144) always pivots.
 * Applies from the next call on the context; any other mode is SCA_EINVAL. */
typedef enum { SCA_PIVOT_PARTIAL = 0, SCA_PIVOT_NONE = 1 } sca_pivot;
sca_status sca_set_pivoting(sca_ctx* ctx, int32_t mode);

/* Arithmetic of the pivoted blocks' panel factorisation (the sub-panel LU with its pivot search,
 * the interchanges with U12 and the rest-of-panel update) on the reduced-precision paths:
 * SCA_PREC_FP32 (default: the blocks' compute type) or SCA_PREC_FP64 (float64 arithmetic on
 * the float32 blocks; the doubled shared-memory panel narrows the sub-panels, e.g. to 4
 * columns at N = 1600).  The pivot-block inverses and the contractions are unchanged.  Float64
 * contexts accept only SCA_PREC_FP64.  Applies from the next call; SCA_EINVAL otherwise. */
sca_status sca_set_panel_precision(sca_ctx* ctx, int32_t prec);

/* SM partitions for the two block groups (driver green contexts).  The pivoted group (the
 * lowest frequencies, a chain of short dependent launches) and the dominant group (bandwidth-
 * bound launches that fill every SM they reach) run side by side on one GPU; with a
 * partition, every launch of the dominant group stays on the SMs outside a set of
 * `pivoted_sms` SMs (rounded up by the driver to its granularity, 8 on this GPU), so the
 * pivoted chain never waits for a dominant CTA to leave an SM.  Modes: 1 the pivoted group
 * may still use any SM (highest stream priority), 2 it is confined to its own set as well,
 * 3 as 1, and the dominant group's pivot-block inverses and prep products run on a second
 * partition that leaves twice as many SMs to the pivoted group, its updates on the first (in
 * between the two sizes, which the driver's 8-SM granularity does not offer).
 * pivoted_sms = 0 removes the partition (the dominant group's persistent tensor-core launches
 * then leave 8 SMs free, 32 above N = 2048, and priorities do the rest).  Contexts with 1024 <= N <= 2048 and at
 * least 64 dominant blocks start with a partition when the driver grants it: 16 SMs in mode 1
 * where the dominant blocks' elimination steps are merged in pairs (the tensor-core path), else
 * 8 SMs in mode 3.
 * Needs the
 * tensor-core path; results do not depend on the partition (tile order and reductions are
 * fixed).  SCA_ECUDA when the driver refuses the partition; the context then keeps its
 * ordinary streams.  sca_sm_partition reports the SM counts in use (0, 0 without one). */
typedef enum {
  SCA_PARTITION_DOMINANT = 1,
  SCA_PARTITION_BOTH = 2,
  SCA_PARTITION_ALTERNATE = 3
} sca_partition_mode;
sca_status sca_set_sm_partition(sca_ctx* ctx, int32_t pivoted_sms, int32_t mode);
sca_status sca_sm_partition(sca_ctx* ctx, int32_t* pivoted_sms, int32_t* dominant_sms);

/* Per-kernel timing.  While enabled, every launch of the context is bracketed by CUDA
 * events on the stream it is launched on, and the elapsed times are accumulated per kernel
 * kind when the calling API function synchronises.  Kinds: 0 assemble, 1 pivoted panel,
 * 2 row interchanges, 3 pivot-block inverse of the pivoted group, 4 rank-nb factors,
 * 5 rank-nb update of the dominant blocks (the dominant contraction), 6 refine (adjoint
 * diag(G)), 7 reduce (+Adam), 8 pivot-block inverse of the dominant blocks, 9 rank-nb update
 * of the pivoted group, 10 fused small-block Adam launch, 11 wall span of the pivoted group on
 * its stream, 12 wall span of the dominant group on the main stream (spans contain the
 * kernels above, so they are not part of any sum), 13 update of the rest of a pivoted outer
 * panel after each sub-panel, 14 rank-nb factors of the pivoted group, 15 the first update of a
 * merged pair of elimination steps of the dominant blocks (only the second step's row and column
 * strips; the merged update of the rest is kind 5).  Enabling resets the
 * counters.  Timing adds a small host overhead per launch; keep it off when measuring
 * throughput.  With the environment variable SCA_PROFILE_TRACE set to a file name, each
 * synchronisation also appends the launches it collected to that file, one line each:
 * kind name, stream index (order of first use), start and duration in ms from the first. */
sca_status sca_profile_enable(sca_ctx* ctx, int32_t enable);
sca_status sca_profile_read(sca_ctx* ctx, int32_t kind, double* total_ms, uint64_t* launches);

/* Algorithmic floating-point operations of one gradient evaluation (all blocks, real flops,
 * complex multiply-add = 8): 8 N^3 per block for the Gauss-Jordan inversion. */
double sca_flops_per_grad(const sca_params* params);

/* Number of blocks that need partial pivoting (omega_n <= 4|t|, the lowest frequencies); the
 * remaining blocks are strictly diagonally dominant by columns. */
int32_t sca_pivoted_blocks(const sca_params* params);

/* ------------------------------------------------------------------ misc -- */

/* Message describing the last failure on the calling thread ("" if none). */
const char* sca_last_error(void);

/* Library version string. */
const char* sca_version(void);

/* Number of kernels this process has launched through the library (all
 * contexts and servers).  For launch accounting. */
uint64_t sca_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* SCA_GB300_H */
