// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>

#include "../../include/sca.h"
#include <nvtx3/nvToolsExt.h>

namespace sca {

// NVTX range over a scope (host-side phases: what each API call and pass enqueues); costs a
// call when no tool listens.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

constexpr int kMaxFusedSteps = 16;  // Adam iterations per fused persistent launch

// Identity of the calling thread's current CUDA context: the driver's unique context id
// (cuCtxGetId, fetched at run time so that the library does not link libcuda), 0 when there is
// no current context or the driver lacks the call.
uint64_t current_context_id();

// One-time set-up per CUDA context.  cudaFuncSetAttribute and similar calls act on the current
// context's copy of a kernel: a process that uses several GPUs repeats them on each, and a
// context that is re-created (after cudaDeviceReset) needs them again.  Each device keeps the
// id of the last context it was set up in; setting an attribute twice is harmless, so two
// threads may both run a set-up, and devices past 63 (or an unknown context) are set up on
// every call.
struct ContextOnce {
  std::atomic<uint64_t> ids[64]{};
  static int device() {
    int d = -1;
    return cudaGetDevice(&d) == cudaSuccess ? d : -1;
  }
  bool done() const {
    const int d = device();
    const uint64_t id = current_context_id();
    return d >= 0 && d < 64 && id != 0 && ids[d].load(std::memory_order_acquire) == id;
  }
  // call after the set-up (which makes the device's context current if it was not)
  void mark() {
    const int d = device();
    if (d >= 0 && d < 64) ids[d].store(current_context_id(), std::memory_order_release);
  }
};

// Counts every kernel launched through the library (sca_kernel_launches()).
extern std::atomic<uint64_t> g_launches;

// Thread-local error message plumbing.
void set_error(const std::string& msg);
sca_status cuda_fail(cudaError_t e, const char* where);

// Arguments of one Adam update (PyTorch's order and bias corrections).
struct AdamStep {
  double lr_over_bc1, sqrt_bc2, beta1, beta2, eps, grad_tol;
};

struct BlockDesc;  // per-slot physics (sca_device.cuh)

// One request of a shared pass (size-bucket batching): its device state and blocks.
struct ReqDesc {
  double *phi, *m, *v, *g, *status;  // N, N, N, N, 8
  const int* slots;                  // nblocks workspace slots, in block order
  int nblocks;
  int do_adam;                       // 0: Omega and gradient only
  double U, T;
  AdamStep adam;
};

// Device buffers and sizes of one parameter set.  Blocks are stored planar:
// for block m of a chunk, the real plane is M + m*mat_stride and the
// imaginary plane follows at + plane_stride; rows have `ldm` elements.
struct Engine {
  sca_params p{};
  int L = 0, N = 0, B = 0;
  int nb = 0;            // Gauss-Jordan / LU block width (diagonally dominant blocks)
  int nb_piv = 0;        // block width of the pivoted group (shared-memory panel)
  int nb_piv64 = 0;      // the same for a float64 panel on float32 blocks
  bool panel_fp64 = false;  // the pivoted group's sub-panels compute in float64 (mixed path)
  bool diag_tc = true;   // dominant pivot-block inverses on the tensor cores (nb = 128)
  int piv_planned = 0;   // piv_blocks under partial pivoting
  int piv_blocks = 0;    // blocks b < piv_blocks need partial pivoting (omega_n <= 4|t|)
  int ldm = 0;           // row stride of a block plane (elements)
  int chunk = 0;         // blocks resident at once
  bool fp64 = false;     // storage and arithmetic of the blocks
  bool refine = false;   // FP64 refinement of diag(G)
  bool tc = false;       // tcgen05 split-precision rank-nb update (3xTF32 or BF16x3)
  bool bf16 = false;     // BF16x3: bf16 hi/lo planes on kind::f16 (else TF32 planes)
  double delta_eff = 0;  // Delta or Delta/2 (ionic convention)
  size_t plane_stride = 0, mat_stride = 0;  // elements
  size_t fw_plane = 0, fw_mat = 0;          // F / W panel strides (elements)

  void* M = nullptr;        // chunk blocks
  void* F = nullptr;        // chunk x 2 planes x N x nb (x2 hi/lo for tc)
  void* W = nullptr;        // same, W^T
  // second factor pair of the merged two-step update (symmetric dominant blocks, tensor cores;
  // null when that path is off), laid out as F and W
  void* F2 = nullptr;
  void* W2 = nullptr;
  bool pair = false;        // merged two-step updates for the symmetric dominant blocks
  void* Tinv = nullptr;     // chunk x 2 x nb x nb complex (compute type)
  float* tt = nullptr;      // chunk x 6 x nb x nb: -T^T split planes (tensor-core prep)
  float* adiag = nullptr;   // chunk x N x 2: Re A_jj = mu - eps_j as a double-float pair
  int* piv = nullptr;       // chunk x N
  int* perm = nullptr;      // chunk x N
  int* flags = nullptr;     // 1 int: nonfinite / singular
  double* ld = nullptr;     // B
  double* d_z = nullptr;    // B: (re, im) of the DOS shifts w_k + mu + i eta (n < B/2)
  double* tr = nullptr;     // B: Im Tr G per block (DOS)
  bool nopiv = false;       // SCA_PIVOT_NONE: no block is pivoted
  bool dos_mode = false;    // blocks use the shifts d_z and end in a trace, not a refine
  const BlockDesc* bd = nullptr;  // per-slot physics of a shared pass (or null)
  double* gd = nullptr;     // B x N
  double* eps_extra = nullptr;  // N or null
  double* d_phi = nullptr;  // N (Adam state)
  double* d_m = nullptr;
  double* d_v = nullptr;
  double* d_g = nullptr;
  double* d_status = nullptr;   // 8 doubles
  double* d_omega = nullptr;    // 1 double scratch
  double* h_status = nullptr;   // pinned 8 doubles
  void* tmap = nullptr;         // host-side tensor-map storage (tc path)
  size_t bytes = 0;
  struct Profiler* prof = nullptr;  // per-kernel event timing (sca_profile_enable)
  cudaStream_t side = nullptr;      // stream of the pivoted group (runs beside the rest)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaStream_t aux = nullptr;       // the dominant group's W planes beside its pivot-block inverse
  cudaEvent_t ev_aux0 = nullptr, ev_aux1 = nullptr;
  // SM partitions (green contexts, sca_partition.cu): the dominant group's streams run on
  // part_sms[1] SMs; the pivoted group keeps part_sms[0] SMs to itself (part_side: a stream
  // confined to them, else the ordinary side stream).
  void* green[2] = {nullptr, nullptr};
  cudaStream_t dom = nullptr, part_aux = nullptr, part_side = nullptr;
  cudaEvent_t ev_join2 = nullptr;
  int part_sms[2] = {0, 0};
  // mode 3: a second dominant partition that leaves twice as many SMs free; the dominant
  // group's elimination steps alternate between the two (odd steps on dom_alt / aux_alt)
  void* green_alt = nullptr;
  cudaStream_t dom_alt = nullptr, aux_alt = nullptr;
  cudaEvent_t ev_alt = nullptr;
  int alt_sms = 0;     // SMs of the second dominant partition
  bool alt_on = false; // set while the dominant group runs on its partition streams
  int alt_policy = 2;  // which launches use the second partition (run_group)
  int* tc_counters = nullptr;       // tile counters of the tensor-core launches of one pass
  int tc_next = 0;
  int tc_cap = 0;                   // CTA cap of the next tensor-core launches (0: one per SM)
  int sm_reserve = 0;               // SMs the dominant group leaves to the pivoted group
  int fused_grid = 0;               // CTAs of the fused small-block kernel (0: not eligible)
  size_t fused_smem = 0;
  unsigned* fused_bar = nullptr;    // grid-barrier counter and generation
  long long wait_cycles = 4000000000ll;  // bound of device-side spin waits
  int* h_flags = nullptr;           // pinned copy of the flags word
};

// Float-plane slots per block of the -T^T split planes (re_hi, im_hi, re_lo, im_lo; a bf16
// plane fills the first half of its slot).
constexpr int kTtPlanes = 4;

// Kernel kinds for per-launch timing.
enum KernelKind {
  kAssemble = 0, kPanel, kSwap, kTrinv, kPrep, kUpdate, kRefine, kReduce,
  kDiag,       // inverse of a dominant pivot block (Gauss-Jordan in registers)
  kUpdatePiv,  // rank-nb update of the pivoted group
  kFused,      // fused small-block Adam launch
  kSpanPiv,    // wall span of the pivoted group on its stream (fork to its last kernel)
  kSpanDom,    // wall span of the dominant group on the main stream (fork to its last kernel)
  kPanelUpd,   // pivoted group: update of the rest of the outer panel after a sub-panel
  kPrepPiv,    // pivoted group: rank-nb factors
  kUpdateCross,  // merged two-step update: the first step's update of the second step's strips
  kKinds
};

// Event bracketing of launches while profiling is on (no-ops otherwise).
struct Profiler {
  bool on = false;
  double ms[kKinds] = {};
  uint64_t n[kKinds] = {};
  struct Rec { int kind; cudaEvent_t a, b; cudaStream_t s; };
  Rec* recs = nullptr;
  int nrec = 0, cap = 0;
  cudaEvent_t* pool = nullptr;
  int npool = 0, used = 0;
};
void prof_begin(Engine& e, int kind, cudaStream_t s);
void prof_end(Engine& e, int kind, cudaStream_t s);
// A span that other records may nest in: begin returns its record (-1 when off).
int prof_span_begin(Engine& e, int kind, cudaStream_t s);
void prof_span_end(Engine& e, int rec, cudaStream_t s);
void prof_collect(Engine& e);  // after a synchronisation: accumulate elapsed times
void prof_free(Engine& e);

// Workspace layout / sizing (no allocation).
sca_status plan(const sca_params& p, Engine& e);
sca_status allocate(Engine& e);
void release(Engine& e);

// Enqueue: evaluate every block for field d_phi; on return (asynchronous),
// e.ld[b] holds ln|det A_b| and, if want_grad, e.gd[b*N+i] holds
// sigma_b Re G_{b,ii}.
bool partition_setup(Engine& e, int piv_sms, int mode);  // false: ordinary streams stay
void partition_release(Engine& e);
sca_status run_blocks(Engine& e, const double* d_phi, bool want_grad, cudaStream_t s,
                      bool refine_stage = true);

// Gradient stage alone, from the inverses left resident by run_blocks(..., want_grad=true,
// refine_stage=false) (requires every block resident: chunk == B).
sca_status run_refine_resident(Engine& e, const double* d_phi, cudaStream_t s);

// Enqueue the reduction of ld / gd into Omega (d_omega) and the gradient
// (d_grad, may be null).  With adam != null also the Adam update of e.d_phi
// (step index `step` >= 1).  Writes status[0..7].

sca_status run_reduce(Engine& e, const double* d_phi, double* d_omega, double* d_grad,
                      const AdamStep* adam, cudaStream_t s);

// Assembled blocks (for sca_debug_assemble).
sca_status run_assemble_only(Engine& e, const double* d_phi, int b0, int count, cudaStream_t s);

// Fused persistent Adam kernel for small blocks (sca_fused.cu).
sca_status fused_prepare(Engine& e);
void fused_release(Engine& e);
bool fused_eligible(const Engine& e);
sca_status run_fused_adam(Engine& e, int nsteps, const AdamStep* steps, bool do_adam,
                          cudaStream_t s);

// Seeded start field on the device.
sca_status run_seed_phi(double* d_phi, int N, uint64_t seed, cudaStream_t s);
// One reduction CTA per request of a shared pass (device table rq of nreq entries).
sca_status run_reduce_batch(Engine& e, const ReqDesc* rq, int nreq, cudaStream_t s);
AdamStep adam_step_args(const sca_adam& a, int32_t step);

// tcgen05 3xTF32 rank-nb update (sca_tc.cu).
bool tc_supported();
sca_status tc_prepare(Engine& e);
void tc_release(Engine& e);
sca_status tc_update(Engine& e, int m0, int cnt, int k0, int kb, int r0, int c0, bool gj,
                     cudaStream_t s, int nbk, bool sym = false);
int tc_sms(const Engine& e);  // CTAs of an uncapped tensor-core launch (one per SM)
sca_status tc_reset_counters(Engine& e, cudaStream_t s);  // before each chunk's launches  // tensor-core maps exist for the pivoted group's width
// F = M[:, K] T on the tensor cores into W scratch planes 4, 5 (rows >= r0).
sca_status tc_prep(Engine& e, int m0, int cnt, int r0, cudaStream_t s);
// the pivoted group's prep product (BF16x3): rows [r0, k0+kb) times T, rows below times inv(L)
// Pivot-block inverse of dominant blocks on the tensor cores (nb = 128, float32 blocks): the
// outputs of the register Gauss-Jordan kernel (T, -T^T split planes, ld += ln|det|).
sca_status tc_diag(const float* M, int ldm, size_t mat_stride, size_t plane_stride, int cnt, int k0,
                   int kb, int nb, int b0, double* ld, void* Tinv, float* TT, int tt_bf16,
                   int* flags, cudaStream_t s);
sca_status tc_prep_piv(Engine& e, int m0, int cnt, int r0, int k0, int kb, bool gj,
                       cudaStream_t s);
// Prep product of the symmetric dominant blocks: F = S (W^T T) written as the four TF32
// planes of F, with S = -1 on the swept rows (< k0) and the rows of K replaced by -T.
sca_status tc_prep_split(Engine& e, int m0, int cnt, int r0, int k0, int kb, bool gj,
                         cudaStream_t s, bool second = false);
// Two adjacent Gauss-Jordan steps K1 = [k1, k1 + kb1), K2 = [k2, k2 + kb2) of the symmetric
// dominant blocks: merge 1 updates only the cross of K2 with F1 W1; merge 2 updates every other
// lower tile with F1 W1 + F2 W2 (the K1 mask) and the cross of K2 with F2 W2 (the K2 mask).
sca_status tc_update_pair(Engine& e, int m0, int cnt, int k1, int kb1, int k2, int kb2, int merge,
                          cudaStream_t s);


// ----------------------------------------------------------- size buckets
// One request served through a size bucket: its parameters, Adam settings and device state
// (phi | m | v | g, N doubles each, then 8 status doubles as in the single-request path).
struct BucketReq {
  sca_params p{};
  sca_adam a{};
  int32_t step = 0;
  int nb = 0, npiv = 0;
  double delta_eff = 0.0;
  double* d = nullptr;
};
struct Bucket;
bool bucketed(const sca_params& p);               // served through a size bucket
sca_params bucket_shape(int32_t L, int32_t prec, int cap);
sca_status bucket_create(int32_t L, int32_t prec, int cap, Bucket** out);
void bucket_destroy(Bucket* b);
cudaStream_t bucket_stream(Bucket* b);
sca_status bucket_req_init(Bucket* b, BucketReq* r, const sca_params& p, const sca_adam& a);
void bucket_req_release(BucketReq* r);
// nsteps gated Adam steps (adam) or one evaluation without update (!adam) for n requests.
sca_status bucket_run(Bucket* b, BucketReq* const* reqs, int n, int nsteps, bool adam);
sca_status bucket_status(Bucket* b, BucketReq* const* reqs, int n, double* out);
sca_status bucket_get_phi(Bucket* b, const BucketReq* r, double* out);
}  // namespace sca

struct sca_ctx {
  sca::Engine e;
  cudaStream_t own = nullptr;     // the context's stream
  cudaStream_t stream = nullptr;  // stream in use (own or the caller's, sca_set_stream)
  double* d_in = nullptr;         // N doubles: host-supplied phi
  sca_adam adam{};
  bool adam_ready = false;
  int32_t step = 0;
  bool kept = false;              // inverses of every block resident from sca_forward_dev
  const double* kept_phi = nullptr;
  // Metropolis chain (sca_metropolis_*): the state is e.d_phi
  double* d_prop = nullptr;       // N: proposal
  double* d_metro = nullptr;      // 4: Omega of the state, accepted, last proposal, non-finite
  double* d_mtrace = nullptr;     // 2 x capacity: per-step Omega and accept flag
  int32_t mtrace_cap = 0;
  double m_delta = 0.0;
  uint64_t m_seed = 0;
  int64_t m_step = 0;             // global step number of the next proposal
  bool metro_ready = false;
};

namespace sca {
sca_status sync_status(sca_ctx* c, cudaStream_t s);  // status -> pinned host, synchronise
sca_status check_finite(sca_ctx* c);                 // status -> SCA_ENONFINITE / ETIMEOUT
sca_status enqueue_adam(sca_ctx* c, int32_t n);      // n gated Adam iterations, no sync
sca_status final_eval(sca_ctx* c);                   // Omega, max|g| at phi (synchronised)
sca_status run_adam_gated(sca_ctx* c, int32_t max_steps, int32_t* applied);  // sca_adam_run
}  // namespace sca
