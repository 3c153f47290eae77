// tcgen05 (5th-generation tensor core) rank-nb update of the Gauss-Jordan / LU sweep on
// sm_103a, in split TF32 ("3xTF32") with float32 accumulation:
//
//   M[i, j] <- mask(i, j) M[i, j] - sum_c F[i, c] W[j, c]          (complex, planar)
//
// Complex product in real MMAs: for a 128-row tile of F and a 128-column tile of W, the
// 128 x 256 real tile [C_re | C_im] is
//   F_re [W_re | W_im] + F_im [-W_im | W_re]:
// the first term is one MMA of width 256 with the 256-row stack (W_re; W_im) as B (the two
// planes sit next to each other in shared memory), the second two MMAs of width 128 into the
// two halves of the accumulator, the one with W_im issued with A negated (instruction
// descriptor bit 13), so no negated copy of W_im is stored or loaded.  Each real product is
// split as hi*hi + hi*lo + lo*hi with hi = the value truncated to TF32 (or rounded to bf16)
// and lo = value - hi (written by the prep kernels): 9 MMAs per K step (3 of N = 256, 6 of
// N = 128), the tensor work of 6 at N = 256.
//
// Kernel structure (persistent, one CTA per SM, 192 threads):
//   warp 0  : TMA producer (cp.async.bulk.tensor, 2-stage shared-memory ring, K = 16 per stage)
//   warp 1  : TMEM allocator and MMA issuer (tcgen05.mma, one elected thread)
//   warps 2-5: epilogue (tcgen05.ld of the accumulator, read-modify-write of M in HBM)
// Accumulators are double buffered in TMEM (2 x 256 columns) so the epilogue of one tile
// overlaps the MMAs of the next.  Every mbarrier wait is bounded; on time-out the kernel
// records an error, stops issuing work, waits (bounded) for its own copies, frees TMEM and
// returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <string>

#include <cuda_bf16.h>

#include "sca_internal.h"

namespace sca {
namespace {

}  // namespace
constexpr int kCounters = 1024;    // tile counters per pass (one per tensor-core launch)
namespace {
constexpr int kBM = 128;           // F rows per tile
constexpr int kBNc = 128;          // complex W columns per tile (real MMA N = 256)
constexpr int kKS = 16;            // K per pipeline stage (SWIZZLE_64B rows of 64 bytes)
constexpr int kStages = 2;
constexpr int kTileBytes = kBM * kKS * 4;             // one 128 x 16 float plane: 8 KB
constexpr int kStageBytes = 8 * kTileBytes;           // 4 F planes + 4 W planes: 64 KB
constexpr int kEpiCols = 32;                          // complex columns per epilogue chunk
constexpr int kEpiPlaneBytes = kBM * kEpiCols * 4;     // 128 x 32 floats, 16 KB
constexpr int kEpiBufBytes = 2 * kEpiPlaneBytes;       // re + im planes
constexpr int kEpiBufs = 2;
constexpr int kRing = 4;                               // tile-id ring (producer -> MMA, epilogue)
constexpr int kSmemBytes = kStages * kStageBytes + kEpiBufs * kEpiBufBytes + 1024 + 256;
constexpr int kThreads = 192;
constexpr uint32_t kTmemCols = 512;                   // 2 accumulators x 256 columns
constexpr long long kWaitCycles = 4000000000ll;       // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: returns false (and raises the CTA's abort flag) if the phase does not
// complete within kWaitCycles, or if another role already aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (mbar_try(bar, parity)) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > kWaitCycles) {
      *abort_flag = 1;
      return false;
    }
  }
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x,
                                            int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, const void* src, int x, int y,
                                             int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(x), "r"(y), "r"(z), "r"(smem_u32(src))
      : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
// Barrier over the 128 epilogue threads that also ANDs a predicate: every thread leaves with
// the same decision, so no thread can be left waiting at the next named barrier.
__device__ __forceinline__ bool epi_all(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "barrier.red.and.pred q, 1, 128, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)(v ? 1 : 0))
      : "memory");
  return r != 0;
}

// Shared-memory matrix descriptor (tcgen05), K-major operand with 64-byte swizzle:
// rows of 64 bytes, 8-row core groups 512 bytes apart (stride byte offset), leading byte
// offset unused for swizzled K-major layouts, descriptor version 1, layout code 4 (64B).
__device__ __forceinline__ uint64_t sdesc_k64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;                 // leading byte offset (16 B, unused)
  d |= (uint64_t)(512 >> 4) << 32;        // stride byte offset
  d |= (uint64_t)1 << 46;                 // descriptor version
  d |= (uint64_t)4 << 61;                 // SWIZZLE_64B
  return d;
}

// Instruction descriptor of tcgen05.mma kind::f16 (A = B = bf16) or kind::tf32 (A = B = tf32):
// D = f32, both operands K-major, M = 128, N = 256 or 128, A optionally negated (bit 13; the
// imaginary-part products of the complex update).
template <bool BF, bool N256, bool NEGA>
__host__ __device__ constexpr uint32_t idesc() {
  return (1u << 4) | ((BF ? 1u : 2u) << 7) | ((BF ? 1u : 2u) << 10) | (NEGA ? (1u << 13) : 0u) |
         (((N256 ? 256u : 128u) >> 3) << 17) | ((128u >> 4) << 24);
}
template <bool BF>
__device__ __forceinline__ void mma_d(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id,
                                      uint32_t acc) {
  if constexpr (BF)
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(id), "r"(acc));
  else
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

struct TcArgs {
  float* M;
  int N, ldm;
  long long mat_stride, plane_stride;  // floats
  int nb;                              // K extent (multiple of 16)
  int r0, c0;                          // first updated row / column
  int k0, kb, gj;                      // masked block K (Gauss-Jordan)
  int tiles_m, tiles_n, tiles;         // per block, and total
  int fplanes, wplanes;                // planes per block in the F / W tensor maps
  int mat0;                            // workspace slot of the first block
  int m_zmul, m_zoff;                  // output map plane index: (mat0+mat)*m_zmul + m_zoff + p
  int* counter;                        // tile counter (zero before the launch)
  int sym;                             // lower-triangle tiles only (tiles_m == tiles_n)
  int per_block;                       // tiles per block
  int* err;                            // device error word (bit 1: wait time-out)
  // Split output (the prep product of the symmetric dominant blocks): no accumulation into
  // the output, v = (A B) row-signed (-1 for rows < k0 when split_neg), rows in K replaced by
  // -T (Gauss-Jordan), stored as the four TF32 planes re_hi, im_hi, re_lo, im_lo.
  int split_out, split_neg;
  const float2* T;                     // pivot-block inverses, (mat0+mat) * t_mat + r * nb + j
  long long t_mat;
};

// Tile t -> (block, tile row, tile column).  With `sym` only tiles on or below the diagonal
// exist (the dominant blocks stay symmetric up to sign, see the host code): rem ->
// (i, j) with rem = i (i + 1) / 2 + j, j <= i.
__device__ __forceinline__ void decode_tile(const TcArgs& a, int t, int& mat, int& tm, int& tn) {
  mat = t / a.per_block;
  const int rem = t - mat * a.per_block;
  if (!a.sym) {
    tm = rem / a.tiles_n;
    tn = rem - tm * a.tiles_n;
    return;
  }
  int i = (int)((sqrtf(8.0f * (float)rem + 1.0f) - 1.0f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= rem) ++i;
  while (i * (i + 1) / 2 > rem) --i;
  tm = i;
  tn = rem - i * (i + 1) / 2;
}

// Shared-memory stage layout (each slot one 128-row plane of 64-byte K rows, 8 KB,
// 1024-aligned):
//   0 F_re_hi  1 F_im_hi  2 F_re_lo  3 F_im_lo  4 W_re_hi  5 W_im_hi  6 W_re_lo  7 W_im_lo
// Global planes: F and W {0 re_hi, 1 im_hi, 2 re_lo, 3 im_lo}.
__constant__ int kFPlaneOfSlot[4] = {0, 1, 2, 3};
__constant__ int kWPlaneOfSlot[4] = {0, 1, 2, 3};  // re_hi, im_hi, re_lo, im_lo

// BF: the operand planes are bf16 (BF16x3 on kind::f16, 32 K-elements per 64-byte stage row)
// instead of TF32-split float32 (16 per row); the stage layout in bytes is the same.
template <bool BF>
__global__ void __launch_bounds__(kThreads, 1)
    k_update_tc(const __grid_constant__ CUtensorMap tmF, const __grid_constant__ CUtensorMap tmW,
                const __grid_constant__ CUtensorMap tmM, TcArgs a) {
  constexpr int kKE = BF ? 32 : kKS;  // K elements per stage
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* epi = smem + kStages * kStageBytes;  // kEpiBufs x (re, im) staging, 128B swizzle
  uint64_t* bars = reinterpret_cast<uint64_t*>(epi + kEpiBufs * kEpiBufBytes);
  uint64_t* full = bars;                 // [kStages]
  uint64_t* empty = bars + kStages;      // [kStages]
  uint64_t* tfull = bars + 2 * kStages;  // [2]
  uint64_t* tempty = tfull + 2;          // [2]
  uint64_t* mdone = tempty + 2;          // [1] all MMAs of this CTA completed
  uint64_t* efull = mdone + 1;           // [kEpiBufs] staging tile of M landed
  uint64_t* rfull = efull + kEpiBufs;    // [kRing] tile id published
  uint64_t* rempty = rfull + kRing;      // [kRing] tile id read by the MMA thread and 4 warps
  int* ring = reinterpret_cast<int*>(rempty + kRing);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(ring + kRing);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&tfull[b], 1); mbar_init(&tempty[b], 4); }
    mbar_init(mdone, 1);
    for (int b = 0; b < kEpiBufs; ++b) mbar_init(&efull[b], 1);
    for (int r = 0; r < kRing; ++r) { mbar_init(&rfull[r], 1); mbar_init(&rempty[r], 5); }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const int ksteps = a.nb / kKE;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int last_parity[kStages];
      for (int s = 0; s < kStages; ++s) last_parity[s] = -1;
      int rslot = 0;
      uint32_t rphase = 0;
      while (true) {
        // claim the next tile and publish it to the MMA thread and the epilogue
        int t = *abort_flag ? -1 : atomicAdd(a.counter, 1);
        if (t >= a.tiles) t = -1;
        if (!mbar_wait(&rempty[rslot], rphase ^ 1, abort_flag)) break;
        ring[rslot] = t;
        mbar_arrive(&rfull[rslot]);
        if (++rslot == kRing) { rslot = 0; rphase ^= 1; }
        if (t < 0) break;
        int mat, tm, tn;
        decode_tile(a, t, mat, tm, tn);
        const int frow = a.r0 + tm * kBM, wrow = a.c0 + tn * kBNc;
        for (int ks = 0; ks < ksteps; ++ks) {
          if (!mbar_wait(&empty[stage], phase ^ 1, abort_flag)) break;
          mbar_expect_tx(&full[stage], kStageBytes);
          unsigned char* st = smem + stage * kStageBytes;
          for (int s = 0; s < 4; ++s)
            tma_load_3d(st + s * kTileBytes, &tmF, &full[stage], ks * kKE, frow,
                        (a.mat0 + mat) * a.fplanes + kFPlaneOfSlot[s]);
          for (int s = 0; s < 4; ++s)
            tma_load_3d(st + (4 + s) * kTileBytes, &tmW, &full[stage], ks * kKE, wrow,
                        (a.mat0 + mat) * a.wplanes + kWPlaneOfSlot[s]);
          last_parity[stage] = (int)phase;
          if (++stage == kStages) { stage = 0; phase ^= 1; }
        }
      }
      // Drain: every copy issued must have landed before the CTA leaves (bounded wait; after
      // a normal run these phases have long completed and the waits return at once).
      volatile int drain_abort = 0;
      for (int s = 0; s < kStages; ++s)
        if (last_parity[s] >= 0) (void)mbar_wait(&full[s], (uint32_t)last_parity[s], &drain_abort);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int rslot = 0;
      uint32_t rphase = 0;
      for (int iter = 0;; ++iter) {
        if (!mbar_wait(&rfull[rslot], rphase, abort_flag)) break;
        const int t = ring[rslot];
        mbar_arrive(&rempty[rslot]);
        if (++rslot == kRing) { rslot = 0; rphase ^= 1; }
        if (t < 0) break;
        const int buf = iter & 1;
        const uint32_t use = (uint32_t)(iter >> 1);  // times this buffer was used before
        if (!mbar_wait(&tempty[buf], (use & 1) ^ 1, abort_flag)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(buf * 256);
        bool ok = true;
        for (int ks = 0; ks < ksteps; ++ks) {
          if (!mbar_wait(&full[stage], phase, abort_flag)) { ok = false; break; }
          tc_fence_after();
          const uint32_t st = smem_u32(smem + stage * kStageBytes);
#pragma unroll
          for (int k8 = 0; k8 < 2; ++k8) {
            const uint32_t off = (uint32_t)(k8 * 32);
            const uint64_t fr_hi = sdesc_k64(st + 0 * kTileBytes + off);
            const uint64_t fi_hi = sdesc_k64(st + 1 * kTileBytes + off);
            const uint64_t fr_lo = sdesc_k64(st + 2 * kTileBytes + off);
            const uint64_t fi_lo = sdesc_k64(st + 3 * kTileBytes + off);
            // B slots: W_re_hi, W_im_hi, W_re_lo, W_im_lo; (W_re; W_im) is one 256-row operand
            const uint64_t bre_hi = sdesc_k64(st + 4 * kTileBytes + off);
            const uint64_t bim_hi = sdesc_k64(st + 5 * kTileBytes + off);
            const uint64_t bre_lo = sdesc_k64(st + 6 * kTileBytes + off);
            const uint64_t bim_lo = sdesc_k64(st + 7 * kTileBytes + off);
            constexpr uint32_t kI256 = idesc<BF, true, false>();
            constexpr uint32_t kI128 = idesc<BF, false, false>();
            constexpr uint32_t kI128n = idesc<BF, false, true>();
            const uint32_t d_im = d_tmem + (uint32_t)kBNc;  // imaginary half of the accumulator
            const uint32_t acc0 = (ks > 0 || k8 > 0) ? 1u : 0u;
            // (re | im) += F_re (W_re; W_im)
            mma_d<BF>(d_tmem, fr_hi, bre_hi, kI256, acc0);
            mma_d<BF>(d_tmem, fr_hi, bre_lo, kI256, 1u);
            mma_d<BF>(d_tmem, fr_lo, bre_hi, kI256, 1u);
            // re += (-F_im) W_im, im += F_im W_re
            mma_d<BF>(d_tmem, fi_hi, bim_hi, kI128n, 1u);
            mma_d<BF>(d_im, fi_hi, bre_hi, kI128, 1u);
            mma_d<BF>(d_tmem, fi_hi, bim_lo, kI128n, 1u);
            mma_d<BF>(d_im, fi_hi, bre_lo, kI128, 1u);
            mma_d<BF>(d_tmem, fi_lo, bim_hi, kI128n, 1u);
            mma_d<BF>(d_im, fi_lo, bre_hi, kI128, 1u);
          }
          mma_commit(&empty[stage]);  // frees the stage once these MMAs have read it
          if (++stage == kStages) { stage = 0; phase ^= 1; }
        }
        if (!ok) break;
        mma_commit(&tfull[buf]);
      }
      // All MMAs issued by this thread complete before TMEM is released.
      mma_commit(mdone);
      volatile int drain_abort = 0;
      (void)mbar_wait(mdone, 0, &drain_abort);
    }
  } else {
    // ------------------------------------------------------------ epilogue (warps 2..5)
    // M is streamed through shared memory in 128 x 32 complex chunks: one thread issues the
    // TMA load of the next chunk while all 128 threads update the current one (thread = row,
    // 128-byte swizzled rows, conflict-free 16-byte accesses), then TMA stores it back.
    const int q = warp & 3;              // TMEM lane quarter this warp may access
    const int row = q * 32 + lane;       // row of the tile owned by this thread
    const bool leader = (warp == 2 && lane == 0);
    const int nchunk = kBNc / kEpiCols;
    int iter = 0;
    uint32_t eph[kEpiBufs] = {0, 0};
    bool pending[kEpiBufs] = {false, false};  // leader: load issued, not yet consumed
    int ebuf = 0;
    bool ok = true;
    // issue the load of chunk c of tile t into staging buffer eb
    auto issue_load = [&](int t, int c, int eb) {
      int mat, tm, tn;
      decode_tile(a, t, mat, tm, tn);
      const int x = a.c0 + tn * kBNc + c * kEpiCols, y = a.r0 + tm * kBM;
      bulk_wait_read0();  // the store that last read this buffer has finished reading it
      pending[eb] = true;
      mbar_expect_tx(&efull[eb], kEpiBufBytes);
      unsigned char* st = epi + eb * kEpiBufBytes;
      const int zb = (a.mat0 + mat) * a.m_zmul + a.m_zoff;
      tma_load_3d(st, &tmM, &efull[eb], x, y, zb);
      tma_load_3d(st + kEpiPlaneBytes, &tmM, &efull[eb], x, y, zb + 1);
    };
    int rslot = 0;
    uint32_t rphase = 0;
    int prefetched = -1;  // tile whose chunk 0 is already loading into staging buffer ebuf
    while (ok) {
      if (!epi_all(mbar_wait(&rfull[rslot], rphase, abort_flag))) { ok = false; break; }
      const int t = ring[rslot];
      __syncwarp();
      if (lane == 0) mbar_arrive(&rempty[rslot]);
      if (++rslot == kRing) { rslot = 0; rphase ^= 1; }
      if (t < 0) break;
      if (leader && !a.split_out && prefetched != t) issue_load(t, 0, ebuf);
      const int buf = iter & 1;
      const uint32_t use = (uint32_t)(iter >> 1);
      int mat, tm, tn;
      decode_tile(a, t, mat, tm, tn);
      const int i = a.r0 + tm * kBM + row;
      const int j0 = a.c0 + tn * kBNc;
      const bool rowk = a.gj && i >= a.k0 && i < a.k0 + a.kb;
      if (!epi_all(mbar_wait(&tfull[buf], use & 1, abort_flag))) { ok = false; break; }
      tc_fence_after();
      const uint32_t tbase = tmem_base + (uint32_t)(buf * 256) + ((uint32_t)(q * 32) << 16);
#pragma unroll 1
      for (int c = 0; c < nchunk; ++c) {
        if (a.split_out) {
          uint32_t cr[32], ci[32];
          tmem_ld32(tbase + (uint32_t)(c * kEpiCols), cr);
          tmem_ld32(tbase + (uint32_t)(kBNc + c * kEpiCols), ci);
          tmem_ld_wait();
          if (leader) bulk_wait_read0();  // the previous chunk's stores have read the staging
          epi_bar();
          const int jc = j0 + c * kEpiCols;
          const bool neg = a.split_neg && i < a.k0;
          const float2* trow =
              rowk ? a.T + (size_t)(a.mat0 + mat) * a.t_mat + (size_t)(i - a.k0) * a.nb : nullptr;
          unsigned char* s0 = epi;
          unsigned char* s1 = epi + kEpiBufBytes;
          if constexpr (BF) {
            // four bf16 planes of 128 rows x 64 bytes (8 KB each) in buffer 0, 64-byte swizzle:
            // 16-byte unit u of row r sits at unit u ^ ((r >> 1) & 3)
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int off = row * 64 + ((u ^ ((row >> 1) & 3)) << 4);
              __nv_bfloat16 h[4][8];
#pragma unroll
              for (int e = 0; e < 8; ++e) {
                const int j = jc + 8 * u + e;
                float vr, vi;
                if (rowk) {
                  const float2 tv = (j < a.kb) ? trow[j] : make_float2(0.f, 0.f);
                  vr = -tv.x;
                  vi = -tv.y;
                } else {
                  vr = -__uint_as_float(cr[8 * u + e]);
                  vi = -__uint_as_float(ci[8 * u + e]);
                  if (neg) { vr = -vr; vi = -vi; }
                }
                h[0][e] = __float2bfloat16_rn(vr);
                h[1][e] = __float2bfloat16_rn(vi);
                h[2][e] = __float2bfloat16_rn(vr - __bfloat162float(h[0][e]));
                h[3][e] = __float2bfloat16_rn(vi - __bfloat162float(h[1][e]));
              }
#pragma unroll
              for (int pl = 0; pl < 4; ++pl)
                *reinterpret_cast<uint4*>(s0 + pl * (kBM * 64) + off) =
                    *reinterpret_cast<const uint4*>(h[pl]);
            }
            fence_proxy_async();
            epi_bar();
            if (leader) {
              const int y = a.r0 + tm * kBM;
              const int zb = (a.mat0 + mat) * a.m_zmul + a.m_zoff;
#pragma unroll
              for (int pl = 0; pl < 4; ++pl) tma_store_3d(&tmM, s0 + pl * (kBM * 64), jc, y, zb + pl);
              bulk_commit();
            }
            continue;
          }
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const int off = row * 128 + ((k ^ (row & 7)) << 4);
            float vr[4], vi[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int j = jc + 4 * k + e;
              if (rowk) {
                const float2 tv = (j < a.kb) ? trow[j] : make_float2(0.f, 0.f);
                vr[e] = -tv.x;
                vi[e] = -tv.y;
              } else {
                vr[e] = -__uint_as_float(cr[4 * k + e]);
                vi[e] = -__uint_as_float(ci[4 * k + e]);
                if (neg) { vr[e] = -vr[e]; vi[e] = -vi[e]; }
              }
            }
            float4 rh, ih, rl, il;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float hr = __uint_as_float(__float_as_uint(vr[e]) & 0xffffe000u);
              const float hi = __uint_as_float(__float_as_uint(vi[e]) & 0xffffe000u);
              (&rh.x)[e] = hr; (&ih.x)[e] = hi; (&rl.x)[e] = vr[e] - hr; (&il.x)[e] = vi[e] - hi;
            }
            *reinterpret_cast<float4*>(s0 + off) = rh;
            *reinterpret_cast<float4*>(s0 + kEpiPlaneBytes + off) = ih;
            *reinterpret_cast<float4*>(s1 + off) = rl;
            *reinterpret_cast<float4*>(s1 + kEpiPlaneBytes + off) = il;
          }
          fence_proxy_async();
          epi_bar();
          if (leader) {
            const int y = a.r0 + tm * kBM;
            const int zb = (a.mat0 + mat) * a.m_zmul + a.m_zoff;
            tma_store_3d(&tmM, s0, jc, y, zb);
            tma_store_3d(&tmM, s0 + kEpiPlaneBytes, jc, y, zb + 1);
            tma_store_3d(&tmM, s1, jc, y, zb + 2);
            tma_store_3d(&tmM, s1 + kEpiPlaneBytes, jc, y, zb + 3);
            bulk_commit();
          }
          continue;
        }
        const int eb = ebuf;
        // prefetch the next chunk (of this tile, or the first of the next tile)
        if (leader) {
          if (c + 1 < nchunk) {
            issue_load(t, c + 1, eb ^ 1);
          } else {
            // the next tile's first chunk, if the producer has already published it
            prefetched = -1;
            if (mbar_try(&rfull[rslot], rphase)) {
              const int t2 = ring[rslot];
              if (t2 >= 0) { issue_load(t2, 0, eb ^ 1); prefetched = t2; }
            }
          }
        }
        uint32_t cr[32], ci[32];
        tmem_ld32(tbase + (uint32_t)(c * kEpiCols), cr);
        tmem_ld32(tbase + (uint32_t)(kBNc + c * kEpiCols), ci);
        tmem_ld_wait();
        if (!epi_all(mbar_wait(&efull[eb], eph[eb], abort_flag))) { ok = false; break; }
        pending[eb] = false;
        eph[eb] ^= 1;
        unsigned char* st = epi + eb * kEpiBufBytes;
        const int jc = j0 + c * kEpiCols;
        const bool colk = a.gj && (jc < a.k0 + a.kb) && (jc + kEpiCols > a.k0);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int off = row * 128 + ((k ^ (row & 7)) << 4);
          float4* pr = reinterpret_cast<float4*>(st + off);
          float4* pi = reinterpret_cast<float4*>(st + kEpiPlaneBytes + off);
          float4 vr = *pr, vi = *pi;
          if (rowk || colk) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int j = jc + 4 * k + e;
              const bool keep = !(rowk || (j >= a.k0 && j < a.k0 + a.kb));
              if (!keep) { (&vr.x)[e] = 0.f; (&vi.x)[e] = 0.f; }
            }
          }
          vr.x -= __uint_as_float(cr[4 * k + 0]); vr.y -= __uint_as_float(cr[4 * k + 1]);
          vr.z -= __uint_as_float(cr[4 * k + 2]); vr.w -= __uint_as_float(cr[4 * k + 3]);
          vi.x -= __uint_as_float(ci[4 * k + 0]); vi.y -= __uint_as_float(ci[4 * k + 1]);
          vi.z -= __uint_as_float(ci[4 * k + 2]); vi.w -= __uint_as_float(ci[4 * k + 3]);
          *pr = vr;
          *pi = vi;
        }
        fence_proxy_async();
        epi_bar();
        if (leader) {
          const int y = a.r0 + tm * kBM;
          const int zb = (a.mat0 + mat) * a.m_zmul + a.m_zoff;
          tma_store_3d(&tmM, st, jc, y, zb);
          tma_store_3d(&tmM, st + kEpiPlaneBytes, jc, y, zb + 1);
          bulk_commit();
        }
        ebuf ^= 1;
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[buf]);
      ++iter;
    }
    if (leader) {
      bulk_wait_all();  // every store of this CTA has completed
      // loads issued but not consumed (only after an abort): wait, bounded, until they land
      volatile int drain_abort = 0;
      for (int b2 = 0; b2 < kEpiBufs; ++b2)
        if (pending[b2]) (void)mbar_wait(&efull[b2], eph[b2], &drain_abort);
    }
  }
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) atomicOr(a.err, 2);
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(kTmemCols)
                 : "memory");
  }
}

// ----------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    (void)cudaGetLastError();
  }
  return fn;
}

struct TcMaps {
  CUtensorMap F, W;    // rank-nb factors, K extent nb
  CUtensorMap M;       // the blocks, for the epilogue
  CUtensorMap TT;      // -T^T split planes (nb x nb per block): B of F = M[:, K] T
  CUtensorMap TL;      // -inv(L)^T bf16 planes of the pivoted group (second halves of TT's)
  CUtensorMap FP;      // planar F = M[:, K] T (W scratch planes 4, 5): output of that product
  CUtensorMap FO;      // the F planes themselves: split output of the symmetric prep product
  int sms = 0;
};

// 3-D map over [blocks*planes][N rows][nbk] elements, box (64 bytes of K) x 128 x 1, 64-byte
// swizzle: float32 planes (16 K-elements per box row) or bf16 planes (32), a bf16 plane
// starting where the float32 plane would (plane stride N nbk x 4 bytes either way).
bool make_fw_map(CUtensorMap* m, void* base, int nbk, int N, long long zdim, bool bf16 = false) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t es_bytes = bf16 ? 2 : 4;
  cuuint64_t dims[3] = {(cuuint64_t)nbk, (cuuint64_t)N, (cuuint64_t)zdim};
  cuuint64_t strides[2] = {(cuuint64_t)nbk * es_bytes, (cuuint64_t)N * nbk * 4};
  cuuint32_t box[3] = {(cuuint32_t)(bf16 ? 32 : kKS), (cuuint32_t)kBM, 1};
  cuuint32_t es[3] = {1, 1, 1};
  return fn(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base,
            dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 3-D map over [z][rows][cols] floats (row stride ld), box 32 x 128 x 1, 128-byte swizzle: the
// epilogue's staging tile.
// bf16: the same rows of bf16 elements (64-byte staging rows, 64-byte swizzle); zstride counts
// float32 elements either way.
bool make_m_map_rows(CUtensorMap* m, void* base, int cols, int rows, int ld, long long zstride,
                     long long z, bool bf16 = false) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)z};
  cuuint64_t strides[2] = {(cuuint64_t)ld * (bf16 ? 2 : 4), (cuuint64_t)zstride * 4};
  cuuint32_t box[3] = {(cuuint32_t)kEpiCols, (cuuint32_t)kBM, 1};
  cuuint32_t es[3] = {1, 1, 1};
  return fn(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base,
            dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            bf16 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The block planes [blocks*2][N rows][N cols] (row stride ldm).
bool make_m_map(CUtensorMap* m, void* base, int N, int ldm, long long plane_stride, long long z) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)N, (cuuint64_t)N, (cuuint64_t)z};
  cuuint64_t strides[2] = {(cuuint64_t)ldm * 4, (cuuint64_t)plane_stride * 4};
  cuuint32_t box[3] = {(cuuint32_t)kEpiCols, (cuuint32_t)kBM, 1};
  cuuint32_t es[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

sca_status tc_reset_counters(Engine& e, cudaStream_t s) {
  e.tc_next = 0;
  if (!e.tc_counters) return SCA_OK;
  cudaError_t err = cudaMemsetAsync(e.tc_counters, 0, kCounters * sizeof(int), s);
  if (err != cudaSuccess) return cuda_fail(err, "tile counters");
  return SCA_OK;
}

bool tc_supported() {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { (void)cudaGetLastError(); return false; }
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return major == 10 && minor == 3 && encode_fn() != nullptr;
}

sca_status tc_prepare(Engine& e) {
  if (e.nb % kKS != 0) {
    set_error("tcgen05 update needs nb to be a multiple of 16");
    return SCA_EINVAL;
  }
  TcMaps* t = new TcMaps();
  std::memset(&t->F, 0, sizeof(t->F));
  std::memset(&t->W, 0, sizeof(t->W));
  std::memset(&t->M, 0, sizeof(t->M));
  const long long zf = (long long)e.chunk * (long long)(e.fw_mat / e.fw_plane);
  if (!make_fw_map(&t->F, e.F, e.nb, e.N, zf, e.bf16) ||
      !make_fw_map(&t->W, e.W, e.nb, e.N, zf, e.bf16) ||
      !make_m_map(&t->M, e.M, e.N, e.ldm, (long long)e.plane_stride, 2ll * e.chunk)) {
    delete t;
    set_error("cuTensorMapEncodeTiled failed for the tensor-core update");
    return SCA_ECUDA;
  }
  {
    // F = M[:, K] T on the tensor cores: A = split pivot columns (W scratch planes 0-3, same
    // map as W), B = -T^T planes, output planar into W scratch planes 4, 5.
    const long long ztt = (long long)e.chunk * kTtPlanes;
    // bf16 planes fill half of a float plane slot: the pivoted group's -inv(L)^T planes sit
    // in the second halves
    float* tl = e.tt ? e.tt + (size_t)e.nb * e.nb / 2 : nullptr;
    bool ok = !e.tt ||
              (make_fw_map(&t->TT, e.tt, e.nb, e.nb, ztt, e.bf16) &&
               (!e.bf16 || make_fw_map(&t->TL, tl, e.nb, e.nb, ztt, true)) &&
               make_m_map_rows(&t->FP, e.W, e.nb, e.N, e.nb, (long long)e.fw_plane, zf) &&
               make_m_map_rows(&t->FO, e.F, e.nb, e.N, e.nb, (long long)e.fw_plane, zf, e.bf16));
    if (!ok) {
      delete t;
      set_error("cuTensorMapEncodeTiled failed for the tensor-core prep product");
      return SCA_ECUDA;
    }
  }
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err == cudaSuccess) err = cudaDeviceGetAttribute(&t->sms, cudaDevAttrMultiProcessorCount, dev);
  if (err == cudaSuccess)
    err = cudaFuncSetAttribute(k_update_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               kSmemBytes);
  if (err == cudaSuccess)
    err = cudaFuncSetAttribute(k_update_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               kSmemBytes);
  if (err != cudaSuccess) {
    delete t;
    return cuda_fail(err, "tcgen05 update set-up");
  }
  err = cudaMalloc((void**)&e.tc_counters, kCounters * sizeof(int));
  if (err == cudaSuccess) err = cudaMemset(e.tc_counters, 0, kCounters * sizeof(int));
  if (err != cudaSuccess) {
    delete t;
    return cuda_fail(err, "tile counters");
  }
  e.tmap = t;
  return SCA_OK;
}

int tc_sms(const Engine& e) {
  const TcMaps* t = static_cast<const TcMaps*>(e.tmap);
  return t ? t->sms : 0;
}

void tc_release(Engine& e) {
  if (e.tc_counters) cudaFree(e.tc_counters);
  e.tc_counters = nullptr;
  TcMaps* t = static_cast<TcMaps*>(e.tmap);
  if (!t) return;
  delete t;
  e.tmap = nullptr;
}

sca_status tc_update(Engine& e, int m0, int cnt, int k0, int kb, int r0, int c0, bool gj,
                     cudaStream_t s, int nbk, bool sym) {
  TcMaps* t = static_cast<TcMaps*>(e.tmap);
  if (!t || nbk != e.nb) {
    set_error("tcgen05 update used before tc_prepare or with an unsupported K extent");
    return SCA_ENOSTATE;
  }
  TcArgs a;
  a.M = static_cast<float*>(e.M) + (size_t)m0 * e.mat_stride;
  a.mat0 = m0;
  a.N = e.N;
  a.ldm = e.ldm;
  a.mat_stride = (long long)e.mat_stride;
  a.plane_stride = (long long)e.plane_stride;
  a.nb = nbk;
  a.r0 = r0;
  a.c0 = c0;
  a.k0 = k0;
  a.kb = kb;
  a.gj = gj ? 1 : 0;
  a.tiles_m = (e.N - r0 + kBM - 1) / kBM;
  a.tiles_n = (e.N - c0 + kBNc - 1) / kBNc;
  a.sym = (sym && r0 == c0) ? 1 : 0;
  a.per_block = a.sym ? a.tiles_m * (a.tiles_m + 1) / 2 : a.tiles_m * a.tiles_n;
  a.tiles = a.per_block * cnt;
  a.fplanes = a.wplanes = (int)(e.fw_mat / ((size_t)e.N * nbk));
  a.m_zmul = 2;
  a.m_zoff = 0;
  a.err = e.flags;
  a.split_out = a.split_neg = 0;
  a.T = nullptr;
  a.t_mat = 0;
  if (a.tiles <= 0) return SCA_OK;
  if (e.tc_next >= kCounters) {
    set_error("too many tensor-core launches in one pass");
    return SCA_EINVAL;
  }
  a.counter = e.tc_counters + e.tc_next++;
  const int grid = std::min(a.tiles, e.tc_cap > 0 ? std::min(e.tc_cap, t->sms) : t->sms);
  if (e.bf16) k_update_tc<true><<<grid, kThreads, kSmemBytes, s>>>(t->F, t->W, t->M, a);
  else k_update_tc<false><<<grid, kThreads, kSmemBytes, s>>>(t->F, t->W, t->M, a);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return cuda_fail(err, "tcgen05 update launch");
  return SCA_OK;
}


sca_status tc_prep(Engine& e, int m0, int cnt, int r0, cudaStream_t s) {
  TcMaps* t = static_cast<TcMaps*>(e.tmap);
  if (!t || !e.tt) {
    set_error("tensor-core prep used before tc_prepare");
    return SCA_ENOSTATE;
  }
  TcArgs a;
  a.M = nullptr;
  a.N = e.N;
  a.ldm = e.nb;
  a.mat_stride = 0;
  a.plane_stride = 0;
  a.nb = e.nb;
  a.r0 = r0;
  a.c0 = 0;
  a.k0 = 0;
  a.kb = 1 << 30;  // every output element masked: the result is -sum F W
  a.gj = 1;
  a.tiles_m = (e.N - r0 + kBM - 1) / kBM;
  a.tiles_n = (e.nb + kBNc - 1) / kBNc;
  a.sym = 0;
  a.per_block = a.tiles_m * a.tiles_n;
  a.tiles = a.per_block * cnt;
  a.fplanes = (int)(e.fw_mat / e.fw_plane);  // A: W scratch planes 0-3
  a.wplanes = kTtPlanes;                           // B: -T^T planes
  a.mat0 = m0;
  a.m_zmul = (int)(e.fw_mat / e.fw_plane);   // output: W scratch planes 4, 5
  a.m_zoff = 4;
  a.err = e.flags;
  a.split_out = a.split_neg = 0;
  a.T = nullptr;
  a.t_mat = 0;
  if (a.tiles <= 0) return SCA_OK;
  if (e.tc_next >= kCounters) {
    set_error("too many tensor-core launches in one pass");
    return SCA_EINVAL;
  }
  a.counter = e.tc_counters + e.tc_next++;
  const int grid = std::min(a.tiles, e.tc_cap > 0 ? std::min(e.tc_cap, t->sms) : t->sms);
  k_update_tc<false><<<grid, kThreads, kSmemBytes, s>>>(t->W, t->TT, t->FP, a);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return cuda_fail(err, "tcgen05 prep launch");
  return SCA_OK;
}

sca_status tc_prep_split(Engine& e, int m0, int cnt, int r0, int k0, int kb, bool gj,
                         cudaStream_t s) {
  TcMaps* t = static_cast<TcMaps*>(e.tmap);
  if (!t || !e.tt) {
    set_error("tensor-core prep used before tc_prepare");
    return SCA_ENOSTATE;
  }
  TcArgs a;
  a.M = nullptr;
  a.N = e.N;
  a.ldm = e.nb;
  a.mat_stride = 0;
  a.plane_stride = 0;
  a.nb = e.nb;
  a.r0 = r0;
  a.c0 = 0;
  a.k0 = k0;
  a.kb = kb;
  a.gj = gj ? 1 : 0;
  a.tiles_m = (e.N - r0 + kBM - 1) / kBM;
  a.tiles_n = (e.nb + kBNc - 1) / kBNc;
  a.sym = 0;
  a.per_block = a.tiles_m * a.tiles_n;
  a.tiles = a.per_block * cnt;
  a.fplanes = (int)(e.fw_mat / e.fw_plane);  // A: W planes 0-3 (re_hi, im_hi, re_lo, im_lo)
  a.wplanes = kTtPlanes;                           // B: -T^T planes
  a.mat0 = m0;
  a.m_zmul = (int)(e.fw_mat / e.fw_plane);   // output: F planes 0-3
  a.m_zoff = 0;
  a.err = e.flags;
  a.split_out = 1;
  a.split_neg = 1;
  a.T = static_cast<const float2*>(e.Tinv);
  a.t_mat = 2ll * e.nb * e.nb;
  if (a.tiles <= 0) return SCA_OK;
  if (e.tc_next >= kCounters) {
    set_error("too many tensor-core launches in one pass");
    return SCA_EINVAL;
  }
  a.counter = e.tc_counters + e.tc_next++;
  const int grid = std::min(a.tiles, e.tc_cap > 0 ? std::min(e.tc_cap, t->sms) : t->sms);
  if (e.bf16) k_update_tc<true><<<grid, kThreads, kSmemBytes, s>>>(t->W, t->TT, t->FO, a);
  else k_update_tc<false><<<grid, kThreads, kSmemBytes, s>>>(t->W, t->TT, t->FO, a);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return cuda_fail(err, "tcgen05 prep launch");
  return SCA_OK;
}

sca_status tc_prep_piv(Engine& e, int m0, int cnt, int r0, int k0, int kb, bool gj,
                       cudaStream_t s) {
  TcMaps* t = static_cast<TcMaps*>(e.tmap);
  if (!t || !e.tt || !e.bf16) {
    set_error("pivoted tensor-core prep needs the BF16x3 planes");
    return SCA_ENOSTATE;
  }
  const int kend = k0 + kb;
  // rows [r0, kend) times T (rows of K: -T), then rows [max(r0, kend), N) times inv(L)
  for (int part = 0; part < 2; ++part) {
    const int ra = part == 0 ? r0 : std::max(r0, kend);
    const int rb = part == 0 ? std::min(kend, e.N) : e.N;
    if (rb <= ra) continue;
    TcArgs a;
    a.M = nullptr;
    a.N = e.N;
    a.ldm = e.nb;
    a.mat_stride = 0;
    a.plane_stride = 0;
    a.nb = e.nb;
    a.r0 = ra;
    a.c0 = 0;
    a.k0 = k0;
    a.kb = kb;
    a.gj = (gj && part == 0) ? 1 : 0;
    a.tiles_m = (rb - ra + kBM - 1) / kBM;
    a.tiles_n = (e.nb + kBNc - 1) / kBNc;
    a.sym = 0;
    a.per_block = a.tiles_m * a.tiles_n;
    a.tiles = a.per_block * cnt;
    a.fplanes = (int)(e.fw_mat / e.fw_plane);  // A: W planes 0-3
    a.wplanes = kTtPlanes;                           // B: -T^T or -inv(L)^T planes
    a.mat0 = m0;
    a.m_zmul = (int)(e.fw_mat / e.fw_plane);   // output: F planes 0-3
    a.m_zoff = 0;
    a.err = e.flags;
    a.split_out = 1;
    a.split_neg = 0;
    a.T = static_cast<const float2*>(e.Tinv);
    a.t_mat = 2ll * e.nb * e.nb;
    if (e.tc_next >= kCounters) {
      set_error("too many tensor-core launches in one pass");
      return SCA_EINVAL;
    }
    a.counter = e.tc_counters + e.tc_next++;
    const int grid = std::min(a.tiles, e.tc_cap > 0 ? std::min(e.tc_cap, t->sms) : t->sms);
    k_update_tc<true><<<grid, kThreads, kSmemBytes, s>>>(t->W, part == 0 ? t->TT : t->TL, t->FO,
                                                          a);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return cuda_fail(err, "tcgen05 pivoted prep launch");
  }
  return SCA_OK;
}

}  // namespace sca
