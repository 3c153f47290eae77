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
#include "sca_device.cuh"

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
// all but the most recent bulk group have finished reading their shared-memory source
__device__ __forceinline__ void bulk_wait_read1() {
  asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
}
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
  // Two Gauss-Jordan steps K1 = [k0, k0 + kb) and K2 = [kc0, kc0 + kcb) in one pass (symmetric
  // blocks, tile row/column cross_t = K2's tiles).  merge 1: only the cross of K2 (tiles
  // (cross_t, j <= cross_t) and (i > cross_t, cross_t)) with F1 W1 from the first map pair;
  // merge 2: every lower tile, K = nb from (F, W) then nb from (F2, W2) with the K1 mask,
  // except the cross of K2, which takes only the second pair with the K2 mask.  merge 0: one
  // step as before.
  int merge, cross_t, kc0, kcb;
};

// Tile t -> (block, tile row, tile column).  With `sym` only tiles on or below the diagonal
// exist (the dominant blocks stay symmetric up to sign, see the host code): rem ->
// (i, j) with rem = i (i + 1) / 2 + j, j <= i.
__device__ __forceinline__ void decode_tile(const TcArgs& a, int t, int& mat, int& tm, int& tn) {
  mat = t / a.per_block;
  const int rem = t - mat * a.per_block;
  if (a.merge == 1) {  // the cross of tile row / column cross_t, lower tiles only
    if (rem <= a.cross_t) { tm = a.cross_t; tn = rem; }
    else { tm = rem; tn = a.cross_t; }
    return;
  }
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

// K stages [ks_lo, ks_hi) of a tile (units of kKE elements; stages from ks_a on come from the
// second map pair) and the Gauss-Jordan mask [mk0, mk0 + mkb) of its epilogue.
__device__ __forceinline__ void tile_k(const TcArgs& a, int tm, int tn, int kke, int& ks_lo,
                                       int& ks_hi, int& mk0, int& mkb) {
  const int ka = a.nb / kke;
  const bool cross = a.merge == 2 && (tm == a.cross_t || tn == a.cross_t);
  ks_lo = cross ? ka : 0;
  ks_hi = a.merge == 2 ? 2 * ka : ka;
  mk0 = cross ? a.kc0 : a.k0;
  mkb = cross ? a.kcb : a.kb;
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
                const __grid_constant__ CUtensorMap tmM, const __grid_constant__ CUtensorMap tmF2,
                const __grid_constant__ CUtensorMap tmW2, TcArgs a) {
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
  const int ka = a.nb / kKE;  // K stages per map pair

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
        int mat, tm, tn, ks_lo, ks_hi, mk0, mkb;
        decode_tile(a, t, mat, tm, tn);
        tile_k(a, tm, tn, kKE, ks_lo, ks_hi, mk0, mkb);
        const int frow = a.r0 + tm * kBM, wrow = a.c0 + tn * kBNc;
        for (int ks = ks_lo; ks < ks_hi; ++ks) {
          if (!mbar_wait(&empty[stage], phase ^ 1, abort_flag)) break;
          mbar_expect_tx(&full[stage], kStageBytes);
          unsigned char* st = smem + stage * kStageBytes;
          const bool second = ks >= ka;
          const CUtensorMap* mf = second ? &tmF2 : &tmF;
          const CUtensorMap* mw = second ? &tmW2 : &tmW;
          const int kx = (second ? ks - ka : ks) * kKE;
          for (int s = 0; s < 4; ++s)
            tma_load_3d(st + s * kTileBytes, mf, &full[stage], kx, frow,
                        (a.mat0 + mat) * a.fplanes + kFPlaneOfSlot[s]);
          for (int s = 0; s < 4; ++s)
            tma_load_3d(st + (4 + s) * kTileBytes, mw, &full[stage], kx, wrow,
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
        int ks_lo, ks_hi;
        {
          int mat, tm, tn, mk0, mkb;
          decode_tile(a, t, mat, tm, tn);
          tile_k(a, tm, tn, kKE, ks_lo, ks_hi, mk0, mkb);
        }
        for (int ks = ks_lo; ks < ks_hi; ++ks) {
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
            const uint32_t acc0 = (ks > ks_lo || k8 > 0) ? 1u : 0u;
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
    int sbuf = 0;  // staging buffer of the next split-output chunk (bf16 planes)
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
      int mat, tm, tn, ks_lo, ks_hi, mk0, mkb;
      decode_tile(a, t, mat, tm, tn);
      tile_k(a, tm, tn, kKE, ks_lo, ks_hi, mk0, mkb);
      const int i = a.r0 + tm * kBM + row;
      const int j0 = a.c0 + tn * kBNc;
      const bool rowk = a.gj && i >= mk0 && i < mk0 + mkb;
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
          // bf16 planes fill one staging buffer: chunks alternate between the two, so a chunk
          // waits only for the stores of the chunk before last (which read this buffer); the
          // float planes fill both buffers and wait for the previous chunk's stores
          if (leader) {
            if constexpr (BF) bulk_wait_read1();
            else bulk_wait_read0();
          }
          epi_bar();
          const int jc = j0 + c * kEpiCols;
          const bool neg = a.split_neg && i < a.k0;
          const float2* trow =
              rowk ? a.T + (size_t)(a.mat0 + mat) * a.t_mat + (size_t)(i - mk0) * a.nb : nullptr;
          unsigned char* s0 = BF ? epi + sbuf * kEpiBufBytes : epi;
          unsigned char* s1 = epi + kEpiBufBytes;
          sbuf ^= 1;
          if constexpr (BF) {
            // four bf16 planes of 128 rows x 64 bytes (8 KB each) in buffer 0, 64-byte swizzle:
            // 16-byte unit u of row r sits at unit u ^ ((r >> 1) & 3)
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int off = row * 64 + ((u ^ ((row >> 1) & 3)) << 4);
              // the 8 entries of this 16-byte unit as bf16 pairs packed in registers (the
              // lower-addressed entry in the low half): planes re_hi, im_hi, re_lo, im_lo
              uint32_t pk[4][4];
#pragma unroll
              for (int e2 = 0; e2 < 4; ++e2) {
                float vr[2], vi[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                  const int e = 2 * e2 + h;
                  const int j = jc + 8 * u + e;
                  if (rowk) {
                    const float2 tv = (j < a.kb) ? trow[j] : make_float2(0.f, 0.f);
                    vr[h] = -tv.x;
                    vi[h] = -tv.y;
                  } else {
                    vr[h] = -__uint_as_float(cr[8 * u + e]);
                    vi[h] = -__uint_as_float(ci[8 * u + e]);
                    if (neg) { vr[h] = -vr[h]; vi[h] = -vi[h]; }
                  }
                }
                const __nv_bfloat162 hr = __floats2bfloat162_rn(vr[0], vr[1]);
                const __nv_bfloat162 hi = __floats2bfloat162_rn(vi[0], vi[1]);
                const float2 hrf = __bfloat1622float2(hr), hif = __bfloat1622float2(hi);
                const __nv_bfloat162 lr = __floats2bfloat162_rn(vr[0] - hrf.x, vr[1] - hrf.y);
                const __nv_bfloat162 li = __floats2bfloat162_rn(vi[0] - hif.x, vi[1] - hif.y);
                pk[0][e2] = *reinterpret_cast<const uint32_t*>(&hr);
                pk[1][e2] = *reinterpret_cast<const uint32_t*>(&hi);
                pk[2][e2] = *reinterpret_cast<const uint32_t*>(&lr);
                pk[3][e2] = *reinterpret_cast<const uint32_t*>(&li);
              }
#pragma unroll
              for (int pl = 0; pl < 4; ++pl)
                *reinterpret_cast<uint4*>(s0 + pl * (kBM * 64) + off) =
                    make_uint4(pk[pl][0], pk[pl][1], pk[pl][2], pk[pl][3]);
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
        const bool colk = a.gj && (jc < mk0 + mkb) && (jc + kEpiCols > mk0);
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
              const bool keep = !(rowk || (j >= mk0 && j < mk0 + mkb));
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

// ------------------------------------------------ pivot-block inverse on the tensor cores
// Gauss-Jordan inverse T = inv(M_KK) of one 128 x 128 diagonally dominant pivot block per CTA
// (no pivoting), the tableau resident in TMEM: lane r = row r, columns 0-127 the real and
// 128-255 the imaginary parts.  It is swept in 8 panels P of 16 pivots; per panel
//   1. the rows of P go to shared memory and one warp inverts M_PP in registers (its pivots
//      are those of the LU, so ln|det M_KK| is the same sum);
//   2. every thread forms its row of F = M[:, P] inv(M_PP) in float32 (rows of P:
//      -inv(M_PP)), and the rows and columns of P are zeroed in TMEM;
//   3. M <- mask(M) - F W (W = M[P, :] with the identity in the columns of P) as real MMAs
//      of M = 128, N = 256, K = 32: A = [F_re | F_im], B rows c: [W_re; -W_im] and rows
//      128 + c: [W_im; W_re], split TF32 (hi*hi + hi*lo + lo*hi), A negated by the
//      instruction descriptor, accumulating into the tableau.
// Two CTAs fit on one SM (256 TMEM columns and ~101 KB of shared memory each), so a launch
// over all dominant blocks is a single wave.  Outputs as the register kernel: T (complex,
// row-major nb x nb, zero outside kb), the -T^T split planes, ld += ln|det M_KK|.
constexpr int kDgThreads = 128;
constexpr int kDgA = 0;                         // A: sub-tile (re, im) x (hi, lo), 128 x 64 B
constexpr int kDgB = 4 * 8192;                  // B: sub-tile (k < 16, k >= 16) x (hi, lo), 256 x 64 B
constexpr int kDgTp = kDgB + 4 * 16384;         // inv(M_PP): 16 x 17 complex
constexpr int kDgPiv = kDgTp + 16 * 17 * 8;     // the 128 pivots (complex)
constexpr int kDgPiv2 = kDgPiv + 128 * 8;       // |pivot|^2 (double)
constexpr int kDgBar = kDgPiv2 + 128 * 8;       // mbarrier, TMEM address, abort flag
constexpr int kDgSmem = kDgBar + 64 + 1024;     // + alignment slack
constexpr int kDgRowStride = 129;               // complex row stride of the panel rows (in A)
constexpr uint32_t kDgTmemCols = 256;

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t* r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
      "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]),
      "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]),
      "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
      "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_st_wait() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// One 64-byte K-major operand row of 16 floats, TF32-split into the hi and lo planes, in the
// 64-byte swizzle (16-byte chunk q of row r at chunk q ^ ((r >> 1) & 3)).
__device__ __forceinline__ void dg_store_row(unsigned char* hi, unsigned char* lo, int row,
                                             const float* v) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      h[e] = __uint_as_float(__float_as_uint(v[4 * q + e]) & 0xffffe000u);
      l[e] = v[4 * q + e] - h[e];
    }
    const int off = row * 64 + ((q ^ ((row >> 1) & 3)) << 4);
    *reinterpret_cast<float4*>(hi + off) = make_float4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<float4*>(lo + off) = make_float4(l[0], l[1], l[2], l[3]);
  }
}

__global__ void __launch_bounds__(kDgThreads, 2)
    k_diag_tc(const float* M, int ldm, long long mat_stride, long long plane_stride, int k0,
              int kb, int b0, double* ld, float2* Tinv, float* TT, int tt_bf16, int* flags) {
  constexpr int KB = 128, PW = 16;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* opA = sm + kDgA;
  unsigned char* opB = sm + kDgB;
  float2* wrow = reinterpret_cast<float2*>(sm + kDgA);  // rows of P, [16][kDgRowStride]
  float2* tp = reinterpret_cast<float2*>(sm + kDgTp);   // inv(M_PP), [16][17]
  float2* pivd = reinterpret_cast<float2*>(sm + kDgPiv);
  double* piv2 = reinterpret_cast<double*>(sm + kDgPiv2);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + kDgBar);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + kDgBar + 8);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + kDgBar + 16);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mat = blockIdx.x, r = tid;
  if (tid == 0) {
    mbar_init(mbar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kDgTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);  // this warp's lane quarter
  const float* re = M + (long long)mat * mat_stride;
  const float* im = re + plane_stride;

  // the pivot block into TMEM (identity outside kb)
#pragma unroll 1
  for (int c0 = 0; c0 < KB; c0 += 32) {
    uint32_t vr[32], vi[32];
    if (r < kb && c0 + 32 <= kb) {
      const float4* pr = reinterpret_cast<const float4*>(re + (size_t)(k0 + r) * ldm + k0 + c0);
      const float4* pi = reinterpret_cast<const float4*>(im + (size_t)(k0 + r) * ldm + k0 + c0);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float4 a4 = pr[q], b4 = pi[q];
        vr[4 * q] = __float_as_uint(a4.x); vr[4 * q + 1] = __float_as_uint(a4.y);
        vr[4 * q + 2] = __float_as_uint(a4.z); vr[4 * q + 3] = __float_as_uint(a4.w);
        vi[4 * q] = __float_as_uint(b4.x); vi[4 * q + 1] = __float_as_uint(b4.y);
        vi[4 * q + 2] = __float_as_uint(b4.z); vi[4 * q + 3] = __float_as_uint(b4.w);
      }
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int c = c0 + i;
        const bool in = r < kb && c < kb;
        const size_t o = (size_t)(k0 + r) * ldm + k0 + c;
        vr[i] = __float_as_uint(in ? re[o] : (r == c ? 1.f : 0.f));
        vi[i] = __float_as_uint(in ? im[o] : 0.f);
      }
    }
    __syncwarp();  // the warp-collective store after a lane-dependent branch
    tmem_st32(trow + (uint32_t)c0, vr);
    tmem_st32(trow + (uint32_t)(KB + c0), vi);
  }
  tmem_st_wait();

  constexpr uint32_t kIdNeg = idesc<false, true, true>();  // tf32, N = 256, A negated
  uint32_t phase = 0;
  bool ok = true;
#pragma unroll 1
  for (int p0 = 0; p0 < KB && ok; p0 += PW) {
    const bool rP = (unsigned)(r - p0) < (unsigned)PW;
    // my row's entries in the panel's columns
    uint32_t xr[16], xi[16];
    tmem_ld16(trow + (uint32_t)p0, xr);
    tmem_ld16(trow + (uint32_t)(KB + p0), xi);
    tmem_ld_wait();
    // the panel's rows to shared memory; in TMEM they are zeroed (mask)
    if (warp == (p0 >> 5)) {
#pragma unroll 1
      for (int c0 = 0; c0 < KB; c0 += 32) {
        uint32_t ur[32], ui[32];
        tmem_ld32(trow + (uint32_t)c0, ur);
        tmem_ld32(trow + (uint32_t)(KB + c0), ui);
        tmem_ld_wait();
        if (rP) {
          float2* w = wrow + (r - p0) * kDgRowStride + c0;
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            w[i] = make_float2(__uint_as_float(ur[i]), __uint_as_float(ui[i]));
            ur[i] = 0u;
            ui[i] = 0u;
          }
        }
        __syncwarp();
        tmem_st32(trow + (uint32_t)c0, ur);
        tmem_st32(trow + (uint32_t)(KB + c0), ui);
      }
      tmem_st_wait();
    }
    __syncthreads();
    // warp 0: inv(M_PP) by Gauss-Jordan in registers; lane owns column lane % 16 of rows
    // lane / 16 + 2 m; the pivot row, column and entry of each step come by shuffle
    if (warp == 0) {
      const int cl = lane & 15, q0 = lane >> 4;
      cpx<float> v[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const float2 t = wrow[(q0 + 2 * m) * kDgRowStride + p0 + cl];
        v[m] = {t.x, t.y};
      }
      // a rolled loop: the pivot's slot is picked by selects and the row update below has no
      // branches, so one short body serves all 16 pivots
#pragma unroll 1
      for (int cc = 0; cc < PW; ++cc) {
        const int own = (cc & 1) * 16, slot = cc >> 1;
        cpx<float> vs = v[0];
#pragma unroll
        for (int m = 1; m < 8; ++m)
          if (m == slot) vs = v[m];
        cpx<float> d, pr, pc[8];
        d.re = __shfl_sync(0xffffffffu, vs.re, own + cc);
        d.im = __shfl_sync(0xffffffffu, vs.im, own + cc);
        pr.re = __shfl_sync(0xffffffffu, vs.re, own + cl);
        pr.im = __shfl_sync(0xffffffffu, vs.im, own + cl);
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          pc[m].re = __shfl_sync(0xffffffffu, v[m].re, q0 * 16 + cc);
          pc[m].im = __shfl_sync(0xffffffffu, v[m].im, q0 * 16 + cc);
        }
        const float m2 = d.re * d.re + d.im * d.im;
        const float rm = (m2 > 0.f) ? 1.f / m2 : 0.f;
        const cpx<float> dinv = {d.re * rm, -d.im * rm};
        if (lane == 0) pivd[p0 + cc] = make_float2(d.re, d.im);
        // new entries: pivot row u = v inv(d) (pivot: inv(d)), pivot column -v inv(d), others
        // v - pc u; chosen by scalar selects (a branch per row serialises the warp)
        const cpx<float> u = cmul(pr, dinv);
        const bool b = cl == cc;
        const float yr = b ? dinv.re : u.re, yi = b ? dinv.im : u.im;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const bool a = q0 + 2 * m == cc;
          const float q2r = pc[m].re * dinv.re - pc[m].im * dinv.im;
          const float q2i = pc[m].re * dinv.im + pc[m].im * dinv.re;
          const float upr = v[m].re - (pc[m].re * u.re - pc[m].im * u.im);
          const float upi = v[m].im - (pc[m].re * u.im + pc[m].im * u.re);
          const float xr = b ? -q2r : upr, xi = b ? -q2i : upi;
          v[m].re = a ? yr : xr;
          v[m].im = a ? yi : xi;
        }
      }
#pragma unroll
      for (int m = 0; m < 8; ++m) tp[(q0 + 2 * m) * 17 + cl] = make_float2(v[m].re, v[m].im);
    }
    // B from the panel's rows: thread c builds rows c and 128 + c of both K sub-tiles
    {
      const int c = tid;
      const bool cP = (unsigned)(c - p0) < (unsigned)PW;
      float wr[16], wi[16], nwi[16];
#pragma unroll
      for (int k = 0; k < PW; ++k) {
        const float2 w = cP ? make_float2(k == c - p0 ? 1.f : 0.f, 0.f)
                            : wrow[k * kDgRowStride + c];
        wr[k] = w.x;
        wi[k] = w.y;
        nwi[k] = -w.y;
      }
      dg_store_row(opB + 0 * 16384, opB + 1 * 16384, c, wr);
      dg_store_row(opB + 0 * 16384, opB + 1 * 16384, KB + c, wi);
      dg_store_row(opB + 2 * 16384, opB + 3 * 16384, c, nwi);
      dg_store_row(opB + 2 * 16384, opB + 3 * 16384, KB + c, wr);
    }
    __syncthreads();  // inv(M_PP) ready; the panel rows are no longer read (A reuses them)
    // my row of F into A, four columns (one 16-byte chunk of each operand row) at a time
#pragma unroll 1
    for (int g = 0; g < 4; ++g) {
      float fr[4], fi[4];
      if (rP) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float2 t = tp[(r - p0) * 17 + 4 * g + k];
          fr[k] = -t.x;
          fi[k] = -t.y;
        }
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) { fr[k] = 0.f; fi[k] = 0.f; }
#pragma unroll
        for (int m = 0; m < PW; ++m) {
          const float xre = __uint_as_float(xr[m]), xim = __uint_as_float(xi[m]);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const float2 t = tp[m * 17 + 4 * g + k];
            fr[k] += xre * t.x - xim * t.y;
            fi[k] += xre * t.y + xim * t.x;
          }
        }
      }
      float hr[4], lr[4], hi[4], li[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        hr[k] = __uint_as_float(__float_as_uint(fr[k]) & 0xffffe000u);
        lr[k] = fr[k] - hr[k];
        hi[k] = __uint_as_float(__float_as_uint(fi[k]) & 0xffffe000u);
        li[k] = fi[k] - hi[k];
      }
      const int off = r * 64 + ((g ^ ((r >> 1) & 3)) << 4);
      *reinterpret_cast<float4*>(opA + 0 * 8192 + off) = make_float4(hr[0], hr[1], hr[2], hr[3]);
      *reinterpret_cast<float4*>(opA + 1 * 8192 + off) = make_float4(lr[0], lr[1], lr[2], lr[3]);
      *reinterpret_cast<float4*>(opA + 2 * 8192 + off) = make_float4(hi[0], hi[1], hi[2], hi[3]);
      *reinterpret_cast<float4*>(opA + 3 * 8192 + off) = make_float4(li[0], li[1], li[2], li[3]);
    }
    __syncwarp();
    {  // the panel's columns of my row zeroed (mask)
      uint32_t z[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) z[i] = 0u;
      tmem_st16(trow + (uint32_t)p0, z);
      tmem_st16(trow + (uint32_t)(KB + p0), z);
    }
    tmem_st_wait();
    fence_proxy_async();  // the operand stores, visible to the tensor core
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int sub = 0; sub < 2; ++sub) {
#pragma unroll
        for (int k8 = 0; k8 < 2; ++k8) {
          const uint32_t off = (uint32_t)(k8 * 32);
          const uint64_t a_hi = sdesc_k64(smem_u32(opA + (2 * sub) * 8192) + off);
          const uint64_t a_lo = sdesc_k64(smem_u32(opA + (2 * sub + 1) * 8192) + off);
          const uint64_t b_hi = sdesc_k64(smem_u32(opB + (2 * sub) * 16384) + off);
          const uint64_t b_lo = sdesc_k64(smem_u32(opB + (2 * sub + 1) * 16384) + off);
          mma_d<false>(tmem, a_hi, b_hi, kIdNeg, 1u);
          mma_d<false>(tmem, a_hi, b_lo, kIdNeg, 1u);
          mma_d<false>(tmem, a_lo, b_hi, kIdNeg, 1u);
        }
      }
      mma_commit(mbar);
    }
    const bool done = mbar_wait(mbar, phase, abort_flag);
    phase ^= 1u;
    tc_fence_after();
    ok = __syncthreads_and(done ? 1 : 0) != 0;
  }
  if (!ok) {
    // a wait ran out: the last commit may still be outstanding; wait for it (bounded)
    volatile int drain_abort = 0;
    if (tid == 0) {
      (void)mbar_wait(mbar, phase ^ 1u, &drain_abort);
      atomicOr(flags, 2);
    }
  } else {
    for (int k = tid; k < kb; k += kDgThreads) {
      const float2 d = pivd[k];
      piv2[k] = (double)d.x * d.x + (double)d.y * d.y;
    }
    __syncthreads();
    const double lsum = logdet_sum<kDgThreads>(piv2, kb, flags);
    if (tid == 0) ld[b0 + mat] += lsum;
    // T (row r) and the -T^T split planes (column r of W_T: coalesced across the warp)
    float2* T = Tinv + (size_t)mat * 2 * KB * KB;
    constexpr size_t P = (size_t)KB * KB;
    float* tt = TT ? TT + (size_t)mat * kTtPlanes * P : nullptr;
#pragma unroll 1
    for (int c0 = 0; c0 < KB; c0 += 32) {
      uint32_t ur[32], ui[32];
      tmem_ld32(trow + (uint32_t)c0, ur);
      tmem_ld32(trow + (uint32_t)(KB + c0), ui);
      tmem_ld_wait();
      float4* trw = reinterpret_cast<float4*>(T + (size_t)r * KB + c0);
#pragma unroll
      for (int i = 0; i < 32; i += 2) {
        const int j = c0 + i;
        const bool in0 = r < kb && j < kb, in1 = r < kb && j + 1 < kb;
        trw[i / 2] = make_float4(in0 ? __uint_as_float(ur[i]) : 0.f,
                                 in0 ? __uint_as_float(ui[i]) : 0.f,
                                 in1 ? __uint_as_float(ur[i + 1]) : 0.f,
                                 in1 ? __uint_as_float(ui[i + 1]) : 0.f);
      }
      if (tt) {
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int j = c0 + i;
          const bool in = r < kb && j < kb;
          const float fr = in ? -__uint_as_float(ur[i]) : 0.f;
          const float fi = in ? -__uint_as_float(ui[i]) : 0.f;
          const size_t o = (size_t)j * KB + r;
          if (tt_bf16) {
            const __nv_bfloat16 hr = __float2bfloat16_rn(fr), hi = __float2bfloat16_rn(fi);
            reinterpret_cast<__nv_bfloat16*>(tt)[o] = hr;
            reinterpret_cast<__nv_bfloat16*>(tt + P)[o] = hi;
            reinterpret_cast<__nv_bfloat16*>(tt + 2 * P)[o] =
                __float2bfloat16_rn(fr - __bfloat162float(hr));
            reinterpret_cast<__nv_bfloat16*>(tt + 3 * P)[o] =
                __float2bfloat16_rn(fi - __bfloat162float(hi));
          } else {
            const float hr = __uint_as_float(__float_as_uint(fr) & 0xffffe000u);
            const float hi = __uint_as_float(__float_as_uint(fi) & 0xffffe000u);
            tt[o] = hr;
            tt[P + o] = hi;
            tt[2 * P + o] = fr - hr;
            tt[3 * P + o] = fi - hi;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kDgTmemCols)
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
  // second factor pair of a merged two-step update of the symmetric dominant blocks (F2, W2
  // planes as F, W) and the split output map of its prep product
  CUtensorMap F2, W2, FO2;
  bool has2 = false;
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
  if (e.F2 && e.W2) {
    if (!make_fw_map(&t->F2, e.F2, e.nb, e.N, zf, e.bf16) ||
        !make_fw_map(&t->W2, e.W2, e.nb, e.N, zf, e.bf16) ||
        !make_m_map_rows(&t->FO2, e.F2, e.nb, e.N, e.nb, (long long)e.fw_plane, zf, e.bf16)) {
      delete t;
      set_error("cuTensorMapEncodeTiled failed for the merged two-step update");
      return SCA_ECUDA;
    }
    t->has2 = true;
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
  a.merge = 0;
  a.cross_t = -1;
  a.kc0 = a.kcb = 0;
  if (a.tiles <= 0) return SCA_OK;
  if (e.tc_next >= kCounters) {
    set_error("too many tensor-core launches in one pass");
    return SCA_EINVAL;
  }
  a.counter = e.tc_counters + e.tc_next++;
  const int grid = std::min(a.tiles, e.tc_cap > 0 ? std::min(e.tc_cap, t->sms) : t->sms);
  if (e.bf16) k_update_tc<true><<<grid, kThreads, kSmemBytes, s>>>(t->F, t->W, t->M, t->F, t->W, a);
  else k_update_tc<false><<<grid, kThreads, kSmemBytes, s>>>(t->F, t->W, t->M, t->F, t->W, a);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return cuda_fail(err, "tcgen05 update launch");
  return SCA_OK;
}


sca_status tc_update_pair(Engine& e, int m0, int cnt, int k1, int kb1, int k2, int kb2, int merge,
                          cudaStream_t s) {
  TcMaps* t = static_cast<TcMaps*>(e.tmap);
  if (!t || !t->has2 || (merge != 1 && merge != 2) || kb1 != e.nb || k2 != k1 + kb1 ||
      kb2 < 1 || kb2 > e.nb || k2 % kBM != 0) {
    set_error("merged tensor-core update: needs the second factor pair and two adjacent steps");
    return SCA_EINVAL;
  }
  TcArgs a;
  a.M = static_cast<float*>(e.M) + (size_t)m0 * e.mat_stride;
  a.mat0 = m0;
  a.N = e.N;
  a.ldm = e.ldm;
  a.mat_stride = (long long)e.mat_stride;
  a.plane_stride = (long long)e.plane_stride;
  a.nb = e.nb;
  a.r0 = 0;
  a.c0 = 0;
  a.k0 = k1;
  a.kb = kb1;
  a.gj = 1;
  a.tiles_m = a.tiles_n = (e.N + kBM - 1) / kBM;
  a.sym = 1;
  a.merge = merge;
  a.cross_t = k2 / kBM;
  a.kc0 = k2;
  a.kcb = kb2;
  a.per_block = merge == 1 ? a.tiles_m : a.tiles_m * (a.tiles_m + 1) / 2;
  a.tiles = a.per_block * cnt;
  a.fplanes = a.wplanes = (int)(e.fw_mat / e.fw_plane);
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
  if (e.bf16)
    k_update_tc<true><<<grid, kThreads, kSmemBytes, s>>>(t->F, t->W, t->M, t->F2, t->W2, a);
  else
    k_update_tc<false><<<grid, kThreads, kSmemBytes, s>>>(t->F, t->W, t->M, t->F2, t->W2, a);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return cuda_fail(err, "tcgen05 merged update launch");
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
  a.merge = 0;
  a.cross_t = -1;
  a.kc0 = a.kcb = 0;
  if (a.tiles <= 0) return SCA_OK;
  if (e.tc_next >= kCounters) {
    set_error("too many tensor-core launches in one pass");
    return SCA_EINVAL;
  }
  a.counter = e.tc_counters + e.tc_next++;
  const int grid = std::min(a.tiles, e.tc_cap > 0 ? std::min(e.tc_cap, t->sms) : t->sms);
  k_update_tc<false><<<grid, kThreads, kSmemBytes, s>>>(t->W, t->TT, t->FP, t->W, t->TT, a);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return cuda_fail(err, "tcgen05 prep launch");
  return SCA_OK;
}

sca_status tc_prep_split(Engine& e, int m0, int cnt, int r0, int k0, int kb, bool gj,
                         cudaStream_t s, bool second) {
  TcMaps* t = static_cast<TcMaps*>(e.tmap);
  if (!t || !e.tt || (second && !t->has2)) {
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
  a.merge = 0;
  a.cross_t = -1;
  a.kc0 = a.kcb = 0;
  if (a.tiles <= 0) return SCA_OK;
  if (e.tc_next >= kCounters) {
    set_error("too many tensor-core launches in one pass");
    return SCA_EINVAL;
  }
  a.counter = e.tc_counters + e.tc_next++;
  const int grid = std::min(a.tiles, e.tc_cap > 0 ? std::min(e.tc_cap, t->sms) : t->sms);
  // A = the W planes of this step (W or W2), output = its F planes (F or F2)
  const CUtensorMap& ta = second ? t->W2 : t->W;
  const CUtensorMap& to = second ? t->FO2 : t->FO;
  if (e.bf16) k_update_tc<true><<<grid, kThreads, kSmemBytes, s>>>(ta, t->TT, to, ta, t->TT, a);
  else k_update_tc<false><<<grid, kThreads, kSmemBytes, s>>>(ta, t->TT, to, ta, t->TT, a);
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
    a.merge = 0;
    a.cross_t = -1;
    a.kc0 = a.kcb = 0;
    if (e.tc_next >= kCounters) {
      set_error("too many tensor-core launches in one pass");
      return SCA_EINVAL;
    }
    a.counter = e.tc_counters + e.tc_next++;
    const int grid = std::min(a.tiles, e.tc_cap > 0 ? std::min(e.tc_cap, t->sms) : t->sms);
    const CUtensorMap& tb = part == 0 ? t->TT : t->TL;
    k_update_tc<true><<<grid, kThreads, kSmemBytes, s>>>(t->W, tb, t->FO, t->W, tb, a);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return cuda_fail(err, "tcgen05 pivoted prep launch");
  }
  return SCA_OK;
}

sca_status tc_diag(const float* M, int ldm, size_t mat_stride, size_t plane_stride, int cnt, int k0,
                   int kb, int nb, int b0, double* ld, void* Tinv, float* TT, int tt_bf16,
                   int* flags, cudaStream_t s) {
  if (nb != 128 || kb < 1 || kb > nb) {
    set_error("tensor-core pivot-block inverse needs nb = 128");
    return SCA_EINVAL;
  }
  static ContextOnce attr;
  if (!attr.done()) {
    cudaError_t err =
        cudaFuncSetAttribute(k_diag_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kDgSmem);
    if (err != cudaSuccess) return cuda_fail(err, "tensor-core pivot-block inverse set-up");
    attr.mark();
  }
  if (cnt <= 0) return SCA_OK;
  k_diag_tc<<<cnt, kDgThreads, kDgSmem, s>>>(M, ldm, (long long)mat_stride,
                                               (long long)plane_stride, k0, kb, b0, ld,
                                               static_cast<float2*>(Tinv), TT, tt_bf16, flags);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return cuda_fail(err, "tensor-core pivot-block inverse launch");
  return SCA_OK;
}

}  // namespace sca
