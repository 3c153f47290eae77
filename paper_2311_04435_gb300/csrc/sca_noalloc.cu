// Allocation-free variant of sca_grad_dev.
//
// Some callers cannot let a library allocate device memory: a process whose device memory is
// reserved up front by its own pool allocator (a cudaMalloc from the library would fail or
// fragment that pool), or a steady-state loop in which allocating is forbidden because
// cudaMalloc / cudaFree can synchronise the whole device.  sca_grad_noalloc_dev serves them:
// its workspace is the file-scope device array below, which every GPU that loads this library
// holds until the process exits, and the call makes no cudaMalloc, cudaFree or other
// allocating call.  It runs the same kernels as sca_grad_dev, on float64 or float32 blocks
// with CUDA-core contractions, and processes the blocks in as many chunks as the array needs.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "sca_internal.h"

namespace sca {
namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;  // 64 MiB per device

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

// Device address of g_scratch on the calling thread's current device.  In host code the symbol
// itself is only a host-side stand-in, so every call asks the runtime for the address: a
// host-side query that allocates nothing and enqueues nothing.  It is not cached, because the
// address belongs to the device's current context and moves when that context is re-created
// (after cudaDeviceReset, for example).
sca_status scratch_address(void** out) {
  void* p = nullptr;
  const cudaError_t err = cudaGetSymbolAddress(&p, g_scratch);
  if (err != cudaSuccess) return cuda_fail(err, "cudaGetSymbolAddress(scratch)");
  *out = p;
  return SCA_OK;
}

}  // namespace
}  // namespace sca

using namespace sca;

extern "C" sca_status sca_grad_noalloc_dev(const sca_params* params, const double* d_phi,
                                           double* d_omega, double* d_grad, void* stream) {
  if (!params || !d_phi || !d_omega || !d_grad) {
    set_error("sca_grad_noalloc_dev: NULL argument");
    return SCA_EINVAL;
  }
  uint64_t unused = 0;
  sca_status st = sca_workspace_bytes(params, &unused);  // validates the parameters
  if (st != SCA_OK) return st;
  if (params->prec != SCA_PREC_FP64 && params->prec != SCA_PREC_FP32) {
    set_error("sca_grad_noalloc_dev: prec must be SCA_PREC_FP64 or SCA_PREC_FP32");
    return SCA_EINVAL;
  }
  Engine e;
  plan(*params, e);
  e.tc = false;
  const size_t S = e.fp64 ? 8 : 4;
  // Fixed part: status, flags, ld (B), gd (B x N).  (Omega goes straight to the caller's
  // d_omega, so the engine's Omega scratch is not carved.)
  const size_t fixed = al256(8 * sizeof(double)) + al256(16) + al256((size_t)e.B * 8) +
                       al256((size_t)e.B * e.N * 8);
  // Per resident block: block planes, F, W, Tinv, piv, perm, diagonal table.
  const size_t per_block = e.mat_stride * S + 2 * e.fw_mat * S + 2 * (size_t)e.nb * e.nb * 2 * S +
                           2 * (size_t)e.N * sizeof(int) + (size_t)e.N * 2 * sizeof(float);
  const size_t room = kScratchBytes > fixed ? kScratchBytes - fixed : 0;
  // every array below is rounded up to 256 bytes: leave 7 x 256 bytes of slack per chunk
  const long long fit = room > 7 * 256 ? (long long)((room - 7 * 256) / per_block) : 0;
  if (fit < 1) {
    set_error("sca_grad_noalloc_dev: problem too large for the " +
              std::to_string(kScratchBytes >> 20) + " MiB static workspace (needs " +
              std::to_string(fixed + per_block) + " bytes for one block)");
    return SCA_EINVAL;
  }
  e.chunk = (int)std::min<long long>(e.B, fit);
  void* base = nullptr;
  if ((st = scratch_address(&base)) != SCA_OK) return st;
  unsigned char* p = static_cast<unsigned char*>(base);
  auto take = [&p](size_t bytes) {
    void* q = p;
    p += al256(bytes);
    return q;
  };
  e.d_status = static_cast<double*>(take(8 * sizeof(double)));
  e.flags = static_cast<int*>(take(16));
  e.ld = static_cast<double*>(take((size_t)e.B * 8));
  e.gd = static_cast<double*>(take((size_t)e.B * e.N * 8));
  e.piv = static_cast<int*>(take((size_t)e.chunk * e.N * sizeof(int)));
  e.perm = static_cast<int*>(take((size_t)e.chunk * e.N * sizeof(int)));
  e.Tinv = take((size_t)e.chunk * 2 * e.nb * e.nb * 2 * S);
  e.adiag = static_cast<float*>(take((size_t)e.chunk * e.N * 2 * sizeof(float)));
  e.F = take((size_t)e.chunk * e.fw_mat * S);
  e.W = take((size_t)e.chunk * e.fw_mat * S);
  e.M = take((size_t)e.chunk * e.mat_stride * S);
  if ((size_t)(p - static_cast<unsigned char*>(base)) > kScratchBytes) {
    set_error("sca_grad_noalloc_dev: internal workspace layout overflow");
    return SCA_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // The array keeps the previous call's contents: clear what the kernels accumulate into.
  cudaError_t err = cudaMemsetAsync(e.d_status, 0, 8 * sizeof(double), s);
  if (err == cudaSuccess) err = cudaMemsetAsync(e.flags, 0, 16, s);
  if (err != cudaSuccess) return cuda_fail(err, "scratch clear");
  if ((st = run_blocks(e, d_phi, true, s)) != SCA_OK) return st;
  return run_reduce(e, d_phi, d_omega, d_grad, nullptr, s);
}
