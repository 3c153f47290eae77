// SM partitions for the two block groups.  The pivoted group is a chain of short dependent
// launches; the dominant group is bandwidth-bound work that fills every SM it can reach.
// Stream priority alone does not keep them apart: a dominant launch of many CTAs (the
// pivot-block inverses, the W planes, the refinement) occupies every SM, and each launch of
// the pivoted chain then waits for one of those CTAs to finish.  Here the dominant group's
// streams live in a green context (driver SM partition) that holds all SMs but `piv_sms`;
// those SMs stay free for the pivoted group, whose own stream keeps the highest priority and
// may use any SM (mode 1) or only its partition (mode 2).
//
// The driver entry points come from cudaGetDriverEntryPointByVersion, so the library does
// not link libcuda.  Any failure leaves the engine on ordinary streams.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>

#include "sca_internal.h"

namespace sca {
namespace {

struct GreenApi {
  CUresult (*device_get)(CUdevice*, int) = nullptr;
  CUresult (*get_resource)(CUdevice, CUdevResource*, CUdevResourceType) = nullptr;
  CUresult (*split)(CUdevResource*, unsigned*, const CUdevResource*, CUdevResource*, unsigned,
                    unsigned) = nullptr;
  CUresult (*make_desc)(CUdevResourceDesc*, CUdevResource*, unsigned) = nullptr;
  CUresult (*ctx_create)(CUgreenCtx*, CUdevResourceDesc, CUdevice, unsigned) = nullptr;
  CUresult (*stream_create)(CUstream*, CUgreenCtx, unsigned, int) = nullptr;
  CUresult (*ctx_destroy)(CUgreenCtx) = nullptr;
  CUresult (*stream_destroy)(CUstream) = nullptr;
  bool ok = false;
};

template <typename F>
bool entry(const char* name, F& fn) {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &p, 12080, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !p) {
    (void)cudaGetLastError();
    return false;
  }
  fn = reinterpret_cast<F>(p);
  return true;
}

const GreenApi& api() {
  static GreenApi a = [] {
    GreenApi g;
    g.ok = entry("cuDeviceGet", g.device_get) && entry("cuDeviceGetDevResource", g.get_resource) &&
           entry("cuDevSmResourceSplitByCount", g.split) &&
           entry("cuDevResourceGenerateDesc", g.make_desc) &&
           entry("cuGreenCtxCreate", g.ctx_create) &&
           entry("cuGreenCtxStreamCreate", g.stream_create) &&
           entry("cuGreenCtxDestroy", g.ctx_destroy) && entry("cuStreamDestroy", g.stream_destroy);
    return g;
  }();
  return a;
}

__global__ void k_partition_probe(int* flag) {
  if (threadIdx.x == 0) *flag = 1;
}

}  // namespace

namespace {

// A green context over all SMs but `free_sms` and two streams on it (probed with one launch
// each and joined back to `join`).  False leaves nothing behind.
bool make_rest_ctx(int free_sms, cudaStream_t join, int* flag, CUgreenCtx* ctx, CUstream* s0,
                   CUstream* s1, int* rest_sms) {
  const GreenApi& g = api();
  int ordinal = 0;
  if (cudaGetDevice(&ordinal) != cudaSuccess) return false;
  CUdevice dev;
  CUdevResource all, part, rest;
  std::memset(&all, 0, sizeof(all));
  std::memset(&part, 0, sizeof(part));
  std::memset(&rest, 0, sizeof(rest));
  unsigned groups = 1;
  if (g.device_get(&dev, ordinal) != CUDA_SUCCESS) return false;
  if (g.get_resource(dev, &all, CU_DEV_RESOURCE_TYPE_SM) != CUDA_SUCCESS) return false;
  if ((unsigned)free_sms >= all.sm.smCount) return false;
  if (g.split(&part, &groups, &all, &rest, 0, (unsigned)free_sms) != CUDA_SUCCESS || groups != 1 ||
      rest.sm.smCount == 0)
    return false;
  CUdevResourceDesc dd = nullptr;
  if (g.make_desc(&dd, &rest, 1) != CUDA_SUCCESS) return false;
  CUgreenCtx gd = nullptr;
  CUstream a = nullptr, b = nullptr;
  bool good = g.ctx_create(&gd, dd, dev, CU_GREEN_CTX_DEFAULT_STREAM) == CUDA_SUCCESS;
  good = good && g.stream_create(&a, gd, CU_STREAM_NON_BLOCKING, 0) == CUDA_SUCCESS;
  good = good && g.stream_create(&b, gd, CU_STREAM_NON_BLOCKING, 0) == CUDA_SUCCESS;
  cudaEvent_t ev = nullptr;
  good = good && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
  for (CUstream st : {a, b}) {
    if (!good) break;
    k_partition_probe<<<1, 32, 0, (cudaStream_t)st>>>(flag);
    good = cudaGetLastError() == cudaSuccess && cudaEventRecord(ev, (cudaStream_t)st) == cudaSuccess &&
           cudaStreamWaitEvent(join, ev, 0) == cudaSuccess &&
           cudaStreamSynchronize(join) == cudaSuccess &&
           cudaStreamSynchronize((cudaStream_t)st) == cudaSuccess;
  }
  if (ev) cudaEventDestroy(ev);
  if (good) good = cudaMemset(flag, 0, sizeof(int)) == cudaSuccess;
  if (!good) {
    (void)cudaGetLastError();
    for (CUstream st : {a, b})
      if (st) g.stream_destroy(st);
    if (gd) g.ctx_destroy(gd);
    return false;
  }
  *ctx = gd;
  *s0 = a;
  *s1 = b;
  *rest_sms = (int)rest.sm.smCount;
  return true;
}

}  // namespace

bool partition_setup(Engine& e, int piv_sms, int mode) {
  const GreenApi& g = api();
  if (!g.ok || piv_sms <= 0 || (mode != 1 && mode != 2 && mode != 3)) return false;
  if (mode == 3) {
    // mode 1, plus a second dominant partition with twice the free SMs for odd steps
    if (!partition_setup(e, piv_sms, 1)) return false;
    CUgreenCtx ga = nullptr;
    CUstream sa = nullptr, sb = nullptr;
    int rest = 0;
    if (cudaEventCreateWithFlags(&e.ev_alt, cudaEventDisableTiming) != cudaSuccess ||
        !make_rest_ctx(2 * e.part_sms[0], e.side, e.flags + 1, &ga, &sa, &sb, &rest) ||
        rest >= e.part_sms[1]) {
      (void)cudaGetLastError();
      if (ga) g.ctx_destroy(ga);
      partition_release(e);
      return false;
    }
    e.green_alt = ga;
    e.dom_alt = (cudaStream_t)sa;
    e.aux_alt = (cudaStream_t)sb;
    e.alt_sms = rest;
    return true;
  }
  int ordinal = 0;
  if (cudaGetDevice(&ordinal) != cudaSuccess) return false;
  CUdevice dev;
  CUdevResource all, part, rest;
  std::memset(&all, 0, sizeof(all));
  std::memset(&part, 0, sizeof(part));
  std::memset(&rest, 0, sizeof(rest));
  unsigned groups = 1;
  if (g.device_get(&dev, ordinal) != CUDA_SUCCESS) return false;
  if (g.get_resource(dev, &all, CU_DEV_RESOURCE_TYPE_SM) != CUDA_SUCCESS) return false;
  if ((unsigned)piv_sms >= all.sm.smCount) return false;
  if (g.split(&part, &groups, &all, &rest, 0, (unsigned)piv_sms) != CUDA_SUCCESS || groups != 1 ||
      rest.sm.smCount == 0)
    return false;
  CUdevResourceDesc dp = nullptr, dd = nullptr;
  if (g.make_desc(&dp, &part, 1) != CUDA_SUCCESS || g.make_desc(&dd, &rest, 1) != CUDA_SUCCESS)
    return false;
  CUgreenCtx gp = nullptr, gd = nullptr;
  CUstream sd = nullptr, sa = nullptr, sp = nullptr;
  int least = 0, greatest = 0;
  bool good = cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess;
  good = good && g.ctx_create(&gd, dd, dev, CU_GREEN_CTX_DEFAULT_STREAM) == CUDA_SUCCESS;
  good = good && g.stream_create(&sd, gd, CU_STREAM_NON_BLOCKING, 0) == CUDA_SUCCESS;
  good = good && g.stream_create(&sa, gd, CU_STREAM_NON_BLOCKING, 0) == CUDA_SUCCESS;
  if (good && mode == 2) {
    good = g.ctx_create(&gp, dp, dev, CU_GREEN_CTX_DEFAULT_STREAM) == CUDA_SUCCESS &&
           g.stream_create(&sp, gp, CU_STREAM_NON_BLOCKING, greatest) == CUDA_SUCCESS;
  }
  // one launch and one event on each new stream, joined back to an ordinary stream
  cudaEvent_t ev = nullptr;
  good = good && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
  for (CUstream s : {sd, sa, sp}) {
    if (!good || !s) continue;
    k_partition_probe<<<1, 32, 0, (cudaStream_t)s>>>(e.flags + 1);
    good = cudaGetLastError() == cudaSuccess &&
           cudaEventRecord(ev, (cudaStream_t)s) == cudaSuccess &&
           cudaStreamWaitEvent(e.side, ev, 0) == cudaSuccess &&
           cudaStreamSynchronize(e.side) == cudaSuccess &&
           cudaStreamSynchronize((cudaStream_t)s) == cudaSuccess;
  }
  if (ev) cudaEventDestroy(ev);
  if (good) good = cudaMemset(e.flags + 1, 0, sizeof(int)) == cudaSuccess;
  if (!good) {
    (void)cudaGetLastError();
    for (CUstream s : {sd, sa, sp})
      if (s) g.stream_destroy(s);
    if (gd) g.ctx_destroy(gd);
    if (gp) g.ctx_destroy(gp);
    return false;
  }
  e.green[0] = gp;
  e.green[1] = gd;
  e.dom = (cudaStream_t)sd;
  e.part_aux = (cudaStream_t)sa;
  e.part_side = (cudaStream_t)sp;
  e.part_sms[0] = (int)part.sm.smCount;
  e.part_sms[1] = (int)rest.sm.smCount;
  return true;
}

void partition_release(Engine& e) {
  const GreenApi& g = api();
  if (!g.ok) return;
  for (cudaStream_t* st : {&e.dom_alt, &e.aux_alt})
    if (*st) {
      cudaStreamSynchronize(*st);
      g.stream_destroy((CUstream)*st);
      *st = nullptr;
    }
  if (e.green_alt) {
    g.ctx_destroy((CUgreenCtx)e.green_alt);
    e.green_alt = nullptr;
  }
  if (e.ev_alt) {
    cudaEventDestroy(e.ev_alt);
    e.ev_alt = nullptr;
  }
  e.alt_sms = 0;
  e.alt_on = false;
  for (cudaStream_t* s : {&e.dom, &e.part_aux, &e.part_side})
    if (*s) {
      cudaStreamSynchronize(*s);
      g.stream_destroy((CUstream)*s);
      *s = nullptr;
    }
  for (void*& c : e.green)
    if (c) {
      g.ctx_destroy((CUgreenCtx)c);
      c = nullptr;
    }
  e.part_sms[0] = e.part_sms[1] = 0;
}

}  // namespace sca
