"""The allocation-free gradient entry point (sca_grad_noalloc_dev) against sca_grad_dev.

sca_grad_noalloc_dev serves callers that cannot let the library allocate device memory
(for example a process whose device memory belongs to its own pool allocator).  Its
workspace is a static 64 MiB device array shared by every call, so the test checks two
calls in a row (the second sees the first call's leftovers), a problem large enough to be
processed in several chunks of that array, and the rejection of a problem whose single block
does not fit, a call after the device's context was re-created (the array's address
moves with the context), and, with the CUDA runtime's allocation calls counted by a
preloaded shim, that the calls themselves allocate nothing.  This file is collected last on
purpose.
"""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2311_04435_gb300 import _lib, api, inputs

pytestmark = pytest.mark.gpu


def _noalloc(params: api.Params, phi_t):
    import torch
    om = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    g = torch.full_like(phi_t, float("nan"))
    st = _lib.lib().sca_grad_noalloc_dev(ctypes.byref(params.c()), ctypes.c_void_p(phi_t.data_ptr()),
                                         ctypes.c_void_p(om.data_ptr()), ctypes.c_void_p(g.data_ptr()),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    _lib.check(st)
    torch.cuda.synchronize()
    return float(om.item()), g.cpu().numpy()


@pytest.mark.parametrize("L,nw,prec", [(4, 16, "fp64"), (8, 8, "fp32"), (10, 128, "fp64")])
def test_noalloc_matches_grad_dev_twice(L, nw, prec):
    torch = pytest.importorskip("torch")
    p = api.Params(L, nw, U=4.0, T=0.1, delta=0.5, prec=prec)
    rel_om, rel_g = (1e-10, 1e-10) if prec == "fp64" else (1e-5, 1e-7)
    with api.Context(p) as c:
        for seed in (1, 2):  # two calls in a row, different fields
            phi = inputs.random_phi(seed, p.N)
            x = torch.tensor(phi, dtype=torch.float64, device="cuda")
            om_ref, g_ref = c.grad_dev(x)
            torch.cuda.synchronize()
            om_ref, g_ref = float(om_ref.item()), g_ref.cpu().numpy()
            om, g = _noalloc(p, x)
            assert om == pytest.approx(om_ref, rel=rel_om)
            assert np.max(np.abs(g - g_ref)) <= rel_g * max(1.0, np.abs(g_ref).max())


def test_noalloc_rejects_problem_beyond_static_workspace():
    torch = pytest.importorskip("torch")
    p = api.Params(64, 4, U=4.0, T=0.1, prec="fp64")  # one 4096^2 complex128 block > 64 MiB
    x = torch.zeros(p.N, dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.SCAError, match="SCA_EINVAL"):
        _noalloc(p, x)
    msg = _lib.lib().sca_last_error().decode()
    assert "too large" in msg


_RESET_CHILD = r"""
import ctypes, os, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2311_04435_gb300 import _lib, api, inputs

lib = _lib.lib()
# the CUDA runtime the library is linked against (already loaded by it)
rt_path = next(ln.split()[-1] for ln in open("/proc/self/maps") if "libcudart.so" in ln)
rt = ctypes.CDLL(rt_path)
vp = ctypes.c_void_p

def ok(err, what):
    assert err == 0, f"{what}: CUDA error {err}"

def noalloc(p, phi):
    n = p.N
    d = [vp(), vp(), vp()]
    for k, size in enumerate((8 * n, 8, 8 * n)):
        ok(rt.cudaMalloc(ctypes.byref(d[k]), ctypes.c_size_t(size)), "cudaMalloc")
    ok(rt.cudaMemcpy(d[0], phi.ctypes.data_as(vp), ctypes.c_size_t(8 * n), 1), "upload")
    _lib.check(lib.sca_grad_noalloc_dev(ctypes.byref(p.c()), d[0], d[1], d[2], None))
    ok(rt.cudaDeviceSynchronize(), "sync")
    om, g = np.zeros(1), np.zeros(n)
    ok(rt.cudaMemcpy(om.ctypes.data_as(vp), d[1], ctypes.c_size_t(8), 2), "read Omega")
    ok(rt.cudaMemcpy(g.ctypes.data_as(vp), d[2], ctypes.c_size_t(8 * n), 2), "read grad")
    for x in d:
        ok(rt.cudaFree(x), "cudaFree")
    return float(om[0]), g

def reference(p, phi):
    with api.Context(p) as c:
        return c.grad(phi)

# 100 sites in float64: the pivoted blocks' panel kernel needs more than 48 KB of shared memory,
# an opt-in that belongs to the context as much as the array's address does
p = api.Params(10, 16, U=4.0, T=0.1, delta=0.5, prec="fp64")
for rnd in range(2):
    phi = inputs.random_phi(60 + rnd, p.N)
    om_ref, g_ref = reference(p, phi)
    om, g = noalloc(p, phi)
    assert abs(om - om_ref) <= 1e-10 * abs(om_ref), (rnd, om, om_ref)
    assert np.max(np.abs(g - g_ref)) <= 1e-10 * max(1.0, np.abs(g_ref).max()), rnd
    if rnd == 0:
        ok(rt.cudaDeviceReset(), "cudaDeviceReset")  # ends this process's context only
print("noalloc-after-reset ok")
"""


def test_noalloc_after_context_reset():
    """In a fresh process: a call, cudaDeviceReset (which re-creates the device's primary
    context, so the array's device address may change), and another call; both match the
    context path."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _RESET_CHILD, root], capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "noalloc-after-reset ok" in r.stdout


# Counts the CUDA runtime's allocating calls made through the dynamic linker (the library
# links libcudart dynamically) and forwards each to the runtime.
_SHIM_SRC = r"""
#define _GNU_SOURCE
#include <dlfcn.h>
#include <stddef.h>

static long g_calls;

long shim_alloc_calls(void) { return __atomic_load_n(&g_calls, __ATOMIC_SEQ_CST); }
void shim_reset(void) { __atomic_store_n(&g_calls, 0, __ATOMIC_SEQ_CST); }

static void* real_fn(const char* name) {
  void* fn = dlsym(RTLD_NEXT, name);
  if (!fn) {  /* the runtime came in with a library loaded RTLD_LOCAL */
    void* h = dlopen("libcudart.so.13", RTLD_NOLOAD | RTLD_LAZY);
    if (h) fn = dlsym(h, name);
  }
  return fn;
}

#define SHIM(name, params, args, types)                             \
  int name params {                                                 \
    __atomic_add_fetch(&g_calls, 1, __ATOMIC_SEQ_CST);              \
    int (*fn) types = (int (*) types)real_fn(#name);                \
    return fn ? fn args : 999; /* cudaErrorUnknown if not found */  \
  }

SHIM(cudaMalloc, (void** p, size_t n), (p, n), (void**, size_t))
SHIM(cudaFree, (void* p), (p), (void*))
SHIM(cudaMallocAsync, (void** p, size_t n, void* s), (p, n, s), (void**, size_t, void*))
SHIM(cudaFreeAsync, (void* p, void* s), (p, s), (void*, void*))
SHIM(cudaMallocManaged, (void** p, size_t n, unsigned fl), (p, n, fl), (void**, size_t, unsigned))
SHIM(cudaMallocPitch, (void** p, size_t* pitch, size_t w, size_t h), (p, pitch, w, h),
     (void**, size_t*, size_t, size_t))
SHIM(cudaMallocHost, (void** p, size_t n), (p, n), (void**, size_t))
SHIM(cudaHostAlloc, (void** p, size_t n, unsigned fl), (p, n, fl), (void**, size_t, unsigned))
SHIM(cudaFreeHost, (void* p), (p), (void*))
"""

_COUNT_CHILD = r"""
import ctypes, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2311_04435_gb300 import _lib, api, inputs

shim = ctypes.CDLL(sys.argv[2])  # the preloaded copy
shim.shim_alloc_calls.restype = ctypes.c_long
lib = _lib.lib()
rt_path = next(ln.split()[-1] for ln in open("/proc/self/maps") if "libcudart.so" in ln)
rt = ctypes.CDLL(rt_path)  # calls through this handle bypass the shim
vp = ctypes.c_void_p

def ok(err, what):
    assert err == 0, f"{what}: CUDA error {err}"

p = api.Params(10, 16, U=4.0, T=0.1, delta=0.5, prec="fp32")
n = p.N
d = [vp(), vp(), vp()]
for k, size in enumerate((8 * n, 8, 8 * n)):
    ok(rt.cudaMalloc(ctypes.byref(d[k]), ctypes.c_size_t(size)), "cudaMalloc")
phis = [inputs.random_phi(70 + k, n) for k in range(2)]
got = []
shim.shim_reset()
for phi in phis:  # the first call on this device and the one after it
    ok(rt.cudaMemcpy(d[0], phi.ctypes.data_as(vp), ctypes.c_size_t(8 * n), 1), "upload")
    _lib.check(lib.sca_grad_noalloc_dev(ctypes.byref(p.c()), d[0], d[1], d[2], None))
    ok(rt.cudaDeviceSynchronize(), "sync")
    om, g = np.zeros(1), np.zeros(n)
    ok(rt.cudaMemcpy(om.ctypes.data_as(vp), d[1], ctypes.c_size_t(8), 2), "read Omega")
    ok(rt.cudaMemcpy(g.ctypes.data_as(vp), d[2], ctypes.c_size_t(8 * n), 2), "read grad")
    got.append((float(om[0]), g))
calls = shim.shim_alloc_calls()
assert calls == 0, f"{calls} allocating runtime calls during sca_grad_noalloc_dev"
for phi, (om, g) in zip(phis, got):
    with api.Context(p) as c:
        om_ref, g_ref = c.grad(phi)
    assert abs(om - om_ref) <= 1e-5 * abs(om_ref), (om, om_ref)
    assert np.max(np.abs(g - g_ref)) <= 1e-7 * max(1.0, np.abs(g_ref).max())
# the context path allocates through the same runtime: the shim saw it
assert shim.shim_alloc_calls() > 0, "the shim did not intercept the runtime's allocation calls"
for x in d:
    ok(rt.cudaFree(x), "cudaFree")
print("noalloc-no-allocating-calls ok")
"""


def test_noalloc_makes_no_allocating_call(tmp_path):
    """In a fresh process whose CUDA runtime allocation calls (cudaMalloc, cudaFree and their
    async, managed, pitched and pinned-host forms) are counted by a preloaded shim: two calls
    of the entry point, the first one on the device included, make none of them, and their
    results match the context path, whose own allocations the shim does see."""
    shim = tmp_path / "libcount_alloc.so"
    src = tmp_path / "count_alloc.c"
    src.write_text(_SHIM_SRC)
    subprocess.run(["gcc", "-O1", "-shared", "-fPIC", "-o", str(shim), str(src), "-ldl"],
                   check=True)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, LD_PRELOAD=str(shim))
    r = subprocess.run([sys.executable, "-c", _COUNT_CHILD, root, str(shim)], capture_output=True,
                       text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "noalloc-no-allocating-calls ok" in r.stdout
