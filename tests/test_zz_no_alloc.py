"""The allocation-free gradient entry point (sca_grad_noalloc_dev) against sca_grad_dev.

sca_grad_noalloc_dev serves callers that cannot let the library allocate device memory
(for example a process whose device memory belongs to its own pool allocator).  Its
workspace is a static 64 MiB device array shared by every call, so the test checks two
calls in a row (the second sees the first call's leftovers), a problem large enough to be
processed in several chunks of that array, and the rejection of a problem whose single block
does not fit.  This file is collected last on purpose.
"""
import ctypes

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
