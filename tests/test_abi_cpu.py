"""CPU-side checks of the C ABI: the library builds, loads, exports every symbol that
include/sca.h declares, and rejects invalid arguments before touching a device."""
import ctypes
import os
import re

import pytest

from paper_2311_04435_gb300 import _lib, api, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "sca.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sca_[a-z0-9_]+)\s*\(", txt)))


def test_library_builds_and_loads():
    so = build.build()
    assert os.path.exists(so)
    l = _lib.lib()
    assert l.sca_version().decode().startswith("sca-gb300")


def test_every_declared_symbol_is_exported():
    names = declared_functions()
    assert len(names) >= 20
    l = ctypes.CDLL(_lib.SO_PATH)
    missing = [n for n in names if not hasattr(l, n)]
    assert not missing, missing
    # and the binding knows every one of them
    bound = {n for n, _, _ in _lib.SIGNATURES}
    assert set(names) <= bound, set(names) - bound


@pytest.mark.parametrize("kw", [dict(L=3), dict(L=0), dict(L=66), dict(n_omega=0), dict(U=0.0),
                                dict(T=-1.0), dict(U=float("nan")), dict(prec="bad")])
def test_invalid_params_rejected_without_device(kw):
    base = dict(L=4, n_omega=8, U=4.0, T=0.1)
    prec = kw.pop("prec", "fp64")
    base.update(kw)
    p = api.Params(**base)
    c = p.c() if prec != "bad" else p.c()
    if prec == "bad":
        c.prec = 7
    out = ctypes.c_uint64()
    st = _lib.lib().sca_workspace_bytes(ctypes.byref(c), ctypes.byref(out))
    assert st == _lib.SCA_EINVAL
    h = ctypes.c_void_p()
    assert _lib.lib().sca_create(ctypes.byref(c), ctypes.byref(h)) == _lib.SCA_EINVAL
    assert not h.value
    assert len(_lib.lib().sca_last_error()) > 0


def test_workspace_sizes_match_layout():
    # 40x40, 128 frequencies: 256 complex64 blocks of 1600^2 resident (5.2 GB) plus panels
    b32 = api.workspace_bytes(api.Params(40, 128, 4.0, 0.1, 1.0, prec="fp32"))
    b64 = api.workspace_bytes(api.Params(40, 128, 4.0, 0.1, 1.0, prec="fp64"))
    assert 256 * 1600 * 1600 * 8 < b32 < 1.2 * 256 * 1600 * 1600 * 8
    assert 256 * 1600 * 1600 * 16 < b64 < 1.2 * 256 * 1600 * 1600 * 16


def test_null_context_calls_fail_cleanly():
    l = _lib.lib()
    om = ctypes.c_double()
    assert l.sca_potential(None, None, ctypes.byref(om)) == _lib.SCA_EINVAL
    assert l.sca_adam_step(None, 1, None, None) == _lib.SCA_EINVAL
    l.sca_destroy(None)
    l.sca_server_destroy(None)
