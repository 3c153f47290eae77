"""FP64 CPU oracle for the SCA+ADAM potential (arXiv 2311.04435, Eq. 1 and Eq. 2).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  The product package never imports it, and it imports nothing from the
product package except the seeded input generators (which hold none of the
method's arithmetic).

The arithmetic lives in ``sca_oracle.c`` (plain C, FP64, dense complex LU with
partial pivoting, explicit inverse columns, a Jacobi eigenvalue route and
explicit Adam); this file compiles it with gcc and exposes it through ctypes.
Every function documents the passage of the paper it follows in the C source.

A second, numpy-level route (``omega_grad_spectral`` / ``adam_run_spectral``) takes the
same Omega and gradient from the eigenvalues of H_sigma (LAPACK's symmetric eigensolver
through ``numpy.linalg.eigh`` as the library step): one diagonalisation per spin replaces
the n_omega LU factorisations, which lets the oracle run Adam to convergence on lattices
of 256..400 sites in seconds.

Parity status: every function here is pinned by tests in
``tests/test_oracle_pins.py`` (Fourier closed forms at phi = 0 and for a
staggered field, the eigenvalue route, finite differences, the Hartree-Fock
gap equation and the paper's printed critical ionic potentials).  The basin
reached by Adam from a random start has no closed form: it is pinned only
through the per-step quantities above ("parity unpinned" for the basin itself).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sca_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libsca_oracle.so")
_lock = threading.Lock()
_lib = None


class Params(ctypes.Structure):
    """Mirror of the physical parameters: lattice L, Matsubara count, precision
    tag (ignored by the oracle), ionic convention (0: -/+Delta as in Eq. 1,
    1: -/+Delta/2), hopping t, interaction U, ionic Delta, temperature T, mu."""

    _fields_ = [("L", ctypes.c_int32), ("n_omega", ctypes.c_int32), ("prec", ctypes.c_int32),
                ("ionic", ctypes.c_int32), ("t", ctypes.c_double), ("U", ctypes.c_double),
                ("delta", ctypes.c_double), ("T", ctypes.c_double), ("mu", ctypes.c_double)]


class Adam(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double), ("grad_tol", ctypes.c_double),
                ("max_steps", ctypes.c_int32), ("seed", ctypes.c_uint64)]


def build(force: bool = False) -> str:
    """Compile sca_oracle.c into _build/libsca_oracle.so (gcc, -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            l = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int32)
            P = ctypes.POINTER(Params)
            l.orc_hamiltonian.argtypes = [P, dp, dp, ctypes.c_int, dp]
            l.orc_omega_grad.argtypes = [P, dp, dp, dp, dp, dp, dp]
            l.orc_omega_grad.restype = ctypes.c_int
            l.orc_omega_grad_eig.argtypes = [P, dp, dp, dp, dp, dp, dp]
            l.orc_omega_grad_eig.restype = ctypes.c_int
            l.orc_block.argtypes = [P, dp, dp, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
            l.orc_block.restype = ctypes.c_int
            l.orc_blocks_sample.argtypes = [P, dp, dp, ctypes.c_int, ip, dp, dp]
            l.orc_blocks_sample.restype = ctypes.c_int
            l.orc_seed_phi.argtypes = [ctypes.c_uint64, ctypes.c_int, dp]
            l.orc_metropolis.argtypes = [P, dp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_uint64,
                                         ctypes.c_int64, dp, ip]
            l.orc_metropolis.restype = ctypes.c_int
            l.orc_metro_normal.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int, ctypes.c_int]
            l.orc_metro_normal.restype = ctypes.c_double
            for fn in (l.orc_dos, l.orc_dos_eig):
                fn.argtypes = [P, dp, dp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_double, dp]
                fn.restype = ctypes.c_int
            l.orc_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            l.orc_splitmix64.restype = ctypes.c_uint64
            l.orc_adam_run.argtypes = [P, dp, ctypes.POINTER(Adam), dp, dp, dp, ip, dp, dp]
            l.orc_adam_run.restype = ctypes.c_int
            l.orc_num_threads.restype = ctypes.c_int
            l.orc_omega_n.argtypes = [P, ctypes.c_int]
            l.orc_omega_n.restype = ctypes.c_double
            _lib = l
    return _lib


def _dp(a):
    if a is None:
        return ctypes.POINTER(ctypes.c_double)()
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_params(L, n_omega, U, T, delta=0.0, t=1.0, mu=0.0, ionic=0, prec=0) -> Params:
    return Params(int(L), int(n_omega), int(prec), int(ionic), float(t), float(U),
                  float(delta), float(T), float(mu))


def num_threads() -> int:
    return int(lib().orc_num_threads())


def hamiltonian(p: Params, phi, sigma: int, eps_extra=None) -> np.ndarray:
    N = p.L * p.L
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    H = np.zeros((N, N))
    ee = None if eps_extra is None else np.ascontiguousarray(eps_extra, dtype=np.float64)
    lib().orc_hamiltonian(ctypes.byref(p), _dp(ee), _dp(phi), int(sigma), _dp(H))
    return H


def omega_grad(p: Params, phi, eps_extra=None, per_block: bool = False):
    """Omega, dOmega/dphi by the LU route; with per_block, also ld[b] and
    sigma*Re G_ii[b, i] for every block b = 2n + s."""
    N, B = p.L * p.L, 2 * p.n_omega
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    ee = None if eps_extra is None else np.ascontiguousarray(eps_extra, dtype=np.float64)
    om = np.zeros(1)
    g = np.zeros(N)
    ld = np.zeros(B) if per_block else None
    gd = np.zeros((B, N)) if per_block else None
    rc = lib().orc_omega_grad(ctypes.byref(p), _dp(ee), _dp(phi), _dp(om), _dp(g), _dp(ld), _dp(gd))
    if rc != 0:
        raise FloatingPointError("oracle: singular block")
    if per_block:
        return float(om[0]), g, ld, gd
    return float(om[0]), g


def omega_only(p: Params, phi, eps_extra=None) -> float:
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    ee = None if eps_extra is None else np.ascontiguousarray(eps_extra, dtype=np.float64)
    om = np.zeros(1)
    rc = lib().orc_omega_grad(ctypes.byref(p), _dp(ee), _dp(phi), _dp(om), None, None, None)
    if rc != 0:
        raise FloatingPointError("oracle: singular block")
    return float(om[0])


def omega_grad_eig(p: Params, phi, eps_extra=None, per_block: bool = False):
    """Same quantities through the Jacobi eigenvalue route."""
    N, B = p.L * p.L, 2 * p.n_omega
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    ee = None if eps_extra is None else np.ascontiguousarray(eps_extra, dtype=np.float64)
    om = np.zeros(1)
    g = np.zeros(N)
    ld = np.zeros(B)
    gd = np.zeros((B, N))
    lib().orc_omega_grad_eig(ctypes.byref(p), _dp(ee), _dp(phi), _dp(om), _dp(g), _dp(ld), _dp(gd))
    if per_block:
        return float(om[0]), g, ld, gd
    return float(om[0]), g


def block(p: Params, phi, n: int, sigma: int, eps_extra=None, full: bool = False):
    """ln|det A_{n,sigma}|, G_ii (complex) and optionally the full inverse."""
    N = p.L * p.L
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    ee = None if eps_extra is None else np.ascontiguousarray(eps_extra, dtype=np.float64)
    ld = np.zeros(1)
    dre, dim = np.zeros(N), np.zeros(N)
    fb = np.zeros((N, N, 2)) if full else None
    rc = lib().orc_block(ctypes.byref(p), _dp(ee), _dp(phi), int(n), int(sigma), _dp(ld),
                         _dp(dre), _dp(dim), _dp(fb))
    if rc != 0:
        raise FloatingPointError("oracle: singular block")
    G = None if fb is None else fb[..., 0] + 1j * fb[..., 1]
    return float(ld[0]), dre + 1j * dim, G


def blocks_sample(p: Params, phi, blocks, eps_extra=None):
    """ld and sigma*Re G_ii for the listed blocks only (OpenMP over blocks)."""
    N = p.L * p.L
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    ee = None if eps_extra is None else np.ascontiguousarray(eps_extra, dtype=np.float64)
    bl = np.ascontiguousarray(blocks, dtype=np.int32)
    ld = np.zeros(len(bl))
    gd = np.zeros((len(bl), N))
    rc = lib().orc_blocks_sample(ctypes.byref(p), _dp(ee), _dp(phi), len(bl),
                                 bl.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(ld), _dp(gd))
    if rc != 0:
        raise FloatingPointError("oracle: singular block")
    return ld, gd


def dos(p: Params, phi, sigma: int, w, eta: float, eps_extra=None, route: str = "lu"):
    """rho_sigma(w) = -(1/(pi N)) Im Tr [(w + i eta + mu) - H_sigma(phi)]^{-1} at the
    frequencies w (the DOS equation of Sec. II); route "lu" (dense pivoted LU and inverse
    columns) or "eig" (Jacobi eigenvalues, a sum of Lorentzians)."""
    N = p.L * p.L
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    ee = None if eps_extra is None else np.ascontiguousarray(eps_extra, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    out = np.zeros(len(w))
    fn = lib().orc_dos if route == "lu" else lib().orc_dos_eig
    rc = fn(ctypes.byref(p), _dp(ee), _dp(phi), int(sigma), len(w), _dp(w), float(eta), _dp(out))
    if rc != 0:
        raise FloatingPointError("oracle: singular resolvent")
    return out


def metropolis(p: Params, phi0, n_steps: int, delta: float, seed: int, step0: int = 0,
               eps_extra=None):
    """Metropolis chain on exp(-Omega/T) from phi0 (Sec. II): returns (phi, Omega trace,
    accept flags) after n_steps steps numbered step0 .. step0 + n_steps - 1."""
    phi = np.array(phi0, dtype=np.float64, copy=True)
    ee = None if eps_extra is None else np.ascontiguousarray(eps_extra, dtype=np.float64)
    om = np.zeros(max(n_steps, 1))
    acc = np.zeros(max(n_steps, 1), dtype=np.int32)
    rc = lib().orc_metropolis(ctypes.byref(p), _dp(ee), _dp(phi), int(n_steps), float(delta),
                              ctypes.c_uint64(seed).value, int(step0), _dp(om),
                              acc.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if rc != 0:
        raise FloatingPointError("oracle: singular block")
    return phi, om[:n_steps], acc[:n_steps].astype(bool)


def metro_normal(seed: int, step: int, N: int, j: int) -> float:
    return float(lib().orc_metro_normal(ctypes.c_uint64(seed).value, int(step), int(N), int(j)))


def seed_phi(seed: int, N: int) -> np.ndarray:
    out = np.zeros(N)
    lib().orc_seed_phi(ctypes.c_uint64(seed), int(N), _dp(out))
    return out


def splitmix64(seed: int, k: int) -> int:
    return int(lib().orc_splitmix64(ctypes.c_uint64(seed), ctypes.c_uint64(k)))


def omega_n(p: Params, n: int) -> float:
    return float(lib().orc_omega_n(ctypes.byref(p), int(n)))


def adam_run(p: Params, lr=0.01, beta1=0.9, beta2=0.999, eps=1e-8, grad_tol=0.0, max_steps=100,
             seed=0, phi0=None, eps_extra=None, history: bool = False):
    """Adam from phi0 (or the seeded start).  Returns (phi, steps, Omega, max|g|)
    plus, with history, the per-step Omega and max|g| arrays."""
    N = p.L * p.L
    phi = seed_phi(seed, N) if phi0 is None else np.array(phi0, dtype=np.float64, copy=True)
    a = Adam(lr, beta1, beta2, eps, grad_tol, int(max_steps), ctypes.c_uint64(seed).value)
    oh = np.zeros(max(max_steps, 1)) if history else None
    gh = np.zeros(max(max_steps, 1)) if history else None
    steps = ctypes.c_int32(0)
    om, gm = np.zeros(1), np.zeros(1)
    ee = None if eps_extra is None else np.ascontiguousarray(eps_extra, dtype=np.float64)
    rc = lib().orc_adam_run(ctypes.byref(p), _dp(ee), ctypes.byref(a), _dp(phi), _dp(oh), _dp(gh),
                            ctypes.byref(steps), _dp(om), _dp(gm))
    if rc != 0:
        raise FloatingPointError("oracle: singular block")
    out = (phi, int(steps.value), float(om[0]), float(gm[0]))
    if history:
        return out + (oh[: steps.value + 1 if steps.value < max_steps else max_steps], gh[: steps.value + 1 if steps.value < max_steps else max_steps])
    return out


# ------------------------------------------------------------ spectral route (numpy)

def omega_grad_spectral(p: Params, phi, eps_extra=None):
    """Omega and dOmega/dphi from the eigen-decomposition H_sigma = V diag(e) V^T.

    Eq. 2 with a real symmetric H_sigma: det[(i w_n + mu) I - H_sigma] = prod_a (i w_n + mu - e_a),
    so with x_a = mu - e_a
        ln|det A_{n,sigma}| = 1/2 sum_a ln(w_n^2 + x_a^2),
        Re G_{n sigma, ii}  = sum_a V_ia^2 x_a / (w_n^2 + x_a^2),
    and Omega = sum_i phi_i^2/U - 2T sum_{n,sigma} ln|det A_{n,sigma}|,
        g_i = 2 phi_i/U - 2T sum_{n,sigma} sigma Re G_{n sigma, ii}
    (the n >= 0 half of the Matsubara sum with the factor 2, as in the LU route).  H_sigma is
    the LU route's own Eq. 1 matrix (orc_hamiltonian); numpy.linalg.eigh is the library step."""
    N = p.L * p.L
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    w = np.array([omega_n(p, n) for n in range(p.n_omega)])
    om = float(np.sum(phi * phi) / p.U)
    g = 2.0 * phi / p.U
    for sg in (1, -1):
        e, V = np.linalg.eigh(hamiltonian(p, phi, sg, eps_extra))
        x = p.mu - e
        den = w[None, :] ** 2 + x[:, None] ** 2          # (a, n)
        om -= 2.0 * p.T * 0.5 * float(np.log(den).sum())
        f = (x[:, None] / den).sum(axis=1)               # sum over n of Re 1/(i w_n + x_a)
        g -= 2.0 * p.T * sg * ((V * V) @ f)
    assert g.shape == (N,)
    return om, g


def adam_run_spectral(p: Params, phi0, lr=0.01, beta1=0.9, beta2=0.999, eps=1e-8, grad_tol=0.0,
                      max_steps=100, eps_extra=None):
    """Adam (Sec. II: ADAM on V(phi); Kingma & Ba 2014, PyTorch's arithmetic order, as
    orc_adam_run) on the spectral-route gradient, from phi0.  The loop evaluates Omega and g at
    phi_k, stops when max|g| < grad_tol or after max_steps updates, else applies update k+1.
    Returns (phi, updates applied, Omega and max|g| at the final phi)."""
    phi = np.array(phi0, dtype=np.float64, copy=True)
    m = np.zeros_like(phi)
    v = np.zeros_like(phi)
    k = 0
    while True:
        om, g = omega_grad_spectral(p, phi, eps_extra)
        gm = float(np.abs(g).max())
        if gm < grad_tol or k >= max_steps:
            break
        k += 1
        step = lr / (1.0 - beta1 ** k)
        sbc2 = math.sqrt(1.0 - beta2 ** k)
        m = beta1 * m + (1.0 - beta1) * g
        v = beta2 * v + (1.0 - beta2) * g * g
        phi -= step * m / (np.sqrt(v) / sbc2 + eps)
    return phi, k, om, gm


def staggered_order(phi, L: int):
    """The two readings of |phi| (the paper leaves the reduction open): the staggered
    magnetisation |N^-1 sum_i s_i phi_i| and the mean magnitude N^-1 sum_i |phi_i|."""
    x, y = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    s = np.where((x + y) % 2 == 0, 1.0, -1.0).reshape(-1)
    phi = np.asarray(phi, dtype=np.float64)
    return float(abs(np.mean(s * phi))), float(np.mean(np.abs(phi)))
