"""Python binding of the SCA+ADAM C ABI (include/sca.h): argument marshalling only.

Every evaluation runs in the CUDA kernels of ``libsca_gb300.so``; PyTorch is used only
for device memory and streams in the ``*_dev`` helpers and the autograd Function.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _lib
from ._lib import CAdam, CParams, check

_dp = ctypes.POINTER(ctypes.c_double)


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class Params:
    """Physical parameters (Eq. 1 lattice L x L, n_omega positive Matsubara frequencies)."""

    L: int
    n_omega: int
    U: float
    T: float
    delta: float = 0.0
    t: float = 1.0
    mu: float = 0.0
    prec: str = "fp64"        # "fp64" | "fp32" | "3xtf32" | "bf16x3"
    ionic: str = "paper"      # "paper" (-/+Delta) | "half" (-/+Delta/2)

    @property
    def N(self) -> int:
        return self.L * self.L

    def c(self) -> CParams:
        return CParams(int(self.L), int(self.n_omega), _lib.PREC[self.prec], _lib.IONIC[self.ionic],
                       float(self.t), float(self.U), float(self.delta), float(self.T), float(self.mu))


@dataclass
class AdamConfig:
    lr: float = 0.01
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    grad_tol: float = 0.0
    max_steps: int = 1000
    seed: int = 0

    def c(self) -> CAdam:
        return CAdam(float(self.lr), float(self.beta1), float(self.beta2), float(self.eps),
                     float(self.grad_tol), int(self.max_steps), ctypes.c_uint64(self.seed).value)


def workspace_bytes(params: Params) -> int:
    out = ctypes.c_uint64(0)
    check(_lib.lib().sca_workspace_bytes(ctypes.byref(params.c()), ctypes.byref(out)))
    return int(out.value)


def flops_per_grad(params: Params) -> float:
    return float(_lib.lib().sca_flops_per_grad(ctypes.byref(params.c())))


def pivoted_blocks(params: Params) -> int:
    return int(_lib.lib().sca_pivoted_blocks(ctypes.byref(params.c())))


def kernel_launches() -> int:
    return int(_lib.lib().sca_kernel_launches())


def version() -> str:
    return _lib.lib().sca_version().decode()


class Context:
    """One parameter set with its device workspace (sca_create / sca_destroy)."""

    def __init__(self, params: Params):
        self.params = params
        self.N = params.N
        self.B = 2 * params.n_omega
        self._h = ctypes.c_void_p()
        self._gen = 0       # bumped by every call that runs work on the context
        self._kept = -1     # generation whose inverses are resident (forward_dev)
        check(_lib.lib().sca_create(ctypes.byref(params.c()), ctypes.byref(self._h)))

    def _bump(self):
        self._gen += 1
        return self._gen

    def close(self):
        if self._h:
            _lib.lib().sca_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def set_site_energy(self, eps_extra=None):
        self._bump()
        if eps_extra is None:
            check(_lib.lib().sca_set_site_energy(self._h, None))
        else:
            e = _f64(eps_extra)
            assert e.shape == (self.N,)
            check(_lib.lib().sca_set_site_energy(self._h, _ptr(e)))

    def potential(self, phi) -> float:
        self._bump()
        phi = _f64(phi)
        om = ctypes.c_double()
        check(_lib.lib().sca_potential(self._h, _ptr(phi), ctypes.byref(om)))
        return om.value

    def grad(self, phi):
        self._bump()
        phi = _f64(phi)
        om = ctypes.c_double()
        g = np.zeros(self.N)
        check(_lib.lib().sca_grad(self._h, _ptr(phi), ctypes.byref(om), _ptr(g)))
        return om.value, g

    def dos(self, phi, w, eta: float):
        """Density of states rho_sigma(w) = -(1/(pi N)) Im Tr[(w + i eta + mu) - H_sigma]^-1
        (Sec. II): returns an array (2, len(w)), spin up first."""
        self._bump()
        phi = _f64(phi)
        w = _f64(w)
        assert phi.shape == (self.N,) and w.ndim == 1 and len(w) > 0
        out = np.zeros(2 * len(w))
        check(_lib.lib().sca_dos(self._h, _ptr(phi), _ptr(w), len(w), float(eta), _ptr(out)))
        return out.reshape(2, len(w))

    def metropolis_init(self, delta: float, seed: int = 0, phi0=None):
        """Start a Metropolis chain on exp(-Omega/T) (Sec. II) at phi0 (or the seeded field)."""
        self._bump()
        p = None if phi0 is None else _f64(phi0)
        check(_lib.lib().sca_metropolis_init(self._h, None if p is None else _ptr(p),
                                             float(delta), ctypes.c_uint64(seed).value))

    def metropolis_step(self, n_steps: int):
        """n_steps further steps: (Omega trace, accept flags, final Omega, accepted since init)."""
        self._bump()
        om_tr = np.zeros(max(n_steps, 1))
        acc = np.zeros(max(n_steps, 1), dtype=np.uint8)
        om = ctypes.c_double()
        tot = ctypes.c_int64()
        check(_lib.lib().sca_metropolis_step(
            self._h, int(n_steps), _ptr(om_tr), acc.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
            ctypes.byref(om), ctypes.byref(tot)))
        return om_tr[:n_steps], acc[:n_steps].astype(bool), om.value, int(tot.value)

    def blocks(self, phi, grad: bool = True):
        """Per block b = 2n+s: ln|det A_b| and (grad) sigma_b Re G_b,ii."""
        self._bump()
        phi = _f64(phi)
        ld = np.zeros(self.B)
        gd = np.zeros((self.B, self.N)) if grad else None
        check(_lib.lib().sca_blocks(self._h, _ptr(phi), _ptr(ld), _ptr(gd) if grad else None))
        return (ld, gd) if grad else ld

    def assemble(self, phi, b0: int = 0, count: int = 1) -> np.ndarray:
        self._bump()
        phi = _f64(phi)
        out = np.zeros((count, self.N, self.N, 2))
        check(_lib.lib().sca_debug_assemble(self._h, _ptr(phi), int(b0), int(count), _ptr(out)))
        return out[..., 0] + 1j * out[..., 1]

    # ---- device-pointer entry points (torch tensors, current stream)
    @staticmethod
    def _stream():
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def potential_dev(self, phi_t, out_t=None):
        import torch
        self._bump()
        assert phi_t.is_cuda and phi_t.dtype == torch.float64 and phi_t.is_contiguous()
        out = out_t if out_t is not None else torch.empty(1, dtype=torch.float64, device=phi_t.device)
        check(_lib.lib().sca_potential_dev(self._h, ctypes.c_void_p(phi_t.data_ptr()),
                                           ctypes.c_void_p(out.data_ptr()), self._stream()))
        return out

    def grad_dev(self, phi_t, omega_t=None, grad_t=None):
        import torch
        self._bump()
        assert phi_t.is_cuda and phi_t.dtype == torch.float64 and phi_t.is_contiguous()
        om = omega_t if omega_t is not None else torch.empty(1, dtype=torch.float64, device=phi_t.device)
        g = grad_t if grad_t is not None else torch.empty_like(phi_t)
        check(_lib.lib().sca_grad_dev(self._h, ctypes.c_void_p(phi_t.data_ptr()),
                                      ctypes.c_void_p(om.data_ptr()), ctypes.c_void_p(g.data_ptr()),
                                      self._stream()))
        return om, g

    def forward_dev(self, phi_t, omega_t) -> int:
        """Omega via the inversion; returns the generation whose inverses stay resident."""
        gen = self._bump()
        check(_lib.lib().sca_forward_dev(self._h, ctypes.c_void_p(phi_t.data_ptr()),
                                         ctypes.c_void_p(omega_t.data_ptr()), self._stream()))
        self._kept = gen
        return gen

    def backward_dev(self, phi_t, grad_t, gen: int | None = None):
        """Adjoint stage from the resident inverses of generation `gen` (default: the
        latest forward_dev).  Raises SCAError(SCA_ENOSTATE) if they are gone."""
        if gen is not None and (gen != self._gen or self._kept != gen):
            raise _lib.SCAError(_lib.SCA_ENOSTATE, "inverses of that forward are no longer resident")
        self._bump()
        self._kept = -1
        check(_lib.lib().sca_backward_dev(self._h, ctypes.c_void_p(phi_t.data_ptr()),
                                          ctypes.c_void_p(grad_t.data_ptr()), self._stream()))

    # ---- streams and per-kernel timing
    KINDS = ["assemble", "panel", "swap", "trinv", "prep", "update", "refine", "reduce", "diag",
             "update_piv", "fused", "span_pivoted", "span_dominant", "panel_update", "prep_piv",
             "update_cross"]

    def set_stream(self, stream=None):
        """Enqueue on a torch.cuda.Stream (or raw handle); None restores the own stream."""
        h = None if stream is None else getattr(stream, "cuda_stream", stream)
        check(_lib.lib().sca_set_stream(self._h, ctypes.c_void_p(h) if h else None))

    def set_wait_limit(self, cycles: int = 0):
        """Bound (SM cycles) of device-side spin waits; 0 restores the default."""
        check(_lib.lib().sca_set_wait_limit(self._h, int(cycles)))

    def set_pivoting(self, mode: str = "partial"):
        """'partial': partial pivoting where diagonal dominance is not guaranteed (default);
        'none': every block eliminated without interchanges (complex-symmetric elimination)."""
        modes = {"partial": 0, "none": 1}
        if mode not in modes:
            raise ValueError(f"pivoting mode must be one of {sorted(modes)}")
        check(_lib.lib().sca_set_pivoting(self._h, modes[mode]))

    def set_panel_precision(self, prec: str = "fp32"):
        """Arithmetic of the pivoted blocks' panel factorisation: 'fp32' (the blocks' compute
        type, default) or 'fp64' (float64 on the float32 blocks of the mixed path)."""
        if prec not in ("fp32", "fp64"):
            raise ValueError("panel precision must be 'fp32' or 'fp64'")
        check(_lib.lib().sca_set_panel_precision(self._h, _lib.PREC[prec]))

    def set_sm_partition(self, pivoted_sms: int = 0, mode: str = "dominant"):
        """Keep the dominant group's launches off `pivoted_sms` SMs (green contexts); mode
        'dominant' leaves the pivoted group free to use any SM, 'both' confines it to its
        set, 'alternate' is 'dominant' with the dominant group's pivot-block inverses and
        prep products on a second partition that leaves twice as many SMs free (the library's
        default where it sets one).  0 removes the partition.
        Returns the SM counts in use (pivoted, dominant)."""
        modes = {"dominant": 1, "both": 2, "alternate": 3}
        if mode not in modes:
            raise ValueError(f"partition mode must be one of {sorted(modes)}")
        check(_lib.lib().sca_set_sm_partition(self._h, int(pivoted_sms), modes[mode]))
        return self.sm_partition()

    def sm_partition(self):
        p, d = ctypes.c_int32(), ctypes.c_int32()
        check(_lib.lib().sca_sm_partition(self._h, ctypes.byref(p), ctypes.byref(d)))
        return p.value, d.value

    def profile(self, enable: bool = True):
        check(_lib.lib().sca_profile_enable(self._h, 1 if enable else 0))

    def profile_read(self) -> dict:
        out = {}
        for k, name in enumerate(self.KINDS):
            ms, n = ctypes.c_double(), ctypes.c_uint64()
            check(_lib.lib().sca_profile_read(self._h, k, ctypes.byref(ms), ctypes.byref(n)))
            out[name] = (ms.value, int(n.value))
        return out

    # ---- Adam state resident on the device
    def adam_init(self, adam: AdamConfig, phi0=None):
        self._bump()
        self._adam = adam
        if phi0 is None:
            check(_lib.lib().sca_adam_init(self._h, ctypes.byref(adam.c()), None))
        else:
            p = _f64(phi0)
            check(_lib.lib().sca_adam_init(self._h, ctypes.byref(adam.c()), _ptr(p)))

    def adam_step(self, nsteps: int = 1):
        self._bump()
        om, gm = ctypes.c_double(), ctypes.c_double()
        check(_lib.lib().sca_adam_step(self._h, int(nsteps), ctypes.byref(om), ctypes.byref(gm)))
        return om.value, gm.value

    def adam_run(self, max_steps: int):
        """Gated Adam until max|g| < grad_tol or max_steps updates (sca_adam_run): returns
        (updates applied, Omega, max|g|) at the final phi."""
        self._bump()
        om, gm = ctypes.c_double(), ctypes.c_double()
        steps = ctypes.c_int32()
        check(_lib.lib().sca_adam_run(self._h, int(max_steps), ctypes.byref(steps), ctypes.byref(om),
                                      ctypes.byref(gm)))
        return int(steps.value), om.value, gm.value

    def phi(self) -> np.ndarray:
        out = np.zeros(self.N)
        check(_lib.lib().sca_get_phi(self._h, _ptr(out)))
        return out

    def get_state(self):
        phi, m, v = np.zeros(self.N), np.zeros(self.N), np.zeros(self.N)
        step = ctypes.c_int32()
        check(_lib.lib().sca_get_state(self._h, _ptr(phi), _ptr(m), _ptr(v), ctypes.byref(step)))
        return {"phi": phi, "m": m, "v": v, "step": int(step.value)}

    def set_state(self, adam: AdamConfig, state: dict):
        self._bump()
        self._adam = adam
        check(_lib.lib().sca_set_state(self._h, ctypes.byref(adam.c()), _ptr(_f64(state["phi"])),
                                       _ptr(_f64(state["m"])), _ptr(_f64(state["v"])),
                                       int(state["step"])))


@dataclass
class SolveResult:
    phi: np.ndarray
    omega: float
    steps: int
    gmax: float


def solve(params: Params, adam: AdamConfig, phi0=None) -> SolveResult:
    """sca_solve: Adam from phi0 (None: SplitMix64 field of adam.seed) to convergence."""
    N = params.N
    phi = np.zeros(N)
    om, gm = ctypes.c_double(), ctypes.c_double()
    steps = ctypes.c_int32()
    p0 = None if phi0 is None else _ptr(_f64(phi0))
    check(_lib.lib().sca_solve(ctypes.byref(params.c()), ctypes.byref(adam.c()), p0, _ptr(phi),
                               ctypes.byref(om), ctypes.byref(steps), ctypes.byref(gm)))
    return SolveResult(phi, om.value, int(steps.value), gm.value)


# ------------------------------------------------------------------ autograd
def _make_function():
    import torch

    class SCAPotential(torch.autograd.Function):
        """Omega(phi) with the hand-written adjoint.  forward: Gauss-Jordan inversion of every
        block (sca_forward_dev; the inverses stay resident), backward: the adjoint stage
        diag(G) -> dOmega/dphi from those inverses (sca_backward_dev).  If the context ran
        anything else in between, backward recomputes through sca_grad_dev."""

        @staticmethod
        def forward(ctx, phi, handle):
            phi = phi.detach().contiguous()
            om = torch.empty(1, dtype=torch.float64, device=phi.device)
            if ctx.needs_input_grad[0]:
                ctx.gen = handle.forward_dev(phi, om)
                ctx.save_for_backward(phi)
                ctx.handle = handle
            else:
                handle.potential_dev(phi, om)
            return om[0]

        @staticmethod
        def backward(ctx, grad_out):
            (phi,) = ctx.saved_tensors
            g = torch.empty_like(phi)
            try:
                ctx.handle.backward_dev(phi, g, ctx.gen)
            except _lib.SCAError as err:
                if err.status != _lib.SCA_ENOSTATE:
                    raise
                ctx.handle.grad_dev(phi, grad_t=g)
            return grad_out * g, None

    return SCAPotential


_FN = None


def sca_potential(phi, handle: Context):
    """Differentiable Omega(phi) for a float64 CUDA tensor phi of N sites."""
    global _FN
    if _FN is None:
        _FN = _make_function()
    return _FN.apply(phi, handle)


# ------------------------------------------------------------------- serving
class Server:
    """Continuous-batching solve server (sca_server_*)."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 64, manual: bool = False):
        """manual=True: no worker thread; drive the rounds with step(now_s) (virtual clock)."""
        self._h = ctypes.c_void_p()
        create = _lib.lib().sca_server_create_manual if manual else _lib.lib().sca_server_create
        check(create(ctypes.c_uint64(int(hbm_budget_bytes)), int(max_slots), ctypes.byref(self._h)))

    def step(self, now_s: float):
        """One round of a manual server at virtual time now_s: (in flight, queued) after it."""
        fl, q = ctypes.c_int32(), ctypes.c_int32()
        check(_lib.lib().sca_server_step(self._h, float(now_s), ctypes.byref(fl), ctypes.byref(q)))
        return fl.value, q.value

    def submit(self, params: Params, adam: AdamConfig) -> int:
        rid = ctypes.c_uint64()
        check(_lib.lib().sca_submit(self._h, ctypes.byref(params.c()), ctypes.byref(adam.c()),
                                    ctypes.byref(rid)))
        return int(rid.value)

    def poll(self, req_id: int, N: int | None = None):
        """None while pending; SolveResult when done; raises on the request's error."""
        om, gm = ctypes.c_double(), ctypes.c_double()
        steps = ctypes.c_int32()
        phi = np.zeros(N) if N else None
        st = _lib.lib().sca_poll(self._h, ctypes.c_uint64(req_id), _ptr(phi) if N else None,
                                 ctypes.byref(om), ctypes.byref(steps), ctypes.byref(gm))
        if st == _lib.SCA_EPENDING:
            return None
        check(st)
        return SolveResult(phi, om.value, int(steps.value), gm.value)

    def times(self, req_id: int):
        v = [ctypes.c_double() for _ in range(4)]
        check(_lib.lib().sca_request_times(self._h, ctypes.c_uint64(req_id), *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def close(self):
        if self._h:
            _lib.lib().sca_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
