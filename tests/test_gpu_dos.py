"""GPU density of states (the DOS equation of Sec. II) against the FP64 oracle.

rho_sigma(w) = -(1/(pi N)) Im Tr[(w + i eta + mu) - H_sigma(phi)]^-1 through the same batched
elimination as the gradient.  Tolerances: float64 path 1e-10 of max rho; the float32 paths
take Im G_ii from the float32 inverse without refinement, whose error is about
kappa(A) * 2^-24 with kappa(A) <= (|w| + 4|t| + max|h_i|) / eta; 2e-5 of max rho covers
kappa <= 100 with a margin.
"""
import numpy as np
import pytest

import oracle
from paper_2311_04435_gb300 import _lib, api, inputs

pytestmark = pytest.mark.gpu


def oparams(p: api.Params):
    return oracle.make_params(p.L, p.n_omega, U=p.U, T=p.T, delta=p.delta, t=p.t, mu=p.mu,
                              ionic=0 if p.ionic == "paper" else 1)


def tol(prec):
    return 1e-10 if prec == "fp64" else 2e-5


@pytest.mark.parametrize("prec", ["fp64", "fp32", "3xtf32", "bf16x3"])
@pytest.mark.parametrize("L,nw,n_w,eta", [(4, 3, 7, 0.1), (10, 4, 9, 0.2), (20, 6, 13, 0.15)])
def test_dos_matches_oracle(prec, L, nw, n_w, eta):
    """Several batches of n_omega frequencies with a short last one; random field plus
    random site energies; blocks of 16, 100 (ragged panels) and 400 (four tiles)."""
    p = api.Params(L, nw, U=4.0, T=0.1, delta=0.6, mu=0.1, prec=prec)
    phi = inputs.random_phi(30 + L, p.N, 1.2)
    ee = inputs.random_phi(40 + L, p.N, 0.4)
    w = np.linspace(-5.5, 5.5, n_w)
    with api.Context(p) as c:
        c.set_site_energy(ee)
        rho = c.dos(phi, w, eta)
    op = oparams(p)
    ref = np.stack([oracle.dos(op, phi, s, w, eta, eps_extra=ee) for s in (1, -1)])
    assert np.max(np.abs(rho - ref)) <= tol(prec) * np.abs(ref).max()


@pytest.mark.parametrize("prec", ["fp64", "3xtf32"])
def test_dos_dominant_and_unpivoted(prec):
    """eta > 4|t| makes every resolvent column diagonally dominant (no pivot search, the
    symmetric update on the tensor cores); SCA_PIVOT_NONE drops the search at small eta."""
    p = api.Params(20, 3, U=4.0, T=0.1, delta=1.0, prec=prec)
    phi = inputs.seed_phi(7, p.N)
    w = np.linspace(-4.0, 4.0, 6)
    op = oparams(p)
    with api.Context(p) as c:
        big = c.dos(phi, w, 4.5)
        c.set_pivoting("none")
        small = c.dos(phi, w, 0.3)
    for eta, got in ((4.5, big), (0.3, small)):
        ref = np.stack([oracle.dos(op, phi, s, w, eta) for s in (1, -1)])
        assert np.max(np.abs(got - ref)) <= tol(prec) * np.abs(ref).max()


def test_dos_staggered_field_spin_split():
    """A staggered field phi_i = phi s_i gives each spin the ionic DOS with Delta + sigma phi
    (closed form), so the spins differ; checked on the float64 path."""
    L, delta, ph = 6, 0.5, 1.1
    p = api.Params(L, 2, U=4.0, T=0.1, delta=delta, prec="fp64")
    x, y = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    s = np.where((x + y) % 2 == 0, 1.0, -1.0).reshape(-1)
    w = np.linspace(-5.0, 5.0, 11)
    k = 2.0 * np.pi * np.arange(L) / L
    kx, ky = np.meshgrid(k, k, indexing="ij")
    ek = (-2.0 * (np.cos(kx) + np.cos(ky))).reshape(-1)
    with api.Context(p) as c:
        rho = c.dos(ph * s, w, 0.2)
    for row, sg in ((0, 1), (1, -1)):
        e = np.sqrt(ek ** 2 + (delta + sg * ph) ** 2)
        lor = 0.2 / ((w[:, None] - e) ** 2 + 0.04) + 0.2 / ((w[:, None] + e) ** 2 + 0.04)
        ref = 0.5 * lor.sum(axis=1) / (np.pi * L * L)
        assert np.allclose(rho[row], ref, rtol=1e-10, atol=1e-13)
    assert np.max(np.abs(rho[0] - rho[1])) > 1e-3


def test_dos_rejects_bad_arguments():
    p = api.Params(4, 2, U=4.0, T=0.1, prec="fp64")
    phi = np.zeros(p.N)
    w = np.array([0.0, 1.0])
    out = np.zeros(4)
    dp = lambda a: a.ctypes.data_as(_lib._dp)
    with api.Context(p) as c:
        for eta, n in ((0.0, 2), (-1.0, 2), (float("nan"), 2), (0.1, 0)):
            assert _lib.lib().sca_dos(c.handle, dp(phi), dp(w), n, eta, dp(out)) == 1
        bad = np.array([0.0, np.inf])
        assert _lib.lib().sca_dos(c.handle, dp(phi), dp(bad), 2, 0.1, dp(out)) == 1
        assert np.all(np.isfinite(c.dos(phi, w, 0.1)))  # the context is still usable
