"""Adam to convergence on the GPU against the oracle's Adam from identical start bits.

Sec. II: the order parameter |phi| is the minimiser of V(phi) (Eq. 2) found by ADAM.  The
mixed-precision tolerances are those of the converged field: stag|phi| and mean|phi| within
1e-6 absolute of the oracle, Omega within 1e-5 relative, the number of updates to
max|g| < 1e-6 within 2.  The FP64 path must follow the oracle's trajectory to rounding: phi
within 1e-9, Omega within 1e-10 relative, the same number of updates (within 1, for the
evaluation that lands next to the gate).  The oracle here is the spectral route
(oracle.adam_run_spectral, pinned against the LU route and the staggered closed form), which
converges these 196- and 256-site lattices in seconds.
"""
import functools
import os

import numpy as np
import pytest

import oracle
from paper_2311_04435_gb300 import api, inputs

pytestmark = pytest.mark.gpu

TOL = 1e-6
MAX_STEPS = 3000

# name: (L, n_omega, U, Delta, T, start field, site-energy seed or None)
CASES = {
    # 256 sites, 12 pivoted + 116 dominant blocks (tensor-core path in the split precisions),
    # random site potential, perturbed Neel start: a non-uniform AF minimum
    "disorder_neel_16x16": (16, 64, 6.0, 0.5, 0.1, "neel", 11),
    # 196 sites (ragged 128-wide tiles), seed-0 random start: a domain-wall minimum
    "random_start_14x14": (14, 32, 6.0, 0.5, 0.1, "seed0", None),
    # the 64x64 workload's parameters on a 16x16 lattice (U = 6, Delta = 0.5, T = 0.2, 64
    # frequencies), seed-0 start
    "rerun_16x16_of_64x64": (16, 64, 6.0, 0.5, 0.2, "seed0", None),
}


def _start(kind, L):
    if kind == "neel":
        return inputs.neel_phi(L, 1.0) + 0.1 * inputs.seed_phi(7, L * L)
    return inputs.seed_phi(0, L * L)


def _ee(seed, N):
    return None if seed is None else inputs.random_phi(seed, N, 0.5)


@functools.lru_cache(maxsize=None)
def _oracle_run(name):
    L, nw, U, De, T, start, es = CASES[name]
    p = oracle.make_params(L, nw, U=U, T=T, delta=De)
    phi, k, om, gm = oracle.adam_run_spectral(p, _start(start, L), lr=0.01, grad_tol=TOL,
                                             max_steps=MAX_STEPS, eps_extra=_ee(es, L * L))
    assert gm < TOL, "the oracle did not converge"
    return phi, k, om, gm


@pytest.mark.parametrize("prec", ["bf16x3", "3xtf32", "fp64"])
@pytest.mark.parametrize("name", list(CASES))
def test_converged_field_matches_oracle(name, prec):
    L, nw, U, De, T, start, es = CASES[name]
    if prec == "fp64" and name != "disorder_neel_16x16":
        pytest.skip("the FP64 trajectory is checked on one case (float64 runs at 1/62 of float32)")
    phi_o, k_o, om_o, gm_o = _oracle_run(name)
    p = api.Params(L, nw, U=U, T=T, delta=De, prec=prec)
    with api.Context(p) as c:
        ee = _ee(es, p.N)
        if ee is not None:
            c.set_site_energy(ee)
        c.adam_init(api.AdamConfig(lr=0.01, grad_tol=TOL, max_steps=MAX_STEPS),
                    _start(start, L))
        k, om, gm = c.adam_run(MAX_STEPS)
        phi = c.phi()
    stag, mean = oracle.staggered_order(phi, L)
    stag_o, mean_o = oracle.staggered_order(phi_o, L)
    assert gm < TOL and k < MAX_STEPS
    if prec == "fp64":
        assert abs(k - k_o) <= 1
        assert np.max(np.abs(phi - phi_o)) < 1e-9
        assert om == pytest.approx(om_o, rel=1e-10)
    else:
        assert abs(k - k_o) <= 2
        assert abs(stag - stag_o) <= 1e-6 and abs(mean - mean_o) <= 1e-6
        assert om == pytest.approx(om_o, rel=1e-5)
        assert np.max(np.abs(phi - phi_o)) <= 1e-5  # every site, not only the averages


def _c2_reference():
    path = os.path.join(os.path.dirname(__file__), "golden", "c2_ionic_20x20_adam3000.txt")
    rows, phi = [], []
    with open(path) as f:
        lines = [ln for ln in f.read().splitlines() if ln and not ln.startswith("#")]
    for ln in lines:
        parts = ln.split()
        if len(parts) == 5:
            rows.append((int(parts[0]),) + tuple(float(x) for x in parts[1:]))
        else:
            phi.append(float(parts[0]))
    return rows, np.array(phi)


@pytest.mark.parametrize("prec", ["bf16x3", "3xtf32"])
def test_c2_20x20_3000_steps_against_oracle(prec):
    """The 20x20 workload (512 blocks of 400 x 400, U = 6, Delta = 0.5, T = 0.1, seed 0):
    3000 plain Adam updates in a mixed precision against the stored FP64 oracle run
    (tests/golden/c2_ionic_20x20_adam3000.txt, written by make_c2_reference.py) at 1000, 2000
    and 3000 updates."""
    rows, phi_ref = _c2_reference()
    wl = inputs.WORKLOADS["ionic_20x20"]
    p = api.Params(wl.L, wl.n_omega, U=wl.U, T=wl.T, delta=wl.delta, prec=prec)
    with api.Context(p) as c:
        c.adam_init(api.AdamConfig(lr=wl.lr, seed=wl.seed))
        done = 0
        for k, om_o, gm_o, stag_o, mean_o in rows:
            c.adam_step(k - done)
            done = k
            phi = c.phi()
            om, g = c.grad(phi)  # Omega at the field after k updates, as the reference
            stag, mean = oracle.staggered_order(phi, wl.L)
            assert om == pytest.approx(om_o, rel=1e-5)
            if k == rows[-1][0]:  # converged by then (max|g| ~ 1e-15 in the oracle)
                assert abs(stag - stag_o) <= 1e-6 and abs(mean - mean_o) <= 1e-6
                assert np.max(np.abs(phi - phi_ref)) <= 1e-5
                assert np.abs(g).max() < 1e-6
