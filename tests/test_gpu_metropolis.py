"""GPU Metropolis chain on exp(-Omega/T) (Sec. II) against the oracle's chain.

Both sides draw from the same counter-based streams (SplitMix64 + Box-Muller for the
proposals, a second stream for the acceptance uniforms), each implemented independently, so
the float64 chain reproduces the oracle's step for step: same accept decisions, the same
states to rounding (1e-12) and Omega to 1e-10.  The mixed-precision chain is checked decision
by decision: every decision must agree with the oracle's Omega unless the acceptance uniform
lies within the mixed path's Omega error of the threshold.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2311_04435_gb300 import _lib, api, inputs

pytestmark = pytest.mark.gpu


def oparams(p: api.Params):
    return oracle.make_params(p.L, p.n_omega, U=p.U, T=p.T, delta=p.delta, t=p.t, mu=p.mu,
                              ionic=0 if p.ionic == "paper" else 1)


@pytest.mark.parametrize("L,nw,delta", [(4, 4, 0.15), (10, 3, 0.05)])
def test_fp64_chain_matches_oracle(L, nw, delta):
    p = api.Params(L, nw, U=4.0, T=0.2, delta=0.6, prec="fp64")
    phi0 = inputs.random_phi(60 + L, p.N, 0.7)
    op = oparams(p)
    with api.Context(p) as c:
        c.metropolis_init(delta, seed=17, phi0=phi0)
        om1, acc1, _, _ = c.metropolis_step(12)
        om2, acc2, om_end, tot = c.metropolis_step(12)  # the chain continues
        phi = c.phi()
    ophi, oom, oacc = oracle.metropolis(op, phi0, 24, delta, 17)
    acc = np.concatenate([acc1, acc2])
    assert np.array_equal(acc, oacc)
    assert 0 < acc.sum() < 24  # both outcomes exercised
    assert np.allclose(np.concatenate([om1, om2]), oom, rtol=1e-10, atol=0)
    assert np.allclose(phi, ophi, rtol=0, atol=1e-12)
    assert tot == acc.sum() and om_end == pytest.approx(oom[-1], rel=1e-10)


def test_mixed_chain_decisions_agree_with_oracle():
    """3xTF32 blocks of 400 x 400: each step's proposal is phi + delta g exactly (the device
    normals equal the oracle's), and each decision agrees with the oracle's Omega unless the
    uniform sits within the mixed path's Omega error (1e-5 relative) of the threshold."""
    p = api.Params(20, 4, U=4.0, T=0.2, delta=0.6, prec="3xtf32")
    op = oparams(p)
    phi = inputs.random_phi(77, p.N, 0.7)
    delta, seed = 0.004, 5
    with api.Context(p) as c:
        c.metropolis_init(delta, seed=seed, phi0=phi)
        om_cur = oracle.omega_grad(op, phi)[0]
        decided = 0
        for t in range(8):
            _, acc, _, _ = c.metropolis_step(1)
            new = c.phi()
            g = np.array([oracle.metro_normal(seed, t, p.N, i) for i in range(p.N)])
            prop = phi + delta * g
            if acc[0]:
                assert np.allclose(new, prop, rtol=1e-15, atol=1e-15)
            else:
                assert np.array_equal(new, phi)
            om_prop = oracle.omega_grad(op, prop)[0]
            u = (oracle.splitmix64(seed + 1, t) >> 11) * 2.0 ** -53
            thr = math.exp(min(0.0, -(om_prop - om_cur) / p.T))
            margin = 2e-5 * (abs(om_prop) + abs(om_cur)) / p.T * max(thr, 1e-300)
            if abs(u - thr) > margin:
                assert acc[0] == (u < thr)
                decided += 1
            if acc[0]:
                phi, om_cur = prop, om_prop
    assert decided >= 4


def test_metropolis_arguments_and_state():
    p = api.Params(4, 2, U=4.0, T=0.2, prec="fp64")
    with api.Context(p) as c:
        assert _lib.lib().sca_metropolis_step(c.handle, 1, None, None, None, None) == 9  # ENOSTATE
        assert _lib.lib().sca_metropolis_init(c.handle, None, -1.0, 0) == 1
        assert _lib.lib().sca_metropolis_init(c.handle, None, float("nan"), 0) == 1
        c.metropolis_init(0.0, seed=3)  # seeded start, zero step: every proposal accepted
        om, acc, om_end, tot = c.metropolis_step(5)
        assert acc.all() and tot == 5
        phi0 = oracle.seed_phi(3, p.N)
        assert np.array_equal(c.phi(), phi0)
        assert om_end == pytest.approx(oracle.omega_grad(oparams(p), phi0)[0], rel=1e-10)
