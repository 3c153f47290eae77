"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, step by step.

Tolerances: float64 path <= 1e-10 relative in Omega and the gradient; reduced precisions
(complex64 blocks, float64 log-det accumulation and float64 refinement of diag(G))
<= 1e-5 relative in Omega; the refined gradient is checked at 1e-7 of max(1, |g|).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2311_04435_gb300 import _lib, api, inputs

pytestmark = pytest.mark.gpu

PRECS = ["fp64", "fp32", "3xtf32", "bf16x3"]


def oparams(p: api.Params):
    return oracle.make_params(p.L, p.n_omega, U=p.U, T=p.T, delta=p.delta, t=p.t, mu=p.mu,
                              ionic=0 if p.ionic == "paper" else 1)


def tol(prec):
    return dict(om=1e-10, ld=1e-10, g=1e-10) if prec == "fp64" else dict(om=1e-5, ld=2e-6, g=1e-7)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("L", [2, 4, 6])
def test_assemble_matches_oracle(prec, L):
    p = api.Params(L, 3, U=5.0, T=0.07, delta=0.4, mu=0.2, prec=prec, ionic="half")
    phi = inputs.random_phi(L, p.N, 1.3)
    with api.Context(p) as c:
        A = c.assemble(phi, 0, 2 * p.n_omega)
    op = oparams(p)
    for b in range(2 * p.n_omega):
        n, sg = b // 2, (1 if b % 2 == 0 else -1)
        H = oracle.hamiltonian(op, phi, sg)
        ref = (p.mu + 1j * oracle.omega_n(op, n)) * np.eye(p.N) - H
        if prec == "fp64":
            assert np.array_equal(A[b], ref)
        else:
            assert np.allclose(A[b], ref.astype(np.complex64), rtol=0, atol=0)


# sizes spanning several panels and a ragged tail (nb = 32 on CUDA cores, 64 on tensor cores)
CASES = [
    (2, 5, 0.0, 0.0),      # accumulated bonds, single tiny panel
    (4, 16, 0.0, 0.0),     # 16x16 blocks
    (6, 7, 0.7, 0.1),      # 36: ragged single panel
    (10, 5, 0.5, 0.0),     # 100: 3 full panels + ragged 4
    (12, 10, 1.0, -0.2),   # 144: 4.5 panels; 6 pivoted + 14 dominant blocks
    (14, 3, 0.5, 0.0),     # 196
]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("L,nw,delta,mu", CASES)
def test_blocks_logdet_and_diag_match_oracle(prec, L, nw, delta, mu):
    p = api.Params(L, nw, U=4.0, T=0.1, delta=delta, mu=mu, prec=prec)
    phi = inputs.random_phi(100 + L, p.N, 1.0)
    with api.Context(p) as c:
        ld, gd = c.blocks(phi, grad=True)
        om_lu = c.potential(phi)
        om, g = c.grad(phi)
    o_om, o_g, o_ld, o_gd = oracle.omega_grad(oparams(p), phi, per_block=True)
    t = tol(prec)
    assert np.allclose(ld, o_ld, rtol=t["ld"], atol=t["ld"])
    scale = max(1.0, np.abs(o_gd).max())
    assert np.max(np.abs(gd - o_gd)) <= t["g"] * scale
    assert om == pytest.approx(o_om, rel=t["om"])
    assert om_lu == pytest.approx(o_om, rel=t["om"])
    assert np.max(np.abs(g - o_g)) <= t["g"] * max(1.0, np.abs(o_g).max()) * 10


@pytest.mark.parametrize("prec", PRECS)
def test_larger_block_20x20_matches_oracle(prec):
    """400 x 400 blocks: pivoted (n < 6) and dominant (n >= 6) groups, ragged last panel."""
    p = api.Params(20, 8, U=6.0, T=0.1, delta=0.5, prec=prec)
    phi = inputs.seed_phi(0, p.N)
    with api.Context(p) as c:
        ld, gd = c.blocks(phi, grad=True)
    o_ld, o_gd = oracle.blocks_sample(oparams(p), phi, list(range(16)))
    t = tol(prec)
    assert np.allclose(ld, o_ld, rtol=t["ld"], atol=t["ld"])
    assert np.max(np.abs(gd - o_gd)) <= t["g"] * max(1.0, np.abs(o_gd).max())


@pytest.mark.parametrize("prec", ["bf16x3", "3xtf32"])
def test_many_dominant_blocks_match_oracle(prec):
    """80 blocks of 256 x 256 (12 pivoted, 68 dominant): Omega (gradient and LU-only passes)
    and the gradient match the oracle, and a repeated evaluation is bit-identical."""
    p = api.Params(16, 40, U=4.0, T=0.1, delta=0.5, prec=prec)
    assert 2 * p.n_omega - api.pivoted_blocks(p) >= 64
    phi = inputs.seed_phi(5, p.N)
    with api.Context(p) as c:
        om, g = c.grad(phi)
        om2, g2 = c.grad(phi)
        om_lu = c.potential(phi)
    o_om, o_g = oracle.omega_grad(oparams(p), phi)
    t = tol(prec)
    assert om == pytest.approx(o_om, rel=t["om"])
    assert om_lu == pytest.approx(o_om, rel=t["om"])
    assert np.max(np.abs(g - o_g)) <= t["g"] * max(1.0, np.abs(o_g).max()) * 10
    assert om2 == om and np.array_equal(g2, g)


@pytest.mark.parametrize("prec", PRECS)
def test_disorder_site_energy_and_half_convention(prec):
    p = api.Params(6, 6, U=3.0, T=0.2, delta=0.9, prec=prec, ionic="half")
    phi = inputs.random_phi(7, p.N)
    ee = inputs.random_phi(8, p.N, 0.5)
    with api.Context(p) as c:
        c.set_site_energy(ee)
        om, g = c.grad(phi)
    o_om, o_g = oracle.omega_grad(oparams(p), phi, eps_extra=ee)
    t = tol(prec)
    assert om == pytest.approx(o_om, rel=t["om"])
    assert np.max(np.abs(g - o_g)) <= 10 * t["g"] * max(1.0, np.abs(o_g).max())


def test_seeded_start_field_is_bit_exact():
    p = api.Params(8, 1, U=4.0, T=0.1)
    with api.Context(p) as c:
        for seed in (0, 1, 2**40 + 3):
            c.adam_init(api.AdamConfig(seed=seed))
            assert np.array_equal(c.phi(), inputs.seed_phi(seed, p.N))


def test_adam_trajectory_4x4_matches_oracle():
    """The 4x4 Hubbard workload (U=6, Delta=0, T=0.1, 64 frequencies: 128 blocks of 16 x 16,
    seed 0, lr=0.01) for its full 2000 Adam steps on the FP64 path: Omega, max|g|, phi and the
    two |phi| readings against the oracle's run."""
    wl = inputs.WORKLOADS["hubbard_4x4"]
    p = api.Params(wl.L, wl.n_omega, U=wl.U, T=wl.T, delta=wl.delta)
    steps = wl.steps
    assert steps == 2000
    ad = api.AdamConfig(lr=wl.lr, max_steps=steps, seed=wl.seed)
    phi_o, k, om_o, gm_o, oh, gh = oracle.adam_run(oparams(p), lr=wl.lr, max_steps=steps,
                                                   seed=wl.seed, history=True)
    with api.Context(p) as c:
        c.adam_init(ad)
        om1, gm1 = c.adam_step(1)
        assert om1 == pytest.approx(oh[0], rel=1e-12)
        assert gm1 == pytest.approx(gh[0], rel=1e-10)
        om, gm = c.adam_step(299)
        assert om == pytest.approx(oh[299], rel=1e-10)
        om, gm = c.adam_step(steps - 300)
        phi = c.phi()
        om_end, g_end = c.grad(phi)
    assert om == pytest.approx(oh[steps - 1], rel=1e-10)
    assert np.max(np.abs(phi - phi_o)) < 1e-9
    assert om_end == pytest.approx(om_o, rel=1e-10)
    assert abs(np.abs(g_end).max() - gm_o) <= 1e-10 * max(1.0, gm_o)
    stag, mean = oracle.staggered_order(phi, wl.L)
    stag_o, mean_o = oracle.staggered_order(phi_o, wl.L)
    assert abs(stag - stag_o) < 1e-9 and abs(mean - mean_o) < 1e-9


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_solve_semantics_match_oracle(prec):
    p = api.Params(4, 16, U=6.0, T=0.1, prec=prec)
    ad = api.AdamConfig(lr=0.02, grad_tol=1e-4, max_steps=700, seed=3)
    r = api.solve(p, ad)
    phi_o, k, om_o, gm_o = oracle.adam_run(oparams(p), lr=0.02, grad_tol=1e-4, max_steps=700, seed=3)
    if prec == "fp64":
        assert r.steps == k
        assert np.max(np.abs(r.phi - phi_o)) < 1e-9
        assert r.omega == pytest.approx(om_o, rel=1e-10)
    else:
        assert abs(r.steps - k) <= 2
        assert np.max(np.abs(r.phi - phi_o)) < 1e-5
        assert r.omega == pytest.approx(om_o, rel=1e-5)
    assert r.gmax < 1e-4 or r.steps == 700


def test_checkpoint_resume_is_bit_identical():
    p = api.Params(4, 8, U=4.0, T=0.2, delta=0.3)
    ad = api.AdamConfig(lr=0.01, seed=5)
    with api.Context(p) as a:
        a.adam_init(ad)
        a.adam_step(40)
        phi_ref = a.phi()
    with api.Context(p) as b:
        b.adam_init(ad)
        b.adam_step(15)
        st = b.get_state()
    with api.Context(p) as c:
        c.set_state(ad, st)
        c.adam_step(25)
        assert np.array_equal(c.phi(), phi_ref)


def test_nonfinite_phi_reported():
    p = api.Params(4, 4, U=4.0, T=0.1)
    phi = np.zeros(p.N)
    phi[3] = np.nan
    with api.Context(p) as c:
        with pytest.raises(Exception, match="SCA_ENONFINITE"):
            c.grad(phi)
        # the context stays usable
        om, g = c.grad(np.zeros(p.N))
        assert np.isfinite(om)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_autograd_function_matches_oracle_and_fd(prec):
    torch = pytest.importorskip("torch")
    p = api.Params(4, 8, U=4.0, T=0.1, delta=0.5, prec=prec)
    phi0 = inputs.random_phi(21, p.N)
    with api.Context(p) as c:
        x = torch.tensor(phi0, dtype=torch.float64, device="cuda", requires_grad=True)
        om = api.sca_potential(x, c)
        om.backward()
        g = x.grad.cpu().numpy()
        o_om, o_g = oracle.omega_grad(oparams(p), phi0)
        t = tol(prec)
        assert float(om) == pytest.approx(o_om, rel=t["om"])
        assert np.max(np.abs(g - o_g)) <= 10 * t["g"] * max(1.0, np.abs(o_g).max())
        if prec == "fp64":
            xx = torch.tensor(phi0[:], dtype=torch.float64, device="cuda", requires_grad=True)
            assert torch.autograd.gradcheck(lambda v: api.sca_potential(v, c), (xx,), eps=1e-6,
                                            atol=1e-6, rtol=1e-5)


def test_forward_backward_entry_points():
    torch = pytest.importorskip("torch")
    p = api.Params(6, 5, U=4.0, T=0.15, delta=0.2, prec="fp32")
    phi0 = inputs.random_phi(5, p.N)
    with api.Context(p) as c:
        x = torch.tensor(phi0, dtype=torch.float64, device="cuda")
        om = torch.empty(1, dtype=torch.float64, device="cuda")
        g = torch.empty_like(x)
        c.forward_dev(x, om)
        c.backward_dev(x, g)
        torch.cuda.synchronize()
        om2, g2 = c.grad(phi0)
        assert float(om) == pytest.approx(om2, rel=1e-12)
        assert np.allclose(g.cpu().numpy(), g2, rtol=1e-12, atol=1e-14)
        with pytest.raises(Exception, match="SCA_ENOSTATE"):
            c.backward_dev(x, g)


@pytest.mark.parametrize("prec", PRECS)
def test_pivot_free_blocks_match_forced_pivoting(prec, monkeypatch):
    """Blocks with omega_n > 4|t| skip the pivot search (column diagonal dominance makes
    partial pivoting keep the diagonal); forcing the pivoted panel on every block must give
    the same results within rounding."""
    p = api.Params(12, 10, U=4.0, T=0.1, delta=0.6, prec=prec)  # 6 pivoted + 14 dominant blocks
    phi = inputs.random_phi(33, p.N)
    with api.Context(p) as c:
        ld_a, gd_a = c.blocks(phi)
    monkeypatch.setenv("SCA_PIVOT_ALL", "1")
    with api.Context(p) as c:
        ld_b, gd_b = c.blocks(phi)
    t = tol(prec)
    assert np.allclose(ld_a, ld_b, rtol=t["ld"], atol=t["ld"])
    assert np.max(np.abs(gd_a - gd_b)) <= t["g"] * max(1.0, np.abs(gd_b).max())
    o_ld, o_gd = oracle.blocks_sample(oparams(p), phi, list(range(2 * p.n_omega)))
    assert np.allclose(ld_a, o_ld, rtol=t["ld"], atol=t["ld"])


@pytest.mark.parametrize("L,nw,prec", [(4, 16, "fp64"), (8, 12, "fp64"), (6, 10, "fp32"), (12, 8, "3xtf32")])
def test_fused_persistent_adam_matches_blocked_path_and_oracle(L, nw, prec, monkeypatch):
    """Small blocks run Adam in one cooperative launch per 16 iterations (blocks in shared
    memory, grid barriers); it must track the blocked multi-launch path and the oracle."""
    p = api.Params(L, nw, U=4.0, T=0.1, delta=0.4, prec=prec)
    ad = api.AdamConfig(lr=0.01, seed=11)
    steps = 40
    with api.Context(p) as c:
        c.adam_init(ad)
        om_f, gm_f = c.adam_step(steps)
        phi_f = c.phi()
    monkeypatch.setenv("SCA_FUSED", "0")
    with api.Context(p) as c:
        c.adam_init(ad)
        om_b, gm_b = c.adam_step(steps)
        phi_b = c.phi()
    phi_o, k, _, _, oh, gh = oracle.adam_run(oparams(p), lr=0.01, max_steps=steps, seed=11,
                                             history=True)
    t = 1e-10 if prec == "fp64" else 1e-6
    assert np.max(np.abs(phi_f - phi_b)) < t
    assert np.max(np.abs(phi_f - phi_o)) < t
    assert om_f == pytest.approx(oh[steps - 1], rel=1e-10 if prec == "fp64" else 1e-6)


def test_device_wait_timeout_is_reported_and_context_survives():
    """Failure detection without a fault: a 1-cycle bound on the fused kernel's grid barrier
    makes the waiting CTAs give up; the call returns SCA_ETIMEOUT (no hang) and the context
    works again once the default bound is restored."""
    p = api.Params(4, 64, U=6.0, T=0.1)  # 128 blocks -> many CTAs meeting at the barrier
    with api.Context(p) as c:
        c.adam_init(api.AdamConfig(lr=0.01, seed=0))
        c.set_wait_limit(1)
        with pytest.raises(Exception, match="SCA_ETIMEOUT"):
            c.adam_step(2)
        c.set_wait_limit(0)
        c.adam_init(api.AdamConfig(lr=0.01, seed=0))
        om, gm = c.adam_step(3)
        assert np.isfinite(om) and np.isfinite(gm)


@pytest.mark.gpu
def test_symmetric_update_matches_full_update(monkeypatch):
    """The dominant blocks' lower-triangle (symmetric) tensor-core update gives the same
    log-dets, diag(G) and gradient as the full update, and both match the oracle.  400 x 400
    blocks span four tiles per side with a ragged last one."""
    p = api.Params(20, 10, U=4.0, T=0.1, delta=0.5, prec="3xtf32")
    phi = inputs.seed_phi(3, p.N)
    res = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("SCA_SYM", flag)
        with api.Context(p) as c:
            ld, gd = c.blocks(phi, grad=True)
            om_lu = c.potential(phi)
            om, g = c.grad(phi)
        res[flag] = (ld, gd, om_lu, om, g)
    o_om, o_g, o_ld, o_gd = oracle.omega_grad(oparams(p), phi, per_block=True)
    t = tol("3xtf32")
    for ld, gd, om_lu, om, g in res.values():
        assert np.allclose(ld, o_ld, rtol=t["ld"], atol=t["ld"])
        assert np.max(np.abs(gd - o_gd)) <= t["g"] * max(1.0, np.abs(o_gd).max())
        assert om == pytest.approx(o_om, rel=t["om"]) and om_lu == pytest.approx(o_om, rel=t["om"])
        assert np.max(np.abs(g - o_g)) <= t["g"] * max(1.0, np.abs(o_g).max()) * 10
    assert np.max(np.abs(res["1"][1] - res["0"][1])) <= 2 * t["g"] * max(1.0, np.abs(o_gd).max())


@pytest.mark.parametrize("prec", ["bf16x3", "3xtf32"])
@pytest.mark.parametrize("L,nw", [(6, 12), (20, 10), (34, 6)])
def test_lower_triangle_refinement_matches_mirrored_rows(L, nw, prec, monkeypatch):
    """diag(G) of the symmetric dominant blocks refined straight from the lower triangle (row
    part, boundary bonds, column part) equals the refinement of whole rows after the mirror
    pass up to summation order, and both match the oracle.  N = 36, 400 and 1156 span one to
    ten 128-wide tiles and 2 to 37 column strips, each with a ragged end; at L = 6 and 34 the
    lattice rows (and so the periodic wraps) fall off the 32-column strip boundaries."""
    monkeypatch.setenv("SCA_FUSED", "0")
    p = api.Params(L, nw, U=4.0, T=0.1, delta=1.0, prec=prec)
    phi = inputs.seed_phi(11, p.N)
    res = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("SCA_REFINE_LOWER", flag)
        with api.Context(p) as c:
            res[flag] = c.blocks(phi, grad=True)
    o_om, o_g, o_ld, o_gd = oracle.omega_grad(oparams(p), phi, per_block=True)
    t = tol(prec)
    for ld, gd in res.values():
        assert np.allclose(ld, o_ld, rtol=t["ld"], atol=t["ld"])
        assert np.max(np.abs(gd - o_gd)) <= t["g"] * max(1.0, np.abs(o_gd).max())
    assert np.array_equal(res["1"][0], res["0"][0])
    scale = np.maximum(1.0, np.abs(res["0"][1]))
    assert np.max(np.abs(res["1"][1] - res["0"][1]) / scale) <= 1e-11


@pytest.mark.parametrize("prec", ["bf16x3", "3xtf32", "fp32"])
@pytest.mark.parametrize("L,nw", [(12, 10), (20, 8), (34, 6)])
def test_blocked_pivoted_inverse_matches_row_solves(L, nw, prec, monkeypatch):
    """The pivoted blocks' pivot-block inverse T = inv(U) inv(L) by blocked triangular inversion
    against the row-solve kernel: both match the oracle, the log-dets agree to float32 rounding
    (each step's T enters the next trailing matrix, hence the later pivots) and diag(G), after
    the refinement, to 1e-9.  N = 144, 400 and 1156 end on a pivot block of 16, 16 and 4 x 16
    rows (128-wide steps and a shorter last one)."""
    monkeypatch.setenv("SCA_FUSED", "0")
    p = api.Params(L, nw, U=4.0, T=0.1, delta=1.0, prec=prec)
    phi = inputs.random_phi(7 + L, p.N, 1.0)
    res = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("SCA_TINV_BLOCKED", flag)
        with api.Context(p) as c:
            res[flag] = c.blocks(phi, grad=True)
    o_om, o_g, o_ld, o_gd = oracle.omega_grad(oparams(p), phi, per_block=True)
    t = tol(prec)
    for ld, gd in res.values():
        assert np.allclose(ld, o_ld, rtol=t["ld"], atol=t["ld"])
        assert np.max(np.abs(gd - o_gd)) <= t["g"] * max(1.0, np.abs(o_gd).max())
    assert np.allclose(res["1"][0], res["0"][0], rtol=1e-7, atol=0.0)
    scale = max(1.0, np.abs(res["0"][1]).max())
    assert np.max(np.abs(res["1"][1] - res["0"][1])) <= 1e-9 * scale


@pytest.mark.parametrize("prec", ["bf16x3", "fp64"])
def test_group_enqueue_order_is_bit_identical(prec, monkeypatch):
    """Without SM partitions (N = 400) the two groups run on their own streams whichever is
    enqueued first: the dominant group first (the default) or the pivoted group first give
    bit-identical log-dets, diag(G) and gradient, and match the oracle."""
    monkeypatch.setenv("SCA_FUSED", "0")
    p = api.Params(20, 8, U=4.0, T=0.1, delta=1.0, prec=prec)
    phi = inputs.random_phi(29, p.N, 1.0)
    res = {}
    for flag in ("0", "1"):
        monkeypatch.setenv("SCA_PIVOTED_FIRST", flag)
        with api.Context(p) as c:
            res[flag] = c.blocks(phi, grad=True) + c.grad(phi)
    o_om, o_g, o_ld, o_gd = oracle.omega_grad(oparams(p), phi, per_block=True)
    t = tol(prec)
    assert np.allclose(res["0"][0], o_ld, rtol=t["ld"], atol=t["ld"])
    assert np.max(np.abs(res["0"][1] - o_gd)) <= t["g"] * max(1.0, np.abs(o_gd).max())
    for a, b in zip(res["0"], res["1"]):
        assert np.array_equal(np.asarray(a), np.asarray(b))


@pytest.mark.parametrize("prec", ["bf16x3", "fp32", "fp64"])
@pytest.mark.parametrize("L,nw", [(6, 12), (20, 8), (34, 6)])
def test_fused_subpanel_interchanges_are_bit_identical(L, nw, prec, monkeypatch):
    """The pivoted sub-panel's interchanges on the rest of its outer panel with the U12 solve
    at the end of the panel launch, and the outer panel's composed interchanges on all other
    columns in one launch afterwards, give bit-identical log-dets, diag(G) and potential to
    the per-sub-panel k_swap_trsm launches (the same entries moved, the same arithmetic), and
    match the oracle.  N = 36, 400 and 1156 cover sub-panels of 16 and a narrower last one;
    the potential alone (LU, no inverse) leaves the columns before the outer panel alone."""
    monkeypatch.setenv("SCA_FUSED", "0")
    p = api.Params(L, nw, U=4.0, T=0.1, delta=1.0, prec=prec)
    phi = inputs.random_phi(5 + L, p.N, 1.0)
    res, pot = {}, {}
    for flag in ("1", "0"):
        monkeypatch.setenv("SCA_FUSED_SWAP", flag)
        with api.Context(p) as c:
            res[flag] = c.blocks(phi, grad=True)
            pot[flag] = c.potential(phi)
    o_om, o_g, o_ld, o_gd = oracle.omega_grad(oparams(p), phi, per_block=True)
    t = tol(prec)
    assert np.allclose(res["1"][0], o_ld, rtol=t["ld"], atol=t["ld"])
    assert np.max(np.abs(res["1"][1] - o_gd)) <= t["g"] * max(1.0, np.abs(o_gd).max())
    assert np.array_equal(res["1"][0], res["0"][0])
    assert np.array_equal(res["1"][1], res["0"][1])
    assert pot["1"] == pot["0"]


@pytest.mark.parametrize("prec", ["bf16x3", "3xtf32"])
def test_tensor_core_pivot_block_inverse_matches_register_kernel(prec, monkeypatch):
    """The dominant pivot-block inverse on the tensor cores (tableau in TMEM, split-TF32
    rank-16 updates) and the register Gauss-Jordan kernel give log-dets, diag(G), Omega and the
    gradient that match the oracle and each other.  400 x 400 blocks: three full 128-wide pivot
    blocks and a ragged 16-wide last one (identity padding inside the 128 x 128 tableau)."""
    p = api.Params(20, 10, U=4.0, T=0.1, delta=0.5, prec=prec)
    phi = inputs.seed_phi(9, p.N)
    res = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("SCA_DIAG_TC", flag)
        with api.Context(p) as c:
            ld, gd = c.blocks(phi, grad=True)
            om_lu = c.potential(phi)
            om, g = c.grad(phi)
        res[flag] = (ld, gd, om_lu, om, g)
    o_om, o_g, o_ld, o_gd = oracle.omega_grad(oparams(p), phi, per_block=True)
    t = tol(prec)
    for ld, gd, om_lu, om, g in res.values():
        assert np.allclose(ld, o_ld, rtol=t["ld"], atol=t["ld"])
        assert np.max(np.abs(gd - o_gd)) <= t["g"] * max(1.0, np.abs(o_gd).max())
        assert om == pytest.approx(o_om, rel=t["om"]) and om_lu == pytest.approx(o_om, rel=t["om"])
        assert np.max(np.abs(g - o_g)) <= t["g"] * max(1.0, np.abs(o_g).max()) * 10
    assert np.allclose(res["1"][0], res["0"][0], rtol=t["ld"], atol=t["ld"])
    assert np.max(np.abs(res["1"][1] - res["0"][1])) <= 2 * t["g"] * max(1.0, np.abs(o_gd).max())


@pytest.mark.parametrize("prec", PRECS)
def test_no_pivoting_matches_oracle(prec):
    """Every block eliminated without interchanges (complex-symmetric elimination), including
    the lowest frequencies (omega_0 = 0.157 < 4t, where the default path pivots), against the
    oracle's partially pivoted LU.  400 x 400 blocks: four tiles per side, ragged last one."""
    p = api.Params(20, 8, U=6.0, T=0.05, delta=0.5, prec=prec)
    assert api.pivoted_blocks(p) > 0
    phi = inputs.seed_phi(5, p.N)
    with api.Context(p) as c:
        with pytest.raises(ValueError):
            c.set_pivoting("rook")
        assert _lib.lib().sca_set_pivoting(c._h, 7) == 1  # SCA_EINVAL, context unchanged
        c.set_pivoting("none")
        ld, gd = c.blocks(phi, grad=True)
        om_lu = c.potential(phi)
        om, g = c.grad(phi)
        c.set_pivoting("partial")
        om_p, g_p = c.grad(phi)
    o_om, o_g, o_ld, o_gd = oracle.omega_grad(oparams(p), phi, per_block=True)
    t = tol(prec)
    assert np.allclose(ld, o_ld, rtol=t["ld"], atol=t["ld"])
    assert np.max(np.abs(gd - o_gd)) <= t["g"] * max(1.0, np.abs(o_gd).max())
    assert om == pytest.approx(o_om, rel=t["om"]) and om_lu == pytest.approx(o_om, rel=t["om"])
    assert om_p == pytest.approx(o_om, rel=t["om"])
    for gg in (g, g_p):
        assert np.max(np.abs(gg - o_g)) <= t["g"] * max(1.0, np.abs(o_g).max()) * 10


@pytest.mark.parametrize("prec", ["3xtf32", "bf16x3"])
def test_full_size_40x40_sampled_blocks(prec):
    """The benchmark's workload at full size (L = 40: 256 blocks of 1600 x 1600, 12 pivoted,
    244 dominant, symmetric tensor-core update, SM reserve and side stream as timed): per-block
    ln|det| and sigma Re G_ii of a sample of pivoted and dominant blocks against the oracle,
    which computes those blocks one by one."""
    wl = inputs.WORKLOADS["ionic_40x40"]
    p = api.Params(wl.L, wl.n_omega, U=wl.U, T=wl.T, delta=wl.delta, t=wl.t, mu=wl.mu, prec=prec)
    assert api.pivoted_blocks(p) == 12
    phi = inputs.seed_phi(wl.seed, p.N)
    with api.Context(p) as c:
        ld, gd = c.blocks(phi, grad=True)
    sample = [0, 1, 11, 12, 13, 128, 255]
    o_ld, o_gd = oracle.blocks_sample(oparams(p), phi, sample)
    t = tol(prec)
    assert np.allclose(ld[sample], o_ld, rtol=t["ld"], atol=t["ld"])
    assert np.max(np.abs(gd[sample] - o_gd)) <= t["g"] * max(1.0, np.abs(o_gd).max())


def test_profile_kinds_and_group_spans():
    """Per-kind event timing (sca_profile_*): with both groups present (12 pivoted + 4
    dominant blocks of 400 x 400) every step records both group spans once, the dominant
    update and pivot-block inverses once per elimination step, and no counts while off."""
    p = api.Params(20, 8, U=6.0, T=0.1, delta=0.5, prec="bf16x3")
    assert api.pivoted_blocks(p) == 12
    phi = inputs.seed_phi(0, p.N)
    with api.Context(p) as c:
        c.grad(phi)  # profiling off
        c.profile(True)
        c.grad(phi)
        prof = c.profile_read()
        c.profile(False)
        c.grad(phi)
        after = c.profile_read()
    steps = -(-p.N // 128)  # elimination steps of width 128
    assert prof["span_pivoted"][1] == 1 and prof["span_dominant"][1] == 1
    # the dominant blocks' steps run in merged pairs: per pair one update of the second step's
    # strips (update_cross) and one merged update; an odd last step updates alone
    pairs = steps // 2
    assert prof["update_cross"][1] == pairs and prof["update"][1] == steps - pairs
    assert prof["diag"][1] == steps
    assert prof["panel"][1] > 0 and prof["refine"][1] >= 2 and prof["reduce"][1] == 1
    # 16-wide sub-panels: the rest of each outer panel is updated after every sub-panel
    assert prof["panel_update"][1] > 0 and prof["prep_piv"][1] == steps
    assert prof["trinv"][1] == steps
    for k in ("span_pivoted", "span_dominant", "update", "panel", "refine"):
        assert prof[k][0] > 0.0
    # spans contain the kernels of their group
    assert prof["span_dominant"][0] >= prof["update"][0]
    assert after == {k: (0.0, 0) for k in after}


def test_profile_timeline_file(tmp_path, monkeypatch):
    """SCA_PROFILE_TRACE: every profiled launch of a call appears in the timeline file with its
    kind, stream, start and duration; the per-kind totals match the file."""
    trace = tmp_path / "timeline.txt"
    monkeypatch.setenv("SCA_PROFILE_TRACE", str(trace))
    p = api.Params(20, 8, U=6.0, T=0.1, delta=0.5, prec="bf16x3")
    with api.Context(p) as c:
        c.profile(True)
        c.grad(inputs.seed_phi(0, p.N))
        prof = c.profile_read()
        c.profile(False)
    lines = trace.read_text().strip().splitlines()
    assert lines[0].startswith("# collection of")
    recs = [ln.split() for ln in lines[1:] if not ln.startswith("#")]
    kinds = {}
    for k, stream, start, dur in recs:
        assert float(start) >= 0.0 and float(dur) >= 0.0 and int(stream) >= 0
        kinds.setdefault(k, [0, 0.0])
        kinds[k][0] += 1
        kinds[k][1] += float(dur)
    for k, (ms, n) in prof.items():
        if n:
            assert kinds[k][0] == n
            assert kinds[k][1] == pytest.approx(ms, rel=1e-3, abs=1e-3)
    # the two groups run on different streams
    streams = {k: s for k, s, _, _ in recs}
    assert streams["span_pivoted"] != streams["span_dominant"]


@pytest.mark.parametrize("mode", ["dominant", "both", "alternate"])
def test_sm_partition_leaves_results_unchanged(mode):
    """SM partitions (green contexts) only move launches between SMs: Omega and the
    gradient are bit-identical with and without them, and removing one restores the plain
    streams."""
    import torch
    p = api.Params(20, 8, U=6.0, T=0.1, delta=0.5, prec="bf16x3")
    phi = inputs.seed_phi(3, p.N)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    with api.Context(p) as c:
        assert c.sm_partition() == (0, 0)
        om0, g0 = c.grad(phi)
        ps, ds = c.set_sm_partition(16, mode)
        assert ps >= 16 and ds > 0 and ps + ds <= sms
        om1, g1 = c.grad(phi)
        assert c.set_sm_partition(0) == (0, 0)
        om2, g2 = c.grad(phi)
    assert om1 == om0 and om2 == om0
    assert np.array_equal(g1, g0) and np.array_equal(g2, g0)


@pytest.mark.parametrize("prec", ["bf16x3", "fp32"])
def test_64x64_staggered_field_closed_form(prec):
    """The 64x64 workload (128 blocks of 4096 x 4096: 6 pivoted with 2-wide shared-memory
    sub-panels, 122 dominant) at a staggered field phi_i = a s_i, where Omega and the gradient
    have the Fourier closed form (spin sigma sees the staggered potential Delta + sigma a)."""
    from test_oracle_pins import G_staggered, ld_staggered, sublattice
    wl = inputs.WORKLOADS["ionic_64x64"]
    p = api.Params(wl.L, wl.n_omega, U=wl.U, T=wl.T, delta=wl.delta, prec=prec)
    assert api.pivoted_blocks(p) == 6
    a, L, N = 0.8, wl.L, wl.L * wl.L
    s = sublattice(L)
    with api.Context(p) as c:
        om, g = c.grad(a * s)
    om_ref = N * a * a / wl.U
    g_a = 2 * a / wl.U  # gradient on an A site (s = +1); B sites carry the opposite sign
    for n in range(wl.n_omega):
        w = (2 * n + 1) * math.pi * wl.T
        for sg in (1, -1):
            D = wl.delta + sg * a
            om_ref -= 2 * wl.T * ld_staggered(L, D, w)
            g_a -= 2 * wl.T * sg * G_staggered(L, D, w, -D).real
    t = tol(prec)
    assert om == pytest.approx(om_ref, rel=t["om"])
    assert np.max(np.abs(g - g_a * s)) <= t["g"] * max(1.0, abs(g_a)) * 10


@pytest.mark.slow
def test_c3_autograd_gradient_matches_central_differences():
    """The 40x40 workload (256 blocks of 1600 x 1600, U = 4, Delta = 1, T = 0.1): the gradient
    from the autograd Function (forward keeps the inverses, backward runs the adjoint diag(G)
    stage) on the FP64 and BF16x3 paths against central differences of the FP64 path,
    h = 1e-6, on 32 seeded random components.  Each difference is formed block by block,
    sum_b [ld_b(phi + h e_i) - ld_b(phi - h e_i)], so the large constant part of Omega cancels
    inside every block (LU-only evaluations)."""
    torch = pytest.importorskip("torch")
    wl = inputs.WORKLOADS["ionic_40x40"]
    phi = inputs.seed_phi(wl.seed, wl.L * wl.L)
    N, h = phi.size, 1e-6
    comps = np.random.default_rng(2311).choice(N, 32, replace=False)
    grads = {}
    for prec in ("fp64", "bf16x3"):
        p = api.Params(wl.L, wl.n_omega, U=wl.U, T=wl.T, delta=wl.delta, prec=prec)
        with api.Context(p) as c:
            x = torch.tensor(phi, dtype=torch.float64, device="cuda", requires_grad=True)
            api.sca_potential(x, c).backward()
            grads[prec] = x.grad.cpu().numpy()
            if prec != "fp64":
                continue
            fd = np.zeros(len(comps))
            for k, i in enumerate(comps):
                e = np.zeros(N)
                e[i] = h
                ld_p = c.blocks(phi + e, grad=False)
                ld_m = c.blocks(phi - e, grad=False)
                quad = ((phi[i] + h) ** 2 - (phi[i] - h) ** 2) / wl.U
                fd[k] = (quad - 2.0 * wl.T * np.sum(ld_p - ld_m)) / (2.0 * h)
    for prec, g in grads.items():
        err = np.abs(g[comps] - fd)
        assert np.all(err <= 1e-5 * np.maximum(1.0, np.abs(fd))), (prec, err.max())
    scale = max(1.0, np.abs(grads["fp64"]).max())
    assert np.max(np.abs(grads["bf16x3"] - grads["fp64"])) <= 1e-6 * scale


@pytest.mark.parametrize("L,nw", [(20, 10), (40, 8)])
def test_fp64_panel_on_the_mixed_path_matches_oracle(L, nw):
    """The pivoted blocks' panel factorisation in float64 on the float32 blocks of the BF16x3
    path (sca_set_panel_precision): per-block ln|det| and diag(G) of every pivoted block (and
    the dominant ones) against the oracle at the mixed tolerances, beside the float32 panel.
    400 sites (16-wide float64 sub-panels) and 1600 sites (4-wide), 12 pivoted blocks each."""
    p = api.Params(L, nw, U=4.0, T=0.1, delta=0.5, prec="bf16x3")
    npiv = api.pivoted_blocks(p)
    assert npiv == 12
    phi = inputs.seed_phi(8, p.N)
    res = {}
    for panel in ("fp32", "fp64"):
        with api.Context(p) as c:
            c.set_panel_precision(panel)
            res[panel] = c.blocks(phi, grad=True)
        with pytest.raises(ValueError):
            c.set_panel_precision("bf16")
    sample = list(range(npiv)) + [npiv, 2 * nw - 1]
    o_ld, o_gd = oracle.blocks_sample(oparams(p), phi, sample)
    t = tol("bf16x3")
    for ld, gd in res.values():
        assert np.allclose(ld[sample], o_ld, rtol=t["ld"], atol=t["ld"])
        assert np.max(np.abs(gd[sample] - o_gd)) <= t["g"] * max(1.0, np.abs(o_gd).max())
