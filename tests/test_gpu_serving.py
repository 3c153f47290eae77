"""Serving loop (sca_server_*): continuous batching of mixed-size solve requests.

Each request's result must be the same alone (sca_solve) and in the mix, bit for bit; the
admission respects the slot count and the HBM budget; bookkeeping errors are reported.
"""
import time

import numpy as np
import pytest

from paper_2311_04435_gb300 import _lib, api

pytestmark = pytest.mark.gpu


def _wait(srv, rid, N, timeout=300.0):
    t0 = time.time()
    while True:
        r = srv.poll(rid, N)
        if r is not None:
            return r
        if time.time() - t0 > timeout:
            raise TimeoutError(rid)
        time.sleep(0.005)


REQS = [
    (api.Params(4, 16, U=6.0, T=0.1, prec="fp64"), api.AdamConfig(lr=0.02, grad_tol=1e-5, max_steps=400, seed=1)),
    (api.Params(6, 8, U=4.0, T=0.2, delta=0.5, prec="fp32"), api.AdamConfig(lr=0.02, grad_tol=1e-5, max_steps=300, seed=2)),
    (api.Params(8, 6, U=3.0, T=0.3, delta=1.0, prec="3xtf32"), api.AdamConfig(lr=0.01, grad_tol=1e-6, max_steps=150, seed=3)),
    (api.Params(12, 10, U=5.0, T=0.1, delta=0.3, prec="3xtf32"), api.AdamConfig(lr=0.01, grad_tol=1e-6, max_steps=40, seed=4)),
    (api.Params(4, 4, U=2.0, T=0.5, prec="fp64"), api.AdamConfig(lr=0.05, grad_tol=1e-3, max_steps=1000, seed=5)),
    (api.Params(10, 5, U=7.0, T=0.15, delta=1.5, prec="fp32"), api.AdamConfig(lr=0.02, grad_tol=1e-6, max_steps=60, seed=6)),
]


def test_results_identical_alone_and_in_the_mix():
    alone = [api.solve(p, a) for p, a in REQS]
    with api.Server(hbm_budget_bytes=8 << 30, max_slots=3) as srv:
        ids = [srv.submit(p, a) for p, a in REQS]
        mixed = [_wait(srv, rid, p.N) for rid, (p, _) in zip(ids, REQS)]
        times = [srv.times(rid) for rid in ids]
    for (p, a), x, y in zip(REQS, alone, mixed):
        assert x.steps == y.steps
        assert np.array_equal(x.phi, y.phi)
        assert x.omega == y.omega and x.gmax == y.gmax
        assert y.gmax < a.grad_tol or y.steps == a.max_steps
    # at most 3 requests between admission and completion at any time
    events = sorted([(t[1], 1) for t in times] + [(t[3], -1) for t in times], key=lambda e: (e[0], e[1]))
    live = peak = 0
    for _, d in events:
        live += d
        peak = max(peak, live)
    assert peak <= 3
    for t in times:
        assert 0 <= t[0] <= t[1] <= t[2] <= t[3]


def test_budget_limits_concurrency():
    p = api.Params(8, 8, U=4.0, T=0.2, prec="fp32")
    a = api.AdamConfig(lr=0.02, grad_tol=0.0, max_steps=80, seed=7)
    b = api.workspace_bytes(p)
    with api.Server(hbm_budget_bytes=2 * b + b // 2, max_slots=8) as srv:
        ids = [srv.submit(p, api.AdamConfig(**{**a.__dict__, "seed": 7 + k})) for k in range(5)]
        for rid in ids:
            _wait(srv, rid, p.N)
        times = [srv.times(rid) for rid in ids]
    events = sorted([(t[1], 1) for t in times] + [(t[3], -1) for t in times], key=lambda e: (e[0], e[1]))
    live = peak = 0
    for _, d in events:
        live += d
        peak = max(peak, live)
    assert peak <= 2
    # admission in arrival order
    admits = [t[1] for t in times]
    assert admits == sorted(admits)


def test_over_budget_and_unknown_ids():
    p = api.Params(20, 64, U=4.0, T=0.1, prec="fp64")
    with api.Server(hbm_budget_bytes=1 << 20, max_slots=2) as srv:
        with pytest.raises(_lib.SCAError, match="SCA_EBUDGET"):
            srv.submit(p, api.AdamConfig())
        with pytest.raises(_lib.SCAError, match="SCA_ENOTFOUND"):
            srv.poll(12345)
        with pytest.raises(_lib.SCAError, match="SCA_EINVAL"):
            srv.submit(api.Params(3, 4, U=4.0, T=0.1), api.AdamConfig())


# Sizes above the fused kernel's share a size bucket per (L, prec): one workspace, one launch
# sequence for all their blocks, one reduction CTA per request.
BUCKETED = [
    (api.Params(16, 8, U=4.0, T=0.1, delta=1.0, prec="bf16x3"), api.AdamConfig(lr=0.01, grad_tol=1e-6, max_steps=40, seed=11)),
    (api.Params(16, 6, U=5.0, T=0.3, delta=0.5, prec="bf16x3"), api.AdamConfig(lr=0.02, grad_tol=1e-4, max_steps=60, seed=12)),
    (api.Params(16, 4, U=3.0, T=0.5, delta=0.0, prec="bf16x3", ionic="half"), api.AdamConfig(lr=0.02, grad_tol=1e-6, max_steps=25, seed=13)),
    (api.Params(10, 5, U=4.0, T=0.2, delta=0.7, prec="fp64"), api.AdamConfig(lr=0.02, grad_tol=1e-6, max_steps=30, seed=14)),
    (api.Params(10, 3, U=6.0, T=0.4, delta=0.2, prec="fp64"), api.AdamConfig(lr=0.02, grad_tol=1e-6, max_steps=35, seed=15)),
    (api.Params(16, 5, U=4.0, T=0.15, delta=0.8, prec="fp32"), api.AdamConfig(lr=0.01, grad_tol=1e-6, max_steps=20, seed=16)),
]


def _check_same(reqs, mixed, alone):
    for (p, a), x, y in zip(reqs, alone, mixed):
        assert x.steps == y.steps
        assert np.array_equal(x.phi, y.phi)
        assert x.omega == y.omega and x.gmax == y.gmax


def test_bucketed_requests_identical_alone_and_shared():
    """Requests sharing a size bucket's passes (pivoted and dominant blocks of several
    requests stacked, different T, n_omega, U, Delta, ionic convention and step counts) give
    bit for bit what each gives alone."""
    alone = [api.solve(p, a) for p, a in BUCKETED]
    with api.Server(hbm_budget_bytes=16 << 30, max_slots=8) as srv:
        ids = [srv.submit(p, a) for p, a in BUCKETED]
        mixed = [_wait(srv, rid, p.N) for rid, (p, _) in zip(ids, BUCKETED)]
    _check_same(BUCKETED, mixed, alone)


def test_bucket_spread_over_passes():
    """A budget that leaves the bucket 16 block slots: three requests of 8 to 12 blocks are
    spread over several passes and still match their solo results."""
    reqs = [(api.Params(16, n, U=4.0, T=0.12, delta=0.6, prec="3xtf32"),
             api.AdamConfig(lr=0.01, grad_tol=1e-6, max_steps=12, seed=20 + n)) for n in (4, 6, 5)]
    alone = [api.solve(p, a) for p, a in reqs]
    ws16 = api.workspace_bytes(api.Params(16, 8, U=1.0, T=1.0, prec="3xtf32"))
    ws32 = api.workspace_bytes(api.Params(16, 16, U=1.0, T=1.0, prec="3xtf32"))
    state = 8 * (4 * 256 + 8)
    budget = ws16 + 3 * state + (ws32 - ws16) // 2  # room for a 16-slot bucket, not 32
    with api.Server(hbm_budget_bytes=budget, max_slots=4) as srv:
        ids = [srv.submit(p, a) for p, a in reqs]
        mixed = [_wait(srv, rid, p.N) for rid, (p, _) in zip(ids, reqs)]
    _check_same(reqs, mixed, alone)


def test_large_bucketed_requests_match_oracle():
    """BF16x3 requests of the serving sweep's larger sizes (L = 24: 576 sites, L = 32: 1024
    sites, tensor-core path with pivoted and dominant blocks) served together in one mix: each
    result after its 25 gated Adam updates matches the oracle's Adam run (spectral route) from
    the same seeded start."""
    import oracle

    reqs = [(api.Params(24, 32, U=4.0, T=0.1, delta=0.6, prec="bf16x3"),
             api.AdamConfig(lr=0.01, grad_tol=1e-6, max_steps=25, seed=31)),
            (api.Params(32, 16, U=5.0, T=0.2, delta=0.3, prec="bf16x3"),
             api.AdamConfig(lr=0.01, grad_tol=1e-6, max_steps=25, seed=32)),
            (api.Params(24, 11, U=6.0, T=0.3, delta=1.2, prec="bf16x3"),
             api.AdamConfig(lr=0.02, grad_tol=1e-6, max_steps=25, seed=33))]
    with api.Server(hbm_budget_bytes=40 << 30, max_slots=4) as srv:
        ids = [srv.submit(p, a) for p, a in reqs]
        mixed = [_wait(srv, rid, p.N) for rid, (p, _) in zip(ids, reqs)]
    for (p, a), r in zip(reqs, mixed):
        op = oracle.make_params(p.L, p.n_omega, U=p.U, T=p.T, delta=p.delta)
        phi_o, k_o, om_o, gm_o = oracle.adam_run_spectral(
            op, oracle.seed_phi(a.seed, p.N), lr=a.lr, grad_tol=a.grad_tol, max_steps=a.max_steps)
        assert r.steps == k_o == a.max_steps
        assert np.max(np.abs(r.phi - phi_o)) <= 1e-6
        assert r.omega == pytest.approx(om_o, rel=1e-5)
        assert r.gmax == pytest.approx(gm_o, rel=1e-4, abs=1e-6)


def _replay(trace, dt, slots, budget):
    """Replays an arrival trace on a manual server: round r runs at virtual time r * dt, after
    the submission of every request that arrived by then.  Returns the per-round (in flight,
    queued) log and, per request, its times, update count and result."""
    reqs = [(api.Params(q.L, q.n_omega, U=q.U, T=q.T, delta=q.delta, prec="bf16x3"),
             api.AdamConfig(lr=0.01, grad_tol=1e-6, max_steps=40, seed=q.seed)) for q in trace]
    log, ids = [], []
    with api.Server(hbm_budget_bytes=budget, max_slots=slots, manual=True) as srv:
        k, r = 0, 0
        while True:
            t = r * dt
            while k < len(trace) and trace[k].arrival_s <= t:
                ids.append(srv.submit(*reqs[k]))
                k += 1
            fl, q = srv.step(t)
            log.append((fl, q))
            assert fl <= slots
            if k == len(trace) and fl == 0 and q == 0:
                break
            r += 1
            assert r < 10000
        out = []
        for rid, (p, _) in zip(ids, reqs):
            res = srv.poll(rid, p.N)
            assert res is not None
            out.append((rid, srv.times(rid), res.steps, res.omega, res.gmax, res.phi))
    return log, out, reqs


def test_replayed_trace_bookkeeping_is_bit_exact():
    """A 14-request slice of the serving trace (L in {8, 12, 16, 20}, BF16x3: fused small
    requests and size buckets) replayed twice on a manual server with a virtual clock: the
    admission order, the in-flight and queued counts of every round, the request times, the
    update counts and the results agree bit for bit; admission follows arrival order and never
    exceeds the slots; each result equals the request solved alone."""
    from paper_2311_04435_gb300 import inputs

    trace = inputs.serving_trace(14, rate_per_s=20.0, seed=77, sizes=(8, 12, 16, 20))
    a = _replay(trace, 0.05, slots=4, budget=6 << 30)
    b = _replay(trace, 0.05, slots=4, budget=6 << 30)
    assert a[0] == b[0]
    for x, y in zip(a[1], b[1]):
        assert x[0] == y[0] and x[1] == y[1] and x[2] == y[2]
        assert x[3] == y[3] and x[4] == y[4] and np.array_equal(x[5], y[5])
    admits = [o[1][1] for o in a[1]]
    assert admits == sorted(admits)
    for o in a[1]:
        sub, adm, st, fin = o[1]
        assert 0 <= sub <= adm <= st <= fin
    assert max(fl for fl, _ in a[0]) == 4  # the slots were the limit at some point
    for (p, ad), o in list(zip(a[2], a[1]))[:4]:
        alone = api.solve(p, ad)
        assert alone.steps == o[2] and np.array_equal(alone.phi, o[5]) and alone.omega == o[3]
