"""Host-side arithmetic of the benchmark line: the algorithmic flop and byte counts of the
dominant update launches, the roofline bound selection and the replica aggregation.

The counts are checked against closed forms of the elimination: one Gauss-Jordan sweep of an
N x N complex block costs 8 N^3 real flops (8 per complex multiply-add, K = N in all), and
4 N^2 (N + 1) when only the lower triangle with its diagonal is updated; merging steps in
pairs changes the number of launches, not the work.
"""
import json
import os

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("N", [36, 400, 1156, 1600, 4096])
@pytest.mark.parametrize("paired", [False, True])
def test_update_flops_sum_to_the_closed_form(N, paired):
    sym = bench.dominant_update_launches("bf16x3", N, 128, True, paired)
    full = bench.dominant_update_launches("bf16x3", N, 128, False, False)
    assert sum(f for _, f, _ in sym) == pytest.approx(4.0 * N * N * (N + 1), rel=1e-12)
    assert sum(f for _, f, _ in full) == pytest.approx(8.0 * N ** 3, rel=1e-12)
    steps = -(-N // 128)
    n_update = sum(1 for k, _, _ in sym if k == "update")
    n_cross = sum(1 for k, _, _ in sym if k == "update_cross")
    if paired:
        assert n_cross == steps // 2 and n_update == steps - steps // 2
    else:
        assert n_cross == 0 and n_update == steps


def test_update_bytes_at_1600_sites():
    """N = 1600 (12 full 128-wide tiles and one of 64): the lower tiles hold
    (N^2 + 12 * 128^2 + 64^2) / 2 complex64 entries, read and written once (22.1 MB), and a
    merged launch reads the F and W split planes of both steps (4 + 4 bf16 planes of
    N x 128 each)."""
    N = 1600
    launches = bench.dominant_update_launches("bf16x3", N, 128, True, True)
    area = (N * N + 12 * 128 ** 2 + 64 ** 2) / 2
    planes = 8.0 * N * 128 * 2
    merged = [b for k, _, b in launches if k == "update"]
    assert merged[0] == pytest.approx(16 * area + 2 * planes)
    assert merged[-1] == pytest.approx(16 * area + planes)  # the odd last step updates alone
    assert len(merged) == 7
    assert 16 * area == pytest.approx(22.09e6, rel=1e-3)


def test_roofline_bound_follows_the_ridge():
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
        pk = json.load(f)
    hbm, peak = pk["hbm_gbs"], pk["bf16_tflops_sustained"] / 3.0
    ridge = peak * 1e3 / hbm  # flop per byte
    # below the ridge: reported against HBM bandwidth
    lo = bench.roofline_for("bf16x3", 0.5 * ridge * 1e12, 1e12, 1.0, None)
    assert lo["bound"] == "hbm" and lo["unit"] == "GB/s"
    assert lo["frac"] == pytest.approx(1e3 / hbm, rel=1e-3)
    # above it: against the split-precision tensor peak
    hi = bench.roofline_for("bf16x3", 2.0 * ridge * 1e12, 1e12, 1.0, 123.0)
    assert hi["bound"] == "tensor" and hi["unit"] == "TFLOP/s" and hi["traffic"] == 123.0
    assert hi["frac"] == pytest.approx(2.0 * ridge / peak, rel=1e-3)
    fp64 = bench.roofline_for("fp64", 1.2e12, 1e9, 1.0, None)
    assert fp64["bound"] == "alu" and fp64["frac"] == pytest.approx(1.0)


def test_single_replica_aggregation():
    ms, value = bench.aggregate_replicas(25.0, 20, 1)
    assert ms == 25.0 and value == pytest.approx(20 / 0.025)
