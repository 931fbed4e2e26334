"""GPU checks of the failure reporting: a kernel that gives up a bounded wait
(or a thin QR that cannot orthogonalize a block) raises a bit in the run's
device status word, and every entry point turns it into TT_ETIMEOUT /
TT_ESINGULAR. The failure is injected on the host: the test hook overwrites
the device status word by a host copy right before the library reads it back,
so no kernel is made to fail and no wait is made to run out."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from tests._gpu import to_dev, const_ranks

pytestmark = pytest.mark.gpu


def _problem():
    dims = [6, 7, 5, 6]
    N = len(dims)
    Ys = [to_dev(synth.gaussian_tt(synth.rng_for(90, j), dims, const_ranks(N, r))) for j, r in enumerate([2, 3])]
    ell = O.clamp_ranks(dims, const_ranks(N, 4))
    return dims, Ys, ell


@pytest.mark.parametrize("bits,code", [(1, 6), (2, 5), (3, 6)])
@pytest.mark.parametrize("tol", [0.0, 1e-6])
def test_eager_sum_rounding_reports_device_status(bits, code, tol):
    import paper_2110_04393_gb300 as tt
    dims, Ys, ell = _problem()
    ref = tt.tt_round_sum_rand(Ys, ell, seed=3, tol=tol)         # clean run
    tt.debug_inject_device_status(bits)
    with pytest.raises(tt.TTError) as ei:
        tt.tt_round_sum_rand(Ys, ell, seed=3, tol=tol)
    assert ei.value.code == code
    again = tt.tt_round_sum_rand(Ys, ell, seed=3, tol=tol)        # the hook disarmed itself
    for a, b in zip(ref, again):
        assert torch.equal(a, b)


def test_other_entry_points_report_device_status():
    import paper_2110_04393_gb300 as tt
    dims, Ys, ell = _problem()
    calls = [lambda: tt.tt_round_det(Ys, tol=1e-8),
             lambda: tt.tt_round_orthrand(Ys, ell, seed=1),
             lambda: tt.tt_round_twosided(Ys, ell, seed=1),
             lambda: tt.tt_round_twosided(Ys, ell, seed=1, precision="mixed"),
             lambda: tt.tt_round_sum_rand(Ys, ell, seed=1, precision="mixed"),
             lambda: tt.tt_gemm_emulated_f64(torch.randn(40, 30, dtype=torch.float64, device="cuda"),
                                             torch.randn(30, 20, dtype=torch.float64, device="cuda"))]
    for f in calls:
        f()
        tt.debug_inject_device_status(1)
        with pytest.raises(tt.TTError) as ei:
            f()
        assert ei.value.code == 6
        f()


def test_plan_replay_reports_device_status():
    import paper_2110_04393_gb300 as tt
    dims, Ys, ell = _problem()
    R = [[1] + [int(c.shape[2]) for c in Y] for Y in Ys]
    plan = tt.SumRoundingPlan(dims, R, ell, tol=0.0, precision="fp64")
    try:
        plan(Ys, seed=2)
        plan.status()
        tt.debug_inject_device_status(1)
        plan(Ys, seed=2)                       # fixed ranks: returns before the replay ends
        with pytest.raises(tt.TTError) as ei:
            plan.status()
        assert ei.value.code == 6
        plan(Ys, seed=2)
        plan.status()
    finally:
        plan.close()
    plan = tt.SumRoundingPlan(dims, R, ell, tol=1e-8, precision="mixed")
    try:
        tt.debug_inject_device_status(2)
        with pytest.raises(tt.TTError) as ei:
            plan(Ys, seed=2)                   # tolerance: the replay is waited for
        assert ei.value.code == 5
        plan(Ys, seed=2)
    finally:
        plan.close()


@pytest.mark.gpu
def test_fp64_rate_probe_in_range():
    # the FP64 FMA rate of a GB300: well above zero and not above the unit-count
    # ceiling (152 SMs x 2 FMA per clock x 2 flops x 2.07 GHz = 1.26 TFLOP/s) by much
    import paper_2110_04393_gb300 as tt
    r = tt.probe_fp64_rate(1 << 12)
    assert 0.3 < r < 1.4
    with pytest.raises(tt.TTError):
        tt.probe_fp64_rate(0)
