"""GPU parity of the Levenberg-Marquardt iteration with adaptive
per-trajectory damping (pes_ieks_run_lm) against the oracle
(orc_iterated_smoother_lm), on models with a positive definite Q."""
import numpy as np
import pytest
import torch

import oracle
from paper_2102_00514_gb300 import pes, synth
from tests.gpu_common import TOL_FP32, TOL_FP64, rel_err, to_dev, workload_to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sm():
    s = pes.Smoother(1 << 16, 64)
    yield s
    s.close()


def starts(wl, seed):
    """Starts off the truth (positions shifted by up to 1.5 units, turn rate by
    up to 3 rad/s), where lightly damped steps overshoot and are rejected."""
    rng = np.random.default_rng(seed)
    off = wl["offsets"]
    x = wl["x_true"].copy()
    for b in range(len(off) - 1):
        sl = slice(int(off[b]), int(off[b + 1]))
        x[:, sl] += np.array([rng.uniform(-1.5, 1.5), rng.uniform(-1.5, 1.5), 0.0, 0.0, rng.uniform(-3, 3)])[:, None]
    return x


@pytest.mark.parametrize("lam0", [1e-4, 1.0])
def test_lm_fp64_matches_oracle(sm, lam0):
    wl = synth.ct_bearings([15, 40, 200, 1000], seed=31, q_form=1, sensor_jitter=0.2)
    x0 = starts(wl, 31)
    model = oracle.Model.from_workload(wl)
    d = workload_to_dev(wl, pes.FP64)
    for iters in (3, 8):
        ref = oracle.iterated_smoother_lm(model, wl["offsets"], wl["y"], wl["m0"], wl["P0"], x_init=x0, iters=iters,
                                          lambda0=lam0, nu=10.0)
        x, P, used, info = sm.ieks_run_lm(d["model"], pes.FP64, d["y"], d["offsets"], d["m0"], d["P0"],
                                          x_init=to_dev(x0), iters=iters, lambda0=lam0, nu=10.0)
        print(f"lam0 {lam0} iters {iters}: kept {info['accepted']} (oracle {ref['accepted']}), "
              f"lambda {info['lam']}")
        assert used == iters
        np.testing.assert_array_equal(info["accepted"], ref["accepted"])
        np.testing.assert_allclose(info["lam"], ref["lam"], rtol=1e-12)
        assert rel_err(x.cpu().numpy(), ref["x"], wl["offsets"]) < TOL_FP64
        assert rel_err(P.cpu().numpy(), ref["P"], wl["offsets"]) < TOL_FP64
    # the case exercises both decisions
    assert (ref["accepted"] < iters).any() and (ref["accepted"] > 0).all()


def test_lm_tolerance_mode_matches_oracle(sm):
    wl = synth.ct_bearings([60, 300], seed=32, q_form=1, sensor_jitter=0.2)
    x0 = starts(wl, 32)
    model = oracle.Model.from_workload(wl)
    d = workload_to_dev(wl, pes.FP64)
    ref = oracle.iterated_smoother_lm(model, wl["offsets"], wl["y"], wl["m0"], wl["P0"], x_init=x0, iters=60,
                                      tol=1e-8, lambda0=1e-2, nu=10.0)
    assert ref["status"] == oracle.OK
    x, P, used, info = sm.ieks_run_lm(d["model"], pes.FP64, d["y"], d["offsets"], d["m0"], d["P0"], x_init=to_dev(x0),
                                      iters=60, tol=1e-8, lambda0=1e-2, nu=10.0)
    # a step whose relative size is within rounding of tol may count on either
    # side of it: the converged iteration agrees to within one
    assert abs(used - ref["iters_used"]) <= 1
    assert np.abs(info["conv_iter"] - ref["conv_iter"]).max() <= 1
    assert rel_err(x.cpu().numpy(), ref["x"], wl["offsets"]) < TOL_FP64
    # at convergence the result is the IEKS fixed point: plain iterations leave it in place
    one = oracle.iterated_smoother(model, oracle.IEKS, wl["offsets"], wl["y"], wl["m0"], wl["P0"], x_init=ref["x"],
                                   iters=1)
    assert rel_err(one["x"], ref["x"], wl["offsets"]) < 1e-7


def test_lm_fp32_matches_oracle(sm):
    """FP32 steps, FP64 objective: the decisions of the first iterations (steps
    far larger than FP32 rounding) agree with the oracle's; near convergence
    the objective of a float trajectory no longer separates a step from the
    nominal, so a longer FP32 run may keep or reject differently there."""
    wl = synth.ct_bearings([40, 200], seed=33, q_form=1, sensor_jitter=0.2)
    x0 = starts(wl, 33)
    model = oracle.Model.from_workload(wl)
    d = workload_to_dev(wl, pes.FP32)
    ref = oracle.iterated_smoother_lm(model, wl["offsets"], wl["y"], wl["m0"], wl["P0"], x_init=x0, iters=3,
                                      lambda0=1.0, nu=10.0)
    x, P, used, info = sm.ieks_run_lm(d["model"], pes.FP32, d["y"], d["offsets"], d["m0"], d["P0"],
                                      x_init=to_dev(x0, torch.float32), iters=3, lambda0=1.0, nu=10.0)
    np.testing.assert_array_equal(info["accepted"], ref["accepted"])
    assert rel_err(x.double().cpu().numpy(), ref["x"], wl["offsets"]) < TOL_FP32
    assert rel_err(P.double().cpu().numpy(), ref["P"], wl["offsets"]) < TOL_FP32


def test_lm_rejects_singular_q_and_bad_arguments(sm):
    wl = synth.ct_bearings([20], seed=34, q_form=0)
    d = workload_to_dev(wl, pes.FP64)
    with pytest.raises(pes.PesError) as ei:
        sm.ieks_run_lm(d["model"], pes.FP64, d["y"], d["offsets"], d["m0"], d["P0"], iters=2)
    assert ei.value.status == pes.UNSUPPORTED
    wl = synth.ct_bearings([20], seed=34, q_form=1)
    d = workload_to_dev(wl, pes.FP64)
    for kw in (dict(lambda0=0.0), dict(nu=1.0), dict(iters=0)):
        with pytest.raises(pes.PesError) as ei:
            sm.ieks_run_lm(d["model"], pes.FP64, d["y"], d["offsets"], d["m0"], d["P0"], **kw)
        assert ei.value.status == pes.INVALID_ARG
