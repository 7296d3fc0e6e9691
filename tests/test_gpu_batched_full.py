"""The batched workload at full size: 4,096 independent trajectories with
lengths uniform in 100..20,000 (about 41 million states), truth turn rates
U(-1, 1) and sensors jittered by U(-0.2, 0.2), all in one launch per method.

The oracle cannot smooth all 41 million states within a test, so parity is
checked on sampled trajectories, each smoothed by the oracle on its own: the
trajectories of a batch are independent (the segment head carries the prior
element, Sec. 2), so the batched result for trajectory b must equal the
oracle's result for trajectory b alone. The sample takes the shortest and the
longest trajectory, the first and the last of the concatenation, and seeded
random ones. Properties checked on every trajectory: finite means, and
symmetric positive diagonal covariances.
"""
import numpy as np
import pytest

from paper_2102_00514_gb300 import pes, synth
from tests.gpu_common import TOL_FP32, TOL_FP64, gpu_run, oracle_run, rel_err

pytestmark = pytest.mark.gpu

ITERS = 10


@pytest.fixture(scope="module")
def batch():
    wl = synth.workload("batch4096")
    off = wl["offsets"]
    T = np.diff(off) - 1
    rng = np.random.default_rng(4096)
    pick = {0, len(T) - 1, int(np.argmin(T)), int(np.argmax(T))}
    pick |= set(int(b) for b in rng.choice(len(T), 4, replace=False))
    return wl, sorted(pick)


@pytest.fixture(scope="module")
def sm(batch):
    wl, _ = batch
    s = pes.Smoother(wl["y"].shape[1], len(wl["offsets"]) - 1)
    yield s
    s.close()


def one_trajectory(wl, b):
    off = wl["offsets"]
    sl = slice(int(off[b]), int(off[b + 1]))
    return dict(wl, offsets=np.array([0, off[b + 1] - off[b]], dtype=np.int64), y=wl["y"][:, sl],
                x_true=wl["x_true"][:, sl], m0=wl["m0"][b:b + 1], P0=wl["P0"][b:b + 1],
                sensors=wl["sensors"][b:b + 1]), sl


def check_properties(x, P):
    assert np.isfinite(x).all() and np.isfinite(P).all()
    # packed upper triangle of 5x5: the diagonal sits at 0, 5, 9, 12, 14
    assert (P[[0, 5, 9, 12, 14]] > 0).all()


@pytest.mark.parametrize("method", [pes.IEKS, pes.CUBATURE])
@pytest.mark.parametrize("prec", [pes.FP32, pes.MIXED, pes.FP64])
def test_batch4096_sampled_trajectories_match_oracle(batch, sm, method, prec):
    wl, pick = batch
    assert wl["y"].shape[1] > 40_000_000 and len(wl["offsets"]) == 4097
    x, P, used, _ = gpu_run(sm, wl, method, prec, iters=ITERS)
    assert used == ITERS
    check_properties(x, P)
    tol = TOL_FP64 if prec == pes.FP64 else TOL_FP32
    worst = (0.0, 0.0)
    for b in pick:
        one, sl = one_trajectory(wl, b)
        ref = oracle_run(one, method, iters=ITERS)
        ex = rel_err(x[:, sl], ref["x"], one["offsets"])
        eP = rel_err(P[:, sl], ref["P"], one["offsets"])
        worst = (max(worst[0], ex), max(worst[1], eP))
        assert ex < tol and eP < tol, (b, int(one["offsets"][1]) - 1, ex, eP)
    print(f"batch4096 method {method} prec {prec}: worst sampled means {worst[0]:.3e} covariances {worst[1]:.3e}")
