"""A batch large enough that the per-state handoff arrays' element offsets pass
2^31: the smoothing-element handoff (50 scalars per state) and the stored
linearisation (65 per state) of 46 million states. Every index into them must
be 64-bit; a 32-bit offset would land the last trajectories' elements at the
wrong place. Those trajectories sit at the highest offsets (a warp's lanes hold
consecutive chunks of the concatenation), so the sample takes the last ones as
well as the first and seeded random ones, each checked against the oracle
smoothing it alone (FP64, 1e-9)."""
import numpy as np
import pytest

from paper_2102_00514_gb300 import pes, synth
from tests.gpu_common import TOL_FP64, gpu_run, oracle_run, rel_err

pytestmark = pytest.mark.gpu

ITERS = 2


@pytest.fixture(scope="module")
def batch():
    wl = synth.workload("batch4600")
    N = wl["y"].shape[1]
    assert 50 * N > 2 ** 31 and 65 * N > 2 ** 31
    B = len(wl["offsets"]) - 1
    rng = np.random.default_rng(4600)
    pick = {0, 1, B - 3, B - 2, B - 1} | set(int(b) for b in rng.choice(B, 3, replace=False))
    return wl, sorted(pick)


@pytest.fixture(scope="module")
def sm(batch):
    wl, _ = batch
    s = pes.Smoother(wl["y"].shape[1], len(wl["offsets"]) - 1)
    yield s
    s.close()


@pytest.mark.parametrize("method", [pes.IEKS, pes.CUBATURE])
def test_offsets_past_two_to_the_31_fp64_sampled_trajectories(batch, sm, method):
    wl, pick = batch
    off = wl["offsets"]
    x, P, used, _ = gpu_run(sm, wl, method, pes.FP64, iters=ITERS)
    assert used == ITERS
    assert np.isfinite(x).all() and np.isfinite(P).all()
    assert (P[[0, 5, 9, 12, 14]] > 0).all()
    for b in pick:
        sl = slice(int(off[b]), int(off[b + 1]))
        one = dict(wl, offsets=np.array([0, off[b + 1] - off[b]], dtype=np.int64), y=wl["y"][:, sl],
                   x_true=wl["x_true"][:, sl], m0=wl["m0"][b:b + 1], P0=wl["P0"][b:b + 1],
                   sensors=wl["sensors"][b:b + 1])
        ref = oracle_run(one, method, iters=ITERS)
        ex = rel_err(x[:, sl], ref["x"], one["offsets"])
        eP = rel_err(P[:, sl], ref["P"], one["offsets"])
        assert ex < TOL_FP64 and eP < TOL_FP64, (b, ex, eP)
