"""The sequential counterpart on the GPU (pes_ieks_run_sequential: one thread
per trajectory) against the oracle and against the parallel path."""
import numpy as np
import pytest
import torch

import oracle
from paper_2102_00514_gb300 import pes, synth
from tests.gpu_common import TOL_FP32, TOL_FP64, gpu_run, oracle_run, rel_err, workload_to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sm():
    s = pes.Smoother(1 << 20, 4096)
    yield s
    s.close()


def seq_run(sm, wl, method, prec, iters=10, tol=0.0):
    d = workload_to_dev(wl, prec)
    x, P, used, st = sm.ieks_run_sequential(d["model"], method, prec, d["y"], d["offsets"], d["m0"], d["P0"],
                                            iters=iters, tol=tol, allow_not_converged=True)
    torch.cuda.synchronize()
    return x.double().cpu().numpy(), P.double().cpu().numpy(), used, st


@pytest.mark.parametrize("method", [pes.IEKS, pes.CUBATURE])
@pytest.mark.parametrize("name", ["ieks_T500", "batch64_T1_400"])
def test_sequential_fp64_matches_oracle(sm, method, name):
    wl = synth.workload(name)
    ref = oracle_run(wl, method, iters=10)
    x, P, used, st = seq_run(sm, wl, method, pes.FP64)
    assert used == 10 and st == pes.OK
    assert rel_err(x, ref["x"], wl["offsets"]) < TOL_FP64
    assert rel_err(P, ref["P"], wl["offsets"]) < TOL_FP64


@pytest.mark.parametrize("method", [pes.IEKS, pes.CUBATURE])
def test_sequential_fp32_matches_oracle(sm, method):
    wl = synth.workload("ipls_T10000")
    ref = oracle_run(wl, method, iters=10)
    x, P, _, _ = seq_run(sm, wl, method, pes.FP32)
    assert rel_err(x, ref["x"], wl["offsets"]) < TOL_FP32
    assert rel_err(P, ref["P"], wl["offsets"]) < TOL_FP32


def test_sequential_equals_parallel(sm):
    wl = synth.workload("batch32_T1_3000")
    for method in (pes.IEKS, pes.CUBATURE):
        xs, Ps, _, _ = seq_run(sm, wl, method, pes.FP64, iters=4)
        xp, Pp, _, _ = gpu_run(sm, wl, method, pes.FP64, iters=4)
        assert rel_err(xs, xp, wl["offsets"]) < 1e-11
        assert rel_err(Ps, Pp, wl["offsets"]) < 1e-11


def test_sequential_stops_each_trajectory_at_its_own_tolerance(sm):
    # every trajectory iterates until its own update meets tol, exactly as the
    # oracle run on that trajectory alone
    wl = synth.workload("batch8_T1_3000")
    x, P, used, st = seq_run(sm, wl, pes.IEKS, pes.FP64, iters=50, tol=1e-6)
    its = sm.traj_iterations(8)
    off = wl["offsets"]
    for b in range(8):
        sl = slice(int(off[b]), int(off[b + 1]))
        one = dict(wl, offsets=np.array([0, off[b + 1] - off[b]]), y=wl["y"][:, sl], m0=wl["m0"][b:b + 1],
                   P0=wl["P0"][b:b + 1], sensors=wl["sensors"][b:b + 1])
        ref = oracle_run(one, pes.IEKS, iters=50, tol=1e-6)
        expect = ref["iters_used"] if ref["status"] == oracle.OK else 0
        assert its[b] == expect, (b, its[b], expect)
        assert rel_err(x[:, sl], ref["x"], one["offsets"]) < TOL_FP64
    assert used == its.max() or (its == 0).any()
    assert (st == pes.OK) == bool((its > 0).all())


def test_sequential_rejects_mixed(sm):
    wl = synth.workload("ieks_T500")
    d = workload_to_dev(wl, pes.FP32)
    with pytest.raises(pes.PesError) as ei:
        sm.ieks_run_sequential(d["model"], pes.IEKS, pes.MIXED, d["y"], d["offsets"], d["m0"], d["P0"], iters=2)
    assert ei.value.status == pes.UNSUPPORTED
