"""GPU parity of the fused iterated smoother (pes_ieks_run) and of the
linearisation (pes_linearize) against the oracle, element by element."""
import numpy as np
import pytest
import torch

import oracle
from paper_2102_00514_gb300 import pes, synth
from tests.gpu_common import (ORACLE_METHOD, TOL_FP32, TOL_FP64, gpu_run, oracle_run, ragged_with_prior_only,
                               rel_err, to_dev, workload_to_dev)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sm():
    s = pes.Smoother(1 << 21, 4096)
    yield s
    s.close()


@pytest.mark.parametrize("method", [pes.IEKS, pes.CUBATURE, pes.UNSCENTED, pes.GAUSS_HERMITE])
@pytest.mark.parametrize("prec", [pes.FP64, pes.FP32])
def test_linearize_matches_oracle(sm, method, prec):
    wl = synth.ct_bearings([40, 1, 300], seed=21, sensor_jitter=0.2, omega0_halfwidth=1.0)
    # a non-trivial nominal: one oracle iteration from the prior
    ut = (0.8, 2.0, 0.5) if method == pes.UNSCENTED else None
    out = oracle_run(wl, method, iters=1, ut=ut)
    om = oracle.Model.from_workload(wl)
    if ut is not None:
        om = om.unscented(*ut)
    ref = oracle.linearize(om, ORACLE_METHOD[method], wl["offsets"], out["x"], out["P"], wl["y"])
    dt = torch.float64 if prec == pes.FP64 else torch.float32
    d = workload_to_dev(wl, prec, ut)
    got = sm.linearize(d["model"], method, prec, to_dev(out["x"], dt), to_dev(out["P"], dt), d["y"], d["offsets"])
    sm.sync()
    tol = 1e-10 if prec == pes.FP64 else 2e-4
    # the offsets c = f - F xbar and d = h - H xbar are differences of terms of
    # the size of f(xbar) and h(xbar): their rounding is measured on that scale
    x = out["x"]
    Fx = np.einsum("ijk,jk->ik", ref["F"].reshape(5, 5, -1), x)
    Hx = np.einsum("ijk,jk->ik", ref["H"].reshape(2, 5, -1), x)
    scales = {"c": np.abs(Fx + ref["c"]).max(), "d": np.abs(Hx + ref["d"]).max()}
    for k in ("F", "c", "Qp", "H", "d", "Rp", "y_used"):
        g = got[k].double().cpu().numpy()
        scale = max(np.abs(ref[k]).max(), scales.get(k, 0.0), 1e-30)
        assert np.abs(g - ref[k]).max() / scale < tol, k


@pytest.mark.parametrize("name,method", [("ieks_T500", pes.IEKS), ("ipls_T10000", pes.CUBATURE),
                                         ("ipls_T10000", pes.IEKS), ("ieks_T500", pes.CUBATURE)])
def test_ieks_run_fp64_matches_oracle(sm, name, method):
    wl = synth.workload(name)
    ref = oracle_run(wl, method, iters=10)
    x, P, used, _ = gpu_run(sm, wl, method, pes.FP64, iters=10)
    assert used == 10
    assert rel_err(x, ref["x"], wl["offsets"]) < TOL_FP64
    assert rel_err(P, ref["P"], wl["offsets"]) < TOL_FP64


UT = [(1.0, 2.0, 1.0), (0.8, 2.0, 0.5)]


@pytest.mark.parametrize("ut", UT)
@pytest.mark.parametrize("name", ["ieks_T500", "ipls_T10000"])
def test_unscented_fp64_matches_oracle(sm, name, ut):
    wl = synth.workload(name)
    ref = oracle_run(wl, pes.UNSCENTED, iters=10, ut=ut)
    x, P, used, _ = gpu_run(sm, wl, pes.UNSCENTED, pes.FP64, iters=10, ut=ut)
    assert used == 10
    assert rel_err(x, ref["x"], wl["offsets"]) < TOL_FP64
    assert rel_err(P, ref["P"], wl["offsets"]) < TOL_FP64


def test_unscented_fp32_matches_oracle(sm):
    wl = synth.workload("ipls_T10000")
    ref = oracle_run(wl, pes.UNSCENTED, iters=10, ut=UT[0])
    x, P, _, _ = gpu_run(sm, wl, pes.UNSCENTED, pes.FP32, iters=10, ut=UT[0])
    assert rel_err(x, ref["x"], wl["offsets"]) < TOL_FP32
    assert rel_err(P, ref["P"], wl["offsets"]) < TOL_FP32


def test_unscented_with_cubature_parameters_equals_cubature(sm):
    wl = synth.workload("batch8_T1_3000")
    xa, Pa, _, _ = gpu_run(sm, wl, pes.UNSCENTED, pes.FP64, iters=3, ut=(1.0, 0.0, 0.0))
    xb, Pb, _, _ = gpu_run(sm, wl, pes.CUBATURE, pes.FP64, iters=3)
    assert rel_err(xa, xb, wl["offsets"]) < 1e-12
    assert rel_err(Pa, Pb, wl["offsets"]) < 1e-12


def test_unscented_sequential_matches_oracle(sm):
    wl = synth.workload("batch8_T1_3000")
    ref = oracle_run(wl, pes.UNSCENTED, iters=5, ut=UT[1])
    d = workload_to_dev(wl, pes.FP64, UT[1])
    x, P, _, _ = sm.ieks_run_sequential(d["model"], pes.UNSCENTED, pes.FP64, d["y"], d["offsets"], d["m0"], d["P0"],
                                        iters=5)
    assert rel_err(x.cpu().numpy(), ref["x"], wl["offsets"]) < TOL_FP64
    assert rel_err(P.cpu().numpy(), ref["P"], wl["offsets"]) < TOL_FP64


def test_unscented_parameters_validated(sm):
    wl = synth.workload("ieks_T500")
    for bad in ((1.0, 0.0, -5.0), (0.0, 2.0, 1.0)):   # n + lambda = 0; alpha = 0
        with pytest.raises(pes.PesError) as ei:
            gpu_run(sm, wl, pes.UNSCENTED, pes.FP64, iters=1, ut=bad)
        assert ei.value.status == pes.INVALID_ARG


@pytest.mark.parametrize("name,method", [("ieks_T500", pes.IEKS), ("ipls_T10000", pes.CUBATURE),
                                         ("ipls_T10000", pes.IEKS)])
def test_ieks_run_fp32_matches_oracle(sm, name, method):
    wl = synth.workload(name)
    ref = oracle_run(wl, method, iters=10)
    x, P, used, _ = gpu_run(sm, wl, method, pes.FP32, iters=10)
    ex = rel_err(x, ref["x"], wl["offsets"])
    eP = rel_err(P, ref["P"], wl["offsets"])
    print(f"{name} method {method} FP32: means {ex:.3e} covariances {eP:.3e}")
    assert ex < TOL_FP32 and eP < TOL_FP32


@pytest.mark.parametrize("method", [pes.IEKS, pes.CUBATURE])
def test_batched_segmented_fp64(sm, method):
    wl = synth.workload("batch64_T1_400")
    ref = oracle_run(wl, method, iters=5)
    x, P, used, _ = gpu_run(sm, wl, method, pes.FP64, iters=5)
    assert rel_err(x, ref["x"], wl["offsets"]) < TOL_FP64
    assert rel_err(P, ref["P"], wl["offsets"]) < TOL_FP64


@pytest.mark.parametrize("method", [pes.IEKS, pes.CUBATURE])
def test_prior_only_trajectories_in_a_ragged_batch(sm, method):
    """Trajectories without a measurement (T_b = 0) beside one-, two-step and
    longer ones: FP64 (persistent and sequential), FP32 and PES_MIXED agree with
    the oracle, and a prior-only trajectory's smoothed moments are its prior,
    exactly (its only element is the prior element)."""
    wl = ragged_with_prior_only()
    off = wl["offsets"]
    ref = oracle_run(wl, method, iters=10)
    heads = [int(off[b]) for b in range(len(off) - 1) if off[b + 1] - off[b] == 1]
    assert len(heads) == 2
    for prec, tol in ((pes.FP64, TOL_FP64), (pes.FP32, TOL_FP32), (pes.MIXED, TOL_FP32)):
        x, P, used, st = gpu_run(sm, wl, method, prec, iters=10)
        assert used == 10 and st == pes.OK
        assert rel_err(x, ref["x"], off) < tol, prec
        assert rel_err(P, ref["P"], off) < tol, prec
        narrow = (lambda a: a) if prec == pes.FP64 else (lambda a: np.float32(a).astype(np.float64))
        for h, b in zip(heads, (0, 4)):
            np.testing.assert_array_equal(x[:, h], narrow(wl["m0"][b]))
            np.testing.assert_array_equal(P[:, h], narrow(wl["P0"][b]))
    d = workload_to_dev(wl, pes.FP64)
    xs, Ps, _, _ = sm.ieks_run_sequential(d["model"], method, pes.FP64, d["y"], d["offsets"], d["m0"], d["P0"],
                                          iters=10)
    assert rel_err(xs.cpu().numpy(), ref["x"], off) < TOL_FP64
    assert rel_err(Ps.cpu().numpy(), ref["P"], off) < TOL_FP64


@pytest.mark.parametrize("method", [pes.IEKS, pes.CUBATURE])
def test_handle_at_exact_capacity_equals_a_larger_handle(sm, method):
    """N = max_states and B = max_batch: every precision runs within the
    handle's workspace (the lane padding and the refinement's workspace at
    their largest) and reproduces, bit for bit, a handle with room to spare
    (the launch shape depends on N alone)."""
    wl = synth.workload("batch8_T1_3000")
    N, B = wl["y"].shape[1], len(wl["offsets"]) - 1
    tight = pes.Smoother(N, B)
    try:
        for prec in (pes.FP64, pes.FP32, pes.MIXED, pes.REFINED):
            d = workload_to_dev(wl, prec)
            args = (d["model"], method, prec, d["y"], d["offsets"], d["m0"], d["P0"])
            xa, Pa, _, _ = sm.ieks_run(*args, iters=4)
            xb, Pb, _, _ = tight.ieks_run(*args, iters=4)
            torch.cuda.synchronize()
            assert torch.equal(xa, xb) and torch.equal(Pa, Pb), prec
    finally:
        tight.close()


def test_batched_equals_separate_runs(sm):
    wl = synth.workload("batch8_T1_3000")
    xb, Pb, _, _ = gpu_run(sm, wl, pes.CUBATURE, pes.FP64, iters=3)
    off = wl["offsets"]
    for b in range(len(off) - 1):
        sl = slice(int(off[b]), int(off[b + 1]))
        one = dict(wl, offsets=np.array([0, off[b + 1] - off[b]]), y=wl["y"][:, sl], m0=wl["m0"][b:b + 1],
                   P0=wl["P0"][b:b + 1], sensors=wl["sensors"][b:b + 1])
        x1, P1, _, _ = gpu_run(sm, one, pes.CUBATURE, pes.FP64, iters=3)
        assert rel_err(x1, xb[:, sl], one["offsets"]) < 1e-11
        assert rel_err(P1, Pb[:, sl], one["offsets"]) < 1e-11


def test_tolerance_mode_matches_oracle_iterations(sm):
    wl = synth.workload("ieks_T500")
    ref = oracle_run(wl, pes.IEKS, iters=50, tol=1e-6)
    x, P, used, st = gpu_run(sm, wl, pes.IEKS, pes.FP64, iters=50, tol=1e-6)
    assert st == pes.OK and used == ref["iters_used"]
    assert rel_err(x, ref["x"], wl["offsets"]) < TOL_FP64
    x, P, used, st = gpu_run(sm, wl, pes.IEKS, pes.FP64, iters=3, tol=1e-6, allow_not_converged=True)
    assert st == pes.NOT_CONVERGED and used == 3


def test_per_trajectory_iterations_match_oracle(sm):
    wl = synth.workload("batch8_T1_3000")
    x, P, used, st = gpu_run(sm, wl, pes.IEKS, pes.FP64, iters=50, tol=1e-6, allow_not_converged=True)
    its = sm.traj_iterations(8)
    off = wl["offsets"]
    for b in range(8):
        sl = slice(int(off[b]), int(off[b + 1]))
        one = dict(wl, offsets=np.array([0, off[b + 1] - off[b]]), y=wl["y"][:, sl], m0=wl["m0"][b:b + 1],
                   P0=wl["P0"][b:b + 1], sensors=wl["sensors"][b:b + 1])
        ref = oracle_run(one, pes.IEKS, iters=50, tol=1e-6)
        expect = ref["iters_used"] if ref["status"] == oracle.OK else 0
        assert its[b] == expect, (b, its[b], expect)
    assert used == (max(its) if (its > 0).all() else 50)
    with pytest.raises(pes.PesError):
        sm.traj_iterations(7)


def test_prior_init_equals_explicit_init(sm):
    wl = synth.workload("ieks_T500")
    d = workload_to_dev(wl, pes.FP64)
    N = wl["y"].shape[1]
    x0 = torch.tensor(np.tile(wl["m0"][0][:, None], (1, N)), dtype=torch.float64, device="cuda")
    P0 = torch.tensor(np.tile(wl["P0"][0][:, None], (1, N)), dtype=torch.float64, device="cuda")
    xa, Pa, _, _ = sm.ieks_run(d["model"], pes.CUBATURE, pes.FP64, d["y"], d["offsets"], d["m0"], d["P0"], iters=2)
    xb, Pb, _, _ = sm.ieks_run(d["model"], pes.CUBATURE, pes.FP64, d["y"], d["offsets"], d["m0"], d["P0"],
                               x_init=x0, P_init=P0, iters=2)
    sm.sync()
    assert torch.equal(xa, xb) and torch.equal(Pa, Pb)


@pytest.mark.parametrize("name,method", [("ieks_T500", pes.IEKS), ("ipls_T10000", pes.CUBATURE),
                                         ("ipls_T10000", pes.IEKS), ("ieks_T500", pes.CUBATURE)])
def test_ieks_run_mixed_matches_oracle(sm, name, method):
    """PES_MIXED: nine FP32 iterations, then the tenth in FP64 from the FP32
    nominal; the result is held to the FP32 bound against the oracle's ten
    FP64 iterations, and the final FP64 iteration equals a plain FP64 run of
    one iteration started from the same nominal."""
    wl = synth.workload(name)
    ref = oracle_run(wl, method, iters=10)
    x, P, used, _ = gpu_run(sm, wl, method, pes.MIXED, iters=10)
    assert used == 10
    ex = rel_err(x, ref["x"], wl["offsets"])
    eP = rel_err(P, ref["P"], wl["offsets"])
    print(f"{name} method {method} MIXED: means {ex:.3e} covariances {eP:.3e}")
    assert ex < TOL_FP32 and eP < TOL_FP32
    # the FP64 step on its own: the FP32 nominal of nine iterations, widened
    x9, P9, _, _ = gpu_run(sm, wl, method, pes.FP32, iters=9)
    r32 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
    wl32 = dict(wl, y=r32(wl["y"]), m0=r32(wl["m0"]), P0=r32(wl["P0"]))   # the float inputs, widened
    one = oracle_run(wl32, method, iters=1, x_init=x9, P_init=P9)
    # the only rounding left is the final narrowing to float
    assert rel_err(x, one["x"], wl["offsets"]) < 1e-6
    assert rel_err(P, one["P"], wl["offsets"]) < 1e-6


def test_host_entry_point_equals_device_entry_point(sm):
    wl = synth.workload("ieks_T500")
    d = workload_to_dev(wl, pes.FP32)
    xd, Pd, _, _ = sm.ieks_run(d["model"], pes.IEKS, pes.FP32, d["y"], d["offsets"], d["m0"], d["P0"], iters=4)
    sm.sync()
    h = lambda a, dt=torch.float32: torch.as_tensor(np.ascontiguousarray(a), dtype=dt).pin_memory()
    xh, Ph, used, _ = sm.ieks_run_host(d["model"], pes.IEKS, pes.FP32, h(wl["y"]), h(wl["offsets"], torch.int64),
                                       h(wl["m0"]), h(wl["P0"]), iters=4,
                                       sensors_host=h(wl["sensors"], torch.float64))
    assert used == 4
    assert torch.equal(xh, xd.cpu()) and torch.equal(Ph, Pd.cpu())


@pytest.mark.parametrize("method,prec", [(pes.IEKS, pes.FP32), (pes.CUBATURE, pes.FP64), (pes.CUBATURE, pes.REFINED)])
def test_host_entry_point_pinned_and_pageable_buffers(sm, method, prec):
    """Pinned or pageable host buffers, mixed, and outputs that are views
    inside larger pinned allocations (written exactly where they lie): the
    results equal the device entry point's bit for bit."""
    wl = synth.workload("ieks_T500")
    dt = torch.float64 if prec == pes.FP64 else torch.float32
    d = workload_to_dev(wl, pes.FP64 if prec == pes.FP64 else pes.FP32)
    xd, Pd, _, _ = sm.ieks_run(d["model"], method, prec, d["y"], d["offsets"], d["m0"], d["P0"], iters=3)
    sm.sync()
    xd, Pd = xd.cpu(), Pd.cpu()
    N = wl["y"].shape[1]
    host = lambda a, t=dt, pin=True: (torch.as_tensor(np.ascontiguousarray(a), dtype=t).pin_memory() if pin
                                      else torch.as_tensor(np.ascontiguousarray(a), dtype=t).clone())
    sens = host(wl["sensors"], torch.float64)
    off, m0, P0 = host(wl["offsets"], torch.int64), host(wl["m0"]), host(wl["P0"])
    big_x = torch.zeros(5 * N + 37, dtype=dt).pin_memory()
    big_P = torch.zeros(15 * N + 11, dtype=dt).pin_memory()
    cases = {
        "pinned": (host(wl["y"]), None, None),
        "pageable": (host(wl["y"], pin=False), torch.empty((5, N), dtype=dt), torch.empty((15, N), dtype=dt)),
        "mixed": (host(wl["y"], pin=False), None, torch.empty((15, N), dtype=dt)),
        "views": (host(wl["y"]), big_x[37:].view(5, N), big_P[11:].view(15, N)),
    }
    for name, (y, xo, Po) in cases.items():
        xh, Ph, used, _ = sm.ieks_run_host(d["model"], method, prec, y, off, m0, P0, iters=3, x_out=xo, P_out=Po,
                                           sensors_host=sens)
        assert used == 3
        assert torch.equal(xh, xd) and torch.equal(Ph, Pd), name
    assert torch.all(big_x[:37] == 0) and torch.all(big_P[:11] == 0)


def test_invalid_arguments_rejected_before_launch(sm):
    wl = synth.workload("ieks_T500")
    d = workload_to_dev(wl, pes.FP64)
    with pytest.raises(pes.PesError) as ei:
        sm.ieks_run(d["model"], pes.IEKS, pes.FP64, d["y"], d["offsets"], d["m0"], d["P0"], iters=0)
    assert ei.value.status == pes.INVALID_ARG
    # PES_MIXED exists for the fused iterated smoother only
    lin = {k: torch.zeros((n, d["y"].shape[1]), dtype=torch.float32, device="cuda")
           for k, n in (("F", 25), ("c", 5), ("Qp", 15), ("H", 10), ("d", 2), ("Rp", 3))}
    with pytest.raises(pes.PesError) as ei:
        sm.filter_scan(pes.MIXED, lin, d["y"].float(), d["m0"].float(), d["P0"].float(), d["offsets"])
    assert ei.value.status == pes.UNSUPPORTED


def test_nonfinite_measurement_reported(sm):
    wl = synth.workload("ieks_T500")
    wl = dict(wl, y=wl["y"].copy())
    wl["y"][0, 250] = np.nan
    with pytest.raises(pes.PesError) as ei:
        gpu_run(sm, wl, pes.IEKS, pes.FP64, iters=2)
    assert ei.value.status in (pes.NONFINITE, pes.NOT_PD)
    # the handle is usable afterwards
    x, P, used, st = gpu_run(sm, synth.workload("ieks_T500"), pes.IEKS, pes.FP64, iters=1)
    assert st == pes.OK


def test_not_positive_definite_prior_reported(sm):
    wl = synth.workload("ieks_T500")
    wl = dict(wl, P0=wl["P0"].copy())
    wl["P0"][0, 0] = -1.0   # P0[0,0] < 0
    with pytest.raises(pes.PesError) as ei:
        gpu_run(sm, wl, pes.CUBATURE, pes.FP64, iters=2)
    assert ei.value.status in (pes.NOT_PD, pes.NONFINITE)


def test_a_grid_barrier_that_cannot_complete_times_out_and_the_context_survives(monkeypatch):
    """The failure path of the smoother kernel's grid barriers, with no GPU
    fault: a handle created with PES_TEST_BARRIER_SHORT starts every launch's
    barrier count one arrival short, so no barrier can complete. With a 50 ms
    limit (PES_BARRIER_TIMEOUT_MS) the first barrier gives up, the others see
    the status and do not wait, the kernel ends, and the call returns
    PES_ERR_TIMEOUT well within a second. A handle created afterwards runs
    normally on the same context."""
    import time
    wl = synth.workload("ieks_T500")
    N = wl["y"].shape[1]
    monkeypatch.setenv("PES_TEST_BARRIER_SHORT", "1")
    monkeypatch.setenv("PES_BARRIER_TIMEOUT_MS", "50")
    bad = pes.Smoother(N, 1)
    monkeypatch.delenv("PES_TEST_BARRIER_SHORT")
    monkeypatch.delenv("PES_BARRIER_TIMEOUT_MS")
    t0 = time.perf_counter()
    with pytest.raises(pes.PesError) as ei:
        gpu_run(bad, wl, pes.IEKS, pes.FP32, iters=3)
    assert ei.value.status == pes.TIMEOUT
    assert time.perf_counter() - t0 < 1.0
    bad.close()
    good = pes.Smoother(N, 1)
    ref = oracle_run(wl, pes.IEKS, iters=3)
    x, P, used, st = gpu_run(good, wl, pes.IEKS, pes.FP64, iters=3)
    assert used == 3 and st == pes.OK
    assert rel_err(x, ref["x"], wl["offsets"]) < TOL_FP64 and rel_err(P, ref["P"], wl["offsets"]) < TOL_FP64
    good.close()


def test_handles_on_concurrent_host_threads_give_the_sequential_results():
    """Handles are independent: two host threads, each with its own handle and
    stream, running the host-buffer entry point at the same time (IEKS on one,
    cubature on the other, several calls each) get bit for bit what the same
    calls give one after the other."""
    import concurrent.futures as cf
    wl = synth.workload("batch8_T100_3000")
    N, B = wl["y"].shape[1], len(wl["offsets"]) - 1
    pin = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt).pin_memory()
    hy, hoff = pin(wl["y"], torch.float32), pin(wl["offsets"], torch.int64)
    hm0, hP0, hs = pin(wl["m0"], torch.float32), pin(wl["P0"], torch.float32), pin(wl["sensors"], torch.float64)
    model = workload_to_dev(wl, pes.FP32)["model"]
    methods = (pes.IEKS, pes.CUBATURE)
    handles = {m: pes.Smoother(N, B) for m in methods}
    streams = {m: torch.cuda.Stream() for m in methods}
    device = torch.cuda.current_device()

    def run(m, prec, reps):
        torch.cuda.set_device(device)
        out = []
        for _ in range(reps):
            x, P, _, _ = handles[m].ieks_run_host(model, m, prec, hy, hoff, hm0, hP0, iters=4, sensors_host=hs,
                                                  stream=streams[m])
            out.append((x.clone(), P.clone()))
        return out

    for prec in (pes.FP32, pes.REFINED):
        seq = {m: run(m, prec, 1)[0] for m in methods}
        with cf.ThreadPoolExecutor(2) as ex:
            conc = dict(zip(methods, ex.map(lambda m: run(m, prec, 3), methods)))
        for m in methods:
            for x, P in conc[m]:
                assert torch.equal(x, seq[m][0]) and torch.equal(P, seq[m][1]), (prec, m)
    for h_ in handles.values():
        h_.close()


def test_autotune_keeps_a_valid_shape_and_results():
    s = pes.Smoother(1 << 16, 64)
    wl = synth.workload("batch16_T100_3000")
    d = workload_to_dev(wl, pes.FP32)
    N = wl["y"].shape[1]
    before = s.launch_shape(pes.CUBATURE, pes.FP32, N)
    nt, min_steps, ms = s.autotune(d["model"], pes.CUBATURE, pes.FP32, d["y"], d["offsets"], d["m0"], d["P0"], iters=2)
    assert nt in (128, 256) and min_steps in (4, 8, 16, 32, 64, 128) and ms > 0
    nb, nt2, L = s.launch_shape(pes.CUBATURE, pes.FP32, N)
    assert nt2 == nt and nb * nt * L >= N
    print(f"autotune: {before} -> {(nb, nt2, L)}, {ms:.3f} ms per run")
    # the other method and precision keep their defaults
    assert s.launch_shape(pes.IEKS, pes.FP32, N)[1] == 256
    # a tuned shape changes only the partition into lanes: FP64 results stay
    # within rounding of the oracle
    d64 = workload_to_dev(wl, pes.FP64)
    s.autotune(d64["model"], pes.CUBATURE, pes.FP64, d64["y"], d64["offsets"], d64["m0"], d64["P0"], iters=2)
    ref = oracle_run(wl, pes.CUBATURE, iters=4)
    x, P, _, _ = gpu_run(s, wl, pes.CUBATURE, pes.FP64, iters=4)
    assert rel_err(x, ref["x"], wl["offsets"]) < TOL_FP64
    assert rel_err(P, ref["P"], wl["offsets"]) < TOL_FP64
    s.close()


def test_tuning_cache_reapplies_a_recorded_shape(tmp_path):
    """A tuning recorded in a cache file is applied by a fresh handle without
    timing: the same launch shape and bit-identical results."""
    cache = str(tmp_path / "tune.json")
    wl = synth.workload("batch16_T100_3000")
    d = workload_to_dev(wl, pes.FP32)
    N = wl["y"].shape[1]
    args = (d["model"], pes.CUBATURE, pes.FP32, d["y"], d["offsets"], d["m0"], d["P0"])
    a = pes.Smoother(1 << 16, 64)
    tuned = a.autotune(*args, iters=2, cache=cache)
    assert len(pes.read_tune_cache(cache)) == 1
    b = pes.Smoother(1 << 16, 64)
    assert b.autotune(*args, iters=2, cache=cache) == tuned
    assert a.launch_shape(pes.CUBATURE, pes.FP32, N) == b.launch_shape(pes.CUBATURE, pes.FP32, N)
    xa, Pa, _, _ = a.ieks_run(*args, iters=3)
    xb, Pb, _, _ = b.ieks_run(*args, iters=3)
    torch.cuda.synchronize()
    assert torch.equal(xa, xb) and torch.equal(Pa, Pb)
    # shapes that are not compiled are refused and the choice stays
    for nt, steps in ((64, 8), (256, 0), (0, 4)):
        with pytest.raises(pes.PesError) as ei:
            b.set_launch_shape(pes.CUBATURE, pes.FP32, nt, steps)
        assert ei.value.status == pes.INVALID_ARG
    with pytest.raises(pes.PesError):
        b.set_launch_shape(pes.CUBATURE, pes.FP64, 256, 8)
    assert b.launch_shape(pes.CUBATURE, pes.FP32, N) == a.launch_shape(pes.CUBATURE, pes.FP32, N)
    b.set_launch_shape(pes.CUBATURE, pes.FP32, 0, 0)   # back to the defaults
    assert b.launch_shape(pes.CUBATURE, pes.FP32, N)[1] == 256
    a.close()
    b.close()


def test_graph_replay_equals_direct_call(sm):
    wl = synth.workload("batch8_T1_3000")
    for method in (pes.IEKS, pes.CUBATURE):
        d = workload_to_dev(wl, pes.FP32)
        x, P, _, _ = sm.ieks_run(d["model"], method, pes.FP32, d["y"], d["offsets"], d["m0"], d["P0"], iters=3)
        sm.sync()
        g = sm.graph(d["model"], method, pes.FP32, d["y"], d["offsets"], d["m0"], d["P0"], iters=3)
        g.launch()
        sm.sync()
        assert torch.equal(g.x, x) and torch.equal(g.P, P)
        # new contents at the same addresses: the replay follows them
        d["y"].mul_(1.0001)
        x2, P2, _, _ = sm.ieks_run(d["model"], method, pes.FP32, d["y"], d["offsets"], d["m0"], d["P0"], iters=3)
        sm.sync()
        g.launch()
        sm.sync()
        assert torch.equal(g.x, x2) and torch.equal(g.P, P2) and not torch.equal(x2, x)
        g.close()


@pytest.mark.parametrize("lm", [1.0, 50.0])
@pytest.mark.parametrize("name,method", [("ieks_T500", pes.IEKS), ("ipls_T10000", pes.CUBATURE),
                                         ("batch64_T1_400", pes.IEKS)])
def test_damped_fp64_matches_oracle(sm, name, method, lm):
    wl = synth.workload(name)
    ref = oracle_run(wl, method, iters=10, lm=lm)
    x, P, used, _ = gpu_run(sm, wl, method, pes.FP64, iters=10, lm=lm)
    assert rel_err(x, ref["x"], wl["offsets"]) < TOL_FP64
    assert rel_err(P, ref["P"], wl["offsets"]) < TOL_FP64


def test_damped_fp32_and_sequential_match_oracle(sm):
    wl = synth.workload("ipls_T10000")
    ref = oracle_run(wl, pes.IEKS, iters=10, lm=10.0)
    x, P, _, _ = gpu_run(sm, wl, pes.IEKS, pes.FP32, iters=10, lm=10.0)
    assert rel_err(x, ref["x"], wl["offsets"]) < TOL_FP32
    assert rel_err(P, ref["P"], wl["offsets"]) < TOL_FP32
    wl = synth.workload("batch8_T1_3000")
    ref = oracle_run(wl, pes.CUBATURE, iters=5, lm=3.0)
    d = workload_to_dev(wl, pes.FP64, lm=3.0)
    x, P, _, _ = sm.ieks_run_sequential(d["model"], pes.CUBATURE, pes.FP64, d["y"], d["offsets"], d["m0"], d["P0"],
                                        iters=5)
    assert rel_err(x.cpu().numpy(), ref["x"], wl["offsets"]) < TOL_FP64
    assert rel_err(P.cpu().numpy(), ref["P"], wl["offsets"]) < TOL_FP64


def test_damping_rejects_negative_lambda(sm):
    wl = synth.workload("ieks_T500")
    with pytest.raises(pes.PesError) as ei:
        gpu_run(sm, wl, pes.IEKS, pes.FP64, iters=1, lm=-1.0)
    assert ei.value.status == pes.INVALID_ARG


def test_mixed_tolerance_mode(sm):
    """PES_MIXED in tolerance mode: FP32 iterations until the tolerance (or
    max_iters - 1), then one FP64 iteration; the result matches the FP64
    oracle iterated to the same tolerance within the FP32 bound."""
    wl = synth.workload("ieks_T500")
    ref = oracle_run(wl, pes.IEKS, iters=50, tol=1e-6)
    x, P, used, st = gpu_run(sm, wl, pes.IEKS, pes.MIXED, iters=50, tol=1e-6, allow_not_converged=True)
    assert st == pes.OK
    assert 2 <= used <= ref["iters_used"] + 3
    assert rel_err(x, ref["x"], wl["offsets"]) < TOL_FP32
    assert rel_err(P, ref["P"], wl["offsets"]) < TOL_FP32


@pytest.mark.parametrize("name,iters", [("ieks_T500", 10), ("ipls_T10000", 10), ("batch64_T1_400", 5)])
def test_gauss_hermite_fp64_matches_oracle(sm, name, iters):
    # the batch holds short trajectories whose iteration has not converged:
    # five iterations, as for the other rules' batched checks
    wl = synth.workload(name)
    ref = oracle_run(wl, pes.GAUSS_HERMITE, iters=iters)
    x, P, used, _ = gpu_run(sm, wl, pes.GAUSS_HERMITE, pes.FP64, iters=iters)
    assert used == iters
    assert rel_err(x, ref["x"], wl["offsets"]) < TOL_FP64
    assert rel_err(P, ref["P"], wl["offsets"]) < TOL_FP64


def test_gauss_hermite_fp32_and_sequential_match_oracle(sm):
    wl = synth.workload("ipls_T10000")
    ref = oracle_run(wl, pes.GAUSS_HERMITE, iters=10)
    x, P, _, _ = gpu_run(sm, wl, pes.GAUSS_HERMITE, pes.FP32, iters=10)
    print(f"Gauss-Hermite FP32: means {rel_err(x, ref['x'], wl['offsets']):.2e} "
          f"covariances {rel_err(P, ref['P'], wl['offsets']):.2e}")
    assert rel_err(x, ref["x"], wl["offsets"]) < TOL_FP32
    assert rel_err(P, ref["P"], wl["offsets"]) < TOL_FP32
    wl = synth.workload("batch8_T1_3000")
    ref = oracle_run(wl, pes.GAUSS_HERMITE, iters=4)
    d = workload_to_dev(wl, pes.FP64)
    x, P, _, _ = sm.ieks_run_sequential(d["model"], pes.GAUSS_HERMITE, pes.FP64, d["y"], d["offsets"], d["m0"],
                                        d["P0"], iters=4)
    assert rel_err(x.cpu().numpy(), ref["x"], wl["offsets"]) < TOL_FP64
    assert rel_err(P.cpu().numpy(), ref["P"], wl["offsets"]) < TOL_FP64
