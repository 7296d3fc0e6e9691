"""The allocation-free entry point pes_ieks_run_noalloc.

It is meant for callers that cannot create a handle because pes_create
allocates device memory (a fixed memory plan after start-up, a framework that
owns every allocation, a latency budget that rules out an allocation that may
synchronise the device). Its results must equal those of pes_ieks_run, which
it shares every kernel with, call after call, although all calls reuse one
fixed scratch array. This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2102_00514_gb300 import pes, synth
from tests.gpu_common import TOL_FP32, TOL_FP64, rel_err, workload_to_dev

pytestmark = pytest.mark.gpu


def run_noalloc(lib, d, method, prec, N, B, iters, tol=0.0, out=None):
    dt = torch.float64 if prec == pes.FP64 else torch.float32
    if out is None:
        out = (torch.empty((5, N), dtype=dt, device="cuda"), torch.empty((15, N), dtype=dt, device="cuda"))
    x, P = out
    used = ctypes.c_int32(0)
    ms = d["model"].as_struct()
    st = lib.pes_ieks_run_noalloc(ctypes.byref(ms), method, prec, d["y"].data_ptr(), d["offsets"].data_ptr(), B, N,
                                  d["m0"].data_ptr(), d["P0"].data_ptr(), None, None, iters, tol, x.data_ptr(),
                                  P.data_ptr(), ctypes.byref(used), torch.cuda.current_stream().cuda_stream)
    return st, x, P, used.value


@pytest.mark.parametrize("prec,tol", [(pes.FP64, TOL_FP64), (pes.FP32, TOL_FP32)])
@pytest.mark.parametrize("method", [pes.IEKS, pes.CUBATURE])
def test_noalloc_matches_handle_entry_point_twice(method, prec, tol):
    lib = pes.load_library()
    for wl in (synth.workload("ieks_T500"), synth.ct_bearings([300, 1, 41], seed=3, sensor_jitter=0.2)):
        d = workload_to_dev(wl, prec)
        N = wl["y"].shape[1]
        B = len(wl["offsets"]) - 1
        sm = pes.Smoother(N, B)
        xr, Pr, _, _ = sm.ieks_run(d["model"], method, prec, d["y"], d["offsets"], d["m0"], d["P0"], iters=4)
        sm.sync()
        ref_x, ref_P = xr.double().cpu().numpy(), Pr.double().cpu().numpy()
        sm.close()
        for _ in range(2):   # two calls in a row share the scratch
            st, x, P, used = run_noalloc(lib, d, method, prec, N, B, 4)
            assert st == pes.OK and used == 4
            assert rel_err(x.double().cpu().numpy(), ref_x, wl["offsets"]) < tol
            assert rel_err(P.double().cpu().numpy(), ref_P, wl["offsets"]) < tol


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = pes.load_library()
    wl = synth.ct_bearings([8192], seed=4)   # N = 8193 states, one more than the limit
    d = workload_to_dev(wl, pes.FP32)
    st, _, _, _ = run_noalloc(lib, d, pes.IEKS, pes.FP32, wl["y"].shape[1], 1, 1)
    assert st == pes.INVALID_ARG


def test_noalloc_rejects_mixed_and_refined_precision():
    # PES_MIXED keeps FP64 copies, PES_REFINED a workspace, that pes_ieks_run allocates
    lib = pes.load_library()
    wl = synth.workload("ieks_T500")
    d = workload_to_dev(wl, pes.FP32)
    for prec in (pes.MIXED, pes.REFINED):
        st, _, _, _ = run_noalloc(lib, d, pes.IEKS, prec, wl["y"].shape[1], 1, 2)
        assert st == pes.UNSUPPORTED


@pytest.mark.parametrize("method", [pes.IEKS, pes.CUBATURE])
def test_noalloc_at_its_limits_allocates_nothing(method):
    """N = PES_NOALLOC_MAX_STATES states in B = PES_NOALLOC_MAX_BATCH
    trajectories (the lane padding closest to the scratch's capacity, the
    per-trajectory arrays full), equal to pes_ieks_run; free device memory as
    cudaMemGetInfo reports it does not change between a first and a second call."""
    lib = pes.load_library()
    B, N = 64, 8192
    wl = synth.ct_bearings(np.full(B, N // B - 1), seed=6, sensor_jitter=0.2, omega0_halfwidth=1.0)
    assert wl["y"].shape[1] == N
    d = workload_to_dev(wl, pes.FP32)
    sm = pes.Smoother(N, B)
    xr, Pr, _, _ = sm.ieks_run(d["model"], method, pes.FP32, d["y"], d["offsets"], d["m0"], d["P0"], iters=3)
    sm.sync()
    ref_x, ref_P = xr.double().cpu().numpy(), Pr.double().cpu().numpy()
    sm.close()
    out = (torch.empty((5, N), dtype=torch.float32, device="cuda"),
           torch.empty((15, N), dtype=torch.float32, device="cuda"))
    st, x, P, used = run_noalloc(lib, d, method, pes.FP32, N, B, 3, out=out)
    assert st == pes.OK and used == 3
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    st, x, P, used = run_noalloc(lib, d, method, pes.FP32, N, B, 3, out=out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before
    assert st == pes.OK and used == 3
    assert rel_err(x.double().cpu().numpy(), ref_x, wl["offsets"]) < TOL_FP32
    assert rel_err(P.double().cpu().numpy(), ref_P, wl["offsets"]) < TOL_FP32


def test_noalloc_tolerance_mode_matches_handle_entry_point():
    lib = pes.load_library()
    wl = synth.workload("ieks_T500")
    N = wl["y"].shape[1]
    d = workload_to_dev(wl, pes.FP64)
    sm = pes.Smoother(N, 1)
    xr, Pr, used_r, _ = sm.ieks_run(d["model"], pes.IEKS, pes.FP64, d["y"], d["offsets"], d["m0"], d["P0"],
                                    iters=40, tol=1e-6)
    ref_x = xr.cpu().numpy()
    sm.close()
    for _ in range(2):
        st, x, P, used = run_noalloc(lib, d, pes.IEKS, pes.FP64, N, 1, 40, tol=1e-6)
        assert st == pes.OK and used == used_r
        assert rel_err(x.cpu().numpy(), ref_x, wl["offsets"]) < TOL_FP64
    # a tolerance the iteration cannot reach: not converged, outputs still set
    st, x, _, used = run_noalloc(lib, d, pes.IEKS, pes.FP64, N, 1, 2, tol=1e-14)
    assert st == pes.NOT_CONVERGED and used == 2 and np.isfinite(x.cpu().numpy()).all()


def test_noalloc_unscented_and_damped_match_handle_entry_point():
    lib = pes.load_library()
    wl = synth.ct_bearings([300, 41], seed=5, sensor_jitter=0.2)
    N, B = wl["y"].shape[1], 2
    d = workload_to_dev(wl, pes.FP64)
    d["model"].ut_alpha, d["model"].ut_beta, d["model"].ut_kappa = 1.0, 2.0, 1.0
    d["model"].lm_lambda = 2.0
    sm = pes.Smoother(N, B)
    xr, Pr, _, _ = sm.ieks_run(d["model"], pes.UNSCENTED, pes.FP64, d["y"], d["offsets"], d["m0"], d["P0"], iters=3)
    sm.sync()
    ref_x, ref_P = xr.cpu().numpy(), Pr.cpu().numpy()
    sm.close()
    st, x, P, used = run_noalloc(lib, d, pes.UNSCENTED, pes.FP64, N, B, 3)
    assert st == pes.OK and used == 3
    assert rel_err(x.cpu().numpy(), ref_x, wl["offsets"]) < 1e-12
    assert rel_err(P.cpu().numpy(), ref_P, wl["offsets"]) < 1e-12
