"""GPU parity of the building-block scans (pes_filter_scan, pes_smooth_scan)
against the oracle's sequential Kalman filter + RTS smoother, for given
linearisation parameters, element by element."""
import zlib

import numpy as np
import pytest
import torch

import oracle
from paper_2102_00514_gb300 import pes
from tests.gpu_common import TOL_FP32, TOL_FP64, random_linear_workload, rel_err, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sm():
    s = pes.Smoother(1 << 18, 4096)
    yield s
    s.close()


CASES = [
    ("one_state", [0]),
    ("one_step", [1]),
    ("short", [37]),
    ("ragged_batch", [0, 3, 1, 250, 17, 0, 99]),
    ("several_blocks", [20011]),                      # spans several blocks with a ragged tail
    ("many_blocks", [100003]),
    ("batch_multi_block", list(range(1, 600, 7))),
]


def _run(sm, prec, T_list, seed, singular_q=False):
    lin, y, m0, P0, off = random_linear_workload(T_list, seed, singular_q)
    ref = oracle.kf_rts(off, lin, y, m0, P0)
    dt = torch.float64 if prec == pes.FP64 else torch.float32
    dlin = {k: to_dev(v, dt) for k, v in lin.items()}
    doff = to_dev(off, torch.int64)
    xf, Pf = sm.filter_scan(prec, dlin, to_dev(y, dt), to_dev(m0, dt), to_dev(P0, dt), doff)
    xs, Ps = sm.smooth_scan(prec, dlin, xf, Pf, doff)
    sm.sync()
    got = {k: v.double().cpu().numpy() for k, v in (("xf", xf), ("Pf", Pf), ("xs", xs), ("Ps", Ps))}
    return got, ref, off


@pytest.mark.parametrize("name,T_list", CASES)
@pytest.mark.parametrize("singular_q", [False, True])
def test_scans_fp64_match_oracle(sm, name, T_list, singular_q):
    got, ref, off = _run(sm, pes.FP64, T_list, seed=zlib.crc32(name.encode()) % 1000, singular_q=singular_q)
    for k in ("xf", "Pf", "xs", "Ps"):
        assert rel_err(got[k], ref[k], off) < TOL_FP64, k


@pytest.mark.parametrize("name,T_list", CASES)
def test_scans_fp32_match_oracle(sm, name, T_list):
    got, ref, off = _run(sm, pes.FP32, T_list, seed=zlib.crc32(name.encode()) % 1000 + 1)
    for k in ("xf", "Pf", "xs", "Ps"):
        assert rel_err(got[k], ref[k], off) < TOL_FP32, k


def test_smoothed_last_state_equals_filtered(sm):
    got, ref, off = _run(sm, pes.FP64, [5, 40, 1], seed=3)
    last = off[1:] - 1
    np.testing.assert_array_equal(got["xs"][:, last], got["xf"][:, last])
    np.testing.assert_array_equal(got["Ps"][:, last], got["Pf"][:, last])


def test_malformed_offsets_rejected(sm):
    lin, y, m0, P0, off = random_linear_workload([4, 4], 0)
    bad = off.copy()
    bad[1] = bad[2]  # empty trajectory: not allowed
    dlin = {k: to_dev(v) for k, v in lin.items()}
    with pytest.raises(pes.PesError) as ei:
        sm.filter_scan(pes.FP64, dlin, to_dev(y), to_dev(m0), to_dev(P0), to_dev(bad, torch.int64))
        sm.sync()
    assert ei.value.status == pes.INVALID_ARG
    # the handle keeps working afterwards
    xf, Pf = sm.filter_scan(pes.FP64, dlin, to_dev(y), to_dev(m0), to_dev(P0), to_dev(off, torch.int64))
    sm.sync()


@pytest.mark.parametrize("name,T_list", CASES)
@pytest.mark.parametrize("prec,tol", [(pes.FP64, TOL_FP64), (pes.FP32, TOL_FP32)])
def test_filter_loglik_matches_oracle(sm, name, T_list, prec, tol):
    lin, y, m0, P0, off = random_linear_workload(T_list, zlib.crc32(name.encode()) % 1000 + 2)
    ref = oracle.kf_loglik(off, lin, y, m0, P0)
    refx = oracle.kf_rts(off, lin, y, m0, P0)
    dt = torch.float64 if prec == pes.FP64 else torch.float32
    dlin = {k: to_dev(v, dt) for k, v in lin.items()}
    xf, Pf, ll = sm.filter_loglik(prec, dlin, to_dev(y, dt), to_dev(m0, dt), to_dev(P0, dt),
                                  to_dev(off, torch.int64))
    sm.sync()
    ll = ll.cpu().numpy()
    for b in range(len(T_list)):
        assert abs(ll[b] - ref[b]) <= tol * max(1.0, abs(ref[b])), (b, ll[b], ref[b])
        if T_list[b] == 0:
            assert ll[b] == 0.0
    # the filtered moments are those of pes_filter_scan
    assert rel_err(xf.double().cpu().numpy(), refx["xf"], off) < tol
    assert rel_err(Pf.double().cpu().numpy(), refx["Pf"], off) < tol
