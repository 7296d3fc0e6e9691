"""Shared helpers of the GPU parity tests (test infrastructure).

Relative errors follow the comparison rule used throughout the tests: per
trajectory, ||M_gpu - M_oracle||_F / ||M_oracle||_F over all its states, for
means [5][T+1] and packed covariances [15][T+1]; the worst trajectory counts.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2102_00514_gb300 import pes, synth

# FP64: rounding-order differences only (1e-9 relative).
TOL_FP64 = 1e-9
# FP32 means and covariances after the final iteration (1e-4 relative).
TOL_FP32 = 1e-4


def rel_err(a: np.ndarray, b: np.ndarray, offsets) -> float:
    """Worst per-trajectory relative Frobenius error of a against b ([ncomp][N])."""
    worst = 0.0
    for i in range(len(offsets) - 1):
        sl = slice(int(offsets[i]), int(offsets[i + 1]))
        num = np.linalg.norm(a[:, sl] - b[:, sl])
        den = np.linalg.norm(b[:, sl])
        worst = max(worst, num / den if den > 0 else num)
    return worst


def to_dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda").contiguous()


def workload_to_dev(wl: dict, prec: int, ut=None, lm: float = 0.0):
    """Device copies of a workload; ut = (alpha, beta, kappa) of the unscented
    rule, lm the Levenberg-Marquardt damping."""
    dt = torch.float64 if prec == pes.FP64 else torch.float32
    model = pes.Model.from_workload(wl)
    model.lm_lambda = lm
    if ut is not None:
        model.ut_alpha, model.ut_beta, model.ut_kappa = ut
    return dict(y=to_dev(wl["y"], dt), offsets=to_dev(wl["offsets"], torch.int64), m0=to_dev(wl["m0"], dt),
                P0=to_dev(wl["P0"], dt), model=model)


ORACLE_METHOD = {pes.IEKS: oracle.IEKS, pes.CUBATURE: oracle.CUBATURE, pes.UNSCENTED: oracle.UNSCENTED,
                 pes.GAUSS_HERMITE: oracle.GAUSS_HERMITE}


def oracle_run(wl: dict, method: int, iters: int = 10, tol: float = 0.0, x_init=None, P_init=None, ut=None,
               lm: float = 0.0):
    model = oracle.Model.from_workload(wl)
    if ut is not None:
        model = model.unscented(*ut)
    if lm:
        model = model.damped(lm)
    om = ORACLE_METHOD[method]
    return oracle.iterated_smoother(model, om, wl["offsets"], wl["y"], wl["m0"], wl["P0"], x_init=x_init,
                                    P_init=P_init, iters=iters, tol=tol)


def gpu_run(sm: pes.Smoother, wl: dict, method: int, prec: int, iters: int = 10, tol: float = 0.0,
            allow_not_converged: bool = False, ut=None, lm: float = 0.0):
    d = workload_to_dev(wl, prec, ut, lm)
    x, P, used, st = sm.ieks_run(d["model"], method, prec, d["y"], d["offsets"], d["m0"], d["P0"], iters=iters,
                                 tol=tol, want_iters=True, allow_not_converged=allow_not_converged)
    torch.cuda.synchronize()
    return x.double().cpu().numpy(), P.double().cpu().numpy(), used, st


def prior_only(wl: dict, bs) -> dict:
    """`wl` with trajectories `bs` cut to their prior state: T_b = 0, one state
    and no measurement (the prior element is the whole trajectory)."""
    off = wl["offsets"]
    keep = np.ones(int(off[-1]), dtype=bool)
    T = np.diff(off) - 1
    for b in bs:
        keep[int(off[b]) + 1:int(off[b + 1])] = False
        T[b] = 0
    return dict(wl, offsets=synth.offsets_from_lengths(T), y=np.ascontiguousarray(wl["y"][:, keep]),
                x_true=np.ascontiguousarray(wl["x_true"][:, keep]))


def ragged_with_prior_only() -> dict:
    """Seven trajectories of 0, 1, 2, 37, 0, 513 and 3,000 measurements."""
    wl = synth.ct_bearings([1, 1, 2, 37, 1, 513, 3000], seed=41, sensor_jitter=0.2, omega0_halfwidth=1.0)
    return prior_only(wl, (0, 4))


def random_linear_workload(T_list, seed: int, singular_q: bool = False):
    """Random per-step affine parameters (SoA, packed) plus data, for the scan
    entry points; returns (lin, y, m0, P0, offsets)."""
    rng = np.random.default_rng(seed)
    T_list = list(T_list)
    offsets = synth.offsets_from_lengths(np.array(T_list))
    N = int(offsets[-1])
    B = len(T_list)
    F = np.zeros((N, 5, 5)); c = np.zeros((N, 5)); Q = np.zeros((N, 5, 5))
    H = np.zeros((N, 2, 5)); d = np.zeros((N, 2)); R = np.zeros((N, 2, 2))
    y = np.zeros((N, 2))
    for b in range(B):
        for k in range(int(offsets[b]), int(offsets[b + 1])):
            if k + 1 < offsets[b + 1]:
                F[k] = np.eye(5) + 0.1 * rng.standard_normal((5, 5))
                c[k] = 0.1 * rng.standard_normal(5)
                A = rng.standard_normal((5, 3 if singular_q else 5))
                Q[k] = 0.02 * A @ A.T
            if k > offsets[b]:
                H[k] = rng.standard_normal((2, 5))
                d[k] = rng.standard_normal(2)
                A = rng.standard_normal((2, 2))
                R[k] = 0.1 * (A @ A.T + 0.5 * np.eye(2))
                y[k] = rng.standard_normal(2)
    lin = dict(F=F.reshape(N, 25).T.copy(), c=c.T.copy(), Qp=oracle.sym_packed(Q).T.copy(),
               H=H.reshape(N, 10).T.copy(), d=d.T.copy(), Rp=oracle.sym_packed(R).T.copy())
    m0 = rng.standard_normal((B, 5))
    P0 = np.stack([oracle.sym_packed(np.eye(5) * (0.5 + rng.random())) for _ in range(B)])
    return lin, y.T.copy(), m0, P0, offsets
