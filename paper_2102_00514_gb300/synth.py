"""Seeded synthetic coordinated-turn / bearings-only workloads (Sec. 5).

This module only makes inputs. Both the CUDA path and the CPU oracle consume
what it returns; it contains no linearisation, filtering or smoothing.

Every workload is a dict of numpy arrays in the library's structure-of-arrays
layout (component-major, ``[ncomp][N]`` with ``N = sum_b (T_b + 1)``):

* ``offsets``  int64 ``[B+1]``: trajectory ``b`` owns states ``offsets[b]..offsets[b+1]-1``;
  state ``offsets[b]`` is its x_0 and has no measurement.
* ``y``        float64 ``[2][N]``: bearings (rad); the x_0 slots hold 0.
* ``x_true``   float64 ``[5][N]``: simulated truth ``[px, py, vx, vy, omega]``.
* ``m0``       float64 ``[B][5]``, ``P0`` float64 ``[B][15]`` (packed upper): the prior.
* ``sensors``  float64 ``[B][4]``: ``(s1x, s1y, s2x, s2y)`` per trajectory.
* scalars ``dt, q_c, q_w, q_form, r_std``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libpes_synth.so")
_lib = None

# Model constants of the simulated experiment (coordinated turn, two bearing
# sensors). Q is diag(0, 0, q_c dt, q_c dt, q_w dt) for q_form 0 and the
# continuous white-acceleration discretisation for q_form 1.
DT = 0.01
Q_C = 0.1
Q_W = 0.01
R_STD = 0.05
SENSORS = (-1.5, 0.5, 1.0, 1.0)
M0 = (0.1, 0.2, 1.0, 0.0, 0.0)
P0_DIAG = (1.0, 1.0, 1.0, 1.0, 1.0)
SEED_BASE = 20210201


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(
                f"{_LIB_PATH} is missing: run __graft_entry__.build() (or "
                "paper_2102_00514_gb300.build.build_all()) first")
        lib = ctypes.CDLL(_LIB_PATH)
        d = ctypes.c_double
        p = ctypes.c_void_p
        i64 = ctypes.c_int64
        lib.synth_lengths.argtypes = [ctypes.c_uint64, i64, i64, i64, p]
        lib.synth_sensors.argtypes = [ctypes.c_uint64, i64, p, d, p]
        lib.synth_ct_bearings.argtypes = [ctypes.c_uint64, i64, p, d, d, d, ctypes.c_int, d,
                                          p, p, d, p, ctypes.c_int, p, p]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def pack_sym(M: np.ndarray) -> np.ndarray:
    """Full symmetric ``[..., n, n]`` -> packed upper ``[..., n(n+1)/2]`` (row-major upper)."""
    n = M.shape[-1]
    iu = np.triu_indices(n)
    return M[..., iu[0], iu[1]]


def unpack_sym(p: np.ndarray, n: int) -> np.ndarray:
    """Packed upper ``[..., n(n+1)/2]`` -> full symmetric ``[..., n, n]``."""
    iu = np.triu_indices(n)
    out = np.zeros(p.shape[:-1] + (n, n), dtype=p.dtype)
    out[..., iu[0], iu[1]] = p
    out[..., iu[1], iu[0]] = p
    return out


def offsets_from_lengths(T: np.ndarray) -> np.ndarray:
    T = np.asarray(T, dtype=np.int64)
    off = np.zeros(len(T) + 1, dtype=np.int64)
    off[1:] = np.cumsum(T + 1)
    return off


def ct_bearings(T, seed: int, *, q_form: int = 0, omega0_halfwidth: float = 0.0,
                sensor_jitter: float = 0.0, dt: float = DT, q_c: float = Q_C,
                q_w: float = Q_W, r_std: float = R_STD) -> dict:
    """Simulate ``len(T)`` coordinated-turn trajectories with ``T[b]`` measurements each.

    Truth x_0 ~ N(M0, diag(P0_DIAG)) (its turn rate U(-hw, hw) when
    ``omega0_halfwidth`` > 0); the filter's prior is (M0, diag(P0_DIAG)) for every
    trajectory.
    """
    lib = _load()
    T = np.atleast_1d(np.asarray(T, dtype=np.int64))
    if np.any(T < 1):
        raise ValueError("every trajectory needs at least one measurement")
    B = len(T)
    offsets = offsets_from_lengths(T)
    N = int(offsets[-1])
    base = np.array(SENSORS, dtype=np.float64)
    sensors = np.empty((B, 4), dtype=np.float64)
    lib.synth_sensors(seed, B, _ptr(base), float(sensor_jitter), _ptr(sensors))
    x0m = np.array(M0, dtype=np.float64)
    x0s = np.sqrt(np.array(P0_DIAG, dtype=np.float64))
    x = np.empty((N, 5), dtype=np.float64)
    y = np.empty((N, 2), dtype=np.float64)
    lib.synth_ct_bearings(seed, B, _ptr(offsets), dt, q_c, q_w, int(q_form), r_std,
                          _ptr(x0m), _ptr(x0s), float(omega0_halfwidth),
                          _ptr(sensors), 1, _ptr(x), _ptr(y))
    m0 = np.tile(x0m, (B, 1))
    P0 = np.tile(pack_sym(np.diag(np.array(P0_DIAG, dtype=np.float64))), (B, 1))
    return dict(offsets=offsets, y=np.ascontiguousarray(y.T), x_true=np.ascontiguousarray(x.T),
                m0=m0, P0=P0, sensors=sensors, dt=dt, q_c=q_c, q_w=q_w, q_form=int(q_form),
                r_std=r_std, seed=int(seed))


def lengths_uniform(B: int, lo: int, hi: int, seed: int) -> np.ndarray:
    lib = _load()
    T = np.empty(B, dtype=np.int64)
    lib.synth_lengths(seed, B, lo, hi, _ptr(T))
    return T


def lengths_log_uniform(B: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """B lengths with log T uniform in [log lo, log hi] (rounded; PCG64 stream)."""
    rng = np.random.default_rng(seed)
    return np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), B))).astype(np.int64).clip(lo, hi)


# Named workloads. The seed of configuration i is SEED_BASE + i.
def workload(name: str) -> dict:
    """Named synthetic workloads.

    * ``ieks_T500``       one trajectory, T = 500 (the IEKS FP64 case)
    * ``ipls_T10000``     one trajectory, T = 10,000 (the cubature case)
    * ``sweep_T<n>``      one trajectory, T = n (the length sweep, n = 2^10 .. 2^20)
    * ``batch<B>``        B trajectories, T_b ~ U{100..20000}, truth turn rate
                          U(-1, 1), sensors jittered by U(-0.2, 0.2)
    * ``batch<B>_T<lo>_<hi>`` the same with other length bounds (test sizes)
    * ``train<n>_T<T>``   n trajectories of T measurements (the learned
                          initialiser's training set; the model of ieks_T500)
    * ``heldout<B>_T<lo>_<hi>`` B trajectories with log T uniform in [lo, hi]
                          (its held-out set; default bounds 1,000 .. 100,000)
    """
    if name == "ieks_T500":
        return ct_bearings([500], SEED_BASE + 1)
    if name == "ipls_T10000":
        return ct_bearings([10000], SEED_BASE + 2)
    if name.startswith("sweep_T"):
        return ct_bearings([int(name[len("sweep_T"):])], SEED_BASE + 3)
    if name.startswith("train"):
        n, T = name[len("train"):].split("_T")
        return ct_bearings(np.full(int(n), int(T)), SEED_BASE + 5)
    if name.startswith("heldout"):
        rest = name[len("heldout"):]
        lo, hi = 1000, 100000
        if "_T" in rest:
            rest, bounds = rest.split("_T")
            lo, hi = (int(v) for v in bounds.split("_"))
        B = int(rest)
        return ct_bearings(lengths_log_uniform(B, lo, hi, SEED_BASE + 6), SEED_BASE + 6)
    if name.startswith("batch"):
        rest = name[len("batch"):]
        lo, hi = 100, 20000
        if "_T" in rest:
            rest, bounds = rest.split("_T")
            lo, hi = (int(v) for v in bounds.split("_"))
        B = int(rest)
        T = lengths_uniform(B, lo, hi, SEED_BASE + 4)
        return ct_bearings(T, SEED_BASE + 4, omega0_halfwidth=1.0, sensor_jitter=0.2)
    raise KeyError(name)
