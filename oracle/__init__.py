"""Python access to the CPU FP64 oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY. The tests, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` are its only users; the product library never imports
it. It shares no code with the product: its own model, linear algebra,
layout conversions and loader.

Array conventions at this interface match the library's structure-of-arrays
layout so results can be compared element by element: per-state arrays are
``[ncomp][N]``, symmetric matrices packed upper-triangular row-major
(15 entries for 5x5, 3 for 2x2), ``H`` row-major 2x5 (10 components), ``F``
row-major 5x5 (25 components). ``m0`` is ``[B][5]``, ``P0`` ``[B][15]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
# A replacement build of oracle.c to load instead: the mutation test points it
# at copies with one planted mistake each, to check that the pins reject them.
# Unset in every other use.
_LIB_OVERRIDE = os.environ.get("PES_ORACLE_LIBRARY")
_lib = None

IEKS = 0
CUBATURE = 1
UNSCENTED = 2
GAUSS_HERMITE = 3
MODEL_CT_BEARINGS = 0
MODEL_LINEAR = 1
OK, NOT_PD, NOT_CONVERGED = 0, 2, 4
NX, NY = 5, 2


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` beside its source with gcc (plain C, -O2)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Model(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("q_form", ctypes.c_int),
                ("dt", ctypes.c_double), ("q_c", ctypes.c_double), ("q_w", ctypes.c_double),
                ("r_std", ctypes.c_double),
                ("sensors", ctypes.c_void_p), ("sensors_per_traj", ctypes.c_int),
                ("F", ctypes.c_double * 25), ("c", ctypes.c_double * 5), ("Q", ctypes.c_double * 25),
                ("H", ctypes.c_double * 10), ("d", ctypes.c_double * 2), ("R", ctypes.c_double * 4),
                ("ut_alpha", ctypes.c_double), ("ut_beta", ctypes.c_double), ("ut_kappa", ctypes.c_double),
                ("lm_lambda", ctypes.c_double)]


class FElem(ctypes.Structure):
    _fields_ = [("A", ctypes.c_double * 25), ("b", ctypes.c_double * 5), ("C", ctypes.c_double * 25),
                ("eta", ctypes.c_double * 5), ("J", ctypes.c_double * 25)]

    def as_dict(self):
        return dict(A=np.array(self.A).reshape(5, 5), b=np.array(self.b), C=np.array(self.C).reshape(5, 5),
                    eta=np.array(self.eta), J=np.array(self.J).reshape(5, 5))

    @classmethod
    def from_arrays(cls, A, b, C, eta, J):
        e = cls()
        e.A[:] = np.ravel(A).tolist()
        e.b[:] = np.ravel(b).tolist()
        e.C[:] = np.ravel(C).tolist()
        e.eta[:] = np.ravel(eta).tolist()
        e.J[:] = np.ravel(J).tolist()
        return e


class SElem(ctypes.Structure):
    _fields_ = [("E", ctypes.c_double * 25), ("g", ctypes.c_double * 5), ("L", ctypes.c_double * 25)]

    def as_dict(self):
        return dict(E=np.array(self.E).reshape(5, 5), g=np.array(self.g), L=np.array(self.L).reshape(5, 5))

    @classmethod
    def from_arrays(cls, E, g, L):
        e = cls()
        e.E[:] = np.ravel(E).tolist()
        e.g[:] = np.ravel(g).tolist()
        e.L[:] = np.ravel(L).tolist()
        return e


def _load():
    global _lib
    if _lib is None:
        if _LIB_OVERRIDE:
            lib = ctypes.CDLL(_LIB_OVERRIDE)
        else:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
        p = ctypes.c_void_p
        i64 = ctypes.c_int64
        d = ctypes.c_double
        i = ctypes.c_int
        mp = ctypes.POINTER(_Model)
        lib.orc_wrap.restype = d
        lib.orc_wrap.argtypes = [d]
        lib.orc_ct_f.argtypes = [p, d, p]
        lib.orc_ct_jacobian.argtypes = [p, d, p]
        lib.orc_bearings_h.argtypes = [p, p, p]
        lib.orc_bearings_jacobian.argtypes = [p, p, p]
        lib.orc_process_noise.argtypes = [mp, p]
        lib.orc_measurement_noise.argtypes = [mp, p]
        lib.orc_slr.argtypes = [mp, i, i64, p, p, p, p, p]
        lib.orc_slr.restype = i
        lib.orc_slr_unscented.argtypes = [mp, i, i64, p, p, p, p, p]
        lib.orc_slr_unscented.restype = i
        lib.orc_slr_gauss_hermite.argtypes = [mp, i, i64, p, p, p, p, p]
        lib.orc_slr_gauss_hermite.restype = i
        lib.orc_linearize.argtypes = [mp, i, i64, p, i64, p, p, p, p, p, p, p, p, p, p]
        lib.orc_linearize.restype = i
        lib.orc_kf_rts.argtypes = [i64, p, i64] + [p] * 13
        lib.orc_kf_rts.restype = i
        lib.orc_kf_loglik.argtypes = [i64, p, i64] + [p] * 10
        lib.orc_kf_loglik.restype = i
        lib.orc_iterated_smoother.argtypes = [mp, i, i64, p, i64, p, p, p, p, p, i, d, p, p, p, p]
        lib.orc_iterated_smoother.restype = i
        lib.orc_map_cost.argtypes = [mp, i64, p, i64, p, p, p, p, p]
        lib.orc_map_cost.restype = i
        lib.orc_iterated_smoother_lm.argtypes = [mp, i64, p, i64, p, p, p, p, i, d, d, d, p, p, p, p, p, p]
        lib.orc_iterated_smoother_lm.restype = i
        lib.orc_filter_element.argtypes = [p] * 7 + [ctypes.POINTER(FElem)]
        lib.orc_filter_element.restype = i
        lib.orc_filter_prior_element.argtypes = [p, p, ctypes.POINTER(FElem)]
        lib.orc_filter_combine.argtypes = [ctypes.POINTER(FElem)] * 3
        lib.orc_filter_combine.restype = i
        lib.orc_smoother_element.argtypes = [p] * 5 + [ctypes.POINTER(SElem)]
        lib.orc_smoother_element.restype = i
        lib.orc_smoother_last_element.argtypes = [p, p, ctypes.POINTER(SElem)]
        lib.orc_smoother_combine.argtypes = [ctypes.POINTER(SElem)] * 3
        lib.orc_filter_by_elements.argtypes = [i64, p, i64] + [p] * 11
        lib.orc_filter_by_elements.restype = i
        lib.orc_smoother_by_elements.argtypes = [i64, p, i64] + [p] * 7
        lib.orc_smoother_by_elements.restype = i
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# ---- packed <-> full symmetric (the oracle's own conversion) ---------------

def _tri_index(n):
    rows, cols = [], []
    for r in range(n):
        for c in range(r, n):
            rows.append(r)
            cols.append(c)
    return np.array(rows), np.array(cols)


def sym_full(packed: np.ndarray, n: int) -> np.ndarray:
    """``[..., n(n+1)/2]`` packed upper -> ``[..., n, n]``."""
    r, c = _tri_index(n)
    out = np.zeros(packed.shape[:-1] + (n, n))
    out[..., r, c] = packed
    out[..., c, r] = packed
    return out


def sym_packed(full: np.ndarray) -> np.ndarray:
    n = full.shape[-1]
    r, c = _tri_index(n)
    return 0.5 * (full[..., r, c] + full[..., c, r])


# ---- model ------------------------------------------------------------------

class Model:
    """A model for the oracle: the coordinated turn + bearings (Sec. 5) or a
    linear-Gaussian one. Keeps the ctypes struct and the arrays it points to."""

    def __init__(self, s: _Model, keep=()):
        self.s = s
        self._keep = keep
        if s.ut_alpha == 0.0:   # the unscented rule's parameters default to the cubature rule's
            s.ut_alpha, s.ut_beta, s.ut_kappa = 1.0, 0.0, 0.0

    def damped(self, lm_lambda: float) -> "Model":
        """The same model with Levenberg-Marquardt damping lm_lambda of the iteration."""
        s = _Model()
        ctypes.pointer(s)[0] = self.s
        s.lm_lambda = lm_lambda
        return Model(s, self._keep)

    def unscented(self, alpha: float, beta: float, kappa: float) -> "Model":
        """The same model with the unscented rule's parameters set."""
        s = _Model()
        ctypes.pointer(s)[0] = self.s
        s.ut_alpha, s.ut_beta, s.ut_kappa = alpha, beta, kappa
        return Model(s, self._keep)

    @classmethod
    def ct_bearings(cls, dt, q_c, q_w, r_std, sensors, q_form=0):
        sensors = _f64(np.atleast_2d(sensors))
        s = _Model()
        s.kind = MODEL_CT_BEARINGS
        s.q_form = int(q_form)
        s.dt, s.q_c, s.q_w, s.r_std = dt, q_c, q_w, r_std
        s.sensors = sensors.ctypes.data
        s.sensors_per_traj = 1 if sensors.shape[0] > 1 else 0
        return cls(s, (sensors,))

    @classmethod
    def from_workload(cls, wl: dict):
        return cls.ct_bearings(wl["dt"], wl["q_c"], wl["q_w"], wl["r_std"], wl["sensors"], wl["q_form"])

    @classmethod
    def linear(cls, F, c, Q, H, d, R):
        s = _Model()
        s.kind = MODEL_LINEAR
        s.F[:] = _f64(F).ravel().tolist()
        s.c[:] = _f64(c).ravel().tolist()
        s.Q[:] = _f64(Q).ravel().tolist()
        s.H[:] = _f64(H).ravel().tolist()
        s.d[:] = _f64(d).ravel().tolist()
        s.R[:] = _f64(R).ravel().tolist()
        return cls(s)

    def Q(self):
        out = np.zeros(25)
        _load().orc_process_noise(ctypes.byref(self.s), _p(out))
        return out.reshape(5, 5)

    def R(self):
        out = np.zeros(4)
        _load().orc_measurement_noise(ctypes.byref(self.s), _p(out))
        return out.reshape(2, 2)


# ---- model functions ----------------------------------------------------------

def wrap(a: float) -> float:
    return _load().orc_wrap(float(a))


def ct_f(x, dt):
    x = _f64(x)
    out = np.zeros(5)
    _load().orc_ct_f(_p(x), dt, _p(out))
    return out


def ct_jacobian(x, dt):
    x = _f64(x)
    out = np.zeros(25)
    _load().orc_ct_jacobian(_p(x), dt, _p(out))
    return out.reshape(5, 5)


def bearings_h(x, s):
    x, s = _f64(x), _f64(s)
    out = np.zeros(2)
    _load().orc_bearings_h(_p(x), _p(s), _p(out))
    return out


def bearings_jacobian(x, s):
    x, s = _f64(x), _f64(s)
    out = np.zeros(10)
    _load().orc_bearings_jacobian(_p(x), _p(s), _p(out))
    return out.reshape(2, 5)


def slr(model: Model, which: int, b: int, xbar, Pbar, method: int = CUBATURE):
    """Sigma-point SLR (Eqs. 7-9) of f (which=0) or h of trajectory b (which=1),
    with the cubature rule or (method=UNSCENTED) the model's unscented rule."""
    nz = 5 if which == 0 else 2
    xbar, Pbar = _f64(xbar), _f64(Pbar)
    G = np.zeros(nz * 5)
    off = np.zeros(nz)
    Lam = np.zeros(nz * nz)
    fn = {UNSCENTED: _load().orc_slr_unscented, GAUSS_HERMITE: _load().orc_slr_gauss_hermite}.get(method,
                                                                                              _load().orc_slr)
    st = fn(ctypes.byref(model.s), which, b, _p(xbar), _p(Pbar), _p(G), _p(off), _p(Lam))
    if st != OK:
        raise np.linalg.LinAlgError(f"orc_slr status {st}")
    return G.reshape(nz, 5), off, Lam.reshape(nz, nz)


# ---- whole-trajectory functions (SoA in, SoA out) -----------------------------

def _aos(soa: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(soa, dtype=np.float64).T)


def _sym_aos(packed_soa: np.ndarray, n: int) -> np.ndarray:
    return np.ascontiguousarray(sym_full(np.asarray(packed_soa, dtype=np.float64).T, n).reshape(-1, n * n))


def _sym_soa(full_aos: np.ndarray, n: int) -> np.ndarray:
    return np.ascontiguousarray(sym_packed(full_aos.reshape(-1, n, n)).T)


def linearize(model: Model, method: int, offsets, xbar, Pbar, y) -> dict:
    """Eqs. 7-10 at every step. Returns SoA: F[25][N], c[5][N], Qp[15][N],
    H[10][N], d[2][N], Rp[3][N], y_used[2][N]."""
    lib = _load()
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    N = int(offsets[-1])
    B = len(offsets) - 1
    xa = _aos(xbar)
    Pa = _sym_aos(Pbar, 5) if Pbar is not None else np.zeros((N, 25))
    ya = _aos(y)
    F = np.zeros((N, 25)); c = np.zeros((N, 5)); Qp = np.zeros((N, 25))
    H = np.zeros((N, 10)); d = np.zeros((N, 2)); Rp = np.zeros((N, 4)); yu = np.zeros((N, 2))
    st = lib.orc_linearize(ctypes.byref(model.s), method, N, _p(offsets), B, _p(xa), _p(Pa), _p(ya),
                           _p(F), _p(c), _p(Qp), _p(H), _p(d), _p(Rp), _p(yu))
    if st != OK:
        raise np.linalg.LinAlgError(f"orc_linearize status {st}")
    return dict(F=np.ascontiguousarray(F.T), c=np.ascontiguousarray(c.T), Qp=_sym_soa(Qp, 5),
                H=np.ascontiguousarray(H.T), d=np.ascontiguousarray(d.T), Rp=_sym_soa(Rp, 2),
                y_used=np.ascontiguousarray(yu.T))


def _lin_aos(lin: dict):
    return (_aos(lin["F"]), _aos(lin["c"]), _sym_aos(lin["Qp"], 5), _aos(lin["H"]), _aos(lin["d"]),
            _sym_aos(lin["Rp"], 2))


def kf_rts(offsets, lin: dict, y, m0, P0) -> dict:
    """The definition: sequential Kalman filter + RTS smoother of the affine model
    given by ``lin``. Returns SoA xf, Pf (packed), xs, Ps (packed)."""
    lib = _load()
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    N = int(offsets[-1])
    B = len(offsets) - 1
    F, c, Qp, H, d, Rp = _lin_aos(lin)
    ya = _aos(y)
    m0a = _f64(m0).reshape(B, 5)
    P0a = np.ascontiguousarray(sym_full(_f64(P0).reshape(B, 15), 5).reshape(B, 25))
    xf = np.zeros((N, 5)); Pf = np.zeros((N, 25)); xs = np.zeros((N, 5)); Ps = np.zeros((N, 25))
    st = lib.orc_kf_rts(N, _p(offsets), B, _p(F), _p(c), _p(Qp), _p(H), _p(d), _p(Rp), _p(ya),
                        _p(m0a), _p(P0a), _p(xf), _p(Pf), _p(xs), _p(Ps))
    if st != OK:
        raise np.linalg.LinAlgError(f"orc_kf_rts status {st}")
    return dict(xf=np.ascontiguousarray(xf.T), Pf=_sym_soa(Pf, 5),
                xs=np.ascontiguousarray(xs.T), Ps=_sym_soa(Ps, 5))


def kf_loglik(offsets, lin: dict, y, m0, P0) -> np.ndarray:
    """log p(y_{1:T_b}) per trajectory under the affine model given by ``lin``
    (prediction error decomposition of the Kalman filter)."""
    lib = _load()
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    N = int(offsets[-1])
    B = len(offsets) - 1
    F, c, Qp, H, d, Rp = _lin_aos(lin)
    ya = _aos(y)
    m0a = _f64(m0).reshape(B, 5)
    P0a = np.ascontiguousarray(sym_full(_f64(P0).reshape(B, 15), 5).reshape(B, 25))
    out = np.zeros(B)
    st = lib.orc_kf_loglik(N, _p(offsets), B, _p(F), _p(c), _p(Qp), _p(H), _p(d), _p(Rp), _p(ya), _p(m0a), _p(P0a),
                           _p(out))
    if st != OK:
        raise np.linalg.LinAlgError(f"orc_kf_loglik status {st}")
    return out


def by_elements(offsets, lin: dict, y, m0, P0) -> dict:
    """The same smoother through the paper's elements and operators (Eqs. 13-19),
    folded sequentially. Returns SoA xf, Pf, xs, Ps."""
    lib = _load()
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    N = int(offsets[-1])
    B = len(offsets) - 1
    F, c, Qp, H, d, Rp = _lin_aos(lin)
    ya = _aos(y)
    m0a = _f64(m0).reshape(B, 5)
    P0a = np.ascontiguousarray(sym_full(_f64(P0).reshape(B, 15), 5).reshape(B, 25))
    xf = np.zeros((N, 5)); Pf = np.zeros((N, 25)); xs = np.zeros((N, 5)); Ps = np.zeros((N, 25))
    st = lib.orc_filter_by_elements(N, _p(offsets), B, _p(F), _p(c), _p(Qp), _p(H), _p(d), _p(Rp), _p(ya),
                                    _p(m0a), _p(P0a), _p(xf), _p(Pf))
    if st != OK:
        raise np.linalg.LinAlgError(f"orc_filter_by_elements status {st}")
    st = lib.orc_smoother_by_elements(N, _p(offsets), B, _p(F), _p(c), _p(Qp), _p(xf), _p(Pf), _p(xs), _p(Ps))
    if st != OK:
        raise np.linalg.LinAlgError(f"orc_smoother_by_elements status {st}")
    return dict(xf=np.ascontiguousarray(xf.T), Pf=_sym_soa(Pf, 5),
                xs=np.ascontiguousarray(xs.T), Ps=_sym_soa(Ps, 5))


def iterated_smoother(model: Model, method: int, offsets, y, m0, P0, x_init=None, P_init=None,
                      iters: int = 10, tol: float = 0.0) -> dict:
    """Sec. 3 iteration. Returns SoA x [5][N], P [15][N], iters_used, rel_history, status."""
    lib = _load()
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    N = int(offsets[-1])
    B = len(offsets) - 1
    ya = _aos(y)
    m0a = _f64(m0).reshape(B, 5)
    P0a = np.ascontiguousarray(sym_full(_f64(P0).reshape(B, 15), 5).reshape(B, 25))
    xi = _aos(x_init) if x_init is not None else None
    Pi = _sym_aos(P_init, 5) if P_init is not None else None
    x = np.zeros((N, 5)); P = np.zeros((N, 25))
    used = ctypes.c_int(0)
    hist = np.zeros(max(iters, 1))
    st = lib.orc_iterated_smoother(ctypes.byref(model.s), method, N, _p(offsets), B, _p(ya), _p(m0a), _p(P0a),
                                   _p(xi) if xi is not None else None, _p(Pi) if Pi is not None else None,
                                   int(iters), float(tol), _p(x), _p(P), ctypes.byref(used), _p(hist))
    if st not in (OK, NOT_CONVERGED):
        raise np.linalg.LinAlgError(f"orc_iterated_smoother status {st}")
    return dict(x=np.ascontiguousarray(x.T), P=_sym_soa(P, 5), iters_used=used.value,
                rel_history=hist[:used.value].copy(), status=st)


def map_cost(model: Model, offsets, y, m0, P0, x) -> np.ndarray:
    """The MAP objective of Eq. 4 per trajectory (positive definite Q), at the
    trajectory x [5][N]."""
    lib = _load()
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    N = int(offsets[-1])
    B = len(offsets) - 1
    m0a = _f64(m0).reshape(B, 5)
    P0a = np.ascontiguousarray(sym_full(_f64(P0).reshape(B, 15), 5).reshape(B, 25))
    out = np.zeros(B)
    st = lib.orc_map_cost(ctypes.byref(model.s), N, _p(offsets), B, _p(_aos(y)), _p(m0a), _p(P0a), _p(_aos(x)),
                          _p(out))
    if st != OK:
        raise np.linalg.LinAlgError(f"orc_map_cost status {st}")
    return out


def iterated_smoother_lm(model: Model, offsets, y, m0, P0, x_init=None, iters: int = 10, tol: float = 0.0,
                         lambda0: float = 1.0, nu: float = 10.0) -> dict:
    """The IEKS with Levenberg-Marquardt steps and adaptive per-trajectory
    damping (Sec. 3). Returns SoA x [5][N], P [15][N], iters_used, and per
    trajectory the final damping, the first converged iteration and the
    number of accepted steps."""
    lib = _load()
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    N = int(offsets[-1])
    B = len(offsets) - 1
    m0a = _f64(m0).reshape(B, 5)
    P0a = np.ascontiguousarray(sym_full(_f64(P0).reshape(B, 15), 5).reshape(B, 25))
    xi = _aos(x_init) if x_init is not None else None
    x = np.zeros((N, 5)); P = np.zeros((N, 25))
    used = ctypes.c_int(0)
    lam = np.zeros(B); conv = np.zeros(B, dtype=np.int32); acc = np.zeros(B, dtype=np.int32)
    st = lib.orc_iterated_smoother_lm(ctypes.byref(model.s), N, _p(offsets), B, _p(_aos(y)), _p(m0a), _p(P0a),
                                      _p(xi) if xi is not None else None, int(iters), float(tol), float(lambda0),
                                      float(nu), _p(x), _p(P), ctypes.byref(used), _p(lam), _p(conv), _p(acc))
    if st not in (OK, NOT_CONVERGED):
        raise np.linalg.LinAlgError(f"orc_iterated_smoother_lm status {st}")
    return dict(x=np.ascontiguousarray(x.T), P=_sym_soa(P, 5), iters_used=used.value, lam=lam, conv_iter=conv,
                accepted=acc, status=st)


# ---- single elements (Eqs. 13-19) ------------------------------------------------

def filter_element(F, c, Qp, H, d, Rp, y) -> FElem:
    e = FElem()
    args = [_f64(a).ravel() for a in (F, c, Qp, H, d, Rp, y)]
    st = _load().orc_filter_element(*[_p(a) for a in args], ctypes.byref(e))
    if st != OK:
        raise np.linalg.LinAlgError("filter element")
    return e


def filter_prior_element(m0, P0) -> FElem:
    e = FElem()
    m0, P0 = _f64(m0).ravel(), _f64(P0).ravel()
    _load().orc_filter_prior_element(_p(m0), _p(P0), ctypes.byref(e))
    return e


def filter_combine(ei: FElem, ej: FElem) -> FElem:
    out = FElem()
    st = _load().orc_filter_combine(ctypes.byref(ei), ctypes.byref(ej), ctypes.byref(out))
    if st != OK:
        raise np.linalg.LinAlgError("filter combine")
    return out


def smoother_element(xf, Pf, F, c, Qp) -> SElem:
    e = SElem()
    args = [_f64(a).ravel() for a in (xf, Pf, F, c, Qp)]
    st = _load().orc_smoother_element(*[_p(a) for a in args], ctypes.byref(e))
    if st != OK:
        raise np.linalg.LinAlgError("smoother element")
    return e


def smoother_last_element(xf, Pf) -> SElem:
    e = SElem()
    xf, Pf = _f64(xf).ravel(), _f64(Pf).ravel()
    _load().orc_smoother_last_element(_p(xf), _p(Pf), ctypes.byref(e))
    return e


def smoother_combine(ei: SElem, ej: SElem) -> SElem:
    out = SElem()
    _load().orc_smoother_combine(ctypes.byref(ei), ctypes.byref(ej), ctypes.byref(out))
    return out
