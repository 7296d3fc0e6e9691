"""Thin Python binding of the C ABI in ``include/pes.h`` (``libpes.so``).

Argument marshalling only: every step of the smoother runs in the library's
CUDA kernels. PyTorch supplies device memory (tensors) and streams. The
binding fails loudly when the library has not been built or no GPU is present;
there is no CPU fallback.

Layouts follow the C ABI: per-state arrays are ``[ncomp][N]`` (component-major),
symmetric matrices packed upper-triangular (15 / 3 components), ``offsets``
int64 ``[B+1]``, priors ``m0 [B][5]``, ``P0 [B][15]``.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpes.so")

OK, INVALID_ARG, NOT_PD, NONFINITE, NOT_CONVERGED, CUDA, UNSUPPORTED, TIMEOUT = range(8)
STATUS_NAMES = {0: "PES_OK", 1: "PES_ERR_INVALID_ARG", 2: "PES_ERR_NOT_PD", 3: "PES_ERR_NONFINITE",
                4: "PES_ERR_NOT_CONVERGED", 5: "PES_ERR_CUDA", 6: "PES_ERR_UNSUPPORTED", 7: "PES_ERR_TIMEOUT"}
IEKS, CUBATURE, UNSCENTED, GAUSS_HERMITE = 0, 1, 2, 3
FP64, FP32, MIXED, REFINED = 0, 1, 2, 3
MODEL_CT_BEARINGS, MODEL_LINEAR = 0, 1

EXPORTED = ["pes_create", "pes_destroy", "pes_last_error", "pes_sync", "pes_linearize", "pes_filter_scan",
            "pes_smooth_scan", "pes_ieks_run", "pes_ieks_run_host", "pes_launch_shape", "pes_measure_fma_peak",
            "pes_debug_phase_times", "pes_ieks_run_noalloc", "pes_traj_iterations", "pes_ieks_run_lm", "pes_filter_loglik", "pes_ieks_run_sequential", "pes_autotune", "pes_set_launch_shape", "pes_ieks_graph_create", "pes_graph_launch", "pes_graph_destroy",
            "pes_init_create", "pes_init_destroy", "pes_init_last_error", "pes_init_set_params",
            "pes_init_get_params", "pes_init_get_state", "pes_init_set_state", "pes_init_forward",
            "pes_init_loss_grad", "pes_init_train_step"]
INIT_NPARAMS = 86661


class PesError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class _Model(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("q_form", ctypes.c_int32), ("dt", ctypes.c_double),
                ("q_c", ctypes.c_double), ("q_w", ctypes.c_double), ("r_std", ctypes.c_double),
                ("sensors", ctypes.c_void_p), ("sensors_per_traj", ctypes.c_int32),
                ("F", ctypes.c_double * 25), ("c", ctypes.c_double * 5), ("Q", ctypes.c_double * 15),
                ("H", ctypes.c_double * 10), ("d", ctypes.c_double * 2), ("R", ctypes.c_double * 3),
                ("ut_alpha", ctypes.c_double), ("ut_beta", ctypes.c_double), ("ut_kappa", ctypes.c_double),
                ("lm_lambda", ctypes.c_double)]


_lib = None


def load_library():
    """Load ``libpes.so`` (built in-tree by ``build.build_cuda``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: the CUDA library has not been built "
                           "(run __graft_entry__.build()); there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    p = ctypes.c_void_p
    i32, i64, d = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    mp = ctypes.POINTER(_Model)
    lib.pes_create.argtypes = [ctypes.POINTER(p), i64, i32]
    lib.pes_destroy.argtypes = [p]
    lib.pes_last_error.argtypes = [p]
    lib.pes_last_error.restype = ctypes.c_char_p
    lib.pes_sync.argtypes = [p, p]
    lib.pes_linearize.argtypes = [p, mp, i32, i32, p, p, p, p, i32, i64, p, p, p, p, p, p, p, p]
    lib.pes_filter_scan.argtypes = [p, i32, p, p, p, p, p, p, p, p, p, p, i32, i64, p, p, p]
    lib.pes_filter_loglik.argtypes = [p, i32, p, p, p, p, p, p, p, p, p, p, i32, i64, p, p, p, p]
    lib.pes_smooth_scan.argtypes = [p, i32, p, p, p, p, p, p, i32, i64, p, p, p]
    lib.pes_ieks_run.argtypes = [p, mp, i32, i32, p, p, i32, i64, p, p, p, p, i32, d, p, p,
                                 ctypes.POINTER(i32), p]
    lib.pes_ieks_run_host.argtypes = lib.pes_ieks_run.argtypes
    lib.pes_ieks_run_sequential.argtypes = lib.pes_ieks_run.argtypes
    lib.pes_ieks_graph_create.argtypes = [p, mp, i32, i32, p, p, i32, i64, p, p, p, p, i32, p, p, ctypes.POINTER(p)]
    lib.pes_graph_launch.argtypes = [p, p]
    lib.pes_graph_destroy.argtypes = [p]
    lib.pes_set_launch_shape.argtypes = [p, i32, i32, i32, i32]
    lib.pes_autotune.argtypes = [p, mp, i32, i32, p, p, i32, i64, p, p, i32, p, p, ctypes.POINTER(i32),
                                 ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_float), p]
    lib.pes_launch_shape.argtypes = [p, i32, i32, i64, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                     ctypes.POINTER(i32)]
    lib.pes_measure_fma_peak.argtypes = [ctypes.POINTER(d), ctypes.POINTER(d)]
    lib.pes_debug_phase_times.argtypes = [p, ctypes.POINTER(d), ctypes.POINTER(d), i32]
    lib.pes_ieks_run_noalloc.argtypes = [mp, i32, i32, p, p, i32, i64, p, p, p, p, i32, d, p, p,
                                         ctypes.POINTER(i32), p]
    lib.pes_traj_iterations.argtypes = [p, ctypes.POINTER(i32), i32, p]
    lib.pes_ieks_run_lm.argtypes = [p, mp, i32, p, p, i32, i64, p, p, p, i32, d, d, d, p, p, ctypes.POINTER(i32),
                                    p, p, p, p]
    lib.pes_init_create.argtypes = [ctypes.POINTER(p), i64, i32]
    lib.pes_init_destroy.argtypes = [p]
    lib.pes_init_last_error.argtypes = [p]
    lib.pes_init_last_error.restype = ctypes.c_char_p
    lib.pes_init_set_params.argtypes = [p, p, p, p]
    lib.pes_init_get_params.argtypes = [p, p]
    lib.pes_init_get_state.argtypes = [p, p, p, p, p, p, ctypes.POINTER(i64)]
    lib.pes_init_set_state.argtypes = [p, p, p, p, p, p, i64]
    lib.pes_init_forward.argtypes = [p, i32, p, p, i32, i64, p, p]
    lib.pes_init_loss_grad.argtypes = [p, i32, p, p, i32, i64, p, p, ctypes.POINTER(d), p]
    lib.pes_init_train_step.argtypes = [p, i32, p, p, i32, i64, p, ctypes.c_float, ctypes.POINTER(d), p]
    for name in EXPORTED:
        if name not in ("pes_last_error", "pes_init_last_error"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


@dataclass
class Model:
    """Model parameters (``pes_model``). For the coordinated-turn / bearings model
    ``sensors`` is a float64 tensor ``[1 or B][4]`` on the device."""
    kind: int = MODEL_CT_BEARINGS
    q_form: int = 0
    dt: float = 0.01
    q_c: float = 0.1
    q_w: float = 0.01
    r_std: float = 0.05
    sensors: torch.Tensor | None = None
    F: tuple = ()
    c: tuple = ()
    Q: tuple = ()
    H: tuple = ()
    d: tuple = ()
    R: tuple = ()
    ut_alpha: float = 1.0   # the unscented rule (UNSCENTED); these values give the cubature rule
    ut_beta: float = 0.0
    ut_kappa: float = 0.0
    lm_lambda: float = 0.0   # Levenberg-Marquardt damping of the iteration (0: none)

    def as_struct(self) -> _Model:
        s = _Model()
        s.kind, s.q_form = self.kind, self.q_form
        s.ut_alpha, s.ut_beta, s.ut_kappa = self.ut_alpha, self.ut_beta, self.ut_kappa
        s.lm_lambda = self.lm_lambda
        s.dt, s.q_c, s.q_w, s.r_std = self.dt, self.q_c, self.q_w, self.r_std
        if self.sensors is not None:
            if self.sensors.dtype != torch.float64:
                raise TypeError("sensors must be float64")
            s.sensors = self.sensors.data_ptr()
            s.sensors_per_traj = 1 if self.sensors.shape[0] > 1 else 0
        for name, n in (("F", 25), ("c", 5), ("Q", 15), ("H", 10), ("d", 2), ("R", 3)):
            v = getattr(self, name)
            if len(v):
                getattr(s, name)[:] = [float(x) for x in v]
        return s

    @classmethod
    def from_workload(cls, wl: dict, device="cuda"):
        sensors = torch.as_tensor(wl["sensors"], dtype=torch.float64, device=device).contiguous()
        return cls(kind=MODEL_CT_BEARINGS, q_form=int(wl["q_form"]), dt=float(wl["dt"]), q_c=float(wl["q_c"]),
                   q_w=float(wl["q_w"]), r_std=float(wl["r_std"]), sensors=sensors)

    @classmethod
    def linear(cls, F, c, Q_packed, H, d, R_packed):
        flat = lambda a: tuple(float(x) for x in torch.as_tensor(a, dtype=torch.float64).reshape(-1).tolist())
        return cls(kind=MODEL_LINEAR, F=flat(F), c=flat(c), Q=flat(Q_packed), H=flat(H), d=flat(d),
                   R=flat(R_packed))


def _dtype(prec: int):
    return torch.float64 if prec == FP64 else torch.float32


def _ptr(t, dtype=None, device=True):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch.Tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected dtype {dtype}, got {t.dtype}")
    if device and not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not device and t.is_cuda:
        raise TypeError("expected a host tensor")
    if not t.is_contiguous():
        raise TypeError("expected a contiguous tensor")
    return t.data_ptr()


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def measure_fma_peak():
    """Measured FP32 and FP64 CUDA-core FMA throughput of the current device, GFLOP/s."""
    lib = load_library()
    f32, f64 = ctypes.c_double(), ctypes.c_double()
    st = lib.pes_measure_fma_peak(ctypes.byref(f32), ctypes.byref(f64))
    if st != OK:
        raise PesError(st, "pes_measure_fma_peak failed")
    return f32.value, f64.value


class Smoother:
    """A ``pes_handle`` on the current CUDA device."""

    def __init__(self, max_states: int, max_batch: int = 1):
        if not torch.cuda.is_available():
            raise RuntimeError("the smoother needs a CUDA GPU; there is no CPU fallback")
        self.lib = load_library()
        torch.cuda.init()
        h = ctypes.c_void_p()
        st = self.lib.pes_create(ctypes.byref(h), int(max_states), int(max_batch))
        if st != OK:
            raise PesError(st, "pes_create failed")
        self.h = h
        self.max_states = int(max_states)
        self.max_batch = int(max_batch)

    def close(self):
        if getattr(self, "h", None):
            self.lib.pes_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int, allow=()):
        if st != OK and st not in allow:
            raise PesError(st, self.lib.pes_last_error(self.h).decode())
        return st

    def last_error(self) -> str:
        return self.lib.pes_last_error(self.h).decode()

    def sync(self, stream=None):
        return self._check(self.lib.pes_sync(self.h, _stream(stream)))

    PHASES = ["fold", "filter up-sweep", "filter barrier", "filter top level", "filter down-sweep", "filter re-run",
              "between passes", "smoother up-sweep", "smoother barrier", "smoother top level", "smoother down-sweep",
              "RTS re-run", "end barrier"]

    def phase_times(self):
        """Per-phase (mean, max) ns of the first iteration of the last launch
        (needs PES_PHASE_TIMES=1 in the environment before the handle is made)."""
        n = len(self.PHASES)
        mean, mx = (ctypes.c_double * n)(), (ctypes.c_double * n)()
        self._check(self.lib.pes_debug_phase_times(self.h, mean, mx, n))
        return {name: (mean[i], mx[i]) for i, name in enumerate(self.PHASES)}

    def traj_iterations(self, B: int, stream=None):
        """Per-trajectory iterations to tolerance of the last tolerance-mode run (0: not reached)."""
        import numpy as np
        out = np.zeros(B, dtype=np.int32)
        self._check(self.lib.pes_traj_iterations(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(B),
                                                 _stream(stream)))
        return out

    def set_launch_shape(self, method: int, prec: int, threads: int, min_steps: int):
        """Keep this launch shape for (method, precision) (pes_set_launch_shape)."""
        self._check(self.lib.pes_set_launch_shape(self.h, method, prec, int(threads), int(min_steps)))

    def autotune(self, model: Model, method: int, prec: int, y, offsets, m0, P0, iters: int = 2, stream=None,
                 cache: str | None = None):
        """Time the candidate launch shapes on this workload and keep the fastest
        for (method, precision); returns (threads, min_steps, ms_per_run). With
        `cache` (a JSON file), a choice recorded there for this GPU, method,
        precision and size class (tune_cache_key) is applied without timing,
        and a new one is recorded."""
        dt = _dtype(prec)
        N = y.shape[1]
        B = offsets.shape[0] - 1
        key = None
        if cache is not None:
            key = tune_cache_key(torch.cuda.get_device_name(y.device), method, prec, N, B)
            hit = read_tune_cache(cache).get(key)
            if hit is not None:
                self.set_launch_shape(method, prec, hit["threads"], hit["min_steps"])
                return hit["threads"], hit["min_steps"], hit["ms_per_run"]
        xs = torch.empty((5, N), dtype=dt, device=y.device)
        Ps = torch.empty((15, N), dtype=dt, device=y.device)
        nt, ms_, t = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
        st = self.lib.pes_autotune(self.h, ctypes.byref(model.as_struct()), method, prec, _ptr(y, dt),
                                   _ptr(offsets, torch.int64), B, N, _ptr(m0, dt), _ptr(P0, dt), int(iters),
                                   _ptr(xs), _ptr(Ps), ctypes.byref(nt), ctypes.byref(ms_), ctypes.byref(t),
                                   _stream(stream))
        self._check(st)
        if key is not None:
            update_tune_cache(cache, key, {"threads": nt.value, "min_steps": ms_.value, "ms_per_run": t.value})
        return nt.value, ms_.value, t.value

    def graph(self, model: Model, method: int, prec: int, y, offsets, m0, P0, x_init=None, P_init=None,
              iters: int = 10, x_out=None, P_out=None):
        """Capture one ieks_run of these arguments into a CUDA graph (see Graph)."""
        dt = _dtype(prec)
        N = y.shape[1]
        B = offsets.shape[0] - 1
        if x_out is None:
            x_out = torch.empty((5, N), dtype=dt, device=y.device)
        if P_out is None:
            P_out = torch.empty((15, N), dtype=dt, device=y.device)
        g = ctypes.c_void_p()
        ms = model.as_struct()
        self._check(self.lib.pes_ieks_graph_create(self.h, ctypes.byref(ms), method, prec, _ptr(y, dt),
                                                   _ptr(offsets, torch.int64), B, N, _ptr(m0, dt), _ptr(P0, dt),
                                                   _ptr(x_init, dt), _ptr(P_init, dt), int(iters), _ptr(x_out, dt),
                                                   _ptr(P_out, dt), ctypes.byref(g)))
        return Graph(self, g, (model, y, offsets, m0, P0, x_init, P_init), x_out, P_out)

    def launch_shape(self, method: int, prec: int, N: int):
        nb, nt, L = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        self._check(self.lib.pes_launch_shape(self.h, method, prec, int(N), ctypes.byref(nb), ctypes.byref(nt),
                                              ctypes.byref(L)))
        return nb.value, nt.value, L.value

    def linearize(self, model: Model, method: int, prec: int, x_nom, P_nom, y, offsets, stream=None):
        dt = _dtype(prec)
        N = x_nom.shape[1]
        B = offsets.shape[0] - 1
        dev = x_nom.device
        out = {name: torch.empty((n, N), dtype=dt, device=dev) for name, n in
               (("F", 25), ("c", 5), ("Qp", 15), ("H", 10), ("d", 2), ("Rp", 3), ("y_used", 2))}
        ms = model.as_struct()
        st = self.lib.pes_linearize(self.h, ctypes.byref(ms), method, prec, _ptr(x_nom, dt), _ptr(P_nom, dt),
                                    _ptr(y, dt), _ptr(offsets, torch.int64), B, N,
                                    *[_ptr(out[k]) for k in ("F", "c", "Qp", "H", "d", "Rp", "y_used")],
                                    _stream(stream))
        self._check(st)
        return out

    def filter_scan(self, prec: int, lin: dict, y, m0, P0, offsets, stream=None):
        dt = _dtype(prec)
        N = y.shape[1]
        B = offsets.shape[0] - 1
        xf = torch.empty((5, N), dtype=dt, device=y.device)
        Pf = torch.empty((15, N), dtype=dt, device=y.device)
        st = self.lib.pes_filter_scan(self.h, prec, *[_ptr(lin[k], dt) for k in ("F", "c", "Qp", "H", "d", "Rp")],
                                      _ptr(y, dt), _ptr(m0, dt), _ptr(P0, dt), _ptr(offsets, torch.int64), B, N,
                                      _ptr(xf), _ptr(Pf), _stream(stream))
        self._check(st)
        return xf, Pf

    def filter_loglik(self, prec: int, lin: dict, y, m0, P0, offsets, stream=None):
        """Filtered moments and per-trajectory log-likelihoods (float64 [B], device)."""
        dt = _dtype(prec)
        N = y.shape[1]
        B = offsets.shape[0] - 1
        xf = torch.empty((5, N), dtype=dt, device=y.device)
        Pf = torch.empty((15, N), dtype=dt, device=y.device)
        ll = torch.empty(B, dtype=torch.float64, device=y.device)
        st = self.lib.pes_filter_loglik(self.h, prec, *[_ptr(lin[k], dt) for k in ("F", "c", "Qp", "H", "d", "Rp")],
                                        _ptr(y, dt), _ptr(m0, dt), _ptr(P0, dt), _ptr(offsets, torch.int64), B, N,
                                        _ptr(xf), _ptr(Pf), _ptr(ll), _stream(stream))
        self._check(st)
        return xf, Pf, ll

    def smooth_scan(self, prec: int, lin: dict, xf, Pf, offsets, stream=None):
        dt = _dtype(prec)
        N = xf.shape[1]
        B = offsets.shape[0] - 1
        xs = torch.empty((5, N), dtype=dt, device=xf.device)
        Ps = torch.empty((15, N), dtype=dt, device=xf.device)
        st = self.lib.pes_smooth_scan(self.h, prec, *[_ptr(lin[k], dt) for k in ("F", "c", "Qp")], _ptr(xf, dt),
                                      _ptr(Pf, dt), _ptr(offsets, torch.int64), B, N, _ptr(xs), _ptr(Ps),
                                      _stream(stream))
        self._check(st)
        return xs, Ps

    def ieks_run(self, model: Model, method: int, prec: int, y, offsets, m0, P0, x_init=None, P_init=None,
                 iters: int = 10, tol: float = 0.0, x_out=None, P_out=None, want_iters: bool = False,
                 stream=None, allow_not_converged: bool = False):
        dt = _dtype(prec)
        N = y.shape[1]
        B = offsets.shape[0] - 1
        if x_out is None:
            x_out = torch.empty((5, N), dtype=dt, device=y.device)
        if P_out is None:
            P_out = torch.empty((15, N), dtype=dt, device=y.device)
        used = ctypes.c_int32(0)
        ms = model.as_struct()
        st = self.lib.pes_ieks_run(self.h, ctypes.byref(ms), method, prec, _ptr(y, dt), _ptr(offsets, torch.int64),
                                   B, N, _ptr(m0, dt), _ptr(P0, dt), _ptr(x_init, dt), _ptr(P_init, dt), int(iters),
                                   float(tol), _ptr(x_out, dt), _ptr(P_out, dt),
                                   ctypes.byref(used) if (want_iters or tol > 0) else None, _stream(stream))
        self._check(st, allow=(NOT_CONVERGED,) if allow_not_converged else ())
        return x_out, P_out, used.value, st

    def ieks_run_lm(self, model: Model, prec: int, y, offsets, m0, P0, x_init=None, iters: int = 20,
                    tol: float = 0.0, lambda0: float = 1.0, nu: float = 10.0, stream=None,
                    allow_not_converged: bool = False):
        """The IEKS with Levenberg-Marquardt steps and per-trajectory adaptive
        damping (pes_ieks_run_lm). Returns x [5][N], P [15][N], iterations,
        and per trajectory the final damping, the steps kept and the converged
        iteration (0: none)."""
        import numpy as np
        dt = _dtype(prec)
        N = y.shape[1]
        B = offsets.shape[0] - 1
        x_out = torch.empty((5, N), dtype=dt, device=y.device)
        P_out = torch.empty((15, N), dtype=dt, device=y.device)
        used = ctypes.c_int32(0)
        lam = np.zeros(B, dtype=np.float64)
        acc = np.zeros(B, dtype=np.int32)
        conv = np.zeros(B, dtype=np.int32)
        ms = model.as_struct()
        st = self.lib.pes_ieks_run_lm(self.h, ctypes.byref(ms), prec, _ptr(y, dt), _ptr(offsets, torch.int64), B, N,
                                      _ptr(m0, dt), _ptr(P0, dt), _ptr(x_init, dt), int(iters), float(tol),
                                      float(lambda0), float(nu), _ptr(x_out, dt), _ptr(P_out, dt),
                                      ctypes.byref(used), lam.ctypes.data, acc.ctypes.data, conv.ctypes.data,
                                      _stream(stream))
        self._check(st, allow=(NOT_CONVERGED,) if allow_not_converged else ())
        return x_out, P_out, used.value, dict(lam=lam, accepted=acc, conv_iter=conv, status=st)

    def ieks_run_sequential(self, model: Model, method: int, prec: int, y, offsets, m0, P0, x_init=None,
                            P_init=None, iters: int = 10, tol: float = 0.0, x_out=None, P_out=None, stream=None,
                            allow_not_converged: bool = False):
        """One thread per trajectory (the sequential method on the GPU); same results as ieks_run."""
        dt = _dtype(prec)
        N = y.shape[1]
        B = offsets.shape[0] - 1
        if x_out is None:
            x_out = torch.empty((5, N), dtype=dt, device=y.device)
        if P_out is None:
            P_out = torch.empty((15, N), dtype=dt, device=y.device)
        used = ctypes.c_int32(0)
        ms = model.as_struct()
        st = self.lib.pes_ieks_run_sequential(self.h, ctypes.byref(ms), method, prec, _ptr(y, dt),
                                              _ptr(offsets, torch.int64), B, N, _ptr(m0, dt), _ptr(P0, dt),
                                              _ptr(x_init, dt), _ptr(P_init, dt), int(iters), float(tol),
                                              _ptr(x_out, dt), _ptr(P_out, dt), ctypes.byref(used), _stream(stream))
        self._check(st, allow=(NOT_CONVERGED,) if allow_not_converged else ())
        return x_out, P_out, used.value, st

    def ieks_run_host(self, model: Model, method: int, prec: int, y, offsets, m0, P0, x_init=None, P_init=None,
                      iters: int = 10, tol: float = 0.0, x_out=None, P_out=None, sensors_host=None, stream=None,
                      allow_not_converged: bool = False):
        """Host tensors in and out (pinned memory recommended); ``sensors_host``
        is a host float64 tensor for the coordinated-turn model."""
        dt = _dtype(prec)
        N = y.shape[1]
        B = offsets.shape[0] - 1
        if x_out is None:
            x_out = torch.empty((5, N), dtype=dt, pin_memory=True)
        if P_out is None:
            P_out = torch.empty((15, N), dtype=dt, pin_memory=True)
        ms = model.as_struct()
        if sensors_host is not None:
            ms.sensors = _ptr(sensors_host, torch.float64, device=False)
            ms.sensors_per_traj = 1 if sensors_host.shape[0] > 1 else 0
        used = ctypes.c_int32(0)
        h = lambda t, d=dt: _ptr(t, d, device=False)
        st = self.lib.pes_ieks_run_host(self.h, ctypes.byref(ms), method, prec, h(y), h(offsets, torch.int64), B, N,
                                        h(m0), h(P0), h(x_init), h(P_init), int(iters), float(tol), h(x_out),
                                        h(P_out), ctypes.byref(used), _stream(stream))
        self._check(st, allow=(NOT_CONVERGED,) if allow_not_converged else ())
        return x_out, P_out, used.value, st


_METHOD_NAMES = {IEKS: "ieks", CUBATURE: "cubature", UNSCENTED: "unscented", GAUSS_HERMITE: "gauss_hermite"}


def tune_cache_key(device_name: str, method: int, prec: int, N: int, B: int) -> str:
    """Key of a launch-shape choice: the GPU's name, the method, the
    precision (FP32 or FP64), and the size class: N and B each rounded up to a
    power of two (the shape a tuning finds depends on the lanes per state,
    which those fix to a factor of two)."""
    up = lambda n: 1 << max(0, int(n - 1).bit_length())
    return f"{device_name}|{_METHOD_NAMES[method]}|{'fp64' if prec == FP64 else 'fp32'}|N<={up(N)}|B<={up(B)}"


def read_tune_cache(path: str) -> dict:
    """The cache's entries; an absent file is an empty cache."""
    import json
    try:
        with open(path) as f:
            return json.load(f)
    except FileNotFoundError:
        return {}


def update_tune_cache(path: str, key: str, entry: dict) -> None:
    """Add or replace one entry: the file is rewritten whole through a
    temporary file and a rename, so a reader never sees half of it."""
    import json
    import os
    data = read_tune_cache(path)
    data[key] = entry
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


class Graph:
    """A captured smoother run (pes_graph); ``launch()`` replays it and the
    results land in ``x`` and ``P``. Keeps the captured tensors alive."""

    def __init__(self, sm: "Smoother", g, keep, x, P):
        self.sm, self.g, self._keep, self.x, self.P = sm, g, keep, x, P

    def launch(self, stream=None):
        st = self.sm.lib.pes_graph_launch(self.g, _stream(stream))
        if st != OK:
            raise PesError(st, "pes_graph_launch failed")

    def close(self):
        if getattr(self, "g", None):
            self.sm.lib.pes_graph_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class InitNet:
    """A ``pes_init_net``: the learned initialiser (include/pes_init.h) on the
    current CUDA device. Parameters are a float32 vector of INIT_NPARAMS."""

    def __init__(self, max_states: int, max_batch: int = 1):
        if not torch.cuda.is_available():
            raise RuntimeError("the learned initialiser needs a CUDA GPU; there is no CPU fallback")
        self.lib = load_library()
        torch.cuda.init()
        h = ctypes.c_void_p()
        st = self.lib.pes_init_create(ctypes.byref(h), int(max_states), int(max_batch))
        if st != OK:
            raise PesError(st, "pes_init_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.pes_init_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int):
        if st != OK:
            raise PesError(st, self.lib.pes_init_last_error(self.h).decode())
        return st

    def set_params(self, params, mu, sigma):
        import numpy as np
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.shape != (INIT_NPARAMS,):
            raise ValueError(f"expected {INIT_NPARAMS} parameters")
        m = np.ascontiguousarray(mu, dtype=np.float64)
        sg = np.ascontiguousarray(sigma, dtype=np.float64)
        self._check(self.lib.pes_init_set_params(self.h, p.ctypes.data, m.ctypes.data, sg.ctypes.data))

    def get_params(self):
        import numpy as np
        p = np.empty(INIT_NPARAMS, dtype=np.float32)
        self._check(self.lib.pes_init_get_params(self.h, p.ctypes.data))
        return p

    def get_state(self) -> dict:
        """The training state (pes_init_get_state): params, mu, sigma, Adam's
        moments m and v, and its step count t."""
        import numpy as np
        st = dict(params=np.empty(INIT_NPARAMS, dtype=np.float32), mu=np.empty(5), sigma=np.empty(5),
                  m=np.empty(INIT_NPARAMS, dtype=np.float32), v=np.empty(INIT_NPARAMS, dtype=np.float32))
        t = ctypes.c_int64()
        self._check(self.lib.pes_init_get_state(self.h, st["params"].ctypes.data, st["mu"].ctypes.data,
                                                st["sigma"].ctypes.data, st["m"].ctypes.data, st["v"].ctypes.data,
                                                ctypes.byref(t)))
        st["t"] = int(t.value)
        return st

    def set_state(self, state: dict):
        """Restore a state from get_state (pes_init_set_state)."""
        import numpy as np
        f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
        f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        p, m, v = f32(state["params"]), f32(state["m"]), f32(state["v"])
        mu, sg = f64(state["mu"]), f64(state["sigma"])
        if p.shape != (INIT_NPARAMS,) or m.shape != p.shape or v.shape != p.shape or mu.shape != (5,) or sg.shape != (5,):
            raise ValueError("malformed training state")
        self._check(self.lib.pes_init_set_state(self.h, p.ctypes.data, mu.ctypes.data, sg.ctypes.data, m.ctypes.data,
                                                v.ctypes.data, int(state["t"])))

    def forward(self, prec: int, y, offsets, x_out=None, stream=None):
        dt = _dtype(prec)
        N = y.shape[1]
        B = offsets.shape[0] - 1
        if x_out is None:
            x_out = torch.empty((5, N), dtype=dt, device=y.device)
        self._check(self.lib.pes_init_forward(self.h, prec, _ptr(y, dt), _ptr(offsets, torch.int64), B, N,
                                              _ptr(x_out, dt), _stream(stream)))
        return x_out

    def loss_grad(self, prec: int, y, offsets, x_target, grad=None, stream=None):
        dt = _dtype(prec)
        N = y.shape[1]
        B = offsets.shape[0] - 1
        if grad is None:
            grad = torch.empty(INIT_NPARAMS, dtype=torch.float32, device=y.device)
        loss = ctypes.c_double()
        self._check(self.lib.pes_init_loss_grad(self.h, prec, _ptr(y, dt), _ptr(offsets, torch.int64), B, N,
                                                _ptr(x_target, dt), _ptr(grad, torch.float32), ctypes.byref(loss),
                                                _stream(stream)))
        return loss.value, grad

    def train_step(self, prec: int, y, offsets, x_target, lr: float, want_loss: bool = True, stream=None):
        dt = _dtype(prec)
        N = y.shape[1]
        B = offsets.shape[0] - 1
        loss = ctypes.c_double()
        self._check(self.lib.pes_init_train_step(self.h, prec, _ptr(y, dt), _ptr(offsets, torch.int64), B, N,
                                                 _ptr(x_target, dt), float(lr),
                                                 ctypes.byref(loss) if want_loss else None, _stream(stream)))
        return loss.value if want_loss else None
