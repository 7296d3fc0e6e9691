#!/usr/bin/env python
"""Benchmark of the parallel iterated smoothers on GB300.

Metric: smoothed steps per second per iteration, i.e. (states smoothed) x
(iterations) / time, for the fused IEKS and cubature IPLS runs (pes_ieks_run).

One *step* = one full pass of the hot path over one batch of synthetic input:
an IEKS run and a cubature IPLS run of 10 iterations each (linearise, filter
scan, smoother scan, re-linearise) on a single coordinated-turn / bearings
trajectory of T = 2^20 measurements, inputs resident in HBM.

The metric counts only at oracle tolerance. Both FP32 and PES_REFINED (FP32
iterations, the final one refined by a Newton step with float-float
residuals) are timed; `value` is the rate of the fastest precision whose
final iteration meets 1e-4 against the oracle in this run's parity check
(`config.precision` names it), and the other rates are reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl pes|reference]
Under torchrun (N > 1) every rank smooths its own replica of the workload
(weak scaling; no data-path collective exists in this method).
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import csv
import hashlib
import io
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "smoothed steps/sec per iteration (FP32 vs FP64, same GPU) at oracle tol; iters saved"
UNIT = "smoothed steps/s per iteration"
# Algorithmic work per state and iteration (FLOP), from the per-step operation
# count of the method (linearise + element build + one combine per scan):
# IEKS ~2,710 FMA, cubature IPLS ~4,260 FMA.
ALG_FLOP = {"ieks": 2 * 2710, "cubature": 2 * 4260}
# CUDA-core FP32 peak from unit counts and clock: SMs x 128 FMA lanes x 2 flops x f_SM.
FP32_LANES_PER_SM = 128


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["pes", "reference"], default="pes")
    ap.add_argument("--T", type=int, default=1 << 20)
    ap.add_argument("--iters", type=int, default=10)
    ap.add_argument("--batch", type=int, default=0,
                    help="B > 0: the batched workload of B trajectories, lengths U{100..20000}, instead of one "
                         "trajectory of length T")
    ap.add_argument("--no-parity", action="store_true", help="skip the full-size oracle parity check")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-learned-init", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--sequential", action="store_true",
                    help="also time the sequential counterpart (one GPU thread per trajectory) on the workload")
    ap.add_argument("--cpu-sample", type=int, default=1 << 17, help="states in the oracle's timed sample")
    ap.add_argument("--profile", choices=["ieks", "cubature", "init", "train"], default=None,
                    help="profiling case: only `warmup` + 1 runs of one method, no JSON line")
    ap.add_argument("--prec", choices=["fp32", "fp64", "refined"], default="fp32", help="precision of --profile")
    ap.add_argument("--sweep", action="store_true",
                    help="the length sweep T = 2^10 .. 2^20: one JSON line per length, no benchmark line")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the 4,096-trajectory batched workload's key in the benchmark line")
    ap.add_argument("--no-length-sweep", action="store_true",
                    help="skip the compact length sweep's key in the benchmark line")
    return ap.parse_args()


def run_profile_case(args):
    """A short, single-method case for ncu captures: `warmup` launches, then one.
    --profile init: forward passes of the learned initialiser on 64 held-out
    trajectories (log T uniform in 1,000 .. 100,000), six GEMM launches each.
    --profile train: `warmup` + `iters` training steps of the learned
    initialiser on one minibatch of 128 trajectories of T = 1,000 (the
    training configuration), the true states as targets."""
    import numpy as np
    import torch

    from paper_2102_00514_gb300 import build, pes, synth
    build.build_all()
    if args.profile == "init":
        from paper_2102_00514_gb300 import learned_init as LI
        wl = synth.workload("heldout64_T1000_100000")
        N = wl["y"].shape[1]
        net = pes.InitNet(N, 64)
        net.set_params(LI.initial_params(0), np.zeros(5), np.ones(5))
        y = torch.as_tensor(wl["y"], dtype=torch.float32, device="cuda")
        o = torch.as_tensor(wl["offsets"], dtype=torch.int64, device="cuda")
        for i in range(args.warmup + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            net.forward(pes.FP32, y, o)
            torch.cuda.synchronize()
            print(f"forward {i}: {N} states, {1e3 * (time.perf_counter() - t0):.3f} ms", flush=True)
        net.close()
        return
    if args.profile == "train":
        from paper_2102_00514_gb300 import learned_init as LI
        wl = synth.workload("train128_T1000")
        N = wl["y"].shape[1]
        xt = wl["x_true"]
        net = pes.InitNet(N, 128)
        net.set_params(LI.initial_params(0), xt.mean(axis=1), xt.std(axis=1) + 1e-3)
        y = torch.as_tensor(wl["y"], dtype=torch.float32, device="cuda")
        o = torch.as_tensor(wl["offsets"], dtype=torch.int64, device="cuda")
        x = torch.as_tensor(xt, dtype=torch.float32, device="cuda")
        n = args.warmup + args.iters
        for i in range(n):
            net.train_step(pes.FP32, y, o, x, 1e-3, want_loss=(i == n - 1))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(n):
            net.train_step(pes.FP32, y, o, x, 1e-3, want_loss=False)
        torch.cuda.synchronize()
        dt_s = (time.perf_counter() - t0) / n
        print(f"train step: {N} states, {1e6 * dt_s:.1f} us, {N / dt_s:.3e} states/s", flush=True)
        net.close()
        return
    wl = synth.workload(f"sweep_T{args.T}")
    N = wl["y"].shape[1]
    prec = {"fp32": pes.FP32, "fp64": pes.FP64, "refined": pes.REFINED}[args.prec]
    dt = torch.float64 if prec == pes.FP64 else torch.float32
    dev = lambda a, d=dt: torch.as_tensor(np.ascontiguousarray(a), dtype=d, device="cuda")
    sm = pes.Smoother(N, 1)
    m = pes.IEKS if args.profile == "ieks" else pes.CUBATURE
    y, off, m0, P0 = dev(wl["y"]), dev(wl["offsets"], torch.int64), dev(wl["m0"]), dev(wl["P0"])
    model = pes.Model.from_workload(wl)
    for i in range(args.warmup + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sm.ieks_run(model, m, prec, y, off, m0, P0, iters=args.iters)
        sm.sync()
        print(f"run {i}: {1e3 * (time.perf_counter() - t0):.3f} ms", flush=True)
    sm.close()


def run_sweep(args):
    """--sweep: one trajectory of each length T = 2^10 .. 2^20, both methods,
    `iters` iterations: milliseconds per run in FP32, MIXED and FP64 (CUDA events,
    median of 5 after 2 warm-up runs, autotuned launch shapes, L2 not flushed),
    and the error of the final iteration (FP32 and MIXED) against one oracle
    iteration from the GPU's own FP32 nominal of the first iters - 1 iterations.
    One JSON line per length."""
    import numpy as np
    import torch

    import oracle
    from paper_2102_00514_gb300 import build, pes, synth
    build.build_all()
    iters = args.iters
    r32 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
    methods = (("ieks", pes.IEKS, oracle.IEKS), ("cubature", pes.CUBATURE, oracle.CUBATURE))
    for e in range(10, 21):
        T = 1 << e
        wl = synth.workload(f"sweep_T{T}")
        N = wl["y"].shape[1]
        sm = pes.Smoother(N, 1)
        model = pes.Model.from_workload(wl)
        dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
        ins = {prec: (dev(wl["y"], dt), dev(wl["offsets"], torch.int64), dev(wl["m0"], dt), dev(wl["P0"], dt))
               for prec, dt in ((pes.FP32, torch.float32), (pes.FP64, torch.float64))}
        ins[pes.MIXED] = ins[pes.FP32]
        line = {"T": T, "iterations": iters, "l2": "not flushed (the sweep is a diagnostic, not the benchmark)"}
        for name, m, om in methods:
            rec = {}
            for prec in (pes.FP32, pes.FP64):
                y, off, m0, P0 = ins[prec]
                sm.autotune(model, m, prec, y, off, m0, P0, iters=2)
            for key, prec in (("fp32", pes.FP32), ("mixed", pes.MIXED), ("fp64", pes.FP64)):
                y, off, m0, P0 = ins[prec]
                ms = []
                for rep_ in range(7):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    sm.ieks_run(model, m, prec, y, off, m0, P0, iters=iters)
                    e1.record()
                    torch.cuda.synchronize()
                    if rep_ >= 2:
                        ms.append(e0.elapsed_time(e1))
                ms_run = statistics.median(ms)
                rec[key] = {"ms_per_run": ms_run, "us_per_iteration": 1e3 * ms_run / iters,
                            "value": T * iters / (ms_run * 1e-3)}
            y, off, m0, P0 = ins[pes.FP32]
            x9, P9 = sm.ieks_run(model, m, pes.FP32, y, off, m0, P0, iters=iters - 1)[:2]
            x, P = sm.ieks_run(model, m, pes.FP32, y, off, m0, P0, iters=iters)[:2]
            xm, Pm = sm.ieks_run(model, m, pes.MIXED, y, off, m0, P0, iters=iters)[:2]
            torch.cuda.synchronize()
            last = oracle.iterated_smoother(oracle.Model.from_workload(wl), om, wl["offsets"], r32(wl["y"]),
                                            r32(wl["m0"]), r32(wl["P0"]), x_init=x9.double().cpu().numpy(),
                                            P_init=P9.double().cpu().numpy(), iters=1)
            o = wl["offsets"]
            rec["final_iteration"] = {
                "fp32_means": rel_err(x.double().cpu().numpy(), last["x"], o),
                "fp32_covs": rel_err(P.double().cpu().numpy(), last["P"], o),
                "mixed_means": rel_err(xm.double().cpu().numpy(), last["x"], o),
                "mixed_covs": rel_err(Pm.double().cpu().numpy(), last["P"], o)}
            rec["launch_fp32"] = dict(zip(("blocks", "threads", "steps_per_thread"), sm.launch_shape(m, pes.FP32, N)))
            line[name] = rec
        print(json.dumps(line), flush=True)
        sm.close()


def peaks_file():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


KERNEL_HEADERS = ("pes_async.cuh", "pes_kernel.cuh", "pes_launch_impl.cuh", "pes_math.cuh", "pes_model.cuh",
                  "pes_ops.cuh")


def kernel_source_hash():
    """Hash of the device code of the persistent smoother kernel (its headers)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2102_00514_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name in KERNEL_HEADERS:
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def traffic_for(method: str, T: int, iters: int):
    """DRAM bytes per launch from the committed ncu capture, if it was taken on
    the current kernel sources (scaled by states x iterations)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except OSError:
        return None
    if rec.get("kernel_source_hash") != kernel_source_hash():
        return None
    per = rec.get("bytes_per_state_iteration", {}).get(method)
    return None if per is None else per * T * iters


class ClockSampler:
    """nvidia-smi samples during the timed region (clocks and throttle reasons)."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self, index: int):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=10)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r for r in csv.reader(io.StringIO(out)) if len(r) >= 9]
        rows = [[c.strip() for c in r] for r in rows if r[0].strip() == str(index)] or \
               [[c.strip() for c in r] for r in rows]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


class NvmlPoller:
    """SM clock and clock-event reasons read through NVML every millisecond on a
    host thread (read-only queries), so that a timed region of a few tens of
    milliseconds still holds samples."""
    # clock-event reason bits of nvml.h
    REASONS = {0x8: "hw_slowdown", 0x40: "hw_thermal_slowdown", 0x20: "sw_thermal_slowdown",
               0x4: "sw_power_cap", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, device: int, fallback_index: int):
        import ctypes
        import threading
        self.ctypes, self.threading = ctypes, threading
        self.lib, self.h, self.thread, self.samples = None, None, None, []
        self.stop_flag = False
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return
            h = ctypes.c_void_p()
            found = False
            try:
                import torch
                pr = torch.cuda.get_device_properties(device)
                for fmt in ("%08x:%02x:%02x.0", "%04x:%02x:%02x.0"):
                    bus = (fmt % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)).encode()
                    if lib.nvmlDeviceGetHandleByPciBusId_v2(bus, ctypes.byref(h)) == 0:
                        found = True
                        break
            except Exception:
                found = False
            if not found and lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(fallback_index), ctypes.byref(h)) != 0:
                return
            self.lib, self.h = lib, h
        except OSError:
            self.lib = None

    def _run(self):
        ct = self.ctypes
        clk, mx, rs = ct.c_uint(), ct.c_uint(), ct.c_ulonglong()
        reasons = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None)
        while not self.stop_flag:
            ok = self.lib.nvmlDeviceGetClockInfo(self.h, 1, ct.byref(clk)) == 0   # NVML_CLOCK_SM
            ok = ok and self.lib.nvmlDeviceGetMaxClockInfo(self.h, 1, ct.byref(mx)) == 0
            ok = ok and reasons is not None and reasons(self.h, ct.byref(rs)) == 0
            if ok:
                self.samples.append((clk.value, mx.value, rs.value))
            time.sleep(0.001)

    def start(self):
        if self.lib is None:
            return
        self.thread = self.threading.Thread(target=self._run, daemon=True)
        self.thread.start()

    def stop(self):
        if self.thread is None:
            return None
        self.stop_flag = True
        self.thread.join()
        if not self.samples:
            return None
        sm = [c for c, _, _ in self.samples]
        reasons = sorted({name for _, _, r in self.samples for bit, name in self.REASONS.items() if r & bit})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(m for _, m, _ in self.samples),
                "reasons": reasons, "samples": len(self.samples), "source": "NVML, every 1 ms during the timed region"}


def per_state_errors(a, b):
    """Per-state relative errors ||a_k - b_k||_2 / ||b_k||_2 ([ncomp][N])."""
    import numpy as np
    num = np.linalg.norm(a - b, axis=0)
    den = np.maximum(np.linalg.norm(b, axis=0), 1e-300)
    return num / den


def per_state_max(a, b):
    """Worst per-state relative error ([ncomp][N])."""
    return float(per_state_errors(a, b).max())


def set_headline(result, key, value, ms):
    """Make precision `key` the headline of the benchmark line: its rate is
    `value`, its step time `ms_per_step`, its host-buffer run `e2e`."""
    result["value"] = value
    result["ms_per_step"] = ms
    result["config"]["precision"] = key
    result["dtype"] = "f32" if key != "mixed" else "f32 (final iteration f64)"
    if key in result:
        result["per_method"] = result[key].get("per_method", result["per_method"])
    e2e = result.get("e2e_by_precision", {}).get(key)
    if e2e is not None:
        result["e2e"] = e2e
    launches = {"fp32": 7, "refined": 12, "mixed": 12}
    result["gpu_launches"] = launches.get(key, 7) * 2 * result["steps"]


def choose_headline(result):
    """`value` is the rate of this run's fastest precision whose final
    iteration meets the tolerance (parity.within_tol); with none, the FP32
    rate stays and `at_oracle_tol` is None."""
    wt = result["parity"]["within_tol"]
    cands = []
    for key in ("fp32", "refined", "mixed"):
        if wt.get(key + "_final_iteration") and key in result:
            cands.append((key, result[key]["value"], result[key]["ms_per_step"]))
    if cands:
        key, v, ms = max(cands, key=lambda c: c[1])
        result["at_oracle_tol"] = {"precision": key, "value": v, "unit": UNIT}
        set_headline(result, key, v, ms)
    else:
        result["at_oracle_tol"] = None
        result["config"]["precision"] = "fp32 (no precision met the tolerance in this run)"


def executed_for(method: str):
    """Executed instructions per state and iteration of the FP32 smoother kernel
    from the committed ncu capture (profiles/traffic.json), if it was taken on
    the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except OSError:
        return None
    if rec.get("kernel_source_hash") != kernel_source_hash():
        return None
    return rec.get("executed", {}).get(method)


def rel_err(a, b, offsets):
    import numpy as np
    worst = 0.0
    for i in range(len(offsets) - 1):
        sl = slice(int(offsets[i]), int(offsets[i + 1]))
        den = np.linalg.norm(b[:, sl])
        worst = max(worst, np.linalg.norm(a[:, sl] - b[:, sl]) / (den if den > 0 else 1.0))
    return float(worst)


def oracle_timed(wl_sample, iters):
    """The oracle as it stands on one host core: both methods on the sample."""
    import oracle
    model = oracle.Model.from_workload(wl_sample)
    out = {}
    for name, m in (("ieks", oracle.IEKS), ("cubature", oracle.CUBATURE)):
        t0 = time.perf_counter()
        oracle.iterated_smoother(model, m, wl_sample["offsets"], wl_sample["y"], wl_sample["m0"], wl_sample["P0"],
                                 iters=iters)
        out[name] = time.perf_counter() - t0
    return out


def max_over_ranks(x: float, dist, device) -> float:
    """The largest value of x over all ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, work_per_step: float, steps: int, seconds: float) -> float:
    """Units all ranks processed per second: every rank does the same work
    (replicas, weak scaling) and the slowest rank's time counts."""
    return world * work_per_step * steps / seconds


def one_trajectory(wl, b):
    """Trajectory b of a workload as a workload of its own, and its state slice."""
    import numpy as np
    off = wl["offsets"]
    sl = slice(int(off[b]), int(off[b + 1]))
    return dict(wl, offsets=np.array([0, off[b + 1] - off[b]], dtype=np.int64), y=wl["y"][:, sl],
                x_true=wl["x_true"][:, sl], m0=wl["m0"][b:b + 1], P0=wl["P0"][b:b + 1],
                sensors=wl["sensors"][b:b + 1]), sl


def sample_workload(wl, S):
    """A bounded sample of about S states: the first S states of a single
    trajectory, or the first whole trajectories of a batch up to S states."""
    import numpy as np
    off = wl["offsets"]
    if len(off) == 2:
        return dict(wl, offsets=np.array([0, S], dtype=np.int64), y=np.ascontiguousarray(wl["y"][:, :S]),
                    x_true=np.ascontiguousarray(wl["x_true"][:, :S]))
    nb = max(1, int(np.searchsorted(off, S, side="right")) - 1)
    n = int(off[nb])
    return dict(wl, offsets=np.ascontiguousarray(off[:nb + 1]), y=np.ascontiguousarray(wl["y"][:, :n]),
                x_true=np.ascontiguousarray(wl["x_true"][:, :n]), m0=wl["m0"][:nb], P0=wl["P0"][:nb],
                sensors=wl["sensors"][:nb])


def parity_units(wl):
    """What the oracle checks: the whole workload for one trajectory; for a
    batch, the first, last, shortest and longest trajectories and four seeded
    random ones, each smoothed alone (the trajectories are independent)."""
    import numpy as np
    B = len(wl["offsets"]) - 1
    if B == 1:
        return [(wl, slice(0, int(wl["offsets"][-1])))]
    T = np.diff(wl["offsets"]) - 1
    pick = {0, B - 1, int(np.argmin(T)), int(np.argmax(T))}
    pick |= set(int(b) for b in np.random.default_rng(B).choice(B, min(4, B), replace=False))
    return [one_trajectory(wl, b) for b in sorted(pick)]


def _final_iteration_errors(sm, pes, oracle, wl, m, om, iters, dev_in, units):
    """Errors of the final iteration of FP32 and PES_REFINED runs against one
    oracle iteration from the GPU's FP32 nominal of iters - 1 iterations (float
    inputs widened), on each unit (trajectory slice) of `units`; worst over units."""
    import numpy as np
    r32 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
    y, off, m0, P0, model = dev_in
    # only the units' slices leave the device
    take = lambda t: [t[:, u[1]].double().cpu().numpy() for u in units]
    x9, P9 = (take(t) for t in sm.ieks_run(model, m, pes.FP32, y, off, m0, P0, iters=iters - 1)[:2])
    outs = {key: tuple(take(t) for t in sm.ieks_run(model, m, prec, y, off, m0, P0, iters=iters)[:2])
            for key, prec in (("fp32", pes.FP32), ("refined", pes.REFINED))}
    err = {}

    def last_of(i):
        one = units[i][0]
        return oracle.iterated_smoother(oracle.Model.from_workload(one), om, one["offsets"], r32(one["y"]),
                                        r32(one["m0"]), r32(one["P0"]), x_init=x9[i], P_init=P9[i], iters=1)

    with cf.ThreadPoolExecutor(min(16, os.cpu_count() or 1)) as ex:
        lasts = list(ex.map(last_of, range(len(units))))
    for key, (xs, Ps) in outs.items():
        err[key + "_means"] = max(rel_err(x, l["x"], u[0]["offsets"]) for x, u, l in zip(xs, units, lasts))
        err[key + "_covs"] = max(rel_err(P, l["P"], u[0]["offsets"]) for P, u, l in zip(Ps, units, lasts))
        err[key + "_covs_worst_state"] = max(per_state_max(P, l["P"]) for P, l in zip(Ps, lasts))
    return err


def _time_runs(sm, pes, m, prec, dev_in, iters, reps=3, warm=1, flush=None):
    import torch
    y, off, m0, P0, model = dev_in
    for _ in range(warm):
        sm.ieks_run(model, m, prec, y, off, m0, P0, iters=iters)
    ms = []
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        sm.ieks_run(model, m, prec, y, off, m0, P0, iters=iters)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    return statistics.median(ms)


def batched_cpu_baseline(wl, iters, budget_states=1 << 20, cores=None):
    """The oracle as it stands on the batched workload, one trajectory per
    thread on all host cores (the C oracle releases the interpreter lock): a
    seeded sample of whole trajectories up to about `budget_states` states, both
    methods, `iters` iterations each. Returns the cpu_baseline record (smoothed
    steps/s per iteration, both methods, like the GPU figure)."""
    import numpy as np

    import oracle
    off = wl["offsets"]
    B = len(off) - 1
    order = np.random.default_rng(B).permutation(B)
    lens = np.diff(off)[order]
    n = max(1, int(np.searchsorted(np.cumsum(lens), budget_states, side="right")))
    picked = sorted(int(b) for b in order[:n])
    units = [one_trajectory(wl, b)[0] for b in picked]
    steps = int(sum(int(u["offsets"][-1]) - 1 for u in units))
    cores = cores or os.cpu_count() or 1

    def run(item):
        u, om = item
        oracle.iterated_smoother(oracle.Model.from_workload(u), om, u["offsets"], u["y"], u["m0"], u["P0"],
                                 iters=iters)

    work = [(u, om) for om in (oracle.IEKS, oracle.CUBATURE) for u in units]
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(cores) as ex:
        list(ex.map(run, work))
    t = time.perf_counter() - t0
    return {"value": 2 * steps * iters / t, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} of {B} trajectories ({steps} steps), one trajectory per thread, IEKS + cubature, "
                      f"{iters} iterations, sequential FP64 oracle", "seconds": t}


def batched_key(args, fp32_peak, flush):
    """The batched workload: 4,096 trajectories, T_b uniform in 100..20,000
    (about 41.9 million states), truth turn rate U(-1, 1), sensors jittered by
    U(-0.2, 0.2); FP32 and PES_REFINED runs of `iters` iterations per method
    (one persistent launch per run; CUDA events, median of 3 after a warm-up,
    L2 flushed before each), the FP32 roofline of each method, and the final
    iteration of both precisions against the oracle on 8 sampled trajectories,
    each smoothed alone."""
    import numpy as np
    import torch

    import oracle
    from paper_2102_00514_gb300 import pes, synth
    iters = args.iters
    wl = synth.workload("batch4096")
    N, B = wl["y"].shape[1], len(wl["offsets"]) - 1
    steps = N - B
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    dev_in = (dev(wl["y"], torch.float32), dev(wl["offsets"], torch.int64), dev(wl["m0"], torch.float32),
              dev(wl["P0"], torch.float32), pes.Model.from_workload(wl))
    sm = pes.Smoother(N, B)
    out = {"workload": f"{B} trajectories, T_b uniform in 100..20000 (sum {steps}), turn rate U(-1,1), sensors "
                       "jittered by U(-0.2,0.2), prior initialisation", "N_states": N, "B": B, "iterations": iters}
    methods = (("ieks", pes.IEKS, oracle.IEKS), ("cubature", pes.CUBATURE, oracle.CUBATURE))
    tot = {"fp32": 0.0, "refined": 0.0}
    units = parity_units(wl)
    for name, m, om in methods:
        rec = {}
        for key, prec in (("fp32", pes.FP32), ("refined", pes.REFINED)):
            ms = _time_runs(sm, pes, m, prec, dev_in, iters, flush=flush)
            tot[key] += ms
            rec[key] = {"ms_per_run": ms, "value": steps * iters / (ms * 1e-3)}
        ach = ALG_FLOP[name] * steps * iters / (rec["fp32"]["ms_per_run"] * 1e-3) / 1e12
        rec["fp32"]["roofline"] = {"bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                                   "frac": ach / fp32_peak}
        rec["launch_fp32"] = dict(zip(("blocks", "threads", "steps_per_thread"), sm.launch_shape(m, pes.FP32, N)))
        rec["final_iteration"] = _final_iteration_errors(sm, pes, oracle, wl, m, om, iters, dev_in, units)
        out[name] = rec
    for key in tot:
        out[key] = {"value": 2 * steps * iters / (tot[key] * 1e-3), "ms_per_step": tot[key]}
    out["parity_scope"] = f"{len(units)} sampled trajectories (first, last, shortest, longest, 4 seeded), each alone"
    sm.close()
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = batched_cpu_baseline(wl, iters)
    return out


def length_sweep_key(args, flush):
    """A compact length sweep, one trajectory per length T = 2^10, 2^12, ...,
    2^18 (2^20 is the main workload): FP32 and PES_REFINED milliseconds per
    run of `iters` iterations (CUDA events, median of 3 after a warm-up,
    launch shapes autotuned per length) and the final iteration of both
    against one oracle iteration from the GPU's own FP32 nominal."""
    import numpy as np
    import torch

    import oracle
    from paper_2102_00514_gb300 import pes, synth
    iters = args.iters
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    out = []
    for e in (10, 12, 14, 16, 18):
        T = 1 << e
        wl = synth.workload(f"sweep_T{T}")
        N = wl["y"].shape[1]
        sm = pes.Smoother(N, 1)
        dev_in = (dev(wl["y"], torch.float32), dev(wl["offsets"], torch.int64), dev(wl["m0"], torch.float32),
                  dev(wl["P0"], torch.float32), pes.Model.from_workload(wl))
        row = {"T": T}
        for name, m, om in (("ieks", pes.IEKS, oracle.IEKS), ("cubature", pes.CUBATURE, oracle.CUBATURE)):
            y, off, m0, P0, model = dev_in
            sm.autotune(model, m, pes.FP32, y, off, m0, P0, iters=2)
            rec = {}
            for key, prec in (("fp32", pes.FP32), ("refined", pes.REFINED)):
                ms = _time_runs(sm, pes, m, prec, dev_in, iters, flush=flush)
                rec[key] = {"ms_per_run": ms, "value": T * iters / (ms * 1e-3)}
            rec["final_iteration"] = _final_iteration_errors(sm, pes, oracle, wl, m, om, iters, dev_in,
                                                             [(wl, slice(0, N))])
            row[name] = rec
        out.append(row)
        sm.close()
    return out


def run_reference(args, rank, world):
    """The reference arm: the CPU oracle, as it stands, on the host cores."""
    if rank != 0:
        return
    from paper_2102_00514_gb300 import build, synth
    build.build_synth()
    import oracle
    oracle.build()
    wl = synth.workload(f"sweep_T{args.T}")
    S = min(args.cpu_sample, wl["y"].shape[1])
    sample = sample_workload(wl, S)
    for _ in range(max(0, min(args.warmup, 1))):
        oracle_timed(sample_workload(wl, min(S, 4096)), 1)
    times = []
    for _ in range(args.steps):
        t = oracle_timed(sample, args.iters)
        times.append(t["ieks"] + t["cubature"])
    total = sum(times)
    value = 2 * S * args.iters * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": f"synthetic coordinated-turn / bearings, seed {wl['seed']}",
            "config": {"workload": f"first {S} states of the T={args.T} trajectory, IEKS + cubature IPLS, "
                                   f"{args.iters} iterations each (sequential FP64 oracle)",
                       "T_sample": S, "iterations": args.iters},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"first {S} of {args.T} states, both methods, {args.iters} iterations"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.profile:
        run_profile_case(args)
        return
    if args.sweep:
        run_sweep(args)
        return

    import numpy as np
    import torch

    from paper_2102_00514_gb300 import build, pes, synth
    build.build_all()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist_mod.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist = dist_mod

    def barrier():
        if dist is not None:
            dist.barrier()

    T, iters = args.T, args.iters
    wl = synth.workload(f"batch{args.batch}" if args.batch > 0 else f"sweep_T{T}")
    N = wl["y"].shape[1]
    B = len(wl["offsets"]) - 1
    steps = N - B   # sum of T_b: every trajectory has one more state than measurements
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    sm = pes.Smoother(N, B)
    methods = (("ieks", pes.IEKS), ("cubature", pes.CUBATURE))

    def device_inputs(prec):
        dt = torch.float32 if prec == pes.FP32 else torch.float64
        return dict(y=dev(wl["y"], dt), offsets=dev(wl["offsets"], torch.int64), m0=dev(wl["m0"], dt),
                    P0=dev(wl["P0"], dt), model=pes.Model.from_workload(wl),
                    x=torch.empty((5, N), dtype=dt, device="cuda"), P=torch.empty((15, N), dtype=dt, device="cuda"))

    def run_step(d, prec, ev=None):
        outs = {}
        for i, (name, m) in enumerate(methods):
            if ev is not None:
                ev[i][0].record()
            sm.ieks_run(d["model"], m, prec, d["y"], d["offsets"], d["m0"], d["P0"], iters=iters,
                        x_out=d["x"], P_out=d["P"])
            if ev is not None:
                ev[i][1].record()
        return outs

    # L2 is flushed before every timed step by writing a buffer larger than L2.
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    d32 = device_inputs(pes.FP32)
    # launch shapes chosen by the library's autotuner on this workload
    tuned = {}
    if not args.no_autotune:
        for name, m in methods:
            nt_, steps_, ms_ = sm.autotune(d32["model"], m, pes.FP32, d32["y"], d32["offsets"], d32["m0"], d32["P0"],
                                           iters=2)
            tuned[name] = {"threads": nt_, "min_steps_per_lane": steps_, "ms_per_2_iterations": ms_}
    timed_precs = (("fp32", pes.FP32), ("refined", pes.REFINED))
    for _ in range(args.warmup):
        for _, prec in timed_precs:
            run_step(d32, prec)
    sm.sync()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()

    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    smi_index = int(vis.split(",")[local]) if vis and vis.split(",")[local].isdigit() else local
    clocks = ClockSampler()
    clocks.start()
    poller = NvmlPoller(torch.cuda.current_device(), smi_index)
    poller.start()
    step_ms = {key: [] for key, _ in timed_precs}
    meth_ms = {key: {name: [] for name, _ in methods} for key, _ in timed_precs}
    for key, prec in timed_precs:
        for _ in range(args.steps):
            flush.zero_()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in methods]
            run_step(d32, prec, ev)
            torch.cuda.synchronize()
            per = [ev[i][0].elapsed_time(ev[i][1]) for i in range(len(methods))]
            for (name, _), ms in zip(methods, per):
                meth_ms[key][name].append(ms)
            step_ms[key].append(sum(per))
    sm.sync()
    torch.cuda.synchronize()
    polled = poller.stop()
    barrier()
    torch.cuda.synchronize()
    smi = clocks.stop(smi_index)
    # the NVML poll is the one with samples inside a short timed region;
    # nvidia-smi (200 ms interval) is kept beside it
    clk = polled if polled is not None else smi
    if clk is not None and polled is not None and smi is not None:
        clk = dict(clk, nvidia_smi=smi)

    work_per_step = len(methods) * steps * iters
    rates = {}
    for key, _ in timed_precs:
        total_ms = max_over_ranks(sum(step_ms[key]), dist, "cuda")
        rates[key] = {"value": whole_job_rate(world, work_per_step, args.steps, total_ms * 1e-3),
                      "ms_per_step": total_ms / args.steps}
    # kernels of one run: FP32 = offsets validation, sensor conversion, y to the
    # lane layout, nominal initialisation, persistent smoother, x and P back to
    # the caller layout; PES_REFINED adds the final iteration's own persistent
    # launch and the refinement's four kernels (forward residuals, forward
    # correction scan, RTS residuals, RTS correction scan)
    launches_per_run = {"fp32": 7, "refined": 12}
    value = rates["fp32"]["value"]
    ms_per_step = rates["fp32"]["ms_per_step"]

    nb, nt, L = sm.launch_shape(pes.IEKS, pes.FP32, N)
    nbc, ntc, Lc = sm.launch_shape(pes.CUBATURE, pes.FP32, N)

    result = None
    if rank == 0:
        peaks = peaks_file()
        props = torch.cuda.get_device_properties(local)
        sm_max = float(peaks.get("sm_max_mhz", 2070.0))
        fp32_peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12   # TFLOP/s
        per_prec = {}
        for key, _ in timed_precs:
            pm = {}
            for name, _ in methods:
                ms = statistics.mean(meth_ms[key][name])
                flop = ALG_FLOP[name] * steps * iters
                pm[name] = {"ms_per_run": ms, "value": steps * iters / (ms * 1e-3),
                            "achieved_tflops": flop / (ms * 1e-3) / 1e12}
            per_prec[key] = pm
        # the roofline is the FP32 smoother kernel's: one launch runs all
        # iterations of an FP32 run (the run's time includes its transposes)
        per_method = per_prec["fp32"]
        dom = max(per_method, key=lambda k: per_method[k]["ms_per_run"])
        achieved = per_method[dom]["achieved_tflops"]
        try:
            probe32, probe64 = pes.measure_fma_peak()
        except Exception:
            probe32, probe64 = None, None
        roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                    "frac": achieved / fp32_peak, "traffic": traffic_for(dom, steps, iters),
                    "kernel": f"pes_persistent_kernel<float, {dom}>",
                    "peak_source": f"{props.multi_processor_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x "
                                   f"{sm_max:.0f} MHz (max SM clock)",
                    "fma_probe_tflops": {"fp32": probe32 / 1e3 if probe32 else None,
                                         "fp64": probe64 / 1e3 if probe64 else None},
                    "alg_flop_per_state_iteration": ALG_FLOP[dom],
                    "timing": "CUDA events around each FP32 pes_ieks_run (the persistent launch plus its layout "
                              "transposes) in the timed region",
                    "executed": executed_for(dom)}
        result = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                  "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                  "vs_baseline": None, "dtype": "f32",
                  "data": f"synthetic coordinated-turn / bearings (seeded, seed {wl['seed']}), inputs resident in HBM",
                  "config": {"workload": (f"single trajectory T={T}" if B == 1 else
                                          f"{B} trajectories, T_b uniform in 100..20000 (sum {steps}), turn rate "
                                          "U(-1,1), sensors jittered by U(-0.2,0.2)") +
                                         f", IEKS + cubature IPLS, {iters} iterations each, FP32, prior initialisation",
                             "T": T if B == 1 else None, "B": B, "N_states": N, "iterations": iters, "methods": ["ieks", "cubature"],
                             "precision": "fp32", "l2": "flushed before every step (512 MB write)",
                             "launch": {"ieks": {"blocks": nb, "threads": nt, "steps_per_thread": L},
                                        "cubature": {"blocks": nbc, "threads": ntc, "steps_per_thread": Lc},
                                        "autotuned": tuned or None}},
                  "roofline": roofline, "per_method": per_method,
                  "fp32": dict(rates["fp32"], per_method=per_prec["fp32"]),
                  "refined": dict(rates["refined"], per_method=per_prec["refined"],
                                  schedule=f"{iters - 1} FP32 iterations, then 1 FP32 iteration refined by a Newton "
                                           "step (float-float residuals, FP32 correction scans)"),
                  "gpu_launches": launches_per_run["fp32"] * len(methods) * args.steps, "clocks": clk}

    # FP64 on the same GPU (the metric compares FP32 with FP64)
    if not args.no_fp64:
        d64 = device_inputs(pes.FP64)
        run_step(d64, pes.FP64)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in methods]
        flush.zero_()
        run_step(d64, pes.FP64, ev)
        torch.cuda.synchronize()
        per = [ev[i][0].elapsed_time(ev[i][1]) for i in range(len(methods))]
        if rank == 0:
            result["fp64"] = {"value": work_per_step / (sum(per) * 1e-3), "ms_per_step": sum(per),
                              "per_method_ms": dict(zip([m for m, _ in methods], per))}
            # the FP64 path is bound by the FP64 pipe: its roofline is the
            # measured FP64 FMA rate (pes_measure_fma_peak)
            p64 = roofline.get("fma_probe_tflops", {}).get("fp64")
            if p64:
                r64 = {}
                for (name, _), ms in zip(methods, per):
                    ach = ALG_FLOP[name] * steps * iters / (ms * 1e-3) / 1e12
                    r64[name] = {"achieved_tflops": ach, "frac": ach / p64}
                result["fp64"]["roofline"] = {"bound": "fp64", "peak_tflops": p64,
                                              "peak_source": "measured FP64 FMA probe", "per_method": r64}
        x64 = {}
        for name, m in methods:
            x, P, _, _ = sm.ieks_run(d64["model"], m, pes.FP64, d64["y"], d64["offsets"], d64["m0"], d64["P0"],
                                     iters=iters)
            x64[name] = (x.cpu().numpy(), P.cpu().numpy())
        del d64

    # FP32 results for the parity check, and the FP32 nominal of the first
    # iters-1 iterations, from which the final iteration is checked on its own
    x32, nom32 = {}, {}
    for name, m in methods:
        x, P, _, _ = sm.ieks_run(d32["model"], m, pes.FP32, d32["y"], d32["offsets"], d32["m0"], d32["P0"],
                                 iters=iters)
        x32[name] = (x.double().cpu().numpy(), P.double().cpu().numpy())
        if iters > 1:
            x, P, _, _ = sm.ieks_run(d32["model"], m, pes.FP32, d32["y"], d32["offsets"], d32["m0"], d32["P0"],
                                     iters=iters - 1)
            nom32[name] = (x.double().cpu().numpy(), P.double().cpu().numpy())
    sm.sync()

    xref = {}
    for name, m in methods:
        x, P, _, _ = sm.ieks_run(d32["model"], m, pes.REFINED, d32["y"], d32["offsets"], d32["m0"], d32["P0"],
                                 iters=iters)
        xref[name] = (x.double().cpu().numpy(), P.double().cpu().numpy())
    sm.sync()

    # the same step replayed from CUDA graphs (one captured run per method)
    graphs = [sm.graph(d32["model"], m, pes.FP32, d32["y"], d32["offsets"], d32["m0"], d32["P0"], iters=iters,
                       x_out=d32["x"], P_out=d32["P"]) for _, m in methods]
    for g in graphs:
        g.launch()
    sm.sync()
    gms = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for g in graphs:
            g.launch()
        e1.record()
        torch.cuda.synchronize()
        gms.append(e0.elapsed_time(e1))
    sm.sync()
    for g in graphs:
        g.close()
    if rank == 0:
        gt = max_over_ranks(sum(gms), None, "cuda")
        result["graph"] = {"value": whole_job_rate(world, work_per_step, args.steps, gt * 1e-3),
                           "ms_per_step": gt / args.steps,
                           "note": "each method's pes_ieks_run captured once (pes_ieks_graph_create), replayed"}

    # the sequential counterpart on the same GPU: one thread per trajectory
    if args.sequential:
        seq = {}
        for name, m in methods:
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            status = "ok"
            try:
                sm.ieks_run_sequential(d32["model"], m, pes.FP32, d32["y"], d32["offsets"], d32["m0"], d32["P0"],
                                       iters=iters, x_out=d32["x"], P_out=d32["P"])
            except pes.PesError as err:   # the run completed; a trajectory's result is flagged
                status = str(err)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            seq[name] = {"ms_per_run": ms, "value": steps * iters / (ms * 1e-3), "status": status}
        if rank == 0:
            result["sequential"] = {"impl": "one GPU thread per trajectory, FP32", "per_method": seq,
                                    "value": work_per_step / (sum(v["ms_per_run"] for v in seq.values()) * 1e-3)}

    # PES_MIXED: the first iters-1 iterations in FP32, the final one in FP64
    xmix = {}
    if not args.no_mixed:
        run_step(d32, pes.MIXED)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in methods]
        flush.zero_()
        run_step(d32, pes.MIXED, ev)
        torch.cuda.synchronize()
        per = [ev[i][0].elapsed_time(ev[i][1]) for i in range(len(methods))]
        if rank == 0:
            result["mixed"] = {"value": work_per_step / (sum(per) * 1e-3), "ms_per_step": sum(per),
                               "per_method_ms": dict(zip([m for m, _ in methods], per)),
                               "schedule": f"{iters - 1} FP32 iterations, then 1 FP64 iteration"}
        for name, m in methods:
            x, P, _, _ = sm.ieks_run(d32["model"], m, pes.MIXED, d32["y"], d32["offsets"], d32["m0"], d32["P0"],
                                     iters=iters)
            xmix[name] = (x.double().cpu().numpy(), P.double().cpu().numpy())
        sm.sync()

    # end-to-end through the host-buffer entry point (copies inside the timed
    # region). A user with both methods to run gives each its own handle, stream
    # and host thread (handles are independent), so that one run's copies
    # overlap the other's kernels; the same calls one after the other on one
    # thread are reported beside it ("serial").
    if not args.no_e2e:
        pin = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt).pin_memory()
        hy, hoff = pin(wl["y"], torch.float32), pin(wl["offsets"], torch.int64)
        hm0, hP0 = pin(wl["m0"], torch.float32), pin(wl["P0"], torch.float32)
        hs = pin(wl["sensors"], torch.float64)
        outs = {name: (torch.empty((5, N), dtype=torch.float32).pin_memory(),
                       torch.empty((15, N), dtype=torch.float32).pin_memory()) for name, _ in methods}
        handles = {name: pes.Smoother(N, wl["offsets"].shape[0] - 1) for name, _ in methods}
        streams = {name: torch.cuda.Stream() for name, _ in methods}
        for name, m in methods:
            if tuned.get(name):
                handles[name].set_launch_shape(m, pes.FP32, tuned[name]["threads"], tuned[name]["min_steps_per_lane"])

        device = torch.cuda.current_device()

        def run_host(name, m, prec, n):
            torch.cuda.set_device(device)   # a worker thread starts on device 0
            hx, hP = outs[name]
            for _ in range(n):
                handles[name].ieks_run_host(d32["model"], m, prec, hy, hoff, hm0, hP0, iters=iters, x_out=hx,
                                            P_out=hP, sensors_host=hs, stream=streams[name])

        def e2e_pipelined(prec, n):
            with cf.ThreadPoolExecutor(len(methods)) as ex:
                for f in [ex.submit(run_host, name, m, prec, n) for name, m in methods]:
                    f.result()

        def e2e_serial(prec, n):
            for _ in range(n):
                for name, m in methods:
                    run_host(name, m, prec, 1)

        e2e_rates = {}
        for key, prec in timed_precs:
            rates = {}
            for mode, fn in (("pipelined", e2e_pipelined), ("serial", e2e_serial)):
                fn(prec, args.warmup)
                barrier()
                t0 = time.perf_counter()
                fn(prec, args.steps)
                e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
                rates[mode] = (whole_job_rate(world, work_per_step, args.steps, e2e_s), 1e3 * e2e_s / args.steps)
            e2e_rates[key] = rates
        for h_ in handles.values():
            h_.close()
        if rank == 0:
            h2d = len(methods) * (hy.numel() * 4 + hoff.numel() * 8 + hm0.numel() * 4 + hP0.numel() * 4 +
                                  hs.numel() * 8)
            d2h = len(methods) * (outs[methods[0][0]][0].numel() * 4 + outs[methods[0][0]][1].numel() * 4)
            result["e2e_by_precision"] = {
                key: {"value": r["pipelined"][0], "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                      "ms_per_step": r["pipelined"][1], "precision": key,
                      "method": "pes_ieks_run_host with pinned host buffers; IEKS and cubature each on its own handle, "
                                "stream and host thread",
                      "serial": {"value": r["serial"][0], "ms_per_step": r["serial"][1]}}
                for key, r in e2e_rates.items()}
            result["e2e"] = result["e2e_by_precision"]["fp32"]

    # iterations saved by the learned initialiser (a reduced run of the full
    # experiment: 8,192 training trajectories, 256 held-out ones)
    if rank == 0 and not args.no_learned_init:
        from paper_2102_00514_gb300 import learned_init as LI
        li = LI.run(n_train=8192, T_train=1000, n_heldout=256, steps=3000, batch_traj=128)
        # the start as the library uses it (network within ten times its
        # training length, prior start beyond, and the prior start again where
        # the network's does not converge), paired over every held-out
        # trajectory with non-converged runs counted at the cap: the policy
        # whose final error is no worse (the metric's "at equal final error")
        result["iters_saved"] = li["ieks"]["gated_fallback"]["iters_saved_capped"]
        result["learned_init"] = li

    if rank == 0:
        import oracle
        oracle.build()
        # CPU baseline: the oracle as it stands on one host core, bounded sample
        if not args.no_cpu_baseline:
            sw = sample_workload(wl, min(args.cpu_sample, N))
            Sn, Sb = sw["y"].shape[1], len(sw["offsets"]) - 1
            t = oracle_timed(sw, iters)
            result["cpu_baseline"] = {"value": 2 * (Sn - Sb) * iters / (t["ieks"] + t["cubature"]), "unit": UNIT,
                                      "cores": 1, "kind": "oracle",
                                      "sample": f"first {Sn} of {N} states ({Sb} trajectories), IEKS + cubature, "
                                                f"{iters} iterations, sequential FP64 oracle"}
        # parity of this very run against the oracle: on the whole workload for
        # one trajectory, on sampled trajectories (each smoothed alone) for a batch
        if not args.no_parity:
            units = parity_units(wl)
            r32 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
            omethods = (("ieks", oracle.IEKS), ("cubature", oracle.CUBATURE))

            def orc(u, m):
                one = u[0]
                return oracle.iterated_smoother(oracle.Model.from_workload(one), m, one["offsets"], one["y"],
                                                one["m0"], one["P0"], iters=iters)

            # the final iteration alone: one FP64 oracle iteration from the GPU's
            # own FP32 nominal, on the float inputs widened to double
            def orc_last(u, name, m):
                one, sl = u
                if name not in nom32:
                    return None
                return oracle.iterated_smoother(oracle.Model.from_workload(one), m, one["offsets"], r32(one["y"]),
                                                r32(one["m0"]), r32(one["P0"]), x_init=nom32[name][0][:, sl],
                                                P_init=nom32[name][1][:, sl], iters=1)

            with cf.ThreadPoolExecutor(min(16, os.cpu_count() or 1)) as ex:
                fut = {(n, i): ex.submit(orc, u, m) for n, m in omethods for i, u in enumerate(units)}
                fut_last = {(n, i): ex.submit(orc_last, u, n, m) for n, m in omethods for i, u in enumerate(units)}
                refs = {k: f.result() for k, f in fut.items()}
                last = {k: f.result() for k, f in fut_last.items()}

            def worst(arr, ref_key, rs, key):
                return max(rel_err(arr[:, u[1]], rs[(ref_key, i)][key], u[0]["offsets"]) for i, u in enumerate(units))

            par = {}
            for name, _ in methods:
                par[name] = {"fp32_means": worst(x32[name][0], name, refs, "x"),
                             "fp32_covs": worst(x32[name][1], name, refs, "P")}
                if not args.no_fp64:
                    par[name]["fp64_means"] = worst(x64[name][0], name, refs, "x")
                    par[name]["fp64_covs"] = worst(x64[name][1], name, refs, "P")
                if name in xmix:
                    par[name]["mixed_means"] = worst(xmix[name][0], name, refs, "x")
                    par[name]["mixed_covs"] = worst(xmix[name][1], name, refs, "P")
                par[name]["refined_means"] = worst(xref[name][0], name, refs, "x")
                par[name]["refined_covs"] = worst(xref[name][1], name, refs, "P")
                par[name]["oracle_final_rel_update"] = max(float(refs[(name, i)]["rel_history"][-1])
                                                           for i in range(len(units)))
                if name in nom32:
                    fi = {"fp32_means": worst(x32[name][0], name, last, "x"),
                          "fp32_covs": worst(x32[name][1], name, last, "P")}
                    if name in xmix:
                        fi["mixed_means"] = worst(xmix[name][0], name, last, "x")
                        fi["mixed_covs"] = worst(xmix[name][1], name, last, "P")
                    fi["refined_means"] = worst(xref[name][0], name, last, "x")
                    fi["refined_covs"] = worst(xref[name][1], name, last, "P")
                    # R12: the worst single state, ||.||_2 relative to the state's own norm
                    fi["refined_means_worst_state"] = max(
                        per_state_max(xref[name][0][:, u[1]], last[(name, i)]["x"]) for i, u in enumerate(units))
                    fi["refined_covs_worst_state"] = max(
                        per_state_max(xref[name][1][:, u[1]], last[(name, i)]["P"]) for i, u in enumerate(units))
                    fi["fp32_covs_worst_state"] = max(
                        per_state_max(x32[name][1][:, u[1]], last[(name, i)]["P"]) for i, u in enumerate(units))
                    # and the median state (R12 reports both)
                    med = lambda arr, c: float(np.median(np.concatenate(
                        [per_state_errors(arr[:, u[1]], last[(name, i)][c]) for i, u in enumerate(units)])))
                    fi["refined_means_median_state"] = med(xref[name][0], "x")
                    fi["refined_covs_median_state"] = med(xref[name][1], "P")
                    fi["fp32_means_median_state"] = med(x32[name][0], "x")
                    fi["fp32_covs_median_state"] = med(x32[name][1], "P")
                    par[name]["final_iteration"] = fi
            scope = ("full workload" if len(units) == 1 else
                     f"{len(units)} sampled trajectories, each smoothed alone by the oracle (worst reported)")

            def within(rows, prefix, tol):
                keys = (prefix + "_means", prefix + "_covs")
                got = [r for r in rows if all(k in r for k in keys)]
                return all(r[k] <= tol for r in got for k in keys) if got else None

            finals = [v["final_iteration"] for v in par.values() if "final_iteration" in v]
            # one outcome per check: the final iteration from a given nominal is what
            # the kernel's precision decides; all iterations also carry the
            # iteration's own amplification wherever the oracle has not converged
            result["parity"] = {"vs": f"CPU FP64 oracle, {scope}; final_iteration: one oracle iteration from "
                                      "the GPU's own FP32 nominal of the first iters-1 iterations",
                                "rel_frobenius": par,
                                "tol": {"fp32": 1e-4, "fp64": 1e-9},
                                "within_tol": {"fp64_all_iterations": within(par.values(), "fp64", 1e-9),
                                               "fp32_final_iteration": within(finals, "fp32", 1e-4),
                                               "mixed_final_iteration": within(finals, "mixed", 1e-4),
                                               "refined_final_iteration": within(finals, "refined", 1e-4),
                                               "fp32_all_iterations": within(par.values(), "fp32", 1e-4),
                                               "mixed_all_iterations": within(par.values(), "mixed", 1e-4)}}
            choose_headline(result)
        if B == 1 and world == 1:
            if not args.no_length_sweep:
                result["length_sweep"] = length_sweep_key(args, flush)
            if not args.no_batched:
                result["batched"] = batched_key(args, roofline["peak"], flush)
        print(json.dumps(result), flush=True)
    sm.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
