"""Training and evaluation of the learned initialiser (include/pes_init.h).

The network maps a trajectory's measurements to the nominal trajectory the
iterated smoother (Sec. 3) starts from. Its training targets are the means the
FP64 smoother itself reaches when iterated to convergence; its use is judged
by the smoother, not by the network's own error: iterations needed to reach a
relative update of 1e-6, and the converged result, against the plain start
from the prior mean.

Everything numerical runs in the library's kernels (the smoother, the
network's forward and backward passes and its Adam steps); this module only
arranges device buffers (PyTorch) and bookkeeping on the host.
"""
from __future__ import annotations

import json
import os
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import pes, synth

TOL_TARGETS = 1e-9      # relative update at which a training target counts as converged
TOL_EVAL = 1e-6         # the tolerance iterations are counted to
MAX_ITERS = 50


def _dev(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def converged_targets(wl: dict, method: int = pes.IEKS, chunk_states: int = 1 << 23, tol: float = TOL_TARGETS,
                      max_iters: int = MAX_ITERS):
    """FP64 smoother means of every trajectory, iterated to `tol` from the prior,
    in chunks of whole trajectories. Returns (x [5][N] float64 host, converged
    bool [B])."""
    off = wl["offsets"]
    B = len(off) - 1
    N = int(off[-1])
    x = np.empty((5, N))
    conv = np.zeros(B, dtype=bool)
    longest = int(np.diff(off).max())
    sm = pes.Smoother(max(chunk_states, longest), B)
    model = pes.Model.from_workload(wl)
    b0 = 0
    while b0 < B:
        b1 = int(np.searchsorted(off, off[b0] + chunk_states, side="right")) - 1
        b1 = max(b1, b0 + 1)
        a, e = int(off[b0]), int(off[b1])
        sub_off = off[b0:b1 + 1] - a
        sub_model = pes.Model.from_workload(dict(wl, sensors=wl["sensors"][b0:b1])) if len(wl["sensors"]) > 1 \
            else model
        xs, _, _, _ = sm.ieks_run(sub_model, method, pes.FP64, _dev(wl["y"][:, a:e], torch.float64),
                                  _dev(sub_off, torch.int64), _dev(wl["m0"][b0:b1], torch.float64),
                                  _dev(wl["P0"][b0:b1], torch.float64), iters=max_iters, tol=tol,
                                  allow_not_converged=True)
        conv[b0:b1] = sm.traj_iterations(b1 - b0) > 0
        x[:, a:e] = xs.cpu().numpy()
        b0 = b1
    sm.close()
    return x, conv


def normalisation(x: np.ndarray):
    mu = x.mean(axis=1)
    sigma = x.std(axis=1)
    return mu, np.where(sigma > 0, sigma, 1.0)


# Packed parameter shapes (include/pes_init.h): 4 conv layers W [64][64][5],
# b [64]; W5 [64][64], b5 [64]; W6 [5][64], b6 [5].
SHAPES = [((64, 64, 5), 64)] * 4 + [((64, 64), 64), ((5, 64), 5)]


def initial_params(seed: int) -> np.ndarray:
    """He-normal weights (fan-in = input channels x taps), zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for ws, nb in SHAPES:
        fan_in = int(np.prod(ws[1:]))
        parts += [rng.standard_normal(int(np.prod(ws))) * np.sqrt(2.0 / fan_in), np.zeros(nb)]
    p = np.concatenate(parts).astype(np.float32)
    assert p.shape == (pes.INIT_NPARAMS,)
    return p


@dataclass
class TrainLog:
    steps: int = 0
    seconds: float = 0.0
    losses: list = field(default_factory=list)


def save_checkpoint(path: str, net, step: int, rng: np.random.Generator, order: np.ndarray) -> None:
    """The training run after `step` steps: the network's training state
    (parameters, normalisation, Adam's moments and step count), the minibatch
    sampler's generator state and its current permutation. Written to a
    temporary file first and renamed over `path`, so that an interrupted save
    leaves the previous checkpoint intact."""
    st = net.get_state()
    rng_state = np.frombuffer(json.dumps(rng.bit_generator.state).encode(), dtype=np.uint8)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "wb") as f:
        np.savez(f, step=np.int64(step), order=np.asarray(order, dtype=np.int64), rng_state=rng_state,
                 params=st["params"], mu=st["mu"], sigma=st["sigma"], adam_m=st["m"], adam_v=st["v"],
                 adam_t=np.int64(st["t"]))
    os.replace(tmp, path)


def load_checkpoint(path: str, net):
    """Restore the network's training state from a checkpoint; returns (step,
    the sampler's generator state, its permutation)."""
    with np.load(path) as z:
        net.set_state(dict(params=z["params"], mu=z["mu"], sigma=z["sigma"], m=z["adam_m"], v=z["adam_v"],
                           t=int(z["adam_t"])))
        return int(z["step"]), json.loads(bytes(z["rng_state"]).decode()), z["order"].copy()


def train(net: pes.InitNet, wl: dict, targets: np.ndarray, keep: np.ndarray, *, batch_traj: int = 128,
          steps: int = 2000, lr: float = 2e-3, lr_final: float = 2e-4, seed: int = 0,
          log_every: int = 100, checkpoint: str | None = None, checkpoint_every: int = 0,
          resume: bool = False, stop_at: int | None = None) -> TrainLog:
    """Adam on minibatches of `batch_traj` whole trajectories of one length,
    the learning rate decayed geometrically from lr to lr_final over `steps`
    steps. Only the trajectories with keep[b] (converged targets) are used. The
    network's parameters and normalisation must be set before (or restored:
    with `resume`, from the checkpoint at `checkpoint`, and the run continues
    at the step it was saved after). With `checkpoint` and `checkpoint_every`,
    the run is saved there every `checkpoint_every` steps and when it stops;
    `stop_at` ends this call after that many steps of the schedule (a job
    split over several calls resumes where the previous one stopped and gives
    the same parameters, bit for bit, as one uninterrupted call)."""
    off = wl["offsets"]
    lens = np.diff(off)
    if not np.all(lens == lens[0]):
        raise ValueError("training trajectories must share one length")
    n1 = int(lens[0])
    idx = np.flatnonzero(keep)
    nmb = len(idx) // batch_traj
    if nmb < 1:
        raise ValueError("fewer kept trajectories than one minibatch")
    idx = idx[:nmb * batch_traj]
    # [minibatch][component][states] so that each minibatch is one contiguous
    # component-major block (the layout of the ABI)
    y = torch.as_tensor(wl["y"], dtype=torch.float32).reshape(2, -1, n1)[:, idx]
    xt = torch.as_tensor(targets, dtype=torch.float32).reshape(5, -1, n1)[:, idx]
    Y = y.reshape(2, nmb, batch_traj * n1).permute(1, 0, 2).contiguous().cuda()
    X = xt.reshape(5, nmb, batch_traj * n1).permute(1, 0, 2).contiguous().cuda()
    moff = _dev(np.arange(batch_traj + 1, dtype=np.int64) * n1, torch.int64)
    rng = np.random.default_rng(seed)
    order = rng.permutation(nmb)
    s0 = 0
    if resume:
        if not checkpoint:
            raise ValueError("resume needs the checkpoint's path")
        s0, rng_state, order = load_checkpoint(checkpoint, net)
        if len(order) != nmb:
            raise ValueError("the checkpoint was taken with another training set or minibatch size")
        rng.bit_generator.state = rng_state
    end = steps if stop_at is None else min(steps, stop_at)
    log = TrainLog()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in range(s0, end):
        if s and s % nmb == 0:
            order = rng.permutation(nmb)
        m = int(order[s % nmb])
        a = lr * (lr_final / lr) ** (s / max(1, steps - 1))
        want = (s % log_every == 0) or s == steps - 1
        loss = net.train_step(pes.FP32, Y[m], moff, X[m], a, want_loss=want)
        if want:
            log.losses.append((s, loss))
        if checkpoint and checkpoint_every and ((s + 1) % checkpoint_every == 0 or s + 1 == end):
            save_checkpoint(checkpoint, net, s + 1, rng, order)
    torch.cuda.synchronize()
    log.seconds = time.perf_counter() - t0
    log.steps = end - s0
    return log


@dataclass
class EvalResult:
    iters_prior: np.ndarray        # per trajectory, 0 = tolerance not reached
    iters_learned: np.ndarray
    err_prior: np.ndarray          # per trajectory RMS position error against the truth
    err_learned: np.ndarray
    rel_diff: np.ndarray           # ||x_learned - x_prior|| / ||x_prior|| per trajectory
    seconds: float
    # with the fallback: trajectories re-run from the prior start, and the
    # iterations the learned policy spent per trajectory (a run that does not
    # reach the tolerance counted at the cap, both runs where there are two)
    fallback: np.ndarray | None = None
    spent_learned: np.ndarray | None = None


def gated_start(x_net: torch.Tensor, wl: dict, t_valid: int) -> torch.Tensor:
    """The start the library uses with the network: the network's nominal for
    trajectories of at most `t_valid` measurements, the prior mean (the plain
    start, which is the fallback) for longer ones. The network sees windows of
    17 measurements; past about ten times its training length the converged
    trajectories leave the range it was trained on (positions hundreds of units
    from the sensors, where two bearings do not fix the range locally) and its
    start lands on another fixed point of the iteration as often as not."""
    off = wl["offsets"]
    x = x_net.clone()
    T = np.diff(off) - 1
    for b in np.flatnonzero(T > t_valid):
        a, e = int(off[b]), int(off[b + 1])
        x[:, a:e] = torch.as_tensor(wl["m0"][b], dtype=x.dtype, device=x.device)[:, None]
    return x


def _subset(wl: dict, idx: np.ndarray) -> dict:
    """The trajectories idx of a workload, packed into one of their own."""
    off = wl["offsets"]
    lens = np.diff(off)[idx]
    cols = np.concatenate([np.arange(off[b], off[b + 1]) for b in idx])
    sub = dict(wl, y=wl["y"][:, cols], offsets=np.concatenate([[0], np.cumsum(lens)]).astype(np.int64),
               m0=wl["m0"][idx], P0=wl["P0"][idx])
    if len(wl["sensors"]) > 1:
        sub["sensors"] = wl["sensors"][idx]
    return sub


def rerun_from_prior(wl: dict, idx: np.ndarray, method: int, tol: float, max_iters: int):
    """The fallback: trajectories idx iterated from the prior start in a batch
    of their own. Returns (x [5][states of idx] float64 host, iterations to
    tol per trajectory, 0 = not reached)."""
    sub = _subset(wl, idx)
    B = len(idx)
    sm = pes.Smoother(int(sub["offsets"][-1]), B)
    xs, _, _, _ = sm.ieks_run(pes.Model.from_workload(sub), method, pes.FP64, _dev(sub["y"], torch.float64),
                              _dev(sub["offsets"], torch.int64), _dev(sub["m0"], torch.float64),
                              _dev(sub["P0"], torch.float64), iters=max_iters, tol=tol, allow_not_converged=True)
    it = sm.traj_iterations(B)
    x = xs.cpu().numpy()
    sm.close()
    return x, it


def evaluate(net: pes.InitNet, wl: dict, method: int = pes.IEKS, tol: float = TOL_EVAL,
             max_iters: int = MAX_ITERS, t_valid: int | None = None, fallback: bool = False,
             judge: bool = False) -> EvalResult:
    """Iterations to `tol` and converged results from the prior start and from
    the network's start (gated by trajectory length when `t_valid` is given),
    every trajectory of `wl` in one FP64 batch each. With `fallback`, the
    trajectories that the network's start (not the prior one it is gated to
    beyond `t_valid`) does not bring to `tol` within `max_iters` are iterated
    again from the prior start in a batch of their own, and that run's result
    replaces theirs; its iterations are added to what the learned policy
    spent. With `judge`, both starts' converged solutions are kept side by side
    and, per trajectory, the one whose filter log-likelihood under its own
    final linearisation (pes_filter_loglik) is higher is the result; the
    policy then spends both runs' iterations (the prior start's run is the
    judge), and `fallback` marks the trajectories where the prior start's
    solution was kept."""
    off = wl["offsets"]
    B = len(off) - 1
    N = int(off[-1])
    sm = pes.Smoother(N, B)
    model = pes.Model.from_workload(wl)
    y = _dev(wl["y"], torch.float64)
    o = _dev(off, torch.int64)
    m0, P0 = _dev(wl["m0"], torch.float64), _dev(wl["P0"], torch.float64)
    t0 = time.perf_counter()
    xa, Pa, _, _ = sm.ieks_run(model, method, pes.FP64, y, o, m0, P0, iters=max_iters, tol=tol,
                               allow_not_converged=True)
    ia = sm.traj_iterations(B)
    x0 = net.forward(pes.FP64, y, o)
    if t_valid is not None:
        x0 = gated_start(x0, wl, t_valid)
    xb, Pb, _, _ = sm.ieks_run(model, method, pes.FP64, y, o, m0, P0, x_init=x0, iters=max_iters, tol=tol,
                               allow_not_converged=True)
    ib = sm.traj_iterations(B)
    lla = llb = None
    if judge:
        def loglik(x, P):
            lin = sm.linearize(model, method, pes.FP64, x, P, y, o)
            _, _, ll = sm.filter_loglik(pes.FP64, lin, lin["y_used"], m0, P0, o)
            return ll.cpu().numpy()
        lla, llb = loglik(xa, Pa), loglik(xb, Pb)
    xa, xb = xa.cpu().numpy(), xb.cpu().numpy()
    sm.close()
    fb = spent = None
    if judge:
        spent = (np.where(ib > 0, ib, max_iters) + np.where(ia > 0, ia, max_iters)).astype(np.int64)
        fb = llb < lla
        for b in np.flatnonzero(fb):
            xb[:, off[b]:off[b + 1]] = xa[:, off[b]:off[b + 1]]
        ib = np.where(fb, ia, ib)
        fallback = False
    if fallback:
        spent = np.where(ib > 0, ib, max_iters).astype(np.int64)
        # only where the network's start was used (beyond t_valid the start
        # already is the prior mean)
        fb = ib == 0
        if t_valid is not None:
            fb &= (np.diff(off) - 1) <= t_valid
        idx = np.flatnonzero(fb)
        if len(idx):
            xf, itf = rerun_from_prior(wl, idx, method, tol, max_iters)
            a = 0
            for j, b in enumerate(idx):
                n = int(off[b + 1] - off[b])
                xb[:, off[b]:off[b + 1]] = xf[:, a:a + n]
                a += n
                spent[b] += itf[j] if itf[j] > 0 else max_iters
            ib = ib.copy()
            ib[idx] = itf
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    xt = wl["x_true"]
    ea, eb, rd = np.zeros(B), np.zeros(B), np.zeros(B)
    for b in range(B):
        sl = slice(int(off[b]), int(off[b + 1]))
        ea[b] = np.sqrt(np.mean((xa[0:2, sl] - xt[0:2, sl]) ** 2) * 2)
        eb[b] = np.sqrt(np.mean((xb[0:2, sl] - xt[0:2, sl]) ** 2) * 2)
        rd[b] = np.linalg.norm(xb[:, sl] - xa[:, sl]) / max(np.linalg.norm(xa[:, sl]), 1e-300)
    return EvalResult(ia, ib, ea, eb, rd, secs, fb, spent)


def summary(r: EvalResult, max_iters: int = MAX_ITERS) -> dict:
    """Paired comparison of the two starts over every trajectory: iterations to
    tolerance with a trajectory that does not get there counted at the cap
    (for the learned policy with the fallback, the iterations of both its runs),
    final position error against the truth (the learned start is "no worse"
    where its error is within 0.1 % of the prior start's), and the same figures
    on the trajectories both starts bring to tolerance."""
    both = (r.iters_prior > 0) & (r.iters_learned > 0)
    ip = np.where(r.iters_prior > 0, r.iters_prior, max_iters)
    il = r.spent_learned if r.spent_learned is not None else np.where(r.iters_learned > 0, r.iters_learned, max_iters)
    no_worse = r.err_learned <= 1.001 * r.err_prior
    out = {"trajectories": int(len(r.iters_prior)),
           "converged_prior": int((r.iters_prior > 0).sum()),
           "converged_learned": int((r.iters_learned > 0).sum()),
           "converged_both": int(both.sum()),
           "mean_iters_prior_capped": float(ip.mean()),
           "mean_iters_learned_capped": float(il.mean()),
           "iters_saved_capped": float((ip - il).mean()),
           "error_no_worse_fraction": float(no_worse.mean()),
           "mean_position_rmse_all_prior": float(r.err_prior.mean()),
           "mean_position_rmse_all_learned": float(r.err_learned.mean()),
           "same_solution_all_within_1e-4": int((r.rel_diff < 1e-4).sum())}
    if r.fallback is not None:
        out["fallback_runs"] = int(r.fallback.sum())
    if both.any():
        out.update({
            "mean_iters_prior": float(r.iters_prior[both].mean()),
            "mean_iters_learned": float(il[both].mean()),
            "iters_saved": float((r.iters_prior[both] - il[both]).mean()),
            "same_solution_within_1e-4": int((r.rel_diff[both] < 1e-4).sum()),
            "median_position_rmse_prior": float(np.median(r.err_prior[both])),
            "median_position_rmse_learned": float(np.median(r.err_learned[both])),
            "mean_position_rmse_prior": float(np.mean(r.err_prior[both])),
            "mean_position_rmse_learned": float(np.mean(r.err_learned[both])),
        })
    return out


def run(n_train: int = 100_000, T_train: int = 1000, n_heldout: int = 1024, heldout_lo: int = 1000,
        heldout_hi: int = 100_000, steps: int = 8000, batch_traj: int = 128, methods=("ieks", "cubature"),
        seed: int = 0) -> dict:
    """The whole experiment: targets, training, evaluation of both methods.
    The defaults are the full-size configuration (10^5 training trajectories
    of T = 1,000; 1,024 held-out trajectories with log T uniform in
    [1,000, 100,000])."""
    out = {"n_train": n_train, "T_train": T_train, "n_heldout": n_heldout,
           "heldout_T": [heldout_lo, heldout_hi], "steps": steps, "batch_traj": batch_traj}
    t0 = time.perf_counter()
    wl = synth.workload(f"train{n_train}_T{T_train}")
    ev = synth.workload(f"heldout{n_heldout}_T{heldout_lo}_{heldout_hi}")
    out["synth_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    x, conv = converged_targets(wl)
    out["targets_s"] = time.perf_counter() - t0
    out["targets_converged"] = float(conv.mean())
    mu, sigma = normalisation(x[:, np.repeat(conv, T_train + 1)])
    net = pes.InitNet(max(ev["y"].shape[1], batch_traj * (T_train + 1)), max(n_heldout, batch_traj))
    net.set_params(initial_params(seed), mu, sigma)
    log = train(net, wl, x, conv, batch_traj=batch_traj, steps=steps, lr=2e-3, lr_final=1e-4, seed=seed)
    out["train_s"] = log.seconds
    out["train_states_per_s"] = steps * batch_traj * (T_train + 1) / log.seconds
    out["loss_first_last"] = [log.losses[0][1], log.losses[-1][1]]
    del x, wl
    # inference throughput on the held-out set (forward pass only)
    y = _dev(ev["y"], torch.float64)
    o = _dev(ev["offsets"], torch.int64)
    net.forward(pes.FP64, y, o)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    net.forward(pes.FP64, y, o)
    e1.record()
    torch.cuda.synchronize()
    out["inference_states_per_s"] = ev["y"].shape[1] / (e0.elapsed_time(e1) * 1e-3)
    t_valid = 10 * T_train
    out["t_valid"] = t_valid
    for name in methods:
        m = pes.IEKS if name == "ieks" else pes.CUBATURE
        r = evaluate(net, ev, method=m)
        out[name] = summary(r)
        out[name]["seconds"] = r.seconds
        # the start as the library uses it: the network within its length
        # domain, the prior start (the fallback) beyond it
        rg = evaluate(net, ev, method=m, t_valid=t_valid)
        out[name]["gated"] = summary(rg)
        # and with the fallback: trajectories the start does not bring to
        # tolerance are iterated again from the prior start
        out[name]["gated_fallback"] = summary(evaluate(net, ev, method=m, t_valid=t_valid, fallback=True))
        # and judged by the converged solutions' log-likelihoods (both runs paid)
        out[name]["gated_judged"] = summary(evaluate(net, ev, method=m, t_valid=t_valid, judge=True))
        T = np.diff(ev["offsets"]) - 1
        inside = T <= t_valid
        if inside.any():
            sub = EvalResult(r.iters_prior[inside], r.iters_learned[inside], r.err_prior[inside],
                             r.err_learned[inside], r.rel_diff[inside], 0.0)
            out[name]["within_t_valid"] = summary(sub)
    net.close()
    return out


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="train and evaluate the learned initialiser")
    ap.add_argument("--n-train", type=int, default=100_000)
    ap.add_argument("--T-train", type=int, default=1000)
    ap.add_argument("--n-heldout", type=int, default=1024)
    ap.add_argument("--steps", type=int, default=8000)
    ap.add_argument("--batch-traj", type=int, default=128)
    a = ap.parse_args()
    from . import build
    build.build_all()
    print(json.dumps(run(a.n_train, a.T_train, a.n_heldout, steps=a.steps, batch_traj=a.batch_traj)), flush=True)
