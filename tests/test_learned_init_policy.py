"""Host logic of the learned initialiser (paper_2102_00514_gb300/learned_init.py),
on the CPU: the packing of a subset of trajectories for the fallback run, the
length gate, the paired summary's iteration accounting when the fallback ran,
and the training checkpoint's file (with a stand-in for the network's state)."""
import numpy as np
import torch

from paper_2102_00514_gb300 import learned_init as L


def small_workload():
    lens = [4, 7, 3]   # states per trajectory
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    N = int(off[-1])
    y = np.arange(2 * N, dtype=np.float64).reshape(2, N)
    m0 = np.arange(15, dtype=np.float64).reshape(3, 5)
    P0 = np.arange(45, dtype=np.float64).reshape(3, 15)
    sensors = np.arange(12, dtype=np.float64).reshape(3, 4)
    return dict(y=y, offsets=off, m0=m0, P0=P0, sensors=sensors)


def test_subset_packs_the_chosen_trajectories_in_order():
    wl = small_workload()
    sub = L._subset(wl, np.array([2, 0]))
    assert sub["offsets"].tolist() == [0, 3, 7]
    assert sub["offsets"].dtype == np.int64
    np.testing.assert_array_equal(sub["y"], np.concatenate([wl["y"][:, 11:14], wl["y"][:, 0:4]], axis=1))
    np.testing.assert_array_equal(sub["m0"], wl["m0"][[2, 0]])
    np.testing.assert_array_equal(sub["P0"], wl["P0"][[2, 0]])
    np.testing.assert_array_equal(sub["sensors"], wl["sensors"][[2, 0]])
    # one shared sensor pair stays shared
    shared = dict(wl, sensors=wl["sensors"][:1])
    assert L._subset(shared, np.array([1]))["sensors"].shape == (1, 4)


def test_gated_start_is_the_prior_mean_beyond_the_valid_length():
    wl = small_workload()
    N = wl["y"].shape[1]
    x_net = torch.arange(5 * N, dtype=torch.float64).reshape(5, N)
    T = np.diff(wl["offsets"]) - 1   # measurements: 3, 6, 2
    xg = L.gated_start(x_net, wl, t_valid=4)
    off = wl["offsets"]
    for b in range(3):
        sl = slice(int(off[b]), int(off[b + 1]))
        if T[b] > 4:
            assert torch.equal(xg[:, sl], torch.as_tensor(wl["m0"][b])[:, None].expand(5, sl.stop - sl.start))
        else:
            assert torch.equal(xg[:, sl], x_net[:, sl])
    assert torch.equal(x_net, torch.arange(5 * N, dtype=torch.float64).reshape(5, N))   # not modified


def test_summary_counts_both_runs_of_a_fallback():
    cap = 50
    ip = np.array([10, 12, 0, 20])            # prior start: trajectory 2 never converges
    # the policy: trajectory 1's network start failed, the fallback converged in 12;
    # trajectory 2 failed both ways
    il = np.array([6, 12, 0, 15])
    spent = np.array([6, cap + 12, cap + cap, 15])
    ep = np.array([1.0, 2.0, 3.0, 4.0])
    el = np.array([1.0, 2.0, 3.5, 3.0])
    r = L.EvalResult(ip, il, ep, el, np.zeros(4), 0.0, fallback=np.array([False, True, True, False]),
                     spent_learned=spent)
    s = L.summary(r, max_iters=cap)
    ip_capped = np.array([10, 12, cap, 20])
    assert s["mean_iters_prior_capped"] == ip_capped.mean()
    assert s["mean_iters_learned_capped"] == spent.mean()
    assert s["iters_saved_capped"] == (ip_capped - spent).mean()
    assert s["converged_prior"] == 3 and s["converged_learned"] == 3 and s["converged_both"] == 3
    assert s["fallback_runs"] == 2
    assert s["error_no_worse_fraction"] == 0.75     # trajectory 2 is worse
    # on the trajectories both converge, the fallback's own iterations count in full
    both = np.array([True, True, False, True])
    assert s["iters_saved"] == (ip[both] - spent[both]).mean()


class _StateHolder:
    """Stands in for pes.InitNet's get_state / set_state."""

    def __init__(self, state=None):
        self.state = state

    def get_state(self):
        return self.state

    def set_state(self, state):
        self.state = state


def test_checkpoint_round_trip_restores_state_and_sampler(tmp_path):
    rng = np.random.default_rng(5)
    n = L.pes.INIT_NPARAMS
    st = dict(params=rng.standard_normal(n).astype(np.float32), mu=rng.standard_normal(5),
              sigma=0.5 + rng.random(5), m=rng.standard_normal(n).astype(np.float32),
              v=rng.random(n).astype(np.float32), t=17)
    g = np.random.default_rng(3)
    order = g.permutation(11)
    g.permutation(11)                        # the sampler has moved on
    path = str(tmp_path / "ckpt.npz")
    L.save_checkpoint(path, _StateHolder(st), 42, g, order)
    expect = g.permutation(11)               # what the uninterrupted sampler draws next
    net = _StateHolder()
    step, rng_state, order2 = L.load_checkpoint(path, net)
    assert step == 42 and np.array_equal(order2, order)
    for k in ("params", "mu", "sigma", "m", "v"):
        assert net.state[k].dtype == st[k].dtype and np.array_equal(net.state[k], st[k]), k
    assert net.state["t"] == 17
    g2 = np.random.default_rng(0)
    g2.bit_generator.state = rng_state
    assert np.array_equal(g2.permutation(11), expect)
    # a second save replaces the file whole
    L.save_checkpoint(path, _StateHolder(dict(st, t=18)), 43, g, order)
    assert L.load_checkpoint(path, net)[0] == 43 and net.state["t"] == 18
