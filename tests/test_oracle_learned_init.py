"""Pins of the learned-initialiser oracle (oracle/learned_init.py) against
what does not depend on it: a library convolution, finite differences of its
own forward pass, the closed form of Adam's first step, and PyTorch's
bfloat16 conversion."""
import numpy as np
import torch

from oracle import learned_init as li


def test_bf16_rounding_equals_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(10000) * 10.0 ** rng.integers(-8, 8, 10000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.005859375, 1.0 + 2 ** -8, 65504.0]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(li.bf16(x), ref)


def test_single_channel_conv_equals_numpy_convolve():
    # one input and one output channel: the layer is a cross-correlation with
    # "same" zero padding, i.e. np.convolve with the flipped kernel
    rng = np.random.default_rng(1)
    h = np.zeros((37, li.C))
    h[:, 0] = rng.standard_normal(37)
    W = np.zeros((li.C, li.C, li.TAPS))
    w = rng.standard_normal(li.TAPS)
    W[0, 0, :] = w
    out = li.conv(h, W, np.zeros(li.C))
    assert np.allclose(out[:, 0], np.convolve(h[:, 0], w[::-1], mode="same"), atol=1e-14)
    assert np.abs(out[:, 1:]).max() == 0.0


def test_conv_multi_channel_brute_force():
    rng = np.random.default_rng(2)
    n = 9
    h = rng.standard_normal((n, li.C))
    W = rng.standard_normal((li.C, li.C, li.TAPS))
    b = rng.standard_normal(li.C)
    out = li.conv(h, W, b)
    for k in (0, 1, 4, n - 1):
        for o in (0, 17, 63):
            acc = b[o]
            for j in range(li.TAPS):
                kk = k + j - 2
                if 0 <= kk < n:
                    acc += sum(W[o, i, j] * h[kk, i] for i in range(li.C))
            assert abs(out[k, o] - acc) < 1e-11


def test_features_on_unit_circle_and_head_marker():
    y = np.vstack([np.linspace(-3, 3, 11), np.linspace(2, -2, 11)])
    phi = li.features(y, 10)
    assert np.allclose(phi[1:, 0] ** 2 + phi[1:, 1] ** 2, 1.0)
    assert np.allclose(np.arctan2(phi[1:, 2], phi[1:, 3]), y[1, 1:])
    assert np.array_equal(phi[0], np.eye(li.C)[5])
    assert np.all(phi[1:, 4] == 1.0) and np.all(phi[:, 6:] == 0.0)


def test_parameter_count_and_packing_roundtrip():
    assert li.NPARAMS == 4 * (64 * 64 * 5 + 64) + 64 * 64 + 64 + 5 * 64 + 5
    p = li.init_params(3)
    assert p.dtype == np.float32 and p.shape == (li.NPARAMS,)
    assert np.array_equal(li.pack(li.unpack(p)), p.astype(np.float64))


def _tiny_problem(seed):
    rng = np.random.default_rng(seed)
    trajs = []
    for T in (6, 3):
        y = rng.uniform(-3, 3, (2, T + 1))
        x = rng.standard_normal((5, T + 1))
        trajs.append((y, x))
    # non-zero biases keep most ReLUs away from their kink
    layers = li.unpack(li.init_params(seed))
    layers = [(W, np.full_like(b, 0.05) + 0.1 * rng.standard_normal(b.shape)) for W, b in layers]
    return li.pack(layers), trajs, rng.standard_normal(5), 0.5 + rng.random(5)


def test_gradient_equals_central_finite_differences():
    params, trajs, mu, sigma = _tiny_problem(4)
    loss, g = li.loss_and_grad(params, trajs, mu, sigma, rounding=False)
    rng = np.random.default_rng(5)
    # offsets of each weight and bias tensor in the flat vector, and a few
    # entries of each (every one of the output layer's five biases)
    sizes = [int(np.prod(t)) for w, b in li.SHAPES for t in (w, b)]
    starts = np.cumsum([0] + sizes)
    idx = []
    for s0, s1 in zip(starts[:-1], starts[1:]):
        idx += list(range(s0, s1)) if s1 - s0 <= 6 else list(rng.integers(s0, s1, 6))
    eps = 1e-6
    for i in idx:
        p1 = params.copy(); p1[i] += eps
        p2 = params.copy(); p2[i] -= eps
        l1, _ = li.loss_and_grad(p1, trajs, mu, sigma, rounding=False)
        l2, _ = li.loss_and_grad(p2, trajs, mu, sigma, rounding=False)
        fd = (l1 - l2) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_loss_is_mean_square_error():
    params, trajs, mu, sigma = _tiny_problem(6)
    loss, _ = li.loss_and_grad(params, trajs, mu, sigma, rounding=False)
    errs = []
    for y, x in trajs:
        o = li.forward(params, y, x.shape[1] - 1, rounding=False)["o"]
        errs.append(((o - (x.T - mu) / sigma) ** 2).ravel())
    assert abs(loss - np.concatenate(errs).mean()) < 1e-14


def test_adam_first_step_closed_form():
    # from zero moments the bias-corrected first step is lr * g / (|g| + eps)
    # (Kingma and Ba: the step divides by sqrt(v_hat) + eps); gradients of the
    # order of eps show where eps enters
    rng = np.random.default_rng(7)
    p = rng.standard_normal(100).astype(np.float32)
    g = rng.standard_normal(100)
    g[:4] = [1e-8, -3e-8, 1e-7, -1e-6]
    opt = li.Adam(lr=1e-2)
    p1 = opt.step(p, g)
    expect = p.astype(np.float64) - 1e-2 * g / (np.abs(g) + 1e-8)
    assert np.allclose(p1, expect.astype(np.float32), rtol=0, atol=1e-6)
    # a constant gradient keeps the step (m_hat = g, v_hat = g^2 exactly): lr
    # where |g| >> eps
    p2 = opt.step(p1, g)
    assert np.allclose(p2.astype(np.float64), p1.astype(np.float64) - 1e-2 * g / (np.abs(g) + 1e-8), atol=1e-6)


def test_a_network_that_outputs_the_normalised_target_gives_the_target():
    """Training compares the output with t = (x - mu) / sigma and inference maps
    the output back: a network whose output is t has zero loss, and its
    initial nominal is x. Zero weights with output bias t0 output t0 at every
    state (a constant target)."""
    rng = np.random.default_rng(9)
    mu, sigma = rng.standard_normal(5), 0.5 + rng.random(5)
    x_star = rng.standard_normal(5)
    layers = [(np.zeros(w), np.zeros(b)) for w, b in li.SHAPES]
    layers[-1] = (layers[-1][0], (x_star - mu) / sigma)
    params = li.pack(layers)
    T = 7
    y = rng.uniform(-3, 3, (2, T + 1))
    target = np.tile(x_star[:, None], (1, T + 1))
    loss, _ = li.loss_and_grad(params, [(y, target)], mu, sigma, rounding=False)
    assert loss < 1e-28
    np.testing.assert_allclose(li.initial_nominal(params, y, T, mu, sigma, rounding=False), target, atol=1e-14)


def test_training_reduces_loss_on_a_fixed_batch():
    params, trajs, mu, sigma = _tiny_problem(8)
    opt = li.Adam(lr=3e-3)
    first, _ = li.loss_and_grad(params, trajs, mu, sigma)
    for _ in range(30):
        _, g = li.loss_and_grad(params, trajs, mu, sigma)
        params = opt.step(params, g)
    last, _ = li.loss_and_grad(params, trajs, mu, sigma)
    assert last < 0.5 * first
