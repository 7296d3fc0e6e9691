"""Plain NumPy oracle of the learned initialiser (the network that maps the
measurements of a trajectory to an initial nominal trajectory for the
iterated smoother of Sec. 3, so that fewer iterations are needed).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU baseline are its only users; the product never imports it.
It shares no code with the CUDA path.

The paper has no such network; it replaces the iteration's starting point,
which the paper leaves open (the plain choice, every state at the prior mean,
stays the fallback). What is computed, for one trajectory with measurements
y_1..y_T (two bearings each) and states k = 0..T:

* features phi_k (64 channels): (sin y_k^1, cos y_k^1, sin y_k^2, cos y_k^2,
  1, 0) for k >= 1 and (0, 0, 0, 0, 0, 1) at k = 0; the other 58 channels 0;
* four convolution layers, l = 1..4, kernel 5, 64 -> 64 channels, "same"
  zero padding at both ends of the trajectory:
  h_l[k, o] = relu(b_l[o] + sum_{j<5} sum_i W_l[o, i, j] h_{l-1}[k + j - 2, i]);
* a per-state MLP head: z_k = relu(W5 h_4[k] + b5) (64 -> 64),
  o_k = W6 z_k + b6 (64 -> 5);
* the initial nominal x_k = mu + sigma * o_k (per-component normalisation of
  the training targets).

Arithmetic: weights, features and the hidden activations h_l and z are
rounded to bfloat16 (round to nearest even) at the points the CUDA path
stores them, every sum is exact here (float64) where the device accumulates
in float32, and the head output o stays unrounded. ``rounding=False`` skips
every bfloat16 rounding, which makes the forward pass smooth for finite
difference checks of the backward pass.

Training: loss = mean over states and the five components of (o - t)^2 with
t = (x* - mu) / sigma; the gradients follow from the chain rule through the
layers above (backward operands rounded to bfloat16 where the device stores
them); parameters are updated by Adam (Kingma and Ba, 2015) with FP32 master
weights.

Parameter packing (float32, this order): for l = 1..4, W_l [64][64][5]
(output channel, input channel, tap) and b_l [64]; W5 [64][64], b5 [64];
W6 [5][64], b6 [5].
"""
from __future__ import annotations

import numpy as np

C = 64          # channels of every hidden layer and of the features
TAPS = 5        # convolution kernel width
NCONV = 4       # convolution layers
NOUT = 5        # state dimension
SHAPES = ([((C, C, TAPS), (C,))] * NCONV) + [((C, C), (C,)), ((NOUT, C), (NOUT,))]
NPARAMS = sum(int(np.prod(w)) + int(np.prod(b)) for w, b in SHAPES)


def bf16(x):
    """Round to bfloat16 (nearest, ties to even) and return float64: the value
    first takes float32, the type the device rounds from."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _r(x, rounding):
    return bf16(x) if rounding else np.asarray(x, dtype=np.float64)


def unpack(params):
    """Flat float32 parameter vector -> list of (W, b) per layer."""
    p = np.asarray(params, dtype=np.float64)
    out, i = [], 0
    for ws, bs in SHAPES:
        nw, nb = int(np.prod(ws)), int(np.prod(bs))
        out.append((p[i:i + nw].reshape(ws), p[i + nw:i + nw + nb].reshape(bs)))
        i += nw + nb
    assert i == NPARAMS
    return out


def pack(layers) -> np.ndarray:
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in layers]).astype(np.float64)


def init_params(seed: int) -> np.ndarray:
    """He-normal weights, zero biases, as float32 (a starting point only)."""
    rng = np.random.default_rng(seed)
    layers = []
    for ws, bs in SHAPES:
        fan_in = int(np.prod(ws[1:]))
        layers.append((rng.standard_normal(ws) * np.sqrt(2.0 / fan_in), np.zeros(bs)))
    return pack(layers).astype(np.float32)


def features(y, T: int) -> np.ndarray:
    """phi [T+1][64] for one trajectory; y is [2][T+1] (column 0 unused)."""
    phi = np.zeros((T + 1, C))
    yy = np.asarray(y, dtype=np.float64)
    phi[1:, 0] = np.sin(yy[0, 1:])
    phi[1:, 1] = np.cos(yy[0, 1:])
    phi[1:, 2] = np.sin(yy[1, 1:])
    phi[1:, 3] = np.cos(yy[1, 1:])
    phi[1:, 4] = 1.0
    phi[0, 5] = 1.0
    return phi


def shift(h, d: int):
    """s[k] = h[k + d] with zeros outside the trajectory."""
    s = np.zeros_like(h)
    n = h.shape[0]
    if d >= 0:
        s[:n - d] = h[d:]
    else:
        s[-d:] = h[:n + d]
    return s


def conv(h, W, b):
    """out[k, o] = b[o] + sum_j sum_i W[o, i, j] h[k + j - 2, i] (pre-activation)."""
    out = np.tile(b, (h.shape[0], 1)).astype(np.float64)
    for j in range(W.shape[2]):
        out += shift(h, j - TAPS // 2) @ W[:, :, j].T
    return out


def forward(params, y, T: int, rounding: bool = True) -> dict:
    """Every stored quantity of the forward pass of one trajectory."""
    layers = [(_r(W, rounding), np.asarray(b, dtype=np.float64)) for W, b in unpack(params)]
    h = [_r(features(y, T), rounding)]
    for l in range(NCONV):
        W, b = layers[l]
        h.append(_r(np.maximum(conv(h[-1], W, b), 0.0), rounding))
    W5, b5 = layers[NCONV]
    z = _r(np.maximum(h[-1] @ W5.T + b5, 0.0), rounding)
    W6, b6 = layers[NCONV + 1]
    o = z @ W6.T + b6
    if rounding:
        o = o.astype(np.float32).astype(np.float64)
    return dict(h=h, z=z, o=o, layers=layers)


def initial_nominal(params, y, T: int, mu, sigma, rounding: bool = True) -> np.ndarray:
    """x [5][T+1] = mu + sigma * o."""
    o = forward(params, y, T, rounding)["o"]
    return (np.asarray(mu)[None, :] + np.asarray(sigma)[None, :] * o).T.copy()


def loss_and_grad(params, trajs, mu, sigma, rounding: bool = True):
    """Loss over a minibatch and its gradient (flat, float64).

    ``trajs`` is a list of (y [2][T+1], x_target [5][T+1]); the loss is the
    mean of (o - t)^2 over all states of all trajectories and the 5 components.
    """
    n_total = sum(int(np.asarray(x).shape[1]) for _, x in trajs)
    grads = [(np.zeros(ws), np.zeros(bs)) for ws, bs in SHAPES]
    loss = 0.0
    mu = np.asarray(mu, dtype=np.float64)
    sigma = np.asarray(sigma, dtype=np.float64)
    for y, xt in trajs:
        xt = np.asarray(xt, dtype=np.float64)
        T = xt.shape[1] - 1
        f = forward(params, y, T, rounding)
        t = (xt.T - mu) / sigma
        e = f["o"] - t
        loss += float(np.sum(e * e))
        dO = _r(2.0 * e / (NOUT * n_total), rounding)           # stored in bf16 for the device GEMMs
        W6, _ = f["layers"][NCONV + 1]
        W5, _ = f["layers"][NCONV]
        z, h = f["z"], f["h"]
        grads[NCONV + 1][0][...] += dO.T @ z
        grads[NCONV + 1][1][...] += dO.sum(axis=0)
        dz = _r((dO @ W6) * (z > 0), rounding)
        grads[NCONV][0][...] += dz.T @ h[NCONV]
        grads[NCONV][1][...] += dz.sum(axis=0)
        dh = _r((dz @ W5) * (h[NCONV] > 0), rounding)
        for l in range(NCONV - 1, -1, -1):      # dh: gradient at the pre-activation of conv layer l+1
            W, _ = f["layers"][l]
            gW, gb = grads[l]
            for j in range(TAPS):
                gW[:, :, j] += dh.T @ shift(h[l], j - TAPS // 2)
            gb += dh.sum(axis=0)
            if l > 0:
                # d h_l[k, i] = sum_j sum_o W[o, i, j] dh[k - j + 2, o]
                back = np.zeros_like(h[l])
                for j in range(TAPS):
                    back += shift(dh, TAPS // 2 - j) @ W[:, :, j]
                dh = _r(back * (h[l] > 0), rounding)
    return loss / (NOUT * n_total), pack(grads)


class Adam:
    """Adam with bias correction; master weights and moments in float32."""

    def __init__(self, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps
        self.m = None
        self.v = None
        self.t = 0

    def step(self, params, grad) -> np.ndarray:
        p = np.asarray(params, dtype=np.float64)
        g = np.asarray(grad, dtype=np.float64)
        if self.m is None:
            self.m = np.zeros_like(p)
            self.v = np.zeros_like(p)
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mhat = self.m / (1 - self.b1 ** self.t)
        vhat = self.v / (1 - self.b2 ** self.t)
        return (p - self.lr * mhat / (np.sqrt(vhat) + self.eps)).astype(np.float32)
