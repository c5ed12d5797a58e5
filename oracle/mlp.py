"""FP64 oracle of the correlation-function emulator: a 4-layer MLP
(5 -> 256 -> 256 -> 256 -> 1, SiLU) trained by Adam on a mean-squared error.

TEST INFRASTRUCTURE ONLY: imported by the test suite, never by the library.

The paper trains no network; the emulator maps cosmological parameters and a
separation to the central sphere's correlation function (the statistic the
simulations are run for, Sec. 1) so that a fit can query it instead of running
a simulation.  Readings fixed here:

* activation SiLU, z * sigmoid(z); linear output layer; loss mean((y - t)^2);
* Adam (Kingma & Ba 2015) with bias correction, beta1 0.9, beta2 0.999,
  eps 1e-8, no weight decay, learning rate given per step;
* BF16 training: every matrix-product operand is rounded to bfloat16 (round to
  nearest, ties to even) -- the inputs, the weights, each hidden activation
  after the SiLU and each back-propagated dZ -- while products are summed
  exactly (FP64 here), biases and their gradients stay unrounded, and the
  master weights and Adam moments are unrounded;
* ``rounding=False`` turns every rounding off: the plain FP64 network, whose
  gradient is pinned against central finite differences.

Parameter order (``PARAM_NAMES``): W1[256][5], b1[256], W2[256][256], b2,
W3[256][256], b3, W4[1][256], b4[1]; packed flat in that order.
"""
from __future__ import annotations

import numpy as np

WIDTHS = (5, 256, 256, 256, 1)
PARAM_NAMES = ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4")
BETA1, BETA2, EPS = 0.9, 0.999, 1e-8


def shapes(widths=WIDTHS):
    out = []
    for l in range(len(widths) - 1):
        out += [(widths[l + 1], widths[l]), (widths[l + 1],)]
    return out


def n_params(widths=WIDTHS) -> int:
    return int(sum(np.prod(s) for s in shapes(widths)))


def unpack(flat, widths=WIDTHS):
    flat = np.asarray(flat, dtype=np.float64)
    out, k = [], 0
    for s in shapes(widths):
        size = int(np.prod(s))
        out.append(flat[k:k + size].reshape(s))
        k += size
    assert k == flat.size
    return out


def pack(params) -> np.ndarray:
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in params])


def bf16(x) -> np.ndarray:
    """Round to the nearest bfloat16 (8 significant bits), ties to even, directly
    from FP64 (no intermediate FP32 rounding); finite normal range only."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)  # x = m * 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.round(m * 256.0) / 256.0, e)  # np.round: half to even


def sigmoid(z):
    return 0.5 * (1.0 + np.tanh(0.5 * z))


def silu(z):
    return z * sigmoid(z)


def silu_grad(z):
    s = sigmoid(z)
    return s * (1.0 + z * (1.0 - s))


def forward(params, x, rounding: bool = True):
    """Network output y[B] and the cache the backward pass needs."""
    r = bf16 if rounding else (lambda v: np.asarray(v, dtype=np.float64))
    nl = len(params) // 2
    a = r(x)
    acts, zs = [a], []
    for l in range(nl):
        W, b = params[2 * l], params[2 * l + 1]
        z = a @ r(W).T + b
        zs.append(z)
        if l < nl - 1:
            a = r(silu(z))
            acts.append(a)
    return zs[-1][:, 0], (acts, zs)


def loss(y, t) -> float:
    return float(np.mean((np.asarray(y) - np.asarray(t)) ** 2))


def backward(params, cache, y, t, rounding: bool = True):
    """Gradients of loss(y, t) with respect to every parameter (same order)."""
    r = bf16 if rounding else (lambda v: np.asarray(v, dtype=np.float64))
    acts, zs = cache
    nl = len(params) // 2
    B = y.shape[0]
    dz = (2.0 / B * (y - t))[:, None]  # dL/dz of the linear output layer
    grads = [None] * len(params)
    for l in range(nl - 1, -1, -1):
        dzr = r(dz)
        grads[2 * l] = dzr.T @ acts[l]  # dW = dZ^T A
        grads[2 * l + 1] = dz.sum(axis=0)  # db from the unrounded dZ
        if l > 0:
            da = dzr @ r(params[2 * l])
            dz = da * silu_grad(zs[l - 1])
    return grads


class Adam:
    """Adam with bias correction on FP64 master parameters."""

    def __init__(self, params):
        self.params = [np.array(p, dtype=np.float64) for p in params]
        self.m = [np.zeros_like(p) for p in self.params]
        self.v = [np.zeros_like(p) for p in self.params]
        self.t = 0

    def step(self, grads, lr: float):
        self.t += 1
        c1, c2 = 1.0 - BETA1 ** self.t, 1.0 - BETA2 ** self.t
        for p, m, v, g in zip(self.params, self.m, self.v, grads):
            m *= BETA1
            m += (1.0 - BETA1) * g
            v *= BETA2
            v += (1.0 - BETA2) * g * g
            p -= lr * (m / c1) / (np.sqrt(v / c2) + EPS)


def train(params, x, t, batches, lrs, rounding: bool = True):
    """Run len(batches) Adam steps; batches[s] are row indices into (x, t).
    Returns the final parameters, the per-step losses and the optimiser."""
    opt = Adam(params)
    losses = []
    for idx, lr in zip(batches, lrs):
        y, cache = forward(opt.params, x[idx], rounding)
        losses.append(loss(y, t[idx]))
        opt.step(backward(opt.params, cache, y, t[idx], rounding), lr)
    return opt.params, np.array(losses), opt


def init_params(seed: int, widths=WIDTHS):
    """Seeded uniform fan-in initial weights (He-uniform for SiLU layers), zero
    biases, as FP32-representable values; the same numbers feed both sides."""
    rng = np.random.default_rng(seed)
    out = []
    for fan_out, fan_in in zip(widths[1:], widths[:-1]):
        lim = np.sqrt(6.0 / fan_in)
        out.append(rng.uniform(-lim, lim, (fan_out, fan_in)).astype(np.float32).astype(np.float64))
        out.append(np.zeros(fan_out))
    return out
