"""Float64 oracle of the learned partitioner's model -- TEST INFRASTRUCTURE ONLY.

Only tests/, the smoke check and bench.py's CPU-baseline leg may import this.

The paper has no learned component; the model is defined by the workload it
serves: a small monotone two-layer network, trained on a sorted sample of the
keys to predict each key's empirical CDF, whose output routes keys to buckets.
This file states that model, its loss and the gradients that the GPU's
backward pass must reproduce, in float64.

Model (H = 32 hidden units, one input)::

    x      = (ord(key) - lo) / (hi - lo)         normalised key order
    d_j    = softplus(delta_j) > 0               knot spacing, j = 0..H-1
    x_j    = x0 + sum_{i<j} d_i                  knots x_0 < x_1 < ... < x_H
    h_j    = ramp((x - x_j) / d_j)               hidden layer; ramp(u) = min(max(u,0),1)
    w      = softmax(beta)                       output weights, w_j >= 0, sum 1
    y      = sum_j w_j h_j                       predicted CDF, in [0, 1]
    bucket = min(floor(y * B), B - 1)

The hidden layer is an affine map with input weight a_j = 1/d_j >= 0 and
bias c_j = -x_j/d_j followed by a monotone activation; the output layer has
non-negative weights, so y is non-decreasing in the key.  The first layer's
weights are tied through the knots so that the ramps tile the key axis: free
ramps, trained on a squared CDF error, open flat stretches between ramps, and
every key in a flat stretch lands in one bucket.

Loss over a sorted sample s_0 <= ... <= s_{m-1}: L = mean_i (y(x_i) - t_i)^2
with targets t_i = (i + 0.5) / m.

Parameters are a flat float64 vector theta = [x0, delta(H), beta(H)].
"""
from __future__ import annotations

import numpy as np

H = 32
NPARAM = 2 * H + 1


def softplus(v):
    v = np.asarray(v, dtype=np.float64)
    return np.where(v > 30.0, v, np.log1p(np.exp(np.minimum(v, 30.0))))


def softplus_inv(a):
    a = np.asarray(a, dtype=np.float64)
    return np.where(a > 30.0, a, np.log(np.expm1(np.maximum(a, 1e-300))))


def sigmoid(v):
    v = np.asarray(v, dtype=np.float64)
    return 0.5 * (1.0 + np.tanh(0.5 * v))


def unpack(theta):
    """theta -> (knots x_0..x_H, spacings d, output weights w)."""
    th = np.asarray(theta, dtype=np.float64)
    x0, delta, beta = th[0], th[1:H + 1], th[H + 1:2 * H + 1]
    d = softplus(delta)
    knots = x0 + np.concatenate([[0.0], np.cumsum(d)])
    e = np.exp(beta - beta.max())
    return knots, d, e / e.sum()


def ord_u32_f32(keys: np.ndarray) -> np.ndarray:
    """float32 -> uint32 whose unsigned order is IEEE-754 totalOrder:
    non-negative patterns get the top bit set; negative patterns are inverted."""
    b = np.ascontiguousarray(keys, dtype=np.float32).view(np.uint32)
    neg = (b >> np.uint32(31)) == 1
    return np.where(neg, ~b, b | np.uint32(0x80000000)).astype(np.uint32)


def normalise(ordv: np.ndarray, lo: float, hi: float) -> np.ndarray:
    span = hi - lo
    if span <= 0:
        return np.zeros(np.shape(ordv), dtype=np.float64)
    return (np.asarray(ordv).astype(np.float64) - lo) / span


def hidden(theta, x):
    """Pre-activations u (m x H) and activations h of the hidden layer."""
    knots, d, _ = unpack(theta)
    u = (np.asarray(x, dtype=np.float64)[:, None] - knots[None, :-1]) / d[None, :]
    return u, np.clip(u, 0.0, 1.0)


def forward(theta, x):
    _, h = hidden(theta, x)
    return h @ unpack(theta)[2]


def loss_and_grad(theta, x, t):
    """L = mean (y - t)^2 and dL/dtheta by the chain rule: the ramp has
    derivative 1 strictly inside (0, 1) and 0 elsewhere; a knot x_j moves with
    x0 and with every spacing d_i, i < j; softplus' = sigmoid; the softmax
    Jacobian is diag(w) - w w^T."""
    th = np.asarray(theta, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    knots, d, w = unpack(th)
    u = (x[:, None] - knots[None, :-1]) / d[None, :]
    h = np.clip(u, 0.0, 1.0)
    y = h @ w
    r = y - t
    L = float(np.mean(r * r))
    g = 2.0 * r / x.size                          # dL/dy_i
    inside = (u > 0.0) & (u < 1.0)
    d_w = h.T @ g                                 # dL/dw_j
    d_beta = w * (d_w - np.dot(w, d_w))
    gu = np.where(inside, g[:, None] * w[None, :], 0.0)   # dL/du_ij
    d_knot = -gu.sum(axis=0) / d                  # dL/dx_j through u_ij, j < H
    d_d = -(gu * u).sum(axis=0) / d               # dL/dd_j through the 1/d_j
    # x_j = x0 + sum_{i<j} d_i: d_i also moves every knot after it
    after = np.concatenate([np.cumsum(d_knot[::-1])[::-1][1:], [0.0]])
    d_d = d_d + after
    d_x0 = d_knot.sum()
    grad = np.concatenate([[d_x0], d_d * sigmoid(th[1:H + 1]), d_beta])
    return L, grad


def targets(m: int) -> np.ndarray:
    return (np.arange(m, dtype=np.float64) + 0.5) / m


def init_from_sample(xs_sorted: np.ndarray, min_gap: float = 1e-7) -> np.ndarray:
    """Quantile start: knots at the sample's 0, 1/H, ..., 1 quantiles (index
    round(j (m-1) / H)) and equal output weights, so y starts as the linear
    interpolation of the empirical CDF between H+1 quantile knots."""
    xs = np.asarray(xs_sorted, dtype=np.float64)
    m = xs.size
    pos = np.rint(np.arange(H + 1) * (m - 1) / H).astype(np.int64)
    kn = xs[pos]
    gaps = np.maximum(np.diff(kn), min_gap)
    return np.concatenate([[kn[0]], softplus_inv(gaps), np.zeros(H)])


def adam_steps(theta, grad_fn, steps: int, lr: float = 3e-3, b1: float = 0.9,
               b2: float = 0.999, eps: float = 1e-8):
    """Adam (Kingma and Ba, 2015, Algorithm 1) in float64: for t = 1..steps,
    g = grad_fn(theta, t); first and second moment estimates
    m = b1 m + (1 - b1) g and v = b2 v + (1 - b2) g^2, both started at 0;
    bias-corrected m^ = m / (1 - b1^t), v^ = v / (1 - b2^t); then
    theta -= lr m^ / (sqrt(v^) + eps), elementwise."""
    th = np.asarray(theta, dtype=np.float64).copy()
    mo = np.zeros_like(th)
    ve = np.zeros_like(th)
    for k in range(1, steps + 1):
        gr = np.asarray(grad_fn(th, k), dtype=np.float64)
        mo = b1 * mo + (1 - b1) * gr
        ve = b2 * ve + (1 - b2) * gr * gr
        mh = mo / (1 - b1 ** k)
        vh = ve / (1 - b2 ** k)
        th = th - lr * mh / (np.sqrt(vh) + eps)
    return th


def adam_train(theta, x, t, steps: int, lr: float = 3e-3, b1: float = 0.9,
               b2: float = 0.999, eps: float = 1e-8):
    """Full-batch Adam on the router's loss over the points (x, t)."""
    return adam_steps(theta, lambda th, k: loss_and_grad(th, x, t)[1], steps, lr, b1, b2, eps)


def buckets(theta, x, num_buckets: int) -> np.ndarray:
    y = forward(theta, x)
    return np.clip(np.floor(y * num_buckets), 0, num_buckets - 1).astype(np.int64)


def equal_width_buckets(x, num_buckets: int) -> np.ndarray:
    """The model-free partition used as the ablation: equal-width buckets over
    the normalised key range."""
    x = np.asarray(x, dtype=np.float64)
    return np.clip(np.floor(x * num_buckets), 0, num_buckets - 1).astype(np.int64)
