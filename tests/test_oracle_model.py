"""Pins the float64 model oracle: gradients against central finite
differences, monotonicity on a dense sweep, the interpolation property of the
quantile start, Adam's descent, and the gain over equal-width buckets."""
import numpy as np
import pytest

from oracle import model as M
import sortrace_inputs as si


def _random_theta(rng):
    return np.concatenate([[rng.normal(0.0, 0.1)], rng.normal(-3.5, 0.5, M.H),
                           rng.normal(0.0, 1.0, M.H)])


def test_gradient_finite_differences():
    rng = np.random.default_rng(0)
    x = rng.random(400)
    t = np.sort(rng.random(400))
    for _ in range(3):
        th = _random_theta(rng)
        _, g = M.loss_and_grad(th, x, t)
        num = np.zeros_like(th)
        eps = 1e-6
        for k in range(th.size):
            e = np.zeros_like(th)
            e[k] = eps
            num[k] = (M.loss_and_grad(th + e, x, t)[0] - M.loss_and_grad(th - e, x, t)[0]) / (2 * eps)
        # kinks of the ramp are met with probability ~0 at these points
        assert np.allclose(g, num, rtol=1e-4, atol=1e-7), np.max(np.abs(g - num))


def test_uniform_knots_is_identity_cdf():
    """Equal spacings 1/H from 0 and equal weights give y(x) = clip(x, 0, 1)
    (the CDF of the uniform distribution); on data whose targets equal their
    inputs the loss and the gradient vanish."""
    th = np.concatenate([[0.0], M.softplus_inv(np.full(M.H, 1.0 / M.H)), np.zeros(M.H)])
    xs = np.linspace(-0.5, 1.5, 2001)
    assert np.allclose(M.forward(th, xs), np.clip(xs, 0, 1), atol=1e-12)
    t = M.targets(1000)
    L, g = M.loss_and_grad(th, t, t)
    assert L < 1e-24 and np.max(np.abs(g)) < 1e-12
    # a pure shift of the data: y = x - 0.01 inside, so L = 1e-4 and dL/dx0 = -2e-2 * (-1)
    L2, g2 = M.loss_and_grad(th, t, t - 0.01)
    assert np.isclose(L2, 1e-4)


def test_monotone_dense_sweep():
    rng = np.random.default_rng(1)
    xs = np.linspace(-0.2, 1.2, 200001)
    for _ in range(5):
        y = M.forward(_random_theta(rng), xs)
        assert np.all(np.diff(y) >= 0)


def test_quantile_start_interpolates_cdf():
    """At the quantile knots the starting model equals j/H exactly (up to
    rounding), i.e. it is the piecewise-linear empirical CDF."""
    rng = np.random.default_rng(5)
    xs = np.sort(rng.random(10000))
    th = M.init_from_sample(xs)
    pos = np.rint(np.arange(M.H + 1) * (xs.size - 1) / M.H).astype(np.int64)
    y = M.forward(th, xs[pos])
    assert np.allclose(y, np.arange(M.H + 1) / M.H, atol=1e-9)


def _lognormal_setup(m=40000, seed=3):
    keys = si.lognormal_f32(m * 100, seed)
    o = M.ord_u32_f32(keys).astype(np.float64)
    sample = np.sort(o[::100])
    lo, hi = sample[0], sample[-1]
    xs = M.normalise(sample, lo, hi)
    return keys, o, lo, hi, xs


def test_adam_lowers_loss_keeps_balance():
    _, o, lo, hi, xs = _lognormal_setup()
    t = M.targets(xs.size)
    th0 = M.init_from_sample(xs)
    L0, _ = M.loss_and_grad(th0, xs, t)
    th = M.adam_train(th0, xs, t, steps=100, lr=3e-3)
    L1, _ = M.loss_and_grad(th, xs, t)
    assert L1 < 0.8 * L0
    x_all = M.normalise(o, lo, hi)
    B = 1 << 16
    m0 = _second_moment(M.buckets(th0, x_all, B), B)
    m1 = _second_moment(M.buckets(th, x_all, B), B)
    assert m1 <= m0 * 1.01


def _second_moment(b, B):
    """sum c_k^2 / (mean^2 B) over the inner buckets: 1 for perfect balance."""
    c = np.bincount(b, minlength=B)[1:-1].astype(np.float64)
    mean = c.sum() / c.size
    return float((c * c).sum() / (mean * mean * c.size))


def test_model_beats_equal_width_buckets():
    """What the trained model gains: on the lognormal mixture at 2^16 buckets
    its bucket sizes are far closer to equal than those of equal-width buckets
    over the key range (the end buckets, which collect the keys beyond the
    sample's extremes, are left out)."""
    _, o, lo, hi, xs = _lognormal_setup()
    B = 1 << 16
    th = M.adam_train(M.init_from_sample(xs), xs, M.targets(xs.size), steps=100, lr=3e-3)
    x_all = M.normalise(o, lo, hi)
    sm = _second_moment(M.buckets(th, x_all, B), B)
    se = _second_moment(M.equal_width_buckets(x_all, B), B)
    assert sm < 1.2 and se > 1.5 * sm, (sm, se)


def test_ord_f32_total_order():
    v = np.array([-np.inf, -2.0, -0.0, 0.0, 1e-45, 3.0, np.inf], dtype=np.float32)
    o = M.ord_u32_f32(v)
    assert np.all(np.diff(o.astype(np.int64)) > 0)


def test_adam_hand_worked_steps():
    """Adam's update (Kingma and Ba, 2015, Algorithm 1) on a worked example
    computed by hand: step size 1, b1 = 0.5, b2 = 0.96, eps = 0, and a fixed
    gradient sequence g = 2, -2, 4 for the first parameter (its mirror for
    the second).
      t=1: m = 1, v = 0.16; m^ = 1/0.5 = 2, v^ = 0.16/0.04 = 4: a step of 1
           (a first bias-corrected step always has the step size's length).
      t=2: m = -0.5, v = 0.3136; m^ = -0.5/0.75 = -2/3, v^ = 0.3136/0.0784 = 4:
           a step of -1/3.
      t=3: m = 1.75, v = 0.941056; m^ = 1.75/0.875 = 2,
           v^ = 0.941056/0.115264 = 14704/1801: a step of 2 sqrt(1801/14704).
    Without the bias correction the first step would be 2.5; with b1 and b2
    swapped the second would be -1/7; eps is checked on its own below."""
    seq = [np.array([2.0, -2.0]), np.array([-2.0, 2.0]), np.array([4.0, -4.0])]
    th0 = np.array([3.0, -1.0])
    run = lambda k: M.adam_steps(th0, lambda th, t: seq[t - 1], k, lr=1.0, b1=0.5, b2=0.96, eps=0.0)
    s3 = 2.0 * np.sqrt(1801.0 / 14704.0)
    for k, want0 in ((1, 3.0 - 1.0), (2, 3.0 - 1.0 + 1.0 / 3.0), (3, 3.0 - 1.0 + 1.0 / 3.0 - s3)):
        got = run(k)
        assert abs(got[0] - want0) < 1e-12, (k, got)
        assert abs(got[1] - (-1.0 - (want0 - 3.0))) < 1e-12, (k, got)
    # eps outside the square root: m^ = 2, v^ = 4, eps = 1 gives a step of
    # 2 / (2 + 1) = 2/3 (inside the root it would be 2 / sqrt(5))
    got = M.adam_steps(np.array([0.0]), lambda th, t: np.array([2.0]), 1, lr=1.0, b1=0.5, b2=0.96, eps=1.0)
    assert abs(got[0] + 2.0 / 3.0) < 1e-12, got
    # adam_train is adam_steps on the router's own gradient
    rng = np.random.default_rng(5)
    xs = np.sort(rng.random(300))
    t = M.targets(xs.size)
    th = M.init_from_sample(xs)
    a = M.adam_train(th, xs, t, steps=3, lr=1e-2)
    b = M.adam_steps(th, lambda p, k: M.loss_and_grad(p, xs, t)[1], 3, lr=1e-2)
    assert np.array_equal(a, b)
