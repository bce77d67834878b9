"""The learned partitioner on the GPU: the router network's device forward and
backward against the float64 oracle, device Adam against the oracle's Adam,
routing monotonicity and agreement with the oracle's buckets, and the learned
sort bit for bit against the oracle (plus the forced fallback, the model-free
ablation and the full-size lognormal workload)."""
import numpy as np
import pytest

import oracle
from oracle import model as M
import sortrace_inputs as si

pytestmark = pytest.mark.gpu

KT = {np.dtype(np.int32): 0, np.dtype(np.uint32): 1, np.dtype(np.float32): 2,
      np.dtype(np.uint64): 3, np.dtype(np.int64): 4}


def _dev(a):
    import torch
    bits = {4: np.int32, 8: np.int64}[a.dtype.itemsize]
    return torch.from_numpy(np.ascontiguousarray(a).view(bits).copy()).cuda()


def _f32dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _learned(sr, a, **opts):
    t = _dev(a)
    sr.sort_keys_learned(t, key_type=KT[a.dtype], **opts)
    return t.cpu().numpy().view(a.dtype), sr.stats()


def _theta(rng):
    return np.concatenate([[rng.normal(0.0, 0.05)], rng.normal(-3.5, 0.4, M.H), rng.normal(0.0, 1.0, M.H)])


def test_device_gradient_matches_oracle(gpu_lib):
    """Forward + backward on the device (float32) against the float64 oracle
    at the same float32-rounded points and parameters."""
    rng = np.random.default_rng(41)
    for trial in range(4):
        x = np.sort(rng.random(3000)).astype(np.float32)
        t = np.sort(rng.random(3000)).astype(np.float32)
        th = _theta(rng).astype(np.float32)
        loss, g = gpu_lib.model_loss_grad(_f32dev(x), _f32dev(t), th)
        L, G = M.loss_and_grad(th.astype(np.float64), x.astype(np.float64), t.astype(np.float64))
        assert abs(loss - L) <= 1e-4 * L + 1e-9, (loss, L)
        G = np.asarray(G)
        g = np.asarray(g)
        scale = np.max(np.abs(G))
        assert np.max(np.abs(g - G)) <= 2e-3 * scale, np.max(np.abs(g - G)) / scale


def test_device_adam_matches_oracle(gpu_lib):
    keys = si.lognormal_f32(200_000, 5)
    o = M.ord_u32_f32(keys).astype(np.float64)
    xs = np.sort(M.normalise(o, o.min(), o.max()))[::50].astype(np.float32)
    ts = ((np.arange(xs.size) + 0.5) / xs.size).astype(np.float32)
    th0 = M.init_from_sample(xs.astype(np.float64)).astype(np.float32)
    L0, _ = M.loss_and_grad(th0.astype(np.float64), xs.astype(np.float64), ts.astype(np.float64))
    th_gpu, loss_gpu = gpu_lib.model_train(_f32dev(xs), _f32dev(ts), th0, steps=30, lr=3e-3)
    th_ref = M.adam_train(th0.astype(np.float64), xs.astype(np.float64), ts.astype(np.float64), steps=30, lr=3e-3)
    L_ref, _ = M.loss_and_grad(th_ref, xs.astype(np.float64), ts.astype(np.float64))
    assert loss_gpu < L0 and L_ref < L0
    assert abs(loss_gpu - L_ref) <= 0.05 * L_ref, (loss_gpu, L_ref)
    assert np.max(np.abs(np.asarray(th_gpu) - th_ref)) < 0.05


def test_device_adam_first_step_exact(gpu_lib):
    """One device Adam step against the oracle's: a bias-corrected first step
    moves every parameter by lr * g / (|g| + eps), i.e. by the step size in
    the direction against its gradient.  Parameters whose float64 gradient
    is at least 1% of the largest (the device gradient is within 0.2% of the
    largest, test above, so its sign is certain there) must land within 1e-6
    of the oracle's (plus float32 rounding of the parameter); the rest move
    by at most the step size."""
    keys = si.lognormal_f32(200_000, 5)
    o = M.ord_u32_f32(keys).astype(np.float64)
    xs = np.sort(M.normalise(o, o.min(), o.max()))[::50].astype(np.float32)
    ts = ((np.arange(xs.size) + 0.5) / xs.size).astype(np.float32)
    th0 = M.init_from_sample(xs.astype(np.float64)).astype(np.float32)
    lr = 3e-3
    th_gpu, _ = gpu_lib.model_train(_f32dev(xs), _f32dev(ts), th0, steps=1, lr=lr)
    x64, t64, th64 = xs.astype(np.float64), ts.astype(np.float64), th0.astype(np.float64)
    th_ref = M.adam_train(th64, x64, t64, steps=1, lr=lr)
    _, g = M.loss_and_grad(th64, x64, t64)
    d = np.abs(np.asarray(th_gpu, dtype=np.float64) - th_ref)
    clear = np.abs(g) > 1e-2 * np.max(np.abs(g))
    assert clear.sum() >= 5, clear.sum()
    tol = 1e-6 + 4e-7 * np.abs(th64)           # float32 rounding of the updated value
    assert np.all(d[clear] < tol[clear]), np.max(d[clear] / tol[clear])
    assert np.max(np.abs(np.asarray(th_gpu, dtype=np.float64) - th64)) <= lr * (1 + 1e-5)


def test_routing_monotone_and_matches_oracle(gpu_lib):
    import torch
    rng = np.random.default_rng(42)
    keys = np.sort(si.lognormal_f32(400_000, 6))
    o = M.ord_u32_f32(keys).astype(np.float64)
    lo, hi = int(o[0]), int(o[-1])
    th = M.init_from_sample(M.normalise(o[::40], lo, hi)).astype(np.float32)
    B = 1 << 16
    out = torch.empty(keys.size, dtype=torch.int32, device="cuda")
    gpu_lib.model_buckets(_dev(keys), th, lo, hi, B, out, key_type=2)
    b = out.cpu().numpy().astype(np.int64)
    assert np.all(np.diff(b) >= 0)                 # sorted keys -> non-decreasing buckets
    ref = M.buckets(th.astype(np.float64), M.normalise(o, lo, hi), B)
    # bucket ids are not pinned bit for bit: the device routes in float32 and a
    # bucket is ~1.5e-5 wide in y at 2^16 buckets, while float32 rounding of
    # x moves y by ~1e-7, so keys this dense land across an edge ~0.3% of
    # the time; never by more than one bucket
    assert np.max(np.abs(b - ref)) <= 1
    assert np.mean(b == ref) > 0.99


@pytest.mark.parametrize("n", [0, 1, 2, 99, 100, 101, 5000, 1 << 20, (1 << 22) + 3])
def test_learned_lognormal_exact(gpu_lib, n):
    a = si.lognormal_f32(n, 7)
    got, st = _learned(gpu_lib, a)
    assert got.view(np.uint32).tobytes() == oracle.sort_keys(a).view(np.uint32).tobytes()
    if n > 1:
        assert st["fallback"] == 0


@pytest.mark.parametrize("kind", list(si.INT32_CLASSES))
def test_learned_int_classes_exact(gpu_lib, kind):
    a = si.int32_input(kind, (1 << 20) + 11, seed=8)
    got, st = _learned(gpu_lib, a)
    assert got.tobytes() == oracle.sort_keys(a).tobytes()
    assert st["fallback"] == 0


def test_learned_other_types_and_degenerate(gpu_lib):
    rng = np.random.default_rng(43)
    cases = [rng.integers(0, 1 << 64, 300_001, dtype=np.uint64),
             rng.integers(-(1 << 62), 1 << 62, 300_001).astype(np.int64),
             rng.integers(0, 1 << 32, 300_001, dtype=np.uint64).astype(np.uint32),
             np.full(123_457, 3.25, np.float32),                     # all equal: one bucket
             np.concatenate([np.full(100_000, -1.0, np.float32), np.full(100_000, 2.0, np.float32)]),
             np.sort(si.lognormal_f32(200_000, 9)),
             np.sort(si.lognormal_f32(200_000, 9))[::-1].copy()]
    for a in cases:
        got, st = _learned(gpu_lib, a)
        assert got.tobytes() == oracle.sort_keys(a).tobytes(), a.dtype
        assert st["fallback"] == 0


def test_forced_bad_router_falls_back_exactly(gpu_lib):
    a = si.lognormal_f32(1 << 20, 10)
    got, st = _learned(gpu_lib, a, model=gpu_lib.MODEL_FORCE_BAD)
    assert st["fallback"] == 1
    assert got.view(np.uint32).tobytes() == oracle.sort_keys(a).view(np.uint32).tobytes()


@pytest.mark.parametrize("model", ["trained", "force_bad"])
def test_learned_in_captured_graph(gpu_lib, model):
    """sr_sort_keys_learned captured whole in the caller's CUDA graph (no host
    read: the plain sort sits behind an IF node that the bucket check sets on
    the device) and replayed on new inputs: every output equals the oracle's;
    with the forced non-monotone router every replay takes the fallback."""
    import torch
    m = gpu_lib.MODEL_TRAINED if model == "trained" else gpu_lib.MODEL_FORCE_BAD
    arrays = [si.lognormal_f32(300_007, seed) for seed in (21, 22, 23)]
    x = _dev(arrays[0])
    gpu_lib.sort_keys_learned(x.clone(), key_type=2, model=m)   # device state exists before the capture
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        gpu_lib.sort_keys_learned(x, key_type=2, model=m, stream=s)
    for a in arrays:
        x.copy_(_dev(a))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert x.cpu().numpy().view(np.uint32).tobytes() == oracle.sort_keys(a).view(np.uint32).tobytes()
        assert gpu_lib.stats()["fallback"] == (1 if model == "force_bad" else 0)


def test_trained_model_gains_over_ablations(gpu_lib):
    """What the trained network gains: on the lognormal mixture its bucket
    sizes are much closer to even than equal-width buckets' (the second moment
    B * sum c^2 / n^2; the largest bucket is about the same for both, set by
    the densest stretch of keys), and training lowers the loss of the quantile
    start; all three give the exact output."""
    a = si.lognormal_f32(1 << 22, 11)
    want = oracle.sort_keys(a).view(np.uint32).tobytes()
    res = {}
    for name, model in (("trained", gpu_lib.MODEL_TRAINED), ("untrained", gpu_lib.MODEL_UNTRAINED),
                        ("equal_width", gpu_lib.MODEL_EQUAL_WIDTH)):
        got, st = _learned(gpu_lib, a, model=model)
        assert got.view(np.uint32).tobytes() == want
        res[name] = st
    assert res["equal_width"]["bucket_imbalance"] > 1.4 * res["trained"]["bucket_imbalance"]
    assert res["trained"]["bucket_imbalance"] < 1.3
    assert res["trained"]["model_loss"] < res["untrained"]["model_loss"]


def test_learned_full_size_matches_plain(gpu_lib, full_size_oracle):
    """2^27 float32 keys of the lognormal mixture: the learned sort's output
    equals the oracle's byte for byte, and the plain GPU sort's too."""
    import torch
    a = si.lognormal_f32(1 << 27, 1)
    x = _dev(a)
    y = x.clone()
    gpu_lib.sort_keys_learned(x, key_type=2)
    st = gpu_lib.stats()
    assert st["fallback"] == 0
    gpu_lib.sort_keys(y, key_type=2)
    assert torch.equal(x, y)
    got = x.cpu().numpy().view(np.float32)
    full_size_oracle("lognormal_f32_2p27_seed1", [a], [got], lambda: [oracle.sort_keys(a)])


def test_every_bucket_config_exact(gpu_lib):
    """The buckets can be sorted under any segmented-sort configuration; the
    output is the same."""
    a = si.lognormal_f32((1 << 21) + 5, 14)
    want = oracle.sort_keys(a).view(np.uint32).tobytes()
    for cfg in gpu_lib.segmented_configs(2):
        got, st = _learned(gpu_lib, a, bucket_config=cfg["index"] + 1)
        assert got.view(np.uint32).tobytes() == want, cfg
        assert st["fallback"] == 0
