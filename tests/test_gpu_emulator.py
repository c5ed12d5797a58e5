"""GPU emulator kernels (bf16 tensor-core products, FP32 accumulation, fused
SiLU/bias epilogues, Adam) against the FP64 oracle network that rounds the
same operands to bfloat16.  Remaining differences come from FP32 sums
(relative 1e-7 per sum) flipping a bfloat16 rounding now and then (one
bfloat16 ulp, 2^-8); the tolerances below are about ten times what an FP32
emulation of the same arithmetic shows."""
import numpy as np
import pytest

from oracle import mlp
from paper_1811_05903_gb300 import steps

pytestmark = pytest.mark.gpu


def make_params(seed):
    rng = np.random.default_rng(seed)
    params = mlp.init_params(seed)
    for p in params[1::2]:
        p[:] = rng.uniform(-0.1, 0.1, p.shape).astype(np.float32)
    return params


def emu(params, batch):
    steps.load(build_if_missing=True)
    return steps.Emulator(mlp.pack(params).astype(np.float32), batch=batch)


@pytest.mark.parametrize("n", [1000, 37, 256])
def test_forward_matches_oracle(n):
    params = make_params(11)
    e = emu(params, 256)
    x = np.random.default_rng(n).uniform(-1, 1, (n, 5)).astype(np.float32)
    y = e.predict(x).astype(np.float64)
    ref, _ = mlp.forward(params, x.astype(np.float64))
    scale = np.abs(ref).max()
    assert np.abs(y - ref).max() <= 5e-3 * scale
    assert np.sqrt(np.mean((y - ref) ** 2)) <= 5e-4 * np.sqrt(np.mean(ref ** 2))
    e.close()


def test_predict_empty_is_noop():
    e = emu(make_params(12), 64)
    assert e.predict(np.zeros((0, 5), np.float32)).shape == (0,)
    e.close()


def test_gradients_match_oracle():
    params = make_params(13)
    B = 1024
    e = emu(params, B)
    rng = np.random.default_rng(14)
    x = rng.uniform(-1, 1, (B, 5)).astype(np.float32)
    t = rng.normal(size=B).astype(np.float32)
    g, loss = e.gradients(x, t)
    y, cache = mlp.forward(params, x.astype(np.float64))
    ref = mlp.backward(params, cache, y, t.astype(np.float64))
    assert abs(loss - mlp.loss(y, t)) <= 1e-4 * mlp.loss(y, t)
    for name, a, b in zip(mlp.PARAM_NAMES, mlp.unpack(g), ref):
        nrel = np.linalg.norm(a - b) / np.linalg.norm(b)
        mrel = np.abs(a - b).max() / np.abs(b).max()
        assert nrel <= 1e-3 and mrel <= 2e-3, (name, nrel, mrel)
    e.close()


def test_one_adam_step_matches_oracle():
    params = make_params(15)
    B, lr = 512, 1e-3
    e = emu(params, B)
    rng = np.random.default_rng(16)
    x = rng.uniform(-1, 1, (B, 5)).astype(np.float32)
    t = rng.normal(size=B).astype(np.float32)
    e.set_data(x, t)
    losses = e.train(np.arange(B, dtype=np.int32)[None], [lr])
    p1, m1, v1, nsteps = e.params()
    assert nsteps == 1
    y, cache = mlp.forward(params, x.astype(np.float64))
    grads = mlp.backward(params, cache, y, t.astype(np.float64))
    assert abs(losses[0] - mlp.loss(y, t)) <= 1e-4 * mlp.loss(y, t)
    opt = mlp.Adam(params)
    opt.step(grads, lr)
    for name, a1, am, av, p0, b1, bm, bv, g in zip(mlp.PARAM_NAMES, mlp.unpack(p1), mlp.unpack(m1),
                                                    mlp.unpack(v1), params, opt.params, opt.m, opt.v, grads):
        big = np.abs(g) >= 1e-2 * np.abs(g).max()  # sign of g certain: the step is -lr sign(g)
        assert np.abs((a1 - p0)[big] - (b1 - p0)[big]).max() <= 1e-3 * lr, name
        assert np.abs(a1 - b1).max() <= 2.01 * lr, name  # never more than a flipped sign apart
        assert np.linalg.norm(am - bm) <= 1e-3 * np.linalg.norm(bm), name
        assert np.linalg.norm(av - bv) <= 2e-3 * np.linalg.norm(bv), name
    e.close()


def test_training_run_tracks_oracle_and_is_deterministic():
    params = make_params(17)
    B, nsteps = 256, 30
    rng = np.random.default_rng(18)
    n = 2048
    x = rng.uniform(-1, 1, (n, 5)).astype(np.float32)
    t = (np.sin(2 * x[:, 0]) * x[:, 4] + 0.3 * x[:, 1] ** 2).astype(np.float32)
    rows = np.stack([rng.choice(n, B, replace=False) for _ in range(nsteps)]).astype(np.int32)
    lr = (1e-3 * 0.5 * (1 + np.cos(np.pi * np.arange(nsteps) / nsteps))).astype(np.float32)
    runs = []
    for _ in range(2):
        e = emu(params, B)
        e.set_data(x, t)
        l1 = e.train(rows[:10], lr[:10])  # two calls: the step table restarts, Adam's t continues
        l2 = e.train(rows[10:], lr[10:])
        runs.append((np.concatenate([l1, l2]), e.params()[0]))
        e.close()
    np.testing.assert_array_equal(runs[0][0], runs[1][0])
    np.testing.assert_array_equal(runs[0][1], runs[1][1])
    ref_params, ref_losses, _ = mlp.train(params, x.astype(np.float64), t.astype(np.float64), rows,
                                          lr.astype(np.float64))
    gl = runs[0][0].astype(np.float64)
    assert np.all(np.abs(gl - ref_losses) <= 1e-2 * ref_losses), np.abs(gl / ref_losses - 1).max()
    p = runs[0][1].astype(np.float64)
    ref = mlp.pack(ref_params)
    init = mlp.pack(params)
    assert np.linalg.norm(p - ref) <= 2e-2 * np.linalg.norm(ref - init)


def test_training_fits_a_smooth_function():
    params = make_params(19)
    B, nsteps, n = 256, 400, 4096
    rng = np.random.default_rng(20)
    x = rng.uniform(-1, 1, (n, 5)).astype(np.float32)
    t = (np.sin(2 * x[:, 0]) * x[:, 4] + 0.3 * x[:, 1] ** 2).astype(np.float32)
    e = emu(params, B)
    e.set_data(x, t)
    rows = rng.integers(0, n, (nsteps, B)).astype(np.int32)
    losses = e.train(rows, np.full(nsteps, 1e-3, np.float32))
    assert losses[-20:].mean() < 0.05 * losses[:5].mean()
    e.close()


def test_emulator_rejects_bad_arguments():
    steps.load(build_if_missing=True)
    p = mlp.pack(make_params(21)).astype(np.float32)
    with pytest.raises(steps.StepsError):
        steps.Emulator(p, batch=100)
    bad = p.copy()
    bad[7] = np.nan
    with pytest.raises(steps.StepsError):
        steps.Emulator(bad, batch=64)
    e = steps.Emulator(p, batch=64)
    with pytest.raises(steps.StepsError):  # no training set yet
        e.train(np.zeros((1, 64), np.int32), [1e-3])
    x = np.zeros((10, 5), np.float32)
    with pytest.raises(steps.StepsError):
        e.set_data(x, np.array([np.inf] + [0.0] * 9, np.float32))
    e.set_data(x, np.zeros(10, np.float32))
    with pytest.raises(steps.StepsError):  # row 10 is outside the set
        e.train(np.full((1, 64), 10, np.int32), [1e-3])
    e.close()
