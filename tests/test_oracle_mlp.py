"""Pins of the FP64 emulator oracle (oracle/mlp.py) against what does not
depend on it: a library bfloat16 cast, central finite differences of the plain
network, closed forms of SiLU and of Adam's bias-corrected update."""
import numpy as np
import pytest

from oracle import mlp


def test_bf16_matches_library_cast_and_ties():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x32 = (rng.standard_normal(20000) * np.exp(rng.uniform(-20, 20, 20000))).astype(np.float32)
    lib = torch.from_numpy(x32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16(x32.astype(np.float64)), lib)
    ulp = 2.0 ** -7  # spacing of bfloat16 just above 1
    assert mlp.bf16(1 + ulp / 2) == 1.0  # tie -> even
    assert mlp.bf16(1 + 1.5 * ulp) == 1 + 2 * ulp  # tie -> even (upwards)
    assert mlp.bf16(1 + 0.51 * ulp) == 1 + ulp
    assert mlp.bf16(-3.0) == -3.0 and mlp.bf16(0.0) == 0.0


def test_silu_closed_forms():
    assert mlp.silu(0.0) == 0.0 and mlp.silu_grad(0.0) == 0.5
    assert abs(mlp.silu(40.0) - 40.0) < 1e-14 and abs(mlp.silu(-40.0)) < 1e-15
    z = np.linspace(-8, 8, 33)
    h = 1e-5
    fd = (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h)
    np.testing.assert_allclose(mlp.silu_grad(z), fd, rtol=0, atol=1e-9)
    np.testing.assert_allclose(mlp.silu(z), z / (1 + np.exp(-z)), rtol=1e-13, atol=1e-300)


@pytest.mark.parametrize("widths", [(5, 16, 12, 8, 1), mlp.WIDTHS])
def test_gradient_matches_finite_differences(widths):
    rng = np.random.default_rng(1)
    params = mlp.init_params(2, widths)
    for p in params[1::2]:
        p[:] = rng.uniform(-0.3, 0.3, p.shape)  # non-zero biases exercise db
    x = rng.uniform(-1, 1, (16, widths[0]))
    t = rng.normal(size=16)
    y, cache = mlp.forward(params, x, rounding=False)
    grads = mlp.backward(params, cache, y, t, rounding=False)
    h = 1e-5
    worst = 0.0
    for k, (p, g) in enumerate(zip(params, grads)):
        flat, gflat = p.reshape(-1), g.reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = mlp.loss(mlp.forward(params, x, rounding=False)[0], t)
            flat[idx] = old - h
            lm = mlp.loss(mlp.forward(params, x, rounding=False)[0], t)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            scale = np.abs(gflat).max()
            worst = max(worst, abs(fd - gflat[idx]) / scale)
    assert worst < 1e-7, worst


def test_rounding_changes_output_by_bf16_amount_only():
    rng = np.random.default_rng(3)
    params = mlp.init_params(4)
    x = rng.uniform(-1, 1, (64, 5))
    y0 = mlp.forward(params, x, rounding=False)[0]
    y1 = mlp.forward(params, x, rounding=True)[0]
    rel = np.abs(y1 - y0).max() / np.abs(y0).max()
    assert 1e-5 < rel < 5e-2, rel


def test_adam_closed_forms():
    p0 = np.array([0.5, -1.0, 2.0, 0.0])
    g1 = np.array([1e-3, -2.0, 0.0, 5.0])
    lr = 1e-2
    opt = mlp.Adam([p0])
    opt.step([g1], lr)  # first step: m_hat = g, v_hat = g^2
    np.testing.assert_allclose(opt.params[0], p0 - lr * g1 / (np.abs(g1) + mlp.EPS), rtol=0, atol=1e-15)
    g2 = np.array([-3e-3, 1.0, 4.0, 5.0])
    opt.step([g2], lr)
    m = 0.09 * g1 + 0.1 * g2  # beta1 (1 - beta1) g1 + (1 - beta1) g2
    v = 0.999 * 0.001 * g1 ** 2 + 0.001 * g2 ** 2
    mh, vh = m / (1 - 0.81), v / (1 - 0.999 ** 2)
    p2 = p0 - lr * g1 / (np.abs(g1) + mlp.EPS) - lr * mh / (np.sqrt(vh) + mlp.EPS)
    np.testing.assert_allclose(opt.params[0], p2, rtol=0, atol=1e-14)
    # a constant gradient keeps m_hat = g, v_hat = g^2 at every step
    opt = mlp.Adam([p0])
    for _ in range(50):
        opt.step([g1], lr)
    np.testing.assert_allclose(opt.params[0], p0 - 50 * lr * g1 / (np.abs(g1) + mlp.EPS), rtol=0, atol=1e-12)


def test_pack_roundtrip_and_size():
    params = mlp.init_params(5)
    assert mlp.n_params() == 5 * 256 + 256 + 2 * (256 * 256 + 256) + 256 + 1
    for a, b in zip(params, mlp.unpack(mlp.pack(params))):
        np.testing.assert_array_equal(a, b)


def test_training_fits_a_smooth_function():
    rng = np.random.default_rng(6)
    widths = (5, 32, 32, 32, 1)
    x = rng.uniform(-1, 1, (512, 5))
    t = np.sin(2 * x[:, 0]) * x[:, 4] + 0.3 * x[:, 1] ** 2
    params = mlp.init_params(7, widths)
    batches = [rng.choice(512, 64, replace=False) for _ in range(400)]
    _, losses, _ = mlp.train(params, x, t, batches, [3e-3] * 400)
    assert losses[-20:].mean() < 0.1 * losses[:5].mean()
