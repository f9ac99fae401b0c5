"""Pins of the proposal network's CPU oracle (oracle/nn.py) against what the
definitions fix: a plain loop, scipy's correlation, the adjoint identities of
linear maps, finite differences and the closed form of Adam."""
import numpy as np
import pytest

from oracle import nn as onn


def _rand(rng, *shape):
    return rng.standard_normal(shape)


def test_conv_matches_plain_loop():
    rng = np.random.default_rng(1)
    for Cin in (2, 3):
        x = _rand(rng, 2, 4, 4, 4, Cin)
        w = _rand(rng, 5, 64, Cin)
        b = _rand(rng, 5)
        assert np.allclose(onn.conv3d_pre(x, w, b), onn.conv3d_loop(x, w, b), rtol=1e-12, atol=1e-12)


def test_conv_matches_scipy_correlate_strided():
    from scipy.signal import correlate
    rng = np.random.default_rng(2)
    D = 8
    x = _rand(rng, 1, D, D, D, 1)
    w = _rand(rng, 1, 64, 1)
    k = w[0, :, 0].reshape(4, 4, 4)          # (kz, ky, kx)
    xp = np.pad(x[0, :, :, :, 0], 1)
    want = correlate(xp, k, mode="valid")[::2, ::2, ::2]
    got = onn.conv3d_pre(x, w)[0, :, :, :, 0]
    assert want.shape == got.shape == (D // 2,) * 3
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12)


def test_backward_data_is_the_adjoint():
    rng = np.random.default_rng(3)
    D, Cin = 6, 4
    x = _rand(rng, 2, D, D, D, Cin)
    w = _rand(rng, 32, 64, Cin)
    g = _rand(rng, 2, D // 2, D // 2, D // 2, 32)
    lhs = np.sum(onn.conv3d_pre(x, w) * g)
    rhs = np.sum(x * onn.conv3d_backward_data(g, w, D))
    assert abs(lhs - rhs) <= 1e-10 * max(1.0, abs(lhs))


def test_backward_weights_is_the_adjoint():
    rng = np.random.default_rng(4)
    D, Cin = 6, 2
    x = _rand(rng, 2, D, D, D, Cin)
    w = _rand(rng, 32, 64, Cin)
    g = _rand(rng, 2, D // 2, D // 2, D // 2, 32)
    lhs = np.sum(onn.conv3d_pre(x, w) * g)
    rhs = np.sum(w * onn.conv3d_backward_weights(x, g))
    assert abs(lhs - rhs) <= 1e-10 * max(1.0, abs(lhs))


def test_backward_data_single_tap_geometry():
    """One output gradient entry spreads to the 4^3 input voxels 2o + k - 1."""
    D = 8
    w = np.zeros((32, 64, 1))
    w[3, :, 0] = np.arange(64) + 1.0
    g = np.zeros((1, 4, 4, 4, 32))
    g[0, 1, 2, 1, 3] = 1.0                    # o = (z 1, y 2, x 1)
    dx = onn.conv3d_backward_data(g, w, D)[0, :, :, :, 0]
    for t, (kz, ky, kx) in enumerate(onn.TAPS):
        iz, iy, ix = 2 * 1 + kz - 1, 2 * 2 + ky - 1, 2 * 1 + kx - 1
        if 0 <= iz < D and 0 <= iy < D and 0 <= ix < D:
            assert dx[iz, iy, ix] == t + 1.0
    assert np.count_nonzero(dx) == 64


def test_gaussian_nll_gradient_finite_differences():
    rng = np.random.default_rng(5)
    out = rng.standard_normal((3, 12))
    y = rng.standard_normal((3, 6))
    _, g = onn.gaussian_nll(out, y)
    h = 1e-6
    num = np.zeros_like(out)
    for i in range(out.shape[0]):
        for j in range(12):
            e = np.zeros_like(out)
            e[i, j] = h
            num[i, j] = (onn.gaussian_nll(out + e, y)[0] - onn.gaussian_nll(out - e, y)[0]) / (2 * h)
    assert np.allclose(g, num, rtol=1e-6, atol=1e-8)


def test_gaussian_nll_minimum_at_the_residual_variance():
    """For fixed mu the loss is minimal at s = log((y - mu)^2)."""
    y = np.array([[0.5, -1.0, 2.0, 0.1, 0.0, 1.0]])
    mu = np.zeros((1, 6))
    s = np.log((y - mu) ** 2 + 1e-300)
    s[0, 4] = 0.0   # zero residual: no finite minimiser; keep it out
    _, g = onn.gaussian_nll(np.concatenate([mu, s], 1), y)
    idx = [0, 1, 2, 3, 5]
    assert np.allclose(g[0, 6 + np.array(idx)], 0.0, atol=1e-12)


def test_adam_constant_gradient_closed_form():
    theta0 = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -0.7, 2.0])
    th, m, v = theta0.copy(), np.zeros(3), np.zeros(3)
    lr, eps = 1e-2, 1e-8
    for t in range(1, 11):
        th, m, v = onn.adam(th, m, v, g, t, lr, eps=eps)
    # bias-corrected moments equal g and g^2 exactly: each step moves lr * g / (|g| + eps)
    assert np.allclose(th, theta0 - 10 * lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-14)


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(6)
    a = (rng.standard_normal(10000) * np.exp(rng.uniform(-20, 20, 10000))).astype(np.float32)
    a[:4] = [1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -1.0 - 2 ** -8, 0.0]   # ties to even
    want = torch.from_numpy(a).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(onn.bf16_round(a), want)
    assert np.array_equal(onn.from_bf16_bits(onn.bf16_bits(want)), want)


def test_layout_counts_the_architecture():
    _, total = onn.layout()
    assert total == 464652


def test_net_backward_matches_finite_differences_without_rounding():
    """With the bf16 roundings switched off, the network gradient equals
    central finite differences of its loss."""
    ident = lambda a: np.asarray(a, np.float64)   # noqa: E731
    rng = np.random.default_rng(9)
    _, total = onn.layout()
    theta = rng.standard_normal(total) * 0.05
    x = np.abs(rng.standard_normal((1, 64, 64, 64, 2))) * 0.5
    y = rng.uniform(-1, 1, (1, 6))
    loss, g = onn.net_backward(theta, x, y, ident)
    off, _ = onn.layout()
    picks = [off["cw0"][0] + 5, off["cw2"][0] + 1000, off["cb3"][0] + 7, off["f1w"][0] + 12345, off["f2b"][0] + 8]
    h = 1e-6   # small enough that no ReLU changes side
    for i in picks:
        e = np.zeros(total)
        e[i] = h
        num = (onn.net_backward(theta + e, x, y, ident)[0] - onn.net_backward(theta - e, x, y, ident)[0]) / (2 * h)
        assert abs(num - g[i]) <= 1e-5 * max(1.0, abs(num)), (i, num, g[i])


def test_box_average_against_loops():
    rng = np.random.default_rng(10)
    vol = rng.integers(0, 256, (11, 13, 17)).astype(np.uint8)
    origin, spacing = np.array([1.5, -2.0, 0.0]), np.array([1.0, 0.8, 1.3])
    box_o, h, G = np.array([0.0, 0.0, 0.0]), np.array([2.5, 1.7, 3.1]), 8
    got = onn.box_average(vol, origin, spacing, box_o, h, G)
    for gz in range(G):
        for gy in range(G):
            for gx in range(G):
                vals = []
                for z in range(vol.shape[0]):
                    for y in range(vol.shape[1]):
                        for x in range(vol.shape[2]):
                            w = origin + spacing * np.array([x, y, z])
                            if all(box_o[d] + h[d] * gg <= w[d] < box_o[d] + h[d] * (gg + 1)
                                   for d, gg in enumerate((gx, gy, gz))):
                                vals.append(vol[z, y, x])
                want = np.mean(vals) / 64.0 if vals else 0.0
                assert abs(got[gz, gy, gx] - want) < 1e-12


def test_abs_bound_is_the_loop_over_absolute_values():
    # the per-output sum of |x| |w| the GPU tests scale their error bounds by
    rng = np.random.default_rng(11)
    x = _rand(rng, 1, 4, 4, 4, 3)
    w = _rand(rng, 2, 64, 3)
    want = onn.conv3d_loop(np.abs(x), np.abs(w), np.zeros(2))
    assert np.allclose(onn.conv3d_abs_bound(x, w), want, rtol=1e-12, atol=1e-12)


def test_network_rounding_is_bf16_at_the_stated_points():
    # net_forward's default rounding: the conv weights and every conv output
    # (after ReLU) are bf16 values; with the identity it is the exact network
    rng = np.random.default_rng(12)
    _, total = onn.layout()
    theta = rng.standard_normal(total) * 0.05
    x = onn.bf16_round(rng.uniform(0, 4, (1, 64, 64, 64, 2)).astype(np.float32)).astype(np.float64)
    out, h, acts = onn.net_forward(theta, x)
    for a in acts:
        assert np.array_equal(a, onn.bf16_round(a.astype(np.float32)).astype(np.float64))
    out_exact, _, _ = onn.net_forward(theta, x, rnd=lambda v: v)
    assert not np.array_equal(out, out_exact)
    assert np.allclose(out, out_exact, rtol=0.05, atol=0.05 * np.abs(out_exact).max())
