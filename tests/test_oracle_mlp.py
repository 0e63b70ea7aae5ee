"""Pins of the proposer network's CPU oracle (oracle/mlp.py) against what
the mathematics fixes, independent of the oracle's own formulas."""
import numpy as np
import pytest
import torch

from oracle import mlp


def _net(rng, n_in, scale=0.3):
    p = np.zeros(mlp.NPARAM)
    p[mlp.OW0:mlp.OB0] = rng.normal(0, scale, mlp.HID * mlp.NIN)
    p[mlp.OB0:mlp.OW1] = rng.normal(0, 0.1, mlp.HID)
    for a, b in ((mlp.OW1, mlp.OB1), (mlp.OW2, mlp.OB2)):
        p[a:b] = rng.normal(0, 1.5 / np.sqrt(mlp.HID), b - a)
    p[mlp.OB1:mlp.OW2] = rng.normal(0, 0.1, mlp.HID)
    p[mlp.OB2:mlp.OW3] = rng.normal(0, 0.1, mlp.HID)
    p[mlp.OW3:mlp.OB3] = rng.normal(0, 0.3, mlp.HID)
    p[mlp.OB3] = 0.2
    return p


@pytest.mark.parametrize("n_in", [30, 7])
def test_gradient_matches_central_differences(n_in):
    """Every block of the chain-rule gradient against (L(p + e) - L(p - e)) / 2e
    on sampled parameters; a transposed operand, a dropped relu mask or a
    missing 1/n fails it."""
    rng = np.random.default_rng(5)
    p = _net(rng, n_in)
    x = rng.normal(0, 1, (23, n_in))
    t = rng.normal(0, 1, 23)
    g, L = mlp.grad(p, x, t)
    assert L == pytest.approx(mlp.loss(p, x, t), rel=1e-14)
    blocks = [(mlp.OW0, mlp.OB0), (mlp.OB0, mlp.OW1), (mlp.OW1, mlp.OB1), (mlp.OB1, mlp.OW2),
              (mlp.OW2, mlp.OB2), (mlp.OB2, mlp.OW3), (mlp.OW3, mlp.OB3), (mlp.OB3, mlp.NPARAM)]
    eps = 1e-6
    for a, b in blocks:
        idx = rng.choice(np.arange(a, b), size=min(12, b - a), replace=False)
        if a == mlp.OW0:   # only columns < n_in take part
            idx = np.array([i for i in range(a, b) if (i - a) % mlp.NIN < n_in][:12])
        for i in idx:
            e = np.zeros(mlp.NPARAM)
            e[i] = eps
            fd = (mlp.loss(p + e, x, t) - mlp.loss(p - e, x, t)) / (2 * eps)
            assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-9), (a, i)
    # W0 columns past n_in do not take part
    gw0 = g[mlp.OW0:mlp.OB0].reshape(mlp.HID, mlp.NIN)
    assert np.all(gw0[:, n_in:] == 0)


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(1)
    v = np.concatenate([rng.normal(0, 1, 5000) * 10.0 ** rng.integers(-30, 30, 5000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.0078125, 1.01171875, 3.0e38, -2.5]])
    want = torch.tensor(v.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(v), want)


def test_exact_fit_has_zero_loss_and_gradient():
    rng = np.random.default_rng(2)
    p = _net(rng, 30)
    x = rng.normal(0, 1, (40, 30))
    y, _ = mlp.forward(p, x)
    g, L = mlp.grad(p, x, y)
    assert L == 0.0 and np.all(g == 0.0)


def test_relu_free_network_is_affine():
    """With all pre-activations positive the network is the affine map
    w3 W2 W1 W0 x + const; the gradient of b3 is then 2 mean(y - t)."""
    rng = np.random.default_rng(3)
    p = np.zeros(mlp.NPARAM)
    p[mlp.OW0:mlp.OB0] = rng.uniform(0.0, 0.1, mlp.HID * mlp.NIN)
    p[mlp.OW1:mlp.OB1] = rng.uniform(0.0, 0.02, mlp.HID * mlp.HID)
    p[mlp.OW2:mlp.OB2] = rng.uniform(0.0, 0.02, mlp.HID * mlp.HID)
    p[mlp.OB0:mlp.OW1] = 1.0
    p[mlp.OW3:mlp.OB3] = rng.normal(0, 1, mlp.HID)
    x = rng.uniform(0, 1, (9, 32))
    P = mlp.unpack(p, 32)
    A = P["w3"] @ P["W2"] @ P["W1"] @ P["W0"]
    c = P["w3"] @ (P["W2"] @ (P["W1"] @ P["b0"] + P["b1"]) + P["b2"]) + P["b3"]
    y, _ = mlp.forward(p, x)
    assert np.allclose(y, x @ A + c, rtol=1e-12)
    t = rng.normal(0, 1, 9)
    g, _ = mlp.grad(p, x, t)
    assert g[mlp.OB3] == pytest.approx(2 * np.mean(y - t), rel=1e-12)


def test_bf16_gradient_is_close_to_the_wide_one():
    rng = np.random.default_rng(4)
    p = _net(rng, 30)
    x = rng.normal(0, 1, (300, 30))
    t = rng.normal(0, 1, 300)
    g64, _ = mlp.grad(p, x, t)
    g16, _ = mlp.grad(p, x, t, bf=True)
    assert np.linalg.norm(g16 - g64) < 0.03 * np.linalg.norm(g64)


def test_features_identities():
    rng = np.random.default_rng(6)
    lo, hi = np.array([-2.0, -1.0, -0.5]), np.array([2.0, 1.0, 0.5])
    p = rng.uniform(lo, hi, (50, 3))
    n = rng.normal(0, 1, (50, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    f = mlp.pin_features(p, n, lo, hi)
    assert f.shape == (50, mlp.N_FEATURES)
    assert np.all(np.abs(f[:, :3]) <= 1.0) and np.allclose(np.abs(f[:, 0]).max(), np.abs(p[:, 0]).max() / 2.0)
    assert np.allclose(f[:, 3:6], n)
    s, c = f[:, 6::2], f[:, 7::2]
    assert np.allclose(s ** 2 + c ** 2, 1.0)
    # octave o + 1 is the double angle of octave o: sin 2a = 2 sin a cos a
    for o in range(3):
        for a in range(3):
            k0, k1 = 6 + 6 * o + 2 * a, 6 + 6 * (o + 1) + 2 * a
            assert np.allclose(f[:, k1], 2 * f[:, k0] * f[:, k0 + 1])
    # the box corner maps to (1, 0.5, 0.25); the diagonal's radius is 2^0
    corner = mlp.pin_features(hi[None], n[:1], lo, hi)[0, :3]
    assert np.allclose(corner, [1.0, 0.5, 0.25])
    assert mlp.radius_target([np.linalg.norm(hi - lo)], lo, hi)[0] == 0.0
