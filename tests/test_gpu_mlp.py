"""The proposer network's tensor-core forward and backward kernels and its
Adam step on the GPU, through the C-ABI, against the CPU oracle
(oracle/mlp.py) run with the same bfloat16 rounding points.

Tolerances: the library accumulates in FP32 on the tensor cores in an order
of its own, so a hidden activation or gradient can land one bfloat16 step
(2^-8 relative) away from the oracle's; that moves outputs and gradients by
about that fraction.  Outputs must agree to 1% in norm, each gradient block
to 3% in norm (cosine above 0.999), the loss to 1e-3.
"""
import numpy as np
import pytest
import torch

from oracle import mlp as ref

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


BLOCKS = {"W0": (ref.OW0, ref.OB0), "b0": (ref.OB0, ref.OW1), "W1": (ref.OW1, ref.OB1), "b1": (ref.OB1, ref.OW2),
          "W2": (ref.OW2, ref.OB2), "b2": (ref.OB2, ref.OW3), "w3": (ref.OW3, ref.OB3), "b3": (ref.OB3, ref.NPARAM)}


def _data(n, n_in, seed):
    rng = np.random.default_rng(seed)
    x = rng.normal(0, 1, (n, n_in)).astype(np.float32)
    t = (np.sin(2 * x[:, 0]) + 0.5 * x[:, 1] ** 2 - 1.0).astype(np.float32)
    return x, t


def _mlp(n_in, seed=3):
    from paper_2403_18761_gb300 import Mlp
    return Mlp(n_in=n_in, seed=seed)


def test_initial_parameters():
    net = _mlp(30)
    p = net.params().cpu().numpy().astype(np.float64)
    P = ref.unpack(p, 32)
    assert np.all(P["W0"][:, 30:] == 0)          # columns past n_in
    assert np.all(P["b0"] == 0) and np.all(P["b1"] == 0) and np.all(P["b2"] == 0) and P["b3"] == 0
    lim0, lim1 = np.sqrt(6.0 / 30), np.sqrt(6.0 / 128)
    assert np.abs(P["W0"][:, :30]).max() <= lim0 and np.abs(P["W0"][:, :30]).max() > 0.9 * lim0
    assert np.abs(P["W1"]).max() <= lim1 and np.abs(P["W2"]).max() <= lim1
    # seeded: the same seed gives the same network
    assert torch.equal(_mlp(30).params(), net.params())


@pytest.mark.parametrize("n,n_in", [(1000, 30), (128, 32), (37, 7)])
def test_forward_matches_oracle(n, n_in):
    """Several 128-row tiles and a ragged last tile; a single full tile; one
    partial tile with a narrow input."""
    net = _mlp(n_in)
    x, _ = _data(n, n_in, 11)
    y = net.forward(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    p = net.params().cpu().numpy().astype(np.float64)
    want, _ = ref.forward(p, x, bf=True)
    assert np.linalg.norm(y - want) <= 0.01 * np.linalg.norm(want)
    assert np.abs(y - want).max() <= 0.05 * np.abs(want).max()


@pytest.mark.parametrize("n,n_in", [(1000, 30), (37, 7)])
def test_gradient_matches_oracle(n, n_in):
    net = _mlp(n_in)
    x, t = _data(n, n_in, 12)
    # a few Adam steps first so no block of the gradient is degenerate
    net.train(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), steps=5, batch=256, lr=1e-3)
    p = net.params().cpu().numpy().astype(np.float64)
    g, loss = net.grad(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    g = g.cpu().numpy().astype(np.float64)
    want, wl = ref.grad(p, x, t, bf=True)
    assert loss == pytest.approx(wl, rel=1e-3)
    for name, (a, b) in BLOCKS.items():
        d, w = g[a:b], want[a:b]
        nw = np.linalg.norm(w)
        assert np.linalg.norm(d - w) <= 0.03 * nw + 1e-7, name
        if nw > 0:
            assert np.dot(d, w) / (np.linalg.norm(d) * nw) > 0.999, name


def test_one_adam_step_moves_each_parameter_by_lr():
    """From zero moments the bias-corrected Adam step is lr g / (|g| + eps):
    every parameter with a clear gradient moves by lr against its sign."""
    net = _mlp(30)
    x, t = _data(512, 30, 13)
    X, T = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    p0 = net.params().cpu().numpy().astype(np.float64)
    want, _ = ref.grad(p0, x, t, bf=True)
    g, _ = net.grad(X, T)
    g = g.cpu().numpy().astype(np.float64)
    lr = 1e-3
    net.train(X, T, steps=1, batch=512, lr=lr)
    step = net.params().cpu().numpy().astype(np.float64) - p0
    # the library's own gradient: -lr g / (|g| + 1e-8), up to FP32 rounding
    # of the update and the order of the gradient's atomic sums
    big = np.abs(g) > 1e-4
    assert big.sum() > 10000
    assert np.allclose(step[big], -lr * g[big] / (np.abs(g[big]) + 1e-8), rtol=2e-3, atol=1e-8)
    # and against the oracle's sign where the gradient is clearly nonzero
    clear = np.abs(want) > 1e-2 * np.abs(want).max()
    assert clear.sum() > 100
    assert np.all(np.sign(step[clear]) == -np.sign(want[clear]))


def test_training_fits_a_smooth_target():
    net = _mlp(30)
    x, t = _data(20000, 30, 14)
    X, T = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    _, l0 = net.grad(X, T)
    net.train(X, T, steps=1500, batch=1024, lr=2e-3)
    _, l1 = net.grad(X, T)
    assert l1 < 0.1 * l0, (l0, l1)


def test_rejects_bad_arguments():
    from paper_2403_18761_gb300 import Mlp, RpdError
    with pytest.raises(RpdError):
        Mlp(n_in=33)
    net = _mlp(30)
    with pytest.raises(RpdError):
        net.set_params(torch.zeros(10, device="cuda"))
    with pytest.raises(RpdError):
        net.train(torch.zeros((4, 30), device="cuda"), torch.zeros(4, device="cuda"), steps=1, batch=4, lr=-1.0)
