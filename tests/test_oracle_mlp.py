"""Pins of the surrogate-network oracle (oracle/mlp.py) against facts outside it: central finite
differences of its own loss, closed forms of degenerate networks, and an independent bfloat16
conversion (PyTorch's)."""
import numpy as np
import pytest

from oracle import mlp as M


def _net(widths, seed, scale=0.5):
    rng = np.random.default_rng(seed)
    return [scale * rng.standard_normal((widths[l + 1], widths[l] + 1))
            for l in range(len(widths) - 1)]


def test_gradient_matches_finite_differences():
    widths = [4, 16, 16, 8]
    mats = _net(widths, 1)
    rng = np.random.default_rng(2)
    X = rng.uniform(-1, 1, (12, 4))
    T = rng.standard_normal((12, 8))
    _, g = M.loss_grad(mats, X, T)
    h = 1e-6
    worst = 0.0
    for l, W in enumerate(mats):
        for idx in [(0, 0), (W.shape[0] - 1, W.shape[1] - 1), (W.shape[0] // 2, 1),
                    (1, W.shape[1] - 1)]:
            Wp = [m.copy() for m in mats]
            Wm = [m.copy() for m in mats]
            Wp[l][idx] += h
            Wm[l][idx] -= h
            fd = (M.loss_grad(Wp, X, T)[0] - M.loss_grad(Wm, X, T)[0]) / (2 * h)
            worst = max(worst, abs(fd - g[l][idx]) / max(1e-3, abs(fd)))
    assert worst < 1e-6, worst


def test_bias_only_network_closed_form():
    """All weights zero: y = b_last for every row, loss = mean (b - t)^2, grad_b = 2 mean (b - t)."""
    widths = [3, 16, 5]
    mats = [np.zeros((16, 4)), np.zeros((5, 17))]
    b = np.array([0.5, -1.0, 2.0, 0.0, 0.25])
    mats[1][:, -1] = b
    rng = np.random.default_rng(3)
    X = rng.standard_normal((7, 3))
    T = rng.standard_normal((7, 5))
    loss, g = M.loss_grad(mats, X, T)
    assert loss == pytest.approx(((b - T) ** 2).mean(), rel=1e-14)
    np.testing.assert_allclose(g[1][:, -1], 2 * (b - T).mean(axis=0) / 5 * 1.0, rtol=1e-13)
    np.testing.assert_allclose(g[1][:, :-1], 0.0)
    np.testing.assert_allclose(g[0], 0.0)   # relu(0) = 0 blocks every path below


def test_linear_network_closed_form():
    """One layer: grad = (2 / (R w)) (Y - T)^T [X | 1]."""
    rng = np.random.default_rng(4)
    W = rng.standard_normal((6, 4))
    X = rng.standard_normal((9, 3))
    T = rng.standard_normal((9, 6))
    loss, g = M.loss_grad([W], X, T)
    Xa = np.hstack([X, np.ones((9, 1))])
    Y = Xa @ W.T
    np.testing.assert_allclose(g[0], 2.0 / (9 * 6) * (Y - T).T @ Xa, rtol=1e-13)
    assert loss == pytest.approx(((Y - T) ** 2).mean(), rel=1e-14)


def test_round_bf16_ties_and_exact_values():
    u = 2.0 ** -7            # one bfloat16 ulp at 1
    vals = np.array([1.0, 1 + u / 2, 1 + 1.5 * u, 1 + u / 2 + 2.0 ** -20, -(1 + 1.5 * u),
                     3.0, 0.0, 2.0 ** -100])
    want = np.array([1.0, 1.0, 1 + 2 * u, 1 + u, -(1 + 2 * u), 3.0, 0.0, 2.0 ** -100])
    np.testing.assert_array_equal(M.round_bf16(vals), want)


def test_round_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    x = rng.standard_normal(100000) * np.exp(rng.uniform(-20, 20, 100000))
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(M.round_bf16(x), ref)


def test_bf16_forward_is_close_to_fp64():
    widths = [4, 32, 32, 8]
    mats = _net(widths, 6, scale=0.3)
    X = np.random.default_rng(7).uniform(-1, 1, (50, 4))
    y64, _ = M.forward(mats, X)
    y16, _ = M.forward(mats, X, bf16=True)
    rel = np.linalg.norm(y16 - y64) / np.linalg.norm(y64)
    assert 1e-5 < rel < 2e-2   # rounding is applied, and stays at bfloat16 level
