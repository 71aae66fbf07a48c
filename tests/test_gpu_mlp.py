"""The surrogate network's BF16 tensor-core kernels against the CPU oracle (oracle/mlp.py):
forward pass, loss and gradients (the oracle rounds to bfloat16 at the same points as the
kernels, so only FP32-vs-FP64 summation differs), training and the ensemble gate."""
import numpy as np
import pytest

from oracle import mlp as OM
from tests._util import rel_fro

pytestmark = pytest.mark.gpu
# Against the bf16-rounding oracle only the summation differs (tensor-core FP32 accumulation vs
# float64), and where that moves a value across a bfloat16 rounding boundary the rounded
# activation differs by one bfloat16 ulp (2^-8 relative); measured ~1e-4 relative at width 256.
BF16_TOL = 2e-3


@pytest.fixture(scope="module")
def M():
    from paper_2509_08968_gb300 import build
    build.build()
    from paper_2509_08968_gb300 import mlp
    return mlp


def _weights(M, widths, E, seed, scale=1.0):
    from paper_2509_08968_gb300.surrogate import init_weights
    W = init_weights(widths, E, seed) * scale
    rng = np.random.default_rng(seed + 99)
    # non-zero biases so that the bias column is exercised
    for e in range(E):
        mats = M.unflatten(W[e], widths)
        for m in mats:
            m[:, -1] = 0.1 * rng.standard_normal(m.shape[0])
    return W


CASES = [([4, 256, 256, 256, 64], 300), ([3, 32, 48, 24], 77), ([4, 16, 8], 1)]


@pytest.mark.parametrize("widths,rows", CASES)
def test_forward_matches_oracle(M, widths, rows):
    E = 3
    W = _weights(M, widths, E, 1)
    X = np.random.default_rng(2).uniform(-1, 1, (rows, widths[0])).astype(np.float32)
    with M.Mlp(widths, W) as net:
        Y = net.forward(X)
    for e in range(E):
        mats = M.unflatten(W[e].astype(np.float64), widths)
        ref16, _ = OM.forward(mats, X, bf16=True)
        ref64, _ = OM.forward(mats, X)
        assert rel_fro(Y[e], ref16) < BF16_TOL, (e, rel_fro(Y[e], ref16))
        assert rel_fro(Y[e], ref64) < 3e-2


@pytest.mark.parametrize("widths,rows", CASES)
def test_gradients_match_oracle(M, widths, rows):
    E = 2
    W = _weights(M, widths, E, 3)
    rng = np.random.default_rng(4)
    X = rng.uniform(-1, 1, (rows, widths[0])).astype(np.float32)
    T = rng.standard_normal((rows, widths[-1])).astype(np.float32)
    with M.Mlp(widths, W) as net:
        loss, G = net.loss_grad(X, T)
    for e in range(E):
        mats = M.unflatten(W[e].astype(np.float64), widths)
        l16, g16 = OM.loss_grad(mats, X, T, bf16=True)
        l64, g64 = OM.loss_grad(mats, X, T)
        assert loss[e] == pytest.approx(l16, rel=BF16_TOL)
        got = M.unflatten(G[e].astype(np.float64), widths)
        for l in range(len(mats)):
            assert rel_fro(got[l], g16[l]) < BF16_TOL, (e, l, rel_fro(got[l], g16[l]))
            assert rel_fro(got[l], g64[l]) < 5e-2, (e, l, rel_fro(got[l], g64[l]))


def test_training_reduces_loss_and_is_reproducible(M):
    widths = [4, 64, 64, 16]
    rng = np.random.default_rng(5)
    X = rng.uniform(-1, 1, (1024, 4)).astype(np.float32)
    T = np.stack([np.sin(X @ rng.standard_normal(4)) for _ in range(16)], axis=1).astype(np.float32)
    W = _weights(M, widths, 2, 6, scale=1.0)
    with M.Mlp(widths, W) as a, M.Mlp(widths, W) as b:
        ha = a.train(X, T, epochs=60, batch=128, lr=3e-3, seed=11)
        hb = b.train(X, T, epochs=60, batch=128, lr=3e-3, seed=11)
        np.testing.assert_array_equal(a.weights(), b.weights())
        assert ha[-1] < 0.1 * ha[0], ha
        # the trained network's own loss agrees with the oracle on the final weights
        Wf = a.weights()
        loss, _ = a.loss_grad(X, T)
        for e in range(2):
            l16, _ = OM.loss_grad(M.unflatten(Wf[e].astype(np.float64), widths), X, T, bf16=True)
            assert loss[e] == pytest.approx(l16, rel=BF16_TOL)


def test_gate_spread_closed_form(M):
    """Bias-only members: v_e = exp(bf16(b_e)); one member off by a factor r gives the relative
    (population) spread 2|r - 1| / (4 + r) for five members."""
    widths = [4, 16, 8]
    E = 5
    P = sum(r * c for r, c in M.param_layout(widths))
    for r_fac, expect_fb in ((1.1, False), (1.2, True)):
        W = np.zeros((E, P), np.float32)
        base = np.linspace(-1.0, 1.0, 8)
        for e in range(E):
            mats = M.unflatten(W[e], widths)
            mats[1][:, -1] = base + (np.log(r_fac) if e == 4 else 0.0)
        with M.Mlp(widths, W) as net:
            X = np.zeros((3, 4), np.float32)
            mean, spread, fb = net.predict(X, np.zeros(8), np.ones(8), 0.05)
        b = OM.round_bf16(np.stack([M.unflatten(W[e], widths)[1][:, -1] for e in range(E)]))
        v = np.exp(b)
        rel = (v.std(axis=0) / v.mean(axis=0)).max()
        np.testing.assert_allclose(spread, rel, rtol=1e-5)
        np.testing.assert_allclose(mean, np.broadcast_to(v.mean(axis=0), mean.shape), rtol=1e-5)
        assert fb.tolist() == [expect_fb] * 3
