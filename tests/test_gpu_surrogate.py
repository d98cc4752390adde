"""Surrogate network kernels (BF16 tensor cores, FP32 accumulation) against the
FP64 network oracle with BF16 operands at the same points.

Tolerance 1e-3 in relative L2: both sides round the same operands to BF16,
but an activation whose FP32 and FP64 values straddle a BF16 rounding
boundary rounds differently (one element off by 2^-8); a few such flips per
128-wide product give errors of order 1e-4."""
import numpy as np
import pytest

from oracle import mlp
from paper_2207_09431_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-3


def relerr(a, b):
    return float(np.linalg.norm(np.asarray(a) - b) / max(np.linalg.norm(b), 1e-30))


@pytest.fixture(scope="module")
def lbm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_09431_gb300 import lbm as _lbm

    _lbm.load_library()
    return _lbm


def test_forward_and_gradients_match_oracle(lbm):
    w = inputs.mlp_init(1, seed=11)
    net = lbm.Surrogate(w, max_batch=256, max_rows=256)
    rng = np.random.default_rng(2)
    for rows in (1, 37, 256):
        X, T = rng.normal(size=(rows, 5)), rng.normal(size=(rows, 2))
        Y, loss, g = net.forward_backward(0, X, T)
        params = inputs.mlp_unflatten(w[0])
        Yo, cache = mlp.forward(params, X)
        go = inputs.mlp_flatten(mlp.backward(params, cache, Yo, T))
        assert relerr(Y, Yo) < TOL
        assert abs(loss - mlp.loss(Yo, T)) <= TOL * mlp.loss(Yo, T)
        assert relerr(g, go) < TOL


def test_one_adam_step_matches_oracle(lbm):
    w = inputs.mlp_init(1, seed=12)
    net = lbm.Surrogate(w, max_batch=128, max_rows=128)
    rng = np.random.default_rng(3)
    X, T = rng.normal(size=(128, 5)), rng.normal(size=(128, 2))
    # surr_train normalises; give it already standardised columns so that the
    # normalisation is (nearly) the identity, then compare with the oracle on
    # the same normalised data
    Xn = (X - X.mean(0)) / X.std(0)
    Tn = (T - T.mean(0)) / T.std(0)
    lr = 1e-3
    net.train(Xn, Tn, epochs=1, batch=128, lr=lr, seed=0)
    w1 = net.weights(0)
    params = inputs.mlp_unflatten(w[0])
    Yo, cache = mlp.forward(params, Xn)
    go = mlp.backward(params, cache, Yo, Tn)
    new, _ = mlp.adam(params, go, mlp.adam_state(params), lr)
    wo = inputs.mlp_flatten(new)
    g = inputs.mlp_flatten(go)
    sure = np.abs(g) > 1e-2 * np.abs(g).max()   # gradient sign far above rounding noise
    assert np.max(np.abs((w1 - w[0])[sure] - (wo - w[0])[sure])) <= 1e-3 * lr
    assert np.max(np.abs(w1 - wo)) <= 2.0 * lr + 1e-7


def test_training_fits_a_smooth_map_and_flags_outside_box(lbm):
    rng = np.random.default_rng(4)
    X = rng.uniform(-1, 1, size=(512, 5))
    Y = np.stack([np.sin(2 * X[:, 0]) + X[:, 1] * X[:, 2], np.cos(X[:, 3]) - 0.5 * X[:, 4] ** 2], axis=1)
    net = lbm.Surrogate(inputs.mlp_init(3, seed=5), max_batch=128, max_rows=512)
    loss = net.train(X, Y, epochs=300, batch=128, lr=3e-3, seed=1)
    Xt = rng.uniform(-0.9, 0.9, size=(64, 5))
    Yt = np.stack([np.sin(2 * Xt[:, 0]) + Xt[:, 1] * Xt[:, 2], np.cos(Xt[:, 3]) - 0.5 * Xt[:, 4] ** 2], axis=1)
    mean, spread, outside = net.predict(Xt)
    assert loss < 5e-3
    assert np.sqrt(np.mean((mean - Yt) ** 2)) < 0.05
    assert not outside.any() and spread.shape == (64, 2)
    _, _, out2 = net.predict(np.array([[0.0, 0.0, 0.0, 0.0, 1.5], [0.1, 0.1, 0.1, 0.1, 0.1]]))
    assert out2.tolist() == [True, False]


def test_local_residual_finds_scattered_labels(lbm):
    """Cross-validated training (surr_train_cv) on a smooth map whose labels
    scatter by 20 % (in the logarithm) where x_0 > 0.5: the local residual is
    large there and small elsewhere, although the ensemble's members agree on
    both sides; k = 1 at a training input is that row's own out-of-fold
    residual, and the residual grows with k."""
    rng = np.random.default_rng(7)
    X = rng.uniform(-1, 1, size=(400, 5))
    Y = np.stack([np.sin(X[:, 0]) + 0.5 * X[:, 1], np.cos(X[:, 2]) - 0.3 * X[:, 3]], axis=1)
    noisy = X[:, 0] > 0.5
    Y[noisy] += rng.normal(scale=0.2, size=(int(noisy.sum()), 2))
    w = inputs.mlp_init(3, seed=6)
    net = lbm.Surrogate(w, max_batch=128, max_rows=400)
    with pytest.raises(lbm.LbmError):
        net.local_residual(X[:2], 3)          # before the cross-validated fit
    net.train_cv(X, Y, 4, 300, 128, 3e-3, 2, w)
    Xq = rng.uniform(-0.9, 0.9, size=(128, 5))
    loc = net.local_residual(Xq, 5)
    hi, lo = Xq[:, 0] > 0.6, Xq[:, 0] < 0.3
    assert np.median(loc[hi]) > 3.0 * np.median(loc[lo])
    _, spread, _ = net.predict(Xq)
    assert np.median(spread[hi].max(1)) < np.median(loc[hi])   # the members do not see the scatter
    own = net.local_residual(X, 1)
    assert np.all(own >= 0) and np.all(np.isfinite(own))
    assert np.median(own[noisy]) > 3.0 * np.median(own[~noisy])
    assert np.all(net.local_residual(Xq, 9) >= loc)
    assert np.allclose(net.local_residual(Xq[:3], 400), own.max())
    # a plain fit forgets the residuals of the earlier set
    net.train(X, Y, epochs=1, batch=128, lr=1e-3, seed=0)
    with pytest.raises(lbm.LbmError):
        net.local_residual(X[:2], 3)
