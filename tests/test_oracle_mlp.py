"""Pins of the oracle's patch network: Table 2 parameter counts, explicit
loops, folded normalisation and the skip rule."""
import os

import numpy as np
import pytest

from paper_2307_14837_gb300 import inputs as I
from oracle import mlp


def test_table2_parameter_counts():
    path = os.path.join(os.path.dirname(__file__), "golden", "table2_parameter_counts.txt")
    rows = [list(map(int, l.split())) for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 4
    for _, n_in, n_h, n_out, count in rows:
        assert mlp.trainable_parameters(n_in, n_h, n_out) == count
    # the counts are not reproduced with linear biases
    for _, n_in, n_h, n_out, count in rows:
        assert mlp.trainable_parameters(n_in, n_h, n_out) + 8 * n_h + n_out != count


def test_forward_matches_explicit_loops():
    widths = (7, 5, 5, 3)
    Ws, ss, ts = I.network_weights(widths, seed=4, scale_shift=True)
    X = I.splitmix_normal(77, 4 * 7).reshape(4, 7)
    Y = mlp.forward(X, Ws, ss, ts, skip=True)
    for r in range(4):
        h = list(X[r])
        for li, W in enumerate(Ws):
            z = []
            for o in range(W.shape[0]):
                acc = 0.0
                for i in range(W.shape[1]):
                    acc += W[o, i] * h[i]
                z.append(acc * ss[li][o] + ts[li][o])
            if li < len(Ws) - 1:
                z = [max(a, 0.0) for a in z]
                if li > 0 and len(z) == len(h):
                    z = [a + b for a, b in zip(z, h)]
            h = z
        assert np.allclose(Y[r], h, rtol=1e-13, atol=1e-14)


def test_folded_batchnorm_equals_unfolded():
    rng = np.random.default_rng(0)
    z = rng.standard_normal((6, 4))
    gamma, beta = rng.uniform(0.5, 2, 4), rng.standard_normal(4)
    mu, s = rng.standard_normal(4), rng.uniform(0.5, 2, 4)
    sc, sh = mlp.fold_batchnorm(gamma, beta, mu, s)
    assert np.allclose(z * sc + sh, (z - mu) / s * gamma + beta, rtol=1e-14, atol=1e-14)


def test_skip_only_where_widths_match():
    widths = (4, 4, 4, 2)
    Ws, ss, ts = I.network_weights(widths, seed=1)
    X = np.abs(I.splitmix_normal(5, 8).reshape(2, 4))
    # identity-like second layer: skip doubles the (non-negative) activation
    Ws = [np.eye(4), np.eye(4), np.ones((2, 4))]
    Y, hid = mlp.forward(X, Ws, ss, ts, skip=True, return_hidden=True)
    assert np.allclose(hid[0], X)            # first layer: no skip
    assert np.allclose(hid[1], 2 * X)        # second layer: relu(x) + x
    assert np.allclose(Y, 2 * X.sum(axis=1, keepdims=True) * np.ones((1, 2)))


def test_training_gradients_match_finite_differences():
    # the oracle's backpropagation against central differences of its loss
    widths = (9, 6, 6, 6, 4)
    Ws, _, _ = I.network_weights(widths, seed=2)
    rng = np.random.default_rng(0)
    bs = [0.1 * rng.standard_normal(w) for w in widths[1:-1]]
    X = rng.standard_normal((7, 9))
    T = rng.standard_normal((7, 4))
    loss, dWs, dbs = mlp.loss_and_grads(X, Ws, bs, T, skip=True)
    eps = 1e-6
    for li in range(len(Ws)):
        for (r, c) in [(0, 0), (1, 2), (Ws[li].shape[0] - 1, Ws[li].shape[1] - 1)]:
            Wp = [w.copy() for w in Ws]
            Wm = [w.copy() for w in Ws]
            Wp[li][r, c] += eps
            Wm[li][r, c] -= eps
            fd = (mlp.loss_and_grads(X, Wp, bs, T)[0] - mlp.loss_and_grads(X, Wm, bs, T)[0]) / (2 * eps)
            assert abs(fd - dWs[li][r, c]) <= 1e-7 * max(1.0, abs(fd))
    for li in range(len(bs)):
        bp = [b.copy() for b in bs]
        bm = [b.copy() for b in bs]
        bp[li][1] += eps
        bm[li][1] -= eps
        fd = (mlp.loss_and_grads(X, Ws, bp, T)[0] - mlp.loss_and_grads(X, Ws, bm, T)[0]) / (2 * eps)
        assert abs(fd - dbs[li][1]) <= 1e-7 * max(1.0, abs(fd))
    # the loss is the forward pass's output error
    Y = mlp.forward(X, Ws, [np.ones(w) for w in widths[1:]], bs + [np.zeros(4)], skip=True)
    assert loss == pytest.approx(np.sum((Y - T) ** 2) / 7, rel=1e-12)
