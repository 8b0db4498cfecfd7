"""Host-side pieces of the training path, on the CPU: the standardisation
made from column statistics (per-column shift and scale, a floor per kind of
column, padding columns untouched) and the target scale."""
import numpy as np

from paper_2307_14837_gb300 import inputs as I
from paper_2307_14837_gb300.train import column_groups, normalization_from_stats


def _stats(n=4096, n_in=228, pad=256, seed=0):
    X = np.zeros((n, pad))
    g = I.splitmix_normal(seed, n * n_in).reshape(n, n_in)
    X[:, :n_in] = 3.0 + g * (1.0 + np.arange(n_in) % 7)   # columns of different spreads
    T = 0.5 * I.splitmix_normal(seed + 1, n * 81).reshape(n, 81) + 0.1
    return X, T, (X.mean(0), X.std(0, ddof=1), T.mean(0), T.std(0, ddof=1))


def test_shift_scale_and_target_scale():
    X, T, (xm, xs, tm, ts_) = _stats()
    mu, sig, ts = normalization_from_stats(xm, xs, tm, ts_, X.shape[0])
    assert np.array_equal(mu[:228], xm[:228]) and np.array_equal(sig[:228], xs[:228])   # no floor active
    assert np.all(mu[228:] == 0.0) and np.all(sig[228:] == 1.0)
    # the root mean square of all target entries, from the column statistics
    assert abs(ts - float(np.sqrt((T ** 2).mean()))) < 1e-12 * ts
    Xn = (X - mu) / sig
    assert np.allclose(Xn[:, :228].mean(0), 0.0, atol=1e-12) and np.allclose(Xn[:, :228].std(0, ddof=1), 1.0)
    assert np.array_equal(Xn[:, 228:], X[:, 228:])


def test_sigma_floor_per_kind_of_column():
    # a near-constant column among columns of its kind is not blown up: its
    # sigma is floored at 5% of the kind's (lower) median spread
    X, T, _ = _stats()
    X[:, 0] = 3.0 + 1e-6 * X[:, 0]                     # u at node 0, nearly constant
    X[:, 216] = 0.25                                    # an edge length, exactly constant
    xs = X.std(0, ddof=1)
    mu, sig, ts = normalization_from_stats(X.mean(0), xs, T.mean(0), T.std(0, ddof=1), X.shape[0])
    kind_u = np.sort(xs[0:108:4])
    assert sig[0] == 0.05 * kind_u[(27 - 1) // 2]
    kind_h = np.sort(xs[216:228])
    assert sig[216] == 0.05 * kind_h[(12 - 1) // 2] > 0.0
    Xn = (X - mu) / sig
    assert np.abs(Xn[:, 0]).max() < 1.0 and np.abs(Xn[:, 216]).max() < 1e-12


def test_column_kinds_cover_the_input_row():
    for n_in in (228, 240):
        cols = sorted(c for g in column_groups(n_in) for c in g)
        assert cols == list(range(n_in))
