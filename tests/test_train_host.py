"""Host-side pieces of the training path, on the CPU: the input
standardisation fitted to a sample (per-column mean and spread, a floor per
kind of column, padding columns untouched) and the target scale."""
import numpy as np
import torch

from paper_2307_14837_gb300 import inputs as I
from paper_2307_14837_gb300.train import fit_normalization, normalize


def _sample(n=4096, n_in=228, pad=256, seed=0):
    X = torch.zeros((n, pad), dtype=torch.float32)
    g = I.splitmix_normal(seed, n * n_in).reshape(n, n_in)
    col_scale = 1.0 + np.arange(n_in) % 7            # columns of different spreads
    X[:, :n_in] = torch.as_tensor(3.0 + g * col_scale, dtype=torch.float32)
    T = torch.as_tensor(0.5 * I.splitmix_normal(seed + 1, n * 81).reshape(n, 81), dtype=torch.float32)
    return X, T


def test_standardised_columns_and_target_scale():
    X, T = _sample()
    mu, sig, ts = fit_normalization(X, T)
    Xn, Tn = normalize(X, (mu, sig, ts), T)
    assert torch.allclose(Xn[:, :228].mean(0), torch.zeros(228), atol=1e-4)
    assert torch.allclose(Xn[:, :228].std(0), torch.ones(228), atol=1e-4)
    assert torch.equal(mu[228:], torch.zeros(28)) and torch.equal(sig[228:], torch.ones(28))
    assert torch.equal(Xn[:, 228:], X[:, 228:])         # padding stays zero
    assert abs(ts - float(torch.sqrt((T ** 2).mean()))) < 1e-6 and abs(float((Tn ** 2).mean()) - 1.0) < 1e-5


def test_sigma_floor_per_kind_of_column():
    # a near-constant column among columns of its kind is not blown up: its
    # sigma is floored at 5% of the kind's median spread
    X, T = _sample()
    X[:, 0] = 3.0 + 1e-6 * X[:, 0]                     # u at node 0, nearly constant
    X[:, 216] = 0.25                                    # an edge length, exactly constant
    mu, sig, ts = fit_normalization(X, T)
    kind_u = sig[0:108:4]
    assert float(sig[0]) >= 0.05 * float(kind_u.median()) - 1e-6
    assert float(sig[216]) > 0.0
    Xn = normalize(X, (mu, sig, ts))
    assert float(Xn[:, 0].abs().max()) < 1.0 and float(Xn[:, 216].abs().max()) < 1e-5


def test_twenty_four_feature_rows():
    X, T = _sample(n_in=240)
    mu, sig, ts = fit_normalization(X, T, n_in=240)
    Xn = normalize(X, (mu, sig, ts))
    assert torch.allclose(Xn[:, :240].std(0), torch.ones(240), atol=1e-4)
    assert torch.equal(Xn[:, 240:], X[:, 240:])
