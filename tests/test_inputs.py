"""The seeded input generators both sides draw from (inputs.py holds no
method arithmetic): the SplitMix64 stream against its published definition,
the derived uniform and normal draws, the weight distribution, and the
meshes' structural promises."""
import os

import numpy as np

from paper_2307_14837_gb300 import inputs as I


def test_splitmix64_first_output_of_state_zero():
    # SplitMix64 (Steele, Lea, Flood 2014) started at state 0 outputs
    # 0xE220A8397B1DCDAF first: the state advances by the golden gamma and is
    # then mixed; stream 0's first uniform is that output's top 53 bits
    first = 0xE220A8397B1DCDAF
    z = I._mix64(np.array([int(I._GOLDEN)], dtype=np.uint64))
    assert int(z[0]) == first
    u = I.splitmix_uniform(0, 3)
    assert u[0] == (first >> 11) / 2.0 ** 53
    assert np.all((u >= 0.0) & (u < 1.0)) and len(set(u.tolist())) == 3


def test_uniform_and_normal_moments():
    u = I.splitmix_uniform(12345, 400_000)
    assert abs(u.mean() - 0.5) < 2e-3 and abs(u.var() - 1.0 / 12.0) < 2e-3
    g = I.splitmix_normal(777, 400_000)
    assert abs(g.mean()) < 1e-2 and abs(g.std() - 1.0) < 1e-2
    assert abs(np.mean(g ** 4) - 3.0) < 0.05                 # Gaussian kurtosis
    # distinct streams are independent draws, the same stream repeats
    assert np.array_equal(I.splitmix_normal(5, 100), I.splitmix_normal(5, 100))
    assert abs(np.corrcoef(I.splitmix_normal(5, 10_000), I.splitmix_normal(6, 10_000))[0, 1]) < 0.05


def test_network_weights_distribution():
    widths = (228, 256, 81)
    Ws, ss, ts = I.network_weights(widths, seed=3, scale_shift=True)
    for i, W in enumerate(Ws):
        assert W.shape == (widths[i + 1], widths[i])
        b = 1.0 / np.sqrt(widths[i])
        assert np.abs(W).max() <= b and np.abs(W).max() > 0.99 * b
        assert abs(W.mean()) < 0.05 * b
    assert np.all((ss[0] >= 0.5) & (ss[0] <= 1.5)) and np.all(np.abs(ts[0]) <= 0.1)
    assert np.array_equal(ss[-1], np.ones(81)) and np.array_equal(ts[-1], np.zeros(81))   # no last bias


def test_cavity_jitter_keeps_the_boundary_and_stays_bounded():
    n, jit = 6, 0.2
    m0 = I.cavity_mesh(n)
    m1 = I.cavity_mesh(n, jitter=jit, seed=9)
    d = m1["xyz"] - m0["xyz"]
    on_b = m0["vertex_bc"] > 0
    assert np.all(d[on_b] == 0.0)
    assert np.abs(d).max() <= jit / n and np.abs(d[~on_b]).max() > 0.5 * jit / n
    assert np.array_equal(m0["cells"], m1["cells"])


def test_smooth_fields_take_the_papers_training_statistics():
    path = os.path.join(os.path.dirname(__file__), "golden", "training_field_statistics.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    mean = np.array([float(r[2]) for r in rows])
    sigma = np.array([float(r[4]) for r in rows])
    assert np.allclose(I.PAPER_FIELD_MEAN, mean, rtol=0, atol=1e-10)
    assert np.allclose(I.PAPER_FIELD_STD, sigma, rtol=0, atol=0)
    m = I.channel_mesh(6, seed=2)
    f = I.smooth_field(m["xyz"], seed=4)
    assert np.allclose(f.mean(axis=0), mean, rtol=0, atol=1e-9)
    assert np.allclose(f.std(axis=0), sigma, rtol=1e-12)
