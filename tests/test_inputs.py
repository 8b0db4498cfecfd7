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


def _coarsen(cells):
    """Parents of consecutive 8-cell groups: corner K of parent g is vertex K
    of child K; the 8 children must share the 27 nodes of a refined hex."""
    g = np.asarray(cells).reshape(-1, 8, 8)
    for t in range(8):
        for k in range(8):
            pos = ((t & 1) + (k & 1)) + 3 * (((t >> 1) & 1) + ((k >> 1) & 1)) + 9 * (((t >> 2) & 1) + ((k >> 2) & 1))
            # any other (t', k') landing on the same node must name the same vertex
            for t2 in range(t + 1, 8):
                for k2 in range(8):
                    pos2 = (((t2 & 1) + (k2 & 1)) + 3 * (((t2 >> 1) & 1) + ((k2 >> 1) & 1))
                            + 9 * (((t2 >> 2) & 1) + ((k2 >> 2) & 1)))
                    if pos2 == pos:
                        assert np.array_equal(g[:, t, k], g[:, t2, k2])
    return np.stack([g[:, K, K] for K in range(8)], axis=1)


def test_nested_meshes_coarsen_to_their_base():
    # a mesh with `levels` = k is the k-th refinement of its base: every 8
    # consecutive cells are the children of one parent, recursively, and the
    # parents' corners are the vertices 0 .. n - 1 of the coarser level
    for m, base in [(I.cavity_mesh(8, levels=3, jitter=0.1, seed=2), I.cavity_mesh(1, grouped=False)),
                    (I.channel_mesh(8, seed=1, levels=2), I.channel_mesh(2, seed=1))]:
        k = m["meta"]["mg_levels"]
        cells = m["cells"]
        for _ in range(k):
            cells = _coarsen(cells)
            nv = cells.max() + 1
            assert np.array_equal(np.unique(cells), np.arange(nv))
        assert cells.shape[0] == base.n_cells and nv == base.n_vertices
        if m["meta"]["kind"] == "channel":
            # the base mesh's vertices, bit for bit, and its boundary kinds
            key = lambda X: np.lexsort(X.T[::-1])   # noqa: E731
            a, b = m["xyz"][:nv], base["xyz"]
            assert np.array_equal(a[key(a)], b[key(b)])
            assert np.array_equal(m["vertex_bc"][:nv][key(a)], base["vertex_bc"][key(b)])


def test_nested_mesh_sizes():
    # cavity n^3 refined from (n/8)^3: (n+1)^3 vertices; channel cells 8^k
    # times the base's
    m = I.cavity_mesh(8, levels=3)
    assert m.n_cells == 512 and m.n_vertices == 729 and m["patch_groups"]
    for nz, k in [(4, 1), (8, 2)]:
        assert I.channel_mesh(nz, seed=0, levels=k).n_cells == 8 ** k * I.channel_mesh(nz >> k, seed=0).n_cells
    # levels = 0 is the unrefined generator
    a, b = I.channel_mesh(6, seed=3), I.channel_mesh(6, seed=3, levels=0)
    assert all(np.array_equal(a[x], b[x]) for x in ("xyz", "cells", "vertex_bc"))
