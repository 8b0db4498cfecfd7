"""Pins of the oracle's local restriction Q, extension L and the DNN-MG
step composition."""
import numpy as np
import pytest

from paper_2307_14837_gb300 import inputs as I
from oracle import dnnmg, fem, mesh, transfer


def _hier(m):
    return mesh.Hierarchy(m["xyz"], m["cells"], m["vertex_bc"])


def test_gather_brute_force_by_position():
    m = I.cavity_mesh(2, jitter=0.15, seed=2)
    h = _hier(m)
    xf = transfer.prolongate(h, I.coarse_state(m, 0))
    r = I.fine_rhs(h.n_fine, 1)
    X = dnnmg.gather(h, xf, r)
    assert X.shape == (8, dnnmg.N_IN)
    for P in range(8):
        corners = m["xyz"][m["cells"][P]]
        for iota in range(27):
            pos = mesh.corner_weights(iota) @ corners
            j = int(np.argmin(np.sum((h.xyz_f - pos) ** 2, axis=1)))
            assert np.array_equal(X[P, 4 * iota:4 * iota + 4], xf[j])
            assert np.array_equal(X[P, 108 + 4 * iota:108 + 4 * iota + 4], r[j])
        for e, (a, b) in enumerate(mesh.LOCAL_EDGES):
            assert X[P, 216 + e] == pytest.approx(np.linalg.norm(corners[b] - corners[a]), rel=1e-15)


@pytest.mark.parametrize("kind", ["constant", "linear"])
def test_extension_preserves_fields(kind):
    m = I.cavity_mesh(4, jitter=0.2, seed=3)
    h = _hier(m)
    if kind == "constant":
        g = np.tile(np.array([0.3, -1.7, 2.5]), (h.n_fine, 1))
    else:
        g = h.xyz_f @ np.array([[1.0, 2.0, -3.0], [0.5, 0.25, 1.0], [-2.0, 1.0, 0.5]]).T + 0.1
    Y = np.empty((h.n_patches, 81))
    for iota in range(27):
        Y[:, 3 * iota:3 * iota + 3] = g[h.patch_map[:, iota]]
    d = dnnmg.extend(h, Y)
    free = ~h.dirichlet_fine()
    assert np.allclose(d[free], g[free], rtol=4e-16, atol=4e-16)
    assert np.all(d[~free] == 0.0)


def test_extension_averages_by_valence():
    m = I.cavity_mesh(2)
    h = _hier(m)
    Y = np.zeros((h.n_patches, 81))
    Y[:, 0] = np.arange(1, h.n_patches + 1)         # u at patch node 0 only
    d = dnnmg.extend(h, Y)
    # node 0 of patch P is its corner vertex cells[P, 0]; that vertex is shared
    # by mult patches of which only those with it as local vertex 0 contribute
    for P in range(h.n_patches):
        j = h.patch_map[P, 0]
        if not h.dirichlet_fine()[j]:
            contrib = [Q + 1 for Q in range(h.n_patches) if h.patch_map[Q, 0] == j]
            assert d[j, 0] == pytest.approx(sum(contrib) / h.mult[j], rel=1e-15)


def test_zero_network_reproduces_plain_coarse_scheme():
    # with W_L = 0 the correction vanishes and the restricted fine rhs equals
    # the coarse rhs, so DNN-MG reproduces the plain scheme on level L
    m = I.cavity_mesh(4)
    h = _hier(m)
    coarse = fem.Level(m["xyz"], m["cells"], m["vertex_bc"], True)
    prm = dict(m=100.0, theta=1.0, nu=0.01, alpha0=0.02, delta0=0.1)
    widths = (228, 32, 32, 81)
    Ws, ss, ts = I.network_weights(widths, seed=0)
    Ws[-1] = np.zeros_like(Ws[-1])
    x0 = np.zeros((m["xyz"].shape[0], 4))
    bcv = lambda t: I.dirichlet_values(m, m["xyz"], m["vertex_bc"], t)
    dn, last = dnnmg.run(h, coarse, (Ws, ss, ts, True), x0, 3, prm, bcv)
    pl = dnnmg.run_plain(coarse, x0, 3, prm, bcv)
    assert np.abs(last["d"]).max() == 0.0
    for a, b in zip(dn, pl):
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
    assert np.abs(pl[-1][:, 0:3]).max() > 0.1              # the flow is moving
    # and a non-zero network changes the trajectory
    Ws2, _, _ = I.network_weights(widths, seed=0)
    dn2, _ = dnnmg.run(h, coarse, (Ws2, ss, ts, True), x0, 2, prm, bcv)
    assert np.abs(dn2[-1] - pl[1]).max() > 1e-6


def test_j2_zero_network_reproduces_plain_coarse_scheme():
    # J = 2: with W_L = 0 and backward Euler (rhs = mass term, which nested
    # Q1 spaces restrict exactly) the two-level patch step gives the plain
    # coarse right-hand side, so the trajectories agree
    m = I.cavity_mesh(2)
    h = mesh.Hierarchy2(m["xyz"], m["cells"], m["vertex_bc"])
    coarse = fem.Level(m["xyz"], m["cells"], m["vertex_bc"], True)
    prm = dict(m=100.0, theta=1.0, nu=0.01, alpha0=0.02, delta0=0.1)
    widths = (1012, 16, 375)
    Ws, ss, ts = I.network_weights(widths, seed=0)
    Ws[-1] = np.zeros_like(Ws[-1])
    x0 = np.zeros((m["xyz"].shape[0], 4))
    bcv = lambda t: I.dirichlet_values(m, m["xyz"], m["vertex_bc"], t)
    dn, last = dnnmg.run(h, coarse, (Ws, ss, ts, True), x0, 2, prm, bcv)
    pl = dnnmg.run_plain(coarse, x0, 2, prm, bcv)
    assert last["X"].shape == (8, 1012) and last["Y"].shape == (8, 375)
    for a, b in zip(dn, pl):
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


def test_j2_gather_by_position():
    m = I.cavity_mesh(2, jitter=0.15, seed=2)
    h = mesh.Hierarchy2(m["xyz"], m["cells"], m["vertex_bc"])
    xf = transfer.prolongate(h, I.coarse_state(m, 0))
    r = I.fine_rhs(h.n_fine, 1)
    X = dnnmg.gather(h, xf, r, features=24)
    assert X.shape == (8, 1024)
    for P in (0, 5):
        for iota in (0, 31, 62, 124):
            t = np.array([iota % 5, (iota // 5) % 5, iota // 25]) / 4.0
            w = np.array([np.prod([t[d] if (k >> d) & 1 else 1 - t[d] for d in range(3)]) for k in range(8)])
            pos = w @ m["xyz"][m["cells"][P]]
            j = int(np.argmin(np.sum((h.xyz_f - pos) ** 2, axis=1)))
            assert np.array_equal(X[P, 4 * iota:4 * iota + 4], xf[j])
            assert np.array_equal(X[P, 500 + 4 * iota:504 + 4 * iota], r[j])
    assert np.allclose(X[:, 1000:], h.geometry(24), rtol=0, atol=0)
