"""Pins of the oracle's mesh hierarchy (refinement, patch map, valences,
boundary kinds) against closed forms and brute force."""
import os

import numpy as np
import pytest

from paper_2307_14837_gb300 import inputs as I
from oracle import fem, mesh


def _hier(m):
    return mesh.Hierarchy(m["xyz"], m["cells"], m["vertex_bc"])


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_counts_closed_form(n):
    m = I.cavity_mesh(n, grouped=False)
    h = _hier(m)
    # (2n+1)^3 fine nodes; 3 n^2 (n+1) edges; 3 n (n+1)^2 faces
    assert h.n_fine == (2 * n + 1) ** 3
    assert h.n_edges == 3 * n * (n + 1) ** 2
    assert h.n_faces == 3 * n * n * (n + 1)
    assert h.mult.sum() == 27 * h.n_patches


@pytest.mark.parametrize("n", [2, 3])
def test_valence_closed_form_and_brute_force(n):
    m = I.cavity_mesh(n, grouped=False)
    h = _hier(m)
    ijk = np.rint(h.xyz_f * 2 * n).astype(int)          # fine grid index 0..2n

    def m1(i):
        return np.where(i % 2 == 1, 1, np.where((i == 0) | (i == 2 * n), 1, 2))
    closed = m1(ijk[:, 0]) * m1(ijk[:, 1]) * m1(ijk[:, 2])
    assert np.array_equal(h.mult, closed)
    # brute force: count coarse cells whose closed box contains the node
    lo = m["xyz"][m["cells"][:, 0]]
    hi = m["xyz"][m["cells"][:, 7]]
    brute = np.array([np.sum(np.all((p >= lo - 1e-12) & (p <= hi + 1e-12), axis=1)) for p in h.xyz_f])
    assert np.array_equal(h.mult, brute)


@pytest.mark.parametrize("jitter", [0.0, 0.2])
def test_patch_map_points_at_trilinear_positions(jitter):
    m = I.cavity_mesh(4, jitter=jitter, seed=3)
    h = _hier(m)
    X = m["xyz"][m["cells"]]                              # [Nc, 8, 3]
    for iota in range(27):
        w = mesh.corner_weights(iota)
        expect = np.einsum("k,nkd->nd", w, X)
        got = h.xyz_f[h.patch_map[:, iota]]
        assert np.allclose(got, expect, rtol=0, atol=1e-15)
    # every patch has 27 distinct nodes
    assert all(len(set(r)) == 27 for r in h.patch_map.tolist())


def test_hierarchical_numbering():
    m = I.cavity_mesh(2, grouped=False)
    h = _hier(m)
    nv = m["xyz"].shape[0]
    # coarse vertices keep their numbers, cell centres come last in cell order
    assert np.array_equal(h.patch_map[:, [0, 2, 6, 8, 18, 20, 24, 26]], m["cells"])
    assert np.array_equal(h.patch_map[:, 13], nv + h.n_edges + h.n_faces + np.arange(8))
    # first cell's 12 edges are numbered first, in local edge order
    e_iota = [1, 7, 19, 25, 3, 5, 21, 23, 9, 11, 15, 17]
    assert np.array_equal(h.patch_map[0, e_iota], nv + np.arange(12))


def test_cavity_fine_boundary_kinds():
    m = I.cavity_mesh(4)
    h = _hier(m)
    x = h.xyz_f
    on_b = np.any((np.abs(x) < 1e-14) | (np.abs(x - 1) < 1e-14), axis=1)
    lid = np.abs(x[:, 2] - 1) < 1e-14
    expect = np.where(lid, 2, np.where(on_b, 1, 0))
    assert np.array_equal(h.bc_f, expect)


def test_channel_kinds_and_positive_jacobians():
    m = I.channel_mesh(4, seed=1)
    h = _hier(m)
    x = h.xyz_f
    H, Lx = I.CHANNEL_HEIGHT, I.CHANNEL_LENGTH
    inflow = np.abs(x[:, 0]) < 1e-12
    out = np.abs(x[:, 0] - Lx) < 1e-12
    walls = (np.abs(x[:, 1]) < 1e-12) | (np.abs(x[:, 1] - H) < 1e-12) | \
        (np.abs(x[:, 2]) < 1e-12) | (np.abs(x[:, 2] - H) < 1e-12)
    assert np.all(h.bc_f[inflow] == 2)
    assert np.all(h.bc_f[out & ~walls] == 3)
    assert np.all(h.bc_f[out & walls] == 1)
    assert np.all(h.bc_f[walls & ~inflow] == 1)
    # every fine cell is a valid (positively oriented) hexahedron
    det, _ = fem.cell_geometry(h.xyz_f[h.cells_f])
    assert det.min() > 0


def test_edge_lengths_cube():
    m = I.cavity_mesh(4)
    h = _hier(m)
    assert np.allclose(h.edge_lengths(), 0.25, rtol=0, atol=1e-15)
    # order: xi-edges measure along x
    m2 = dict(m)
    xyz = m["xyz"] * np.array([1.0, 2.0, 3.0])
    h2 = mesh.Hierarchy(xyz, m["cells"], m["vertex_bc"])
    e = h2.edge_lengths()
    assert np.allclose(e[:, 0:4], 0.25) and np.allclose(e[:, 4:8], 0.5) and np.allclose(e[:, 8:12], 0.75)


def _one_cell(X):
    """A single hexahedron with corners X[k], k = k0 + 2 k1 + 4 k2."""
    return mesh.Hierarchy(np.asarray(X, dtype=np.float64), np.arange(8, dtype=np.int32)[None, :],
                          np.ones(8, dtype=np.int32))


def _parallelepiped(a, b, c, origin=(0.0, 0.0, 0.0)):
    o = np.asarray(origin, dtype=np.float64)
    return [o + (k & 1) * np.asarray(a) + ((k >> 1) & 1) * np.asarray(b) + ((k >> 2) & 1) * np.asarray(c)
            for k in range(8)]


def test_geometry_features_cube_and_box():
    h = _one_cell(_parallelepiped((0.3, 0, 0), (0, 0.5, 0), (0, 0, 0.7)))
    g = h.geometry(24)
    assert g.shape == (1, 24)
    assert np.allclose(g[0, 12:16], np.sqrt(0.3 ** 2 + 0.5 ** 2 + 0.7 ** 2), rtol=0, atol=1e-15)
    assert np.allclose(g[0, 16:24], np.pi / 2, rtol=0, atol=1e-14)
    assert np.array_equal(h.geometry(12), g[:, :12])


def test_face_angles_sheared_cell_closed_form():
    # a parallelepiped sheared in the xy-plane by the angle phi: the faces
    # through the z-edge at vertex 0 meet at phi, the other pairs at pi/2;
    # at vertex 1 the z-edge pair meets at pi - phi
    phi = 1.1
    a, b, c = np.array([1.0, 0, 0]), np.array([np.cos(phi), np.sin(phi), 0]), np.array([0, 0, 1.0])
    h = _one_cell(_parallelepiped(a, b, c))
    ang = h.face_angles()[0]
    assert abs(ang[0] - (np.pi + phi) / 3) < 1e-14
    assert abs(ang[1] - (2 * np.pi - phi) / 3) < 1e-14
    assert abs(ang[2] - (2 * np.pi - phi) / 3) < 1e-14     # vertex b: edges -b, a, c
    assert abs(ang[3] - (np.pi + phi) / 3) < 1e-14         # vertex a + b: edges -a, -b, c
    d = h.diagonals()[0]
    for k, ref in enumerate([a + b + c, b + c - a, a + c - b, c - a - b]):
        assert abs(d[k] - np.linalg.norm(ref)) < 1e-14


def test_geometry_features_invariance():
    # a general (non-planar-faced) hexahedron: lengths scale with the cell,
    # angles do not; both are unchanged by a rotation and a translation
    rng = np.random.default_rng(4)
    X = np.array(_parallelepiped((1, 0, 0), (0, 1, 0), (0, 0, 1))) + 0.15 * rng.standard_normal((8, 3))
    g = _one_cell(X).geometry(24)[0]
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    g_rot = _one_cell(X @ q.T + np.array([3.0, -1.0, 2.0])).geometry(24)[0]
    assert np.allclose(g_rot, g, rtol=1e-12, atol=1e-13)
    g_scaled = _one_cell(2.5 * X).geometry(24)[0]
    assert np.allclose(g_scaled[:16], 2.5 * g[:16], rtol=1e-13)
    assert np.allclose(g_scaled[16:], g[16:], rtol=1e-12)
    # a skewed cell is not a box: some mean angle differs from pi / 2
    assert np.abs(g[16:] - np.pi / 2).max() > 1e-3


def test_golden_patch_sizes():
    path = os.path.join(os.path.dirname(__file__), "golden", "patch_sizes.txt")
    rows = [list(map(int, l.split())) for l in open(path) if l.strip() and not l.startswith("#")]
    J1 = rows[0]
    assert J1[1] == 27 and J1[2] == 4 * 27 and J1[4] == 2 * J1[2] + J1[3] and J1[5] == 3 * 27
    # the build's patches: 27 and 125 nodes per coarse cell, input rows of
    # 2 N_dof^P + n_Geo with the 24 geometry features
    m = I.cavity_mesh(2)
    h = _hier(m)
    assert h.patch_map.shape[1] == J1[1]
    J2 = rows[1]
    assert J2[0] == 2 and J2[5] == 3 * J2[1] and J2[4] == 2 * J2[2] + J2[3]
    h2 = mesh.Hierarchy2(m["xyz"], m["cells"], m["vertex_bc"])
    assert h2.patch_map.shape[1] == J2[1]
    from oracle import dnnmg
    X = dnnmg.gather(h2, np.zeros((h2.n_fine, 4)), np.zeros((h2.n_fine, 4)), features=J2[3])
    assert X.shape[1] == J2[4]
    assert dnnmg.gather(h, np.zeros((h.n_fine, 4)), np.zeros((h.n_fine, 4)), features=J1[3]).shape[1] == J1[4]


@pytest.mark.parametrize("n", [1, 2])
def test_j2_counts_valences_closed_form(n):
    # twofold refinement of the n^3 cavity: the (4n+1)^3 grid; a node lies in
    # 2 patches per axis where its grid index is an interior multiple of 4
    m = I.cavity_mesh(n, grouped=False)
    h = mesh.Hierarchy2(m["xyz"], m["cells"], m["vertex_bc"])
    assert h.n_fine == (4 * n + 1) ** 3 and h.patch_map.shape == (n ** 3, 125)
    ijk = np.rint(h.xyz_f * 4 * n).astype(int)

    def m1(i):
        return np.where(i % 4 != 0, 1, np.where((i == 0) | (i == 4 * n), 1, 2))
    assert np.array_equal(h.mult, m1(ijk[:, 0]) * m1(ijk[:, 1]) * m1(ijk[:, 2]))
    assert all(len(set(r)) == 125 for r in h.patch_map.tolist())


def test_j2_patch_map_points_at_trilinear_positions():
    m = I.cavity_mesh(2, jitter=0.2, seed=5)
    h = mesh.Hierarchy2(m["xyz"], m["cells"], m["vertex_bc"])
    X = m["xyz"][m["cells"]]
    for iota in range(125):
        t = np.array([iota % 5, (iota // 5) % 5, iota // 25]) / 4.0
        w = np.array([np.prod([t[d] if (k >> d) & 1 else 1 - t[d] for d in range(3)]) for k in range(8)])
        assert np.allclose(h.xyz_f[h.patch_map[:, iota]], np.einsum("k,nkd->nd", w, X), rtol=0, atol=1e-15)
    # every fine node of level L+2 belongs to some patch, Dirichlet kinds on the lid
    assert np.array_equal(np.unique(h.patch_map), np.arange(h.n_fine))
    top = np.isclose(h.xyz_f[:, 2], 1.0)
    assert np.all(h.bc_f[top] > 0)
