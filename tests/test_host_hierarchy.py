"""The library's C++ mesh hierarchy, built on the host alone
(dnnmg_hierarchy_build, no GPU), against the oracle's: patch maps and
valences bit for bit, boundary kinds, node coordinates and the geometry
features, for one- and two-level patches on the cavity and the channel."""
import numpy as np
import pytest

from oracle import mesh as omesh
from paper_2307_14837_gb300 import build, capi, inputs as I


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    capi.load()


CASES = {
    "cavity4_jitter": lambda: I.cavity_mesh(4, jitter=0.2, seed=3),
    "cavity3": lambda: I.cavity_mesh(3, grouped=False),
    "channel4": lambda: I.channel_mesh(4, seed=1),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("features", [12, 24])
def test_one_level_hierarchy_matches_oracle(case, features):
    m = CASES[case]()
    h = omesh.Hierarchy(m["xyz"], m["cells"], m["vertex_bc"])
    lib = capi.HostHierarchy(m, features=features, patch_levels=1)
    assert lib.sizes["n_patches"] == h.n_patches and lib.sizes["n_fine_nodes"] == h.n_fine
    assert lib.sizes["n_in"] == 216 + features and lib.sizes["n_out"] == 81 and lib.sizes["precision"] == -1
    assert np.array_equal(lib.data(capi.PATCH_MAP), h.patch_map)
    assert np.array_equal(lib.data(capi.VALENCE), h.mult)
    assert np.array_equal(lib.data(capi.FINE_KIND), h.bc_f)
    assert np.allclose(lib.data(capi.FINE_XYZ), h.xyz_f, rtol=0, atol=1e-15)
    g = h.geometry(features)
    assert np.allclose(lib.data(capi.GEOMETRY), g, rtol=1e-13, atol=1e-14)
    assert np.allclose(lib.data(capi.EDGE_LENGTHS), g[:, :12], rtol=1e-13, atol=1e-14)
    lib.close()


@pytest.mark.parametrize("case", ["cavity4_jitter", "channel4"])
def test_two_level_hierarchy_matches_oracle(case):
    m = CASES[case]()
    h2 = omesh.Hierarchy2(m["xyz"], m["cells"], m["vertex_bc"])
    lib = capi.HostHierarchy(m, features=24, patch_levels=2)
    assert lib.sizes["n_in"] == 1024 and lib.sizes["n_out"] == 375 and lib.sizes["n_in_padded"] == 1024
    assert np.array_equal(lib.data(capi.PATCH_MAP), h2.patch_map)
    assert np.array_equal(lib.data(capi.VALENCE), h2.mult)
    assert np.array_equal(lib.data(capi.FINE_KIND), h2.bc_f)
    assert np.allclose(lib.data(capi.FINE_XYZ), h2.xyz_f, rtol=0, atol=1e-15)
    assert np.allclose(lib.data(capi.GEOMETRY), h2.geometry(24), rtol=1e-13, atol=1e-14)
    lib.close()


def test_invalid_meshes_and_arguments_are_refused():
    m = I.cavity_mesh(2)
    with pytest.raises(capi.DnnmgError) as e:
        capi.HostHierarchy(m, features=13)
    assert e.value.status == -1
    with pytest.raises(capi.DnnmgError):
        capi.HostHierarchy(m, patch_levels=3)
    bad = dict(m, cells=np.array(m["cells"]).copy())
    bad["cells"][0, 0] = len(m["xyz"])                  # a vertex index past the end
    with pytest.raises(capi.DnnmgError):
        capi.HostHierarchy(bad)
    twice = dict(m, cells=np.array(m["cells"]).copy())
    twice["cells"][0, 1] = twice["cells"][0, 0]         # a repeated vertex
    with pytest.raises(capi.DnnmgError):
        capi.HostHierarchy(twice)


def test_multigrid_levels_of_nested_meshes():
    # the solver's coarsening (parents of the 27-node groups) recovers every
    # level of a nested mesh; level L+1 coarsens to level L first
    # (a coarser level needs 8 nodes of free velocity: the cavity stops at 4^3,
    # as 2^3 has only its centre)
    m = I.cavity_mesh(8, levels=3)
    h = capi.HostHierarchy(m)
    assert h.mg_nodes(0, 16) == [729, 125]
    assert h.mg_nodes(0, 1) == [729, 125]
    assert h.mg_nodes(0, 0) == [729]
    assert h.mg_nodes(1, 16) == [17 ** 3, 729, 125]
    assert h.mg_nodes(1, 0) == [17 ** 3]
    h.close()
    m = I.channel_mesh(8, seed=0, levels=2)
    nv = [m.n_vertices]
    cells = m["cells"]
    for _ in range(2):
        g = cells.reshape(-1, 8, 8)
        cells = np.stack([g[:, K, K] for K in range(8)], axis=1)
        nv.append(int(cells.max()) + 1)
    h = capi.HostHierarchy(m)
    assert h.mg_nodes(0, 16) == nv
    h.close()
    # a mesh that is not nested has no level below L (and L+1 only L)
    m = I.channel_mesh(4, seed=1)
    h = capi.HostHierarchy(m)
    assert h.mg_nodes(0, 16) == [m.n_vertices]
    assert h.mg_nodes(1, 16) == [h.sizes["n_fine_nodes"], m.n_vertices]
    h.close()


def test_two_level_fine_level_multigrid_and_injection():
    # level L+2 of a J = 2 context over L = 4^3 (nested over 2^3): the solver
    # coarsens it through L+1 (9^3 nodes) and L (5^3); 3^3 has one free
    # velocity node and stops the hierarchy
    m = I.cavity_mesh(4, levels=1)
    j2 = capi.HostHierarchy(m, patch_levels=2)
    j1 = capi.HostHierarchy(m, patch_levels=1)
    assert j2.mg_nodes(level=capi.LEVEL_FINE) == [17 ** 3, 9 ** 3, 5 ** 3]
    # the first nodes of level L+2 are level L+1's, in the J = 1 numbering:
    # injection onto level L+1 is a prefix of the rows
    n1 = j1.sizes["n_fine_nodes"]
    assert np.array_equal(j2.data(capi.FINE_XYZ)[:n1], j1.data(capi.FINE_XYZ))
    assert np.array_equal(j2.data(capi.FINE_KIND)[:n1], j1.data(capi.FINE_KIND))
    # and on the nested channel: L+2 -> L+1 -> L -> L-1
    c = I.channel_mesh(4, seed=2, levels=1)
    c2 = capi.HostHierarchy(c, patch_levels=2)
    c1 = capi.HostHierarchy(c, patch_levels=1)
    nodes = c2.mg_nodes(level=capi.LEVEL_FINE)
    assert nodes[1] == c1.sizes["n_fine_nodes"] and nodes[2] == c["xyz"].shape[0] and len(nodes) == 4
    assert np.array_equal(c2.data(capi.FINE_XYZ)[:nodes[1]], c1.data(capi.FINE_XYZ))
    for h in (j2, j1, c2, c1):
        h.close()
