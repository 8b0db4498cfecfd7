"""Uniform refinement of a hexahedral mesh and the patch data of DNN-MG.

A patch is one cell M of the coarse level L together with its 8 children on
level L+1 (the J = 1 patch of Sec. 5.2).  Its 27 fine nodes carry the local
index  iota = a + 3 b + 9 c,  (a, b, c) in {0,1,2}^3  along the coarse cell's
reference axes; the map dof(P, iota) of Sec. 5.2 is ``patch_map[P, iota]``.

Fine node numbering (hierarchical): the coarse vertices keep their numbers;
then one node per coarse edge, per coarse face and per coarse cell, each
numbered in order of first appearance when the cells are visited in order and
their edges / faces in the local order below.

Boundary kinds of fine nodes: vertices keep their kind; a coarse boundary
face (a face of exactly one cell) takes the lowest-priority kind among its
four vertices, with priority outflow(3) < wall(1) < driven(2); a fine node
on a boundary edge takes the highest-priority kind among the boundary faces
containing that edge; a face-centre node takes its face's kind; all other
nodes are interior (0).

Pinned by: closed-form valences and node counts on n^3 meshes, the
sum of valences = 27 N_c, brute-force containment counts, and exact
reproduction of trilinear fields through the prolongation.
"""
from __future__ import annotations

import numpy as np

# local edges (pairs of local vertices), xi-edges then eta-edges then zeta-edges
LOCAL_EDGES = ((0, 1), (2, 3), (4, 5), (6, 7),
               (0, 2), (1, 3), (4, 6), (5, 7),
               (0, 4), (1, 5), (2, 6), (3, 7))
# local faces, vertices listed lexicographically in the two free coordinates
LOCAL_FACES = ((0, 2, 4, 6), (1, 3, 5, 7),
               (0, 1, 4, 5), (2, 3, 6, 7),
               (0, 1, 2, 3), (4, 5, 6, 7))

_RANK = {3: 0, 1: 1, 2: 2}
_UNRANK = {0: 3, 1: 1, 2: 2}


def local_entity(iota: int):
    """Which coarse entity patch node ``iota`` sits on: ('v', k), ('e', e),
    ('f', f) or ('c', 0), with k / e / f local indices."""
    a, b, c = iota % 3, (iota // 3) % 3, iota // 9
    ones = (a == 1) + (b == 1) + (c == 1)
    if ones == 0:
        return ("v", a // 2 + 2 * (b // 2) + 4 * (c // 2))
    if ones == 1:
        if a == 1:
            return ("e", 0 + b // 2 + 2 * (c // 2))
        if b == 1:
            return ("e", 4 + a // 2 + 2 * (c // 2))
        return ("e", 8 + a // 2 + 2 * (b // 2))
    if ones == 2:
        if a != 1:
            return ("f", 0 + a // 2)
        if b != 1:
            return ("f", 2 + b // 2)
        return ("f", 4 + c // 2)
    return ("c", 0)


def corner_weights(iota: int) -> np.ndarray:
    """Trilinear weights of the 8 coarse corners at patch node ``iota``
    (its reference point is (a/2, b/2, c/2))."""
    a, b, c = iota % 3, (iota // 3) % 3, iota // 9
    p = (a / 2.0, b / 2.0, c / 2.0)
    w = np.empty(8)
    for k in range(8):
        bits = (k & 1, (k >> 1) & 1, (k >> 2) & 1)
        w[k] = np.prod([p[d] if bits[d] else 1.0 - p[d] for d in range(3)])
    return w


def child_nodes():
    """CH[t][a]: patch index of vertex a of child cell t = i + 2 j + 4 k."""
    CH = np.empty((8, 8), dtype=np.int64)
    for t in range(8):
        i, j, k = t & 1, (t >> 1) & 1, (t >> 2) & 1
        for a in range(8):
            di, dj, dk = a & 1, (a >> 1) & 1, (a >> 2) & 1
            CH[t, a] = (i + di) + 3 * (j + dj) + 9 * (k + dk)
    return CH


class Hierarchy:
    """Coarse mesh (level L) and its uniform refinement (level L+1)."""

    def __init__(self, xyz, cells, vertex_bc):
        xyz = np.asarray(xyz, dtype=np.float64)
        cells = np.asarray(cells, dtype=np.int64)
        vertex_bc = np.asarray(vertex_bc, dtype=np.int64)
        nv, nc = xyz.shape[0], cells.shape[0]
        self.xyz_c, self.cells_c, self.bc_c = xyz, cells, vertex_bc
        self.n_coarse_vertices, self.n_patches = nv, nc

        # -- boundary faces of the coarse mesh
        face_count: dict = {}
        for c in range(nc):
            for f in LOCAL_FACES:
                key = tuple(sorted(int(cells[c, k]) for k in f))
                face_count[key] = face_count.get(key, 0) + 1
        bface_kind: dict = {}
        for key, cnt in face_count.items():
            if cnt == 1:
                ks = [int(vertex_bc[v]) for v in key]
                if min(ks) == 0:
                    raise ValueError("boundary face with an interior-marked vertex")
                bface_kind[key] = _UNRANK[min(_RANK[k] for k in ks)]
        bedge_kind: dict = {}
        for c in range(nc):
            for f in LOCAL_FACES:
                key = tuple(sorted(int(cells[c, k]) for k in f))
                if key not in bface_kind:
                    continue
                fk = bface_kind[key]
                v = [int(cells[c, k]) for k in f]
                for (p, q) in ((v[0], v[1]), (v[2], v[3]), (v[0], v[2]), (v[1], v[3])):
                    e = (min(p, q), max(p, q))
                    old = bedge_kind.get(e)
                    if old is None or _RANK[fk] > _RANK[old]:
                        bedge_kind[e] = fk

        # -- number edges, faces, cells in order of first appearance
        edge_id: dict = {}
        edge_par: list = []
        for c in range(nc):
            for (p, q) in LOCAL_EDGES:
                a, b = int(cells[c, p]), int(cells[c, q])
                key = (min(a, b), max(a, b))
                if key not in edge_id:
                    edge_id[key] = nv + len(edge_par)
                    edge_par.append((a, b))
        ne = len(edge_par)
        face_id: dict = {}
        face_par: list = []
        for c in range(nc):
            for f in LOCAL_FACES:
                vs = tuple(int(cells[c, k]) for k in f)
                key = tuple(sorted(vs))
                if key not in face_id:
                    face_id[key] = nv + ne + len(face_par)
                    face_par.append(vs)
        nf = len(face_par)
        self.n_edges, self.n_faces = ne, nf
        n_fine = nv + ne + nf + nc
        self.n_fine = n_fine

        # -- patch map dof(P, iota)
        pm = np.empty((nc, 27), dtype=np.int64)
        for c in range(nc):
            for iota in range(27):
                kind, idx = local_entity(iota)
                if kind == "v":
                    pm[c, iota] = cells[c, idx]
                elif kind == "e":
                    p, q = LOCAL_EDGES[idx]
                    a, b = int(cells[c, p]), int(cells[c, q])
                    pm[c, iota] = edge_id[(min(a, b), max(a, b))]
                elif kind == "f":
                    key = tuple(sorted(int(cells[c, k]) for k in LOCAL_FACES[idx]))
                    pm[c, iota] = face_id[key]
                else:
                    pm[c, iota] = nv + ne + nf + c
        self.patch_map = pm

        # -- parents (coarse vertices a fine node interpolates from)
        parents = [None] * n_fine
        for v in range(nv):
            parents[v] = (v,)
        for i, (a, b) in enumerate(edge_par):
            parents[nv + i] = (a, b)
        for i, vs in enumerate(face_par):
            parents[nv + ne + i] = vs
        for c in range(nc):
            parents[nv + ne + nf + c] = tuple(int(v) for v in cells[c])
        self.parents = parents

        # -- fine coordinates: mean of the parents' coordinates
        xf = np.empty((n_fine, 3))
        for j, par in enumerate(parents):
            s = np.zeros(3)
            for v in par:
                s = s + xyz[v]
            xf[j] = s / len(par)
        self.xyz_f = xf

        # -- valence (multiplicity): number of patches containing each node
        mult = np.zeros(n_fine, dtype=np.int64)
        for c in range(nc):
            for iota in range(27):
                mult[pm[c, iota]] += 1
        self.mult = mult

        # -- boundary kinds of fine nodes
        kind = np.zeros(n_fine, dtype=np.int64)
        kind[:nv] = vertex_bc
        for i, (a, b) in enumerate(edge_par):
            kind[nv + i] = bedge_kind.get((min(a, b), max(a, b)), 0)
        for i, vs in enumerate(face_par):
            kind[nv + ne + i] = bface_kind.get(tuple(sorted(vs)), 0)
        self.bc_f = kind

        # -- fine cells: child t = i + 2 j + 4 k of patch c is cell 8 c + t
        CH = child_nodes()
        self.cells_f = np.empty((8 * nc, 8), dtype=np.int64)
        for c in range(nc):
            for t in range(8):
                self.cells_f[8 * c + t] = pm[c, CH[t]]

    # ------------------------------------------------------------------
    def dirichlet_fine(self) -> np.ndarray:
        """True at fine nodes whose velocity is prescribed (kinds 1 and 2)."""
        return (self.bc_f == 1) | (self.bc_f == 2)

    def dirichlet_coarse(self) -> np.ndarray:
        return (self.bc_c == 1) | (self.bc_c == 2)

    def edge_lengths(self) -> np.ndarray:
        """Geometry input h^c of Sec. 5.2 (network inputs): the 12 edge lengths of each coarse
        cell, in LOCAL_EDGES order.  [N_c, 12]"""
        out = np.empty((self.n_patches, 12))
        for c in range(self.n_patches):
            for e, (p, q) in enumerate(LOCAL_EDGES):
                d = self.xyz_c[self.cells_c[c, q]] - self.xyz_c[self.cells_c[c, p]]
                out[c, e] = np.sqrt(np.sum(d * d))
        return out

    def diagonals(self) -> np.ndarray:
        """The 4 diagonals of each coarse cell that join vertices sharing no
        face (Sec. 5.2, network inputs): vertex k to vertex 7 - k, k = 0..3.
        [N_c, 4]"""
        out = np.empty((self.n_patches, 4))
        for c in range(self.n_patches):
            X = self.xyz_c[self.cells_c[c]]
            for k in range(4):
                out[c, k] = np.linalg.norm(X[7 - k] - X[k])
        return out

    def face_angles(self) -> np.ndarray:
        """For each vertex of each coarse cell the mean of the 3 angles
        between the cell's faces that meet at the vertex (Sec. 5.2, network
        inputs), in radians.  Two faces through vertex v share one of the
        three edges e at v; their angle is the angle between their normals at
        v, e x u and e x w, where u and w are the other two edges at v (the
        interior angle: u and w point into the cell's side of each face).
        [N_c, 8], vertex order k = 0..7."""
        out = np.empty((self.n_patches, 8))
        for c in range(self.n_patches):
            X = self.xyz_c[self.cells_c[c]]
            for v in range(8):
                edges = [X[v ^ (1 << a)] - X[v] for a in range(3)]
                angles = []
                for a in range(3):
                    e, u, w = edges[a], edges[(a + 1) % 3], edges[(a + 2) % 3]
                    n1, n2 = np.cross(e, u), np.cross(e, w)
                    cs = np.dot(n1, n2) / (np.linalg.norm(n1) * np.linalg.norm(n2))
                    angles.append(np.arccos(np.clip(cs, -1.0, 1.0)))
                out[c, v] = np.mean(angles)
        return out

    def geometry(self, n_features: int = 12) -> np.ndarray:
        """Geometry part of the network input row: the 12 edge lengths, or
        with n_features = 24 the edge lengths, the 4 diagonals and the 8 mean
        face angles (the three kinds of Sec. 5.2; Table 2's N_in = 240 =
        2 x 108 + 24).  [N_c, n_features]"""
        if n_features == 12:
            return self.edge_lengths()
        if n_features == 24:
            return np.concatenate([self.edge_lengths(), self.diagonals(), self.face_angles()], axis=1)
        raise ValueError("n_features must be 12 or 24")

    def fine_mesh(self) -> dict:
        """Level L+1 as a mesh in the same format as the input (cells come in
        patch groups of 8 children)."""
        return dict(xyz=self.xyz_f, cells=self.cells_f, vertex_bc=self.bc_f,
                    patch_groups=True)


class Hierarchy2:
    """Patches of J = 2 (Sec. 5.2): each coarse cell of level L with the
    64 cells and 125 nodes of its twofold refinement.  Level L+2 is level
    L+1 (``Hierarchy``, with its fine cells as the mesh: cell 8 P + t is
    child t of coarse cell P) refined once more by the same rules, so its
    node numbering, boundary kinds and cell grouping follow from those of
    one refinement.  The patch node iota = a + 5 b + 25 c, (a, b, c) in
    {0..4}^3 along the coarse cell's reference axes, is node (a - 2 i,
    b - 2 j, c - 2 k) of child (i, j, k), i = min(a // 2, 1) etc. (nodes on
    the children's common faces are the same node in either child).

    Pinned by the same closed forms as ``Hierarchy`` (node counts, valences,
    trilinear node positions) on twofold refinements; see
    tests/test_oracle_mesh.py."""

    J = 2

    def __init__(self, xyz, cells, vertex_bc):
        self.h1 = Hierarchy(xyz, cells, vertex_bc)
        self.h2 = Hierarchy(self.h1.xyz_f, self.h1.cells_f, self.h1.bc_f)
        self.levels = (self.h1, self.h2)
        h1, h2 = self.h1, self.h2
        self.n_patches = h1.n_patches
        self.n_coarse_vertices = h1.n_coarse_vertices
        self.xyz_c, self.cells_c = h1.xyz_c, h1.cells_c
        self.n_fine = h2.n_fine
        self.xyz_f, self.cells_f, self.bc_f = h2.xyz_f, h2.cells_f, h2.bc_f
        nc = self.n_patches
        pm = np.empty((nc, 125), dtype=np.int64)
        for P in range(nc):
            for iota in range(125):
                a, b, c = iota % 5, (iota // 5) % 5, iota // 25
                i, j, k = min(a // 2, 1), min(b // 2, 1), min(c // 2, 1)
                child = i + 2 * j + 4 * k
                local = (a - 2 * i) + 3 * (b - 2 * j) + 9 * (c - 2 * k)
                pm[P, iota] = h2.patch_map[8 * P + child, local]
        self.patch_map = pm
        self.mult = np.bincount(pm.ravel(), minlength=self.n_fine)

    def dirichlet_fine(self) -> np.ndarray:
        return self.h2.dirichlet_fine()

    def dirichlet_coarse(self) -> np.ndarray:
        return self.h1.dirichlet_coarse()

    def edge_lengths(self) -> np.ndarray:
        return self.h1.edge_lengths()

    def geometry(self, n_features: int = 12) -> np.ndarray:
        return self.h1.geometry(n_features)

    def fine_mesh(self) -> dict:
        return self.h2.fine_mesh()

