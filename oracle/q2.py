"""Q2/Q2 finite elements with one-level local projection stabilisation
(oracle), the discretisation the paper itself uses (Sec. 3.2).

TEST INFRASTRUCTURE ONLY, like the rest of this package.

Element: equal-order triquadratic velocity and pressure on hexahedra whose
geometry is the trilinear map of the cell's 8 vertices (the 27 nodes sit at
the trilinear images of (a/2, b/2, c/2), a, b, c in {0, 1, 2}; local node
iota = a + 3 b + 9 c).  The 1D Lagrange basis on the nodes 0, 1/2, 1 is
  L0 = 2 (x - 1/2)(x - 1),  L1 = -4 x (x - 1),  L2 = 2 x (x - 1/2)
and phi_iota = L_a(xi) L_b(eta) L_c(zeta).

Operator: the same theta-scheme as the Q1 oracle (Eqs. (6), (9); see
oracle.fem for the terms), with the stabilisation of Eq. (5) as the paper
states it: pi_h is the projection Q2 -> Q1 on each cell, here the Q1
interpolant at the cell's 8 vertices (a Q2 function with nodal values
sum_K w(vertex K) N_K(node)), kappa_h = id - pi_h, and
  s_h(x; phi) = sum_T delta_T (v.grad v - pi v.grad pi v, v.grad phi - pi v.grad pi phi)_T
  s_h(x; xi)  = sum_T alpha_T (grad(p - pi p), grad(xi - pi xi))_T
with alpha_T, delta_T of Eq. (8) (h_T = the cell's largest vertex distance,
|v|_inf,T = the largest Euclidean |v| over the cell's 27 nodes).  The terms
vanish for velocity and pressure in Q1 on every cell.

Integrals use the 3x3x3 Gauss rule on the reference cube.

Transfer: the refined mesh's Q2 space contains the coarse one (nested
trilinear geometry), so prolongation is evaluation of the coarse
triquadratic function at the fine nodes, (a/4, b/4, c/4) in the coarse
cell; restriction is its transpose.

Pinned by: the Lagrange property and exactness of the basis for
triquadratics, mass rows summing to the volume, exactness of the operator's
terms on polynomial fields, vanishing of the stabilisation on Q1 fields,
exact prolongation of coarse Q2 functions, complex-step Jacobian against
finite differences, and manufactured-solution convergence rates (velocity
L2 ~ h^3, H1 ~ h^2, pressure L2 ~ h^2); tests/test_oracle_q2.py.
"""
from __future__ import annotations

import numpy as np

from .fem import CORNERS, WPI, _diameter, gauss_points, q1_basis


def lagrange2(x):
    """Values [3] and derivatives [3] of the 1D quadratic Lagrange basis on
    the nodes 0, 1/2, 1 at x."""
    v = np.array([2.0 * (x - 0.5) * (x - 1.0), -4.0 * x * (x - 1.0), 2.0 * x * (x - 0.5)])
    d = np.array([4.0 * x - 3.0, 4.0 - 8.0 * x, 4.0 * x - 1.0])
    return v, d


def q2_basis(xi):
    """Values phi[27] and reference gradients dphi[27, 3] at xi in [0,1]^3."""
    (vx, dx), (vy, dy), (vz, dz) = (lagrange2(xi[d]) for d in range(3))
    phi = np.empty(27)
    dphi = np.empty((27, 3))
    for iota in range(27):
        a, b, c = iota % 3, (iota // 3) % 3, iota // 9
        phi[iota] = vx[a] * vy[b] * vz[c]
        dphi[iota] = (dx[a] * vy[b] * vz[c], vx[a] * dy[b] * vz[c], vx[a] * vy[b] * dz[c])
    return phi, dphi


_QP, _QW = gauss_points(3)
QW = np.array(_QW)                                        # [27] weights on [0,1]^3
PHI2 = np.array([q2_basis(p)[0] for p in _QP])            # [27 q, 27 i]
DPHI2 = np.array([q2_basis(p)[1] for p in _QP])           # [27 q, 27 i, 3]
DPHI1 = np.array([q1_basis(p)[1] for p in _QP])           # [27 q, 8 k, 3] (geometry)


def cell_geometry(X8):
    """det J [n, 27] and physical Q2 basis gradients [n, 27 q, 27 i, 3] at the
    Gauss points of cells with vertices X8 [n, 8, 3] (trilinear map)."""
    n = X8.shape[0]
    det = np.empty((n, 27))
    grads = np.empty((n, 27, 27, 3))
    for q in range(27):
        J = np.einsum("nkd,ke->nde", X8, DPHI1[q])           # dx_d / dxi_e
        det[:, q] = np.linalg.det(J)
        Jinv = np.linalg.inv(J)
        grads[:, q] = np.einsum("ie,ned->nid", DPHI2[q], Jinv)
    return det, grads


def cell_operator(X8, U, m, theta, nu):
    """Galerkin part of A_h per cell: [n, 27, 4] for nodal values U [n, 27, 4]."""
    det, G = cell_geometry(X8)
    R = np.zeros(U.shape, dtype=U.dtype)
    for q in range(27):
        w = QW[q] * det[:, q]
        phi, g = PHI2[q], G[:, q]
        v = np.einsum("i,nic->nc", phi, U[:, :, 0:3])
        p = np.einsum("i,ni->n", phi, U[:, :, 3])
        Dv = np.einsum("nic,nid->ncd", U[:, :, 0:3], g)
        conv = np.einsum("nd,ncd->nc", v, Dv)
        div = Dv[:, 0, 0] + Dv[:, 1, 1] + Dv[:, 2, 2]
        mom = (m * v[:, None, :] * phi[None, :, None]
               + theta * conv[:, None, :] * phi[None, :, None]
               + theta * nu * np.einsum("ncd,nid->nic", Dv, g)
               - p[:, None, None] * g)
        R[:, :, 0:3] += w[:, None, None] * mom
        R[:, :, 3] += w[:, None] * div[:, None] * phi[None, :]
    return R


def cell_rhs(X8, V, m, theta, nu, f_new=None, f_old=None):
    """b(v_old) per cell: [n, 27, 4] (pressure rows zero); V [n, 27, 3]."""
    det, G = cell_geometry(X8)
    B = np.zeros(V.shape[:2] + (4,), dtype=V.dtype)
    for q in range(27):
        w = QW[q] * det[:, q]
        phi, g = PHI2[q], G[:, q]
        v = np.einsum("i,nic->nc", phi, V)
        Dv = np.einsum("nic,nid->ncd", V, g)
        conv = np.einsum("nd,ncd->nc", v, Dv)
        val = (m * v[:, None, :] * phi[None, :, None]
               - (1.0 - theta) * (conv[:, None, :] * phi[None, :, None]
                                  + nu * np.einsum("ncd,nid->nic", Dv, g)))
        if f_new is not None:
            f = theta * np.einsum("i,nic->nc", phi, f_new)
            if f_old is not None:
                f = f + (1.0 - theta) * np.einsum("i,nic->nc", phi, f_old)
            val = val + f[:, None, :] * phi[None, :, None]
        B[:, :, 0:3] += w[:, None, None] * val
    return B


def cell_lps(X8, U, m, nu, alpha0, delta0, Vref=None):
    """Local projection terms per cell: [n, 27, 4] (pressure rows: alpha
    term, velocity rows: delta term).  pi_h U takes the vertex values to
    the 27 nodes with the trilinear weights; the test side's pi_h phi_a is
    the vertex function N_K for a = vertex K and 0 otherwise, so its part is
    gathered onto the vertex rows with the same weights."""
    PU = np.einsum("ik,nkc->nic", WPI, U[:, CORNERS, :])
    h = _diameter(X8)
    Vs = U if Vref is None else Vref
    vmax = np.max(np.sqrt(np.sum(np.real(Vs[:, :, 0:3]) ** 2, axis=2)), axis=1)
    denom = nu / h ** 2 + vmax / h + m
    aT, dT = alpha0 / denom, delta0 / denom
    det, G = cell_geometry(X8)
    sp = np.zeros(U.shape[:2], dtype=U.dtype)
    s1 = np.zeros(U.shape[:2] + (3,), dtype=U.dtype)
    s2 = np.zeros(U.shape[:2] + (3,), dtype=U.dtype)
    kp = U[:, :, 3] - PU[:, :, 3]
    for q in range(27):
        w = QW[q] * det[:, q]
        phi, g = PHI2[q], G[:, q]
        v = np.einsum("i,nic->nc", phi, U[:, :, 0:3])
        pv = np.einsum("i,nic->nc", phi, PU[:, :, 0:3])
        Dv = np.einsum("nic,nid->ncd", U[:, :, 0:3], g)
        Dpv = np.einsum("nic,nid->ncd", PU[:, :, 0:3], g)
        gkp = np.einsum("ni,nid->nd", kp, g)
        sp += (aT * w)[:, None] * np.einsum("nd,nad->na", gkp, g)
        gv = np.einsum("nd,ncd->nc", v, Dv) - np.einsum("nd,ncd->nc", pv, Dpv)
        s1 += (dT * w)[:, None, None] * gv[:, None, :] * np.einsum("nd,nad->na", v, g)[:, :, None]
        s2 += (dT * w)[:, None, None] * gv[:, None, :] * np.einsum("nd,nad->na", pv, g)[:, :, None]
    R = np.zeros(U.shape, dtype=U.dtype)
    R[:, :, 3] += sp
    R[:, CORNERS, 3] -= np.einsum("ak,na->nk", WPI, sp)
    R[:, :, 0:3] += s1
    R[:, CORNERS, 0:3] -= np.einsum("ak,nac->nkc", WPI, s2)
    return R


def cells_of_patches(patch_map):
    """The Q2 cells of a mesh refined once, from the patch map of a twice
    refined hierarchy [nc, 125] (node a + 5 b + 25 c): coarse cell P holds
    the fine cells (i, j, k) in {0, 1}^3 (order i + 2 j + 4 k) whose nodes
    are (2 i + a, 2 j + b, 2 k + c), a, b, c in {0, 1, 2}."""
    nc = patch_map.shape[0]
    cells = np.empty((nc, 8, 27), dtype=np.int64)
    for t in range(8):
        i, j, k = t & 1, (t >> 1) & 1, (t >> 2) & 1
        for iota in range(27):
            a, b, c = iota % 3, (iota // 3) % 3, iota // 9
            cells[:, t, iota] = patch_map[:, (2 * i + a) + 5 * (2 * j + b) + 25 * (2 * k + c)]
    return cells.reshape(8 * nc, 27)


class LevelQ2:
    """One Q2 mesh level: nodes xyz [n, 3], cells [nc, 27] (local node
    a + 3 b + 9 c), node boundary kinds [n] (0 interior, 1 no-slip, 2
    prescribed inflow / lid, 3 do-nothing).  The interface matches
    oracle.fem.Level, so oracle.solve.newton solves on it."""

    def __init__(self, xyz, cells, node_bc):
        self.xyz = np.asarray(xyz, dtype=np.float64)
        self.cells = np.asarray(cells, dtype=np.int64)
        self.bc = np.asarray(node_bc, dtype=np.int64)
        self.n = self.xyz.shape[0]
        self.X8 = self.xyz[self.cells[:, CORNERS]]
        self.dirichlet = (self.bc == 1) | (self.bc == 2)
        self.pressure_mean_zero = not np.any(self.bc == 3)

    def local_operator(self, U, prm):
        R = cell_operator(self.X8, U, prm["m"], prm["theta"], prm["nu"])
        if prm.get("lps", True):
            vref = prm.get("vref")
            R = R + cell_lps(self.X8, U, prm["m"], prm["nu"], prm["alpha0"], prm["delta0"],
                             None if vref is None else vref[self.cells])
        return R

    def operator(self, x, prm):
        Rl = self.local_operator(x[self.cells], prm)
        out = np.zeros((self.n, 4), dtype=Rl.dtype)
        np.add.at(out, self.cells.ravel(), Rl.reshape(-1, 4))
        return out

    def rhs(self, v_old, prm, f_new=None, f_old=None):
        Fn = None if f_new is None else f_new[self.cells]
        Fo = None if f_old is None else f_old[self.cells]
        Bl = cell_rhs(self.X8, v_old[self.cells], prm["m"], prm["theta"], prm["nu"], Fn, Fo)
        out = np.zeros((self.n, 4))
        np.add.at(out, self.cells.ravel(), Bl.reshape(-1, 4))
        out[self.dirichlet, 0:3] = 0.0
        return out

    def residual(self, x, F, prm):
        r = F - self.operator(x, prm)
        r[self.dirichlet, 0:3] = 0.0
        return r

    def jacobian(self, x, prm, h=1e-30):
        """dA_h/dx (stabilisation parameters frozen) by complex-step
        differentiation of the local contributions, [4n, 4n] sparse, unknown
        4 * node + component."""
        import scipy.sparse as sp
        nodes = self.cells
        U = x[nodes].astype(np.complex128)
        ndir = 4 * 27
        cols = []
        for d in range(ndir):     # |v|_inf takes the real part: the parameters stay frozen
            Up = U.copy()
            Up[:, d // 4, d % 4] += 1j * h
            cols.append(np.imag(self.local_operator(Up, prm)).reshape(U.shape[0], ndir) / h)
        Jl = np.stack(cols, axis=2)
        gdof = (4 * nodes[:, :, None] + np.arange(4)[None, None, :]).reshape(nodes.shape[0], ndir)
        rows = np.repeat(gdof[:, :, None], ndir, axis=2)
        colm = np.repeat(gdof[:, None, :], ndir, axis=1)
        return sp.csr_matrix((Jl.ravel(), (rows.ravel(), colm.ravel())), shape=(4 * self.n, 4 * self.n))

    def lumped_mass(self):
        """The integral of each basis function."""
        det, _ = cell_geometry(self.X8)
        ml = np.einsum("nq,qi->ni", QW[None, :] * det, PHI2)
        out = np.zeros(self.n)
        np.add.at(out, self.cells.ravel(), ml.ravel())
        return out

    def evaluate(self, x, xi):
        """Values [nc, 4] of the nodal field x [n, 4] at reference point xi
        of every cell, and the physical points [nc, 3]."""
        phi, _ = q2_basis(xi)
        phi1, _ = q1_basis(xi)
        return np.einsum("i,nic->nc", phi, x[self.cells]), np.einsum("k,nkd->nd", phi1, self.X8)


def coarse_level(hier):
    """The Q2 level on a mesh: its nodes are those of the mesh refined once
    (hier = oracle.mesh.Hierarchy of the mesh), its cells the coarse cells
    with their 27 patch nodes."""
    return LevelQ2(hier.xyz_f, hier.patch_map, hier.bc_f)


def fine_level(hier2):
    """The Q2 level on the refined mesh (hier2 = oracle.mesh.Hierarchy2 of
    the coarse mesh: the nodes of two refinements)."""
    return LevelQ2(hier2.xyz_f, cells_of_patches(hier2.patch_map), hier2.bc_f)


def prolongate(hier, hier2, xc):
    """P x: the coarse Q2 field xc [n_coarse_q2, k] (nodes of hier's fine
    level) evaluated at the Q2 nodes of the refined mesh (hier2's fine
    level).  Each fine node is set from a coarse cell containing it; the
    field is continuous, so every such cell gives the same value."""
    out = np.zeros((hier2.n_fine,) + xc.shape[1:], dtype=xc.dtype)
    Uc = xc[hier.patch_map]                                  # [nc, 27, k]
    for iota in range(125):
        a, b, c = iota % 5, (iota // 5) % 5, iota // 25
        phi, _ = q2_basis((a / 4.0, b / 4.0, c / 4.0))
        out[hier2.patch_map[:, iota]] = np.einsum("i,ni...->n...", phi, Uc)
    return out


def prolongation_matrix(hier, hier2):
    """P as a sparse [n_fine_q2, n_coarse_q2] matrix (rows set once per fine
    node, from the first coarse cell that contains it)."""
    import scipy.sparse as sp
    nf, ncq = hier2.n_fine, hier.n_fine
    rows, cols, vals = [], [], []
    seen = np.zeros(nf, dtype=bool)
    for P in range(hier.patch_map.shape[0]):
        for iota in range(125):
            j = hier2.patch_map[P, iota]
            if seen[j]:
                continue
            seen[j] = True
            a, b, c = iota % 5, (iota // 5) % 5, iota // 25
            phi, _ = q2_basis((a / 4.0, b / 4.0, c / 4.0))
            for i in np.flatnonzero(np.abs(phi) > 0):
                rows.append(j)
                cols.append(hier.patch_map[P, i])
                vals.append(phi[i])
    return sp.csr_matrix((vals, (rows, cols)), shape=(nf, ncq))


# ---- DNN-MG with Q2 elements (Alg. 1 on the paper's element) ----------------
#
# The coarse level is Q2 on the mesh (nodes: the mesh refined once, hier);
# the fine level L+1 is Q2 on the refined mesh (nodes: the mesh refined
# twice, hier2).  A patch is a coarse cell with its 125 fine Q2 nodes, the
# node set and order of a two-level patch, so the local restriction Q and
# the extension L are those of oracle.dnnmg applied to hier2.

def restrict(hier, hier2, b_fine):
    """R b = P^T b, then zero velocity rows at coarse Dirichlet nodes."""
    P = prolongation_matrix(hier, hier2)
    out = np.asarray(P.T @ b_fine)
    dirc = (hier.bc_f == 1) | (hier.bc_f == 2)
    out[dirc, 0:3] = 0.0
    return out


def hot_path_step(hier, hier2, net, x_coarse, F, prm, fine=None, features=12):
    """The patch-correction steps of Alg. 1 with Q2 elements: x~ = P x^L,
    r = F - A_{L+1}(x~), X = Q(x~) | Q(r) | geometry, Y = N(X),
    d = L(Y), b = Rhs(v~ + d), b^L = R b.  Every intermediate as a dict."""
    from . import dnnmg, mlp
    lev = fine if fine is not None else fine_level(hier2)
    x_f = prolongate(hier, hier2, x_coarse)
    r = lev.residual(x_f, F, prm)
    X = dnnmg.gather(hier2, x_f, r, features)
    Ws, ss, ts, skip = net
    Y = mlp.forward(X, Ws, ss, ts, skip=skip)
    d = dnnmg.extend(hier2, Y)
    b_f = lev.rhs(x_f[:, 0:3] + d, prm)
    return dict(x_fine=x_f, r=r, X=X, Y=Y, d=d, b_fine=b_f, b_coarse=restrict(hier, hier2, b_f))


def run(hier, hier2, net, x0, n_steps, prm, bc_values, newton_tol=1e-13, features=12):
    """DNN-MG time stepping with Q2 elements: Newton on the coarse Q2 level,
    then the patch correction on the fine one.  x0 [n_coarse_q2, 4];
    bc_values(t) -> [n_coarse_q2, 3].  Returns the coarse states."""
    from .solve import newton
    coarse, fine = coarse_level(hier), fine_level(hier2)
    x = np.array(x0, dtype=np.float64)
    F = fine.rhs(prolongate(hier, hier2, x[:, 0:3]), prm)
    b = restrict(hier, hier2, F)
    states = []
    for n in range(1, n_steps + 1):
        t = n / prm["m"] if prm["m"] > 0 else float(n)
        xi = x.copy()
        xi[coarse.dirichlet, 0:3] = bc_values(t)[coarse.dirichlet]
        x, _ = newton(coarse, xi, b, prm, tol=newton_tol)
        states.append(x.copy())
        last = hot_path_step(hier, hier2, net, x, F, prm, fine=fine, features=features)
        F, b = last["b_fine"], last["b_coarse"]
    return states


def run_plain(hier, x0, n_steps, prm, bc_values, newton_tol=1e-13):
    """The plain Q2 scheme on the coarse level: rhs b_L(v_{n-1}) each step."""
    from .solve import newton
    coarse = coarse_level(hier)
    x = np.array(x0, dtype=np.float64)
    states = []
    for n in range(1, n_steps + 1):
        t = n / prm["m"] if prm["m"] > 0 else float(n)
        b = coarse.rhs(x[:, 0:3], prm)
        xi = x.copy()
        xi[coarse.dirichlet, 0:3] = bc_values(t)[coarse.dirichlet]
        x, _ = newton(coarse, xi, b, prm, tol=newton_tol)
        states.append(x.copy())
    return states
