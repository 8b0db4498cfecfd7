"""Q1/Q1 finite elements with local projection stabilisation (oracle).

Reading of the paper used here: the paper discretises with equal-order Q2/Q2
and a projection pi_h : Q2 -> Q1 on each cell (Sec. 3.2, Eq. (5)).  The hot path of
this project uses equal-order Q1/Q1 on a mesh whose cells come in groups of 8
children of a parent cell; pi_h is then the interpolation onto Q1 of the
parent cell (the two-level local projection of the works cited in Sec. 3.2),
defined nodally: (pi_h w)(node) = sum over the parent's 8 corners K of
w(corner K) * trilinear weight of K at the node.  A group of 8 children has
the same 27 nodes as one Q2 cell, so this is the Q1 analogue of the paper's
construction.

The discrete operator A_h of Eqs. (6) and (9) (theta-scheme, theta = 1/2 is the
paper's Crank-Nicolson, theta = 1 backward Euler), per velocity test
function phi e_c and pressure test function xi:

  A_c(x; phi) = m (v, phi)_c + theta (v.grad v, phi)_c
                + theta nu (grad v_c, grad phi) - (p, d_c phi)
                + sum_T delta_T (v.grad v - pi v.grad pi v, v.grad phi - pi v.grad pi phi)_c
  A_p(x; xi)  = (div v, xi) + sum_T alpha_T (grad(p - pi p), grad(xi - pi xi))

with m = 1/k.  The right-hand side b(v_old) of Eq. (6):

  b_c(phi) = m (v_old, phi)_c - (1-theta) [(v_old.grad v_old, phi)_c
              + nu (grad v_old_c, grad phi)] + (theta f_new + (1-theta) f_old, phi)_c
  b_p = 0.

The stabilisation parameters of Eq. (8):
  alpha_T = alpha0 / (nu/h_T^2 + |v|_inf,T / h_T + m),  delta_T likewise with delta0;
h_T = largest distance between two vertices of T, |v|_inf,T = largest
Euclidean |v| over T's nodes (from the real part, i.e. frozen under complex
differentiation, as the paper freezes them in the Jacobian).

Integrals use the 2x2x2 Gauss rule on the reference cube [0,1]^3 and the
trilinear map of each cell; f is the nodal interpolant (f_h of Sec. 3.2).

Pinned by: manufactured-solution convergence rates (velocity L2 ~ h^2,
H1 ~ h, pressure L2 ~ h), complex-step Jacobian vs finite differences of the
global residual on a 4^3 mesh, closed forms (sum of mass rows = volume,
constant fields in the stiffness kernel), and the vanishing of the
stabilisation on prolongated fields.
"""
from __future__ import annotations

import math

import numpy as np

from .mesh import child_nodes, corner_weights

_g = 0.5 / math.sqrt(3.0)
GAUSS_1D = (0.5 - _g, 0.5 + _g)
GAUSS_W = 1.0 / 8.0          # weight of each of the 8 points on [0,1]^3


def q1_basis(xi):
    """Values phi[8] and reference gradients dphi[8, 3] at xi in [0,1]^3."""
    phi = np.empty(8)
    dphi = np.empty((8, 3))
    for k in range(8):
        bits = (k & 1, (k >> 1) & 1, (k >> 2) & 1)
        f = [xi[d] if bits[d] else 1.0 - xi[d] for d in range(3)]
        df = [1.0 if bits[d] else -1.0 for d in range(3)]
        phi[k] = f[0] * f[1] * f[2]
        dphi[k, 0] = df[0] * f[1] * f[2]
        dphi[k, 1] = f[0] * df[1] * f[2]
        dphi[k, 2] = f[0] * f[1] * df[2]
    return phi, dphi


def gauss_points(n1d=2):
    if n1d == 2:
        pts1, w1 = GAUSS_1D, (0.5, 0.5)
    elif n1d == 3:
        s = 0.5 * math.sqrt(3.0 / 5.0)
        pts1, w1 = (0.5 - s, 0.5, 0.5 + s), (5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0)
    else:
        raise ValueError(n1d)
    pts, ws = [], []
    for c in range(n1d):
        for b in range(n1d):
            for a in range(n1d):
                pts.append((pts1[a], pts1[b], pts1[c]))
                ws.append(w1[a] * w1[b] * w1[c])
    return pts, ws


_QP, _QW = gauss_points(2)
PHI = np.array([q1_basis(p)[0] for p in _QP])      # [8 q, 8 k]
DPHI = np.array([q1_basis(p)[1] for p in _QP])     # [8 q, 8 k, 3]


def cell_geometry(X, dphi=DPHI):
    """Per quadrature point: det J [n, nq] and physical basis gradients
    [n, nq, 8, 3] for cells with vertex coordinates X [n, 8, 3]."""
    nq = dphi.shape[0]
    det = np.empty((X.shape[0], nq))
    grads = np.empty((X.shape[0], nq, 8, 3))
    for q in range(nq):
        J = np.einsum("nkd,ke->nde", X, dphi[q])          # J[d, e] = dx_d / dxi_e
        det[:, q] = np.linalg.det(J)
        Jinv = np.linalg.inv(J)                          # Jinv[e, d] = dxi_e / dx_d
        grads[:, q] = np.einsum("ke,ned->nkd", dphi[q], Jinv)
    return det, grads


def cell_operator(X, U, m, theta, nu):
    """Galerkin part of A_h on each cell: [n, 8, 4] local contributions for
    cells X [n, 8, 3] with nodal values U [n, 8, 4] = (u, v, w, p)."""
    det, G = cell_geometry(X)
    R = np.zeros(U.shape, dtype=U.dtype)
    for q in range(8):
        w = GAUSS_W * det[:, q]
        phi, g = PHI[q], G[:, q]
        v = np.einsum("k,nkc->nc", phi, U[:, :, 0:3])
        p = np.einsum("k,nk->n", phi, U[:, :, 3])
        Dv = np.einsum("nkc,nkd->ncd", U[:, :, 0:3], g)   # Dv[c, d] = dv_c/dx_d
        conv = np.einsum("nd,ncd->nc", v, Dv)
        div = Dv[:, 0, 0] + Dv[:, 1, 1] + Dv[:, 2, 2]
        mom = (m * v[:, None, :] * phi[None, :, None]
               + theta * conv[:, None, :] * phi[None, :, None]
               + theta * nu * np.einsum("ncd,nkd->nkc", Dv, g)
               - p[:, None, None] * g)
        R[:, :, 0:3] += w[:, None, None] * mom
        R[:, :, 3] += w[:, None] * div[:, None] * phi[None, :]
    return R


def cell_rhs(X, V, m, theta, nu, f_new=None, f_old=None):
    """b(v_old) on each cell: [n, 8, 4] (pressure rows zero).  V [n, 8, 3]
    is the old velocity, f_new / f_old [n, 8, 3] nodal forces or None."""
    det, G = cell_geometry(X)
    B = np.zeros(V.shape[:2] + (4,), dtype=V.dtype)
    for q in range(8):
        w = GAUSS_W * det[:, q]
        phi, g = PHI[q], G[:, q]
        v = np.einsum("k,nkc->nc", phi, V)
        Dv = np.einsum("nkc,nkd->ncd", V, g)
        conv = np.einsum("nd,ncd->nc", v, Dv)
        val = (m * v[:, None, :] * phi[None, :, None]
               - (1.0 - theta) * (conv[:, None, :] * phi[None, :, None]
                                  + nu * np.einsum("ncd,nkd->nkc", Dv, g)))
        if f_new is not None:
            f = theta * np.einsum("k,nkc->nc", phi, f_new)
            if f_old is not None:
                f = f + (1.0 - theta) * np.einsum("k,nkc->nc", phi, f_old)
            val = val + f[:, None, :] * phi[None, :, None]
        B[:, :, 0:3] += w[:, None, None] * val
    return B


CH = child_nodes()                                   # [8 children, 8 vertices]
CORNERS = np.array([2 * (k & 1) + 6 * ((k >> 1) & 1) + 18 * ((k >> 2) & 1) for k in range(8)])
WPI = np.array([corner_weights(i) for i in range(27)])  # [27, 8]


def _diameter(X):
    d = np.zeros(X.shape[0])
    for a in range(8):
        for b in range(a + 1, 8):
            d = np.maximum(d, np.sqrt(np.sum((X[:, a] - X[:, b]) ** 2, axis=1)))
    return d


def group_lps(Xg, Ug, m, nu, alpha0, delta0, Vref=None):
    """Local projection terms of A_h for groups of 8 children.

    Xg [n, 27, 3], Ug [n, 27, 4]: coordinates and values at the 27 group
    nodes.  Returns [n, 27, 4] contributions (pressure row: alpha term,
    velocity rows: delta term).  The parameters alpha_T, delta_T take
    |v|_inf from Vref [n, 27, 4] when given (frozen), else from Ug."""
    Uc = Ug[:, CORNERS, :]
    PU = np.einsum("ik,nkc->nic", WPI, Uc)            # pi_h U at the 27 nodes
    R = np.zeros(Ug.shape, dtype=Ug.dtype)
    for t in range(8):
        idx = CH[t]
        X, U, P = Xg[:, idx], Ug[:, idx], PU[:, idx]
        h = _diameter(X)
        Vs = U if Vref is None else Vref[:, idx]
        vmax = np.max(np.sqrt(np.sum(np.real(Vs[:, :, 0:3]) ** 2, axis=2)), axis=1)
        denom = nu / h ** 2 + vmax / h + m
        aT, dT = alpha0 / denom, delta0 / denom
        WK = WPI[idx]                                  # [8 a, 8 K]
        det, G = cell_geometry(X)
        sp = np.zeros(U.shape[:2], dtype=U.dtype)
        s1 = np.zeros(U.shape[:2] + (3,), dtype=U.dtype)
        s2 = np.zeros(U.shape[:2] + (3,), dtype=U.dtype)
        kp = U[:, :, 3] - P[:, :, 3]
        for q in range(8):
            w = GAUSS_W * det[:, q]
            phi, g = PHI[q], G[:, q]
            v = np.einsum("k,nkc->nc", phi, U[:, :, 0:3])
            pv = np.einsum("k,nkc->nc", phi, P[:, :, 0:3])
            Dv = np.einsum("nkc,nkd->ncd", U[:, :, 0:3], g)
            Dpv = np.einsum("nkc,nkd->ncd", P[:, :, 0:3], g)
            gkp = np.einsum("nk,nkd->nd", kp, g)
            sp += (aT * w)[:, None] * np.einsum("nd,nad->na", gkp, g)
            gv = np.einsum("nd,ncd->nc", v, Dv) - np.einsum("nd,ncd->nc", pv, Dpv)
            vg = np.einsum("nd,nad->na", v, g)          # v . grad phi_a
            pvg = np.einsum("nd,nad->na", pv, g)        # pi v . grad phi_a
            s1 += (dT * w)[:, None, None] * gv[:, None, :] * vg[:, :, None]
            s2 += (dT * w)[:, None, None] * gv[:, None, :] * pvg[:, :, None]
        R[:, idx, 3] += sp
        R[:, CORNERS, 3] -= np.einsum("ak,na->nk", WK, sp)
        R[:, idx, 0:3] += s1
        R[:, CORNERS, 0:3] -= np.einsum("ak,nac->nkc", WK, s2)
    return R


class Level:
    """One mesh level for the operator: cells (optionally in patch groups)."""

    def __init__(self, xyz, cells, vertex_bc, patch_groups: bool):
        self.xyz = np.asarray(xyz, dtype=np.float64)
        self.cells = np.asarray(cells, dtype=np.int64)
        self.bc = np.asarray(vertex_bc, dtype=np.int64)
        self.n = self.xyz.shape[0]
        self.grouped = bool(patch_groups)
        if self.grouped:
            ng = self.cells.shape[0] // 8
            nodes = np.empty((ng, 27), dtype=np.int64)
            for t in range(8):
                nodes[:, CH[t]] = self.cells[t::8]
            self.groups = nodes
        self.dirichlet = (self.bc == 1) | (self.bc == 2)
        # the pressure is fixed only up to a constant when there is no
        # do-nothing boundary (Sec. 2.1, space L)
        self.pressure_mean_zero = not np.any(self.bc == 3)

    # -- local evaluations ---------------------------------------------
    def local_operator(self, U, prm):
        """[ng, 27, 4] (grouped) or [nc, 8, 4] local contributions of A_h."""
        m, th, nu = prm["m"], prm["theta"], prm["nu"]
        if self.grouped:
            Xg = self.xyz[self.groups]
            R = np.zeros(U.shape, dtype=U.dtype)
            for t in range(8):
                R[:, CH[t]] += cell_operator(Xg[:, CH[t]], U[:, CH[t]], m, th, nu)
            if prm.get("lps", True):
                vref = prm.get("vref")
                R += group_lps(Xg, U, m, nu, prm["alpha0"], prm["delta0"],
                               None if vref is None else vref[self.groups])
            return R
        return cell_operator(self.xyz[self.cells], U, m, th, nu)

    def local_nodes(self):
        return self.groups if self.grouped else self.cells

    def operator(self, x, prm):
        """A_h(x) assembled: [n, 4]."""
        nodes = self.local_nodes()
        Rl = self.local_operator(x[nodes], prm)
        out = np.zeros((self.n, 4), dtype=Rl.dtype)
        np.add.at(out, nodes.ravel(), Rl.reshape(-1, 4))
        return out

    def rhs(self, v_old, prm, f_new=None, f_old=None):
        """b(v_old) assembled: [n, 4], pressure rows 0, Dirichlet velocity rows 0."""
        X = self.xyz[self.cells]
        Fn = None if f_new is None else f_new[self.cells]
        Fo = None if f_old is None else f_old[self.cells]
        Bl = cell_rhs(X, v_old[self.cells], prm["m"], prm["theta"], prm["nu"], Fn, Fo)
        out = np.zeros((self.n, 4))
        np.add.at(out, self.cells.ravel(), Bl.reshape(-1, 4))
        out[self.dirichlet, 0:3] = 0.0
        return out

    def residual(self, x, F, prm):
        """r = F - A_h(x), velocity rows zero at Dirichlet nodes."""
        r = F - self.operator(x, prm)
        r[self.dirichlet, 0:3] = 0.0
        return r

    def jacobian(self, x, prm, h=1e-30):
        """dA_h/dx (stabilisation parameters frozen) by complex-step
        differentiation of the local contributions, assembled as a sparse
        [4n, 4n] matrix with unknown ordering 4 * node + component."""
        import scipy.sparse as sp
        nodes = self.local_nodes()
        nl = nodes.shape[1]
        U = x[nodes].astype(np.complex128)
        ndir = 4 * nl
        cols = []
        for d in range(ndir):
            Up = U.copy()
            Up[:, d // 4, d % 4] += 1j * h
            cols.append(np.imag(self.local_operator(Up, prm)).reshape(U.shape[0], ndir) / h)
        Jl = np.stack(cols, axis=2)                      # [ne, rows, cols]
        gdof = (4 * nodes[:, :, None] + np.arange(4)[None, None, :]).reshape(nodes.shape[0], ndir)
        rows = np.repeat(gdof[:, :, None], ndir, axis=2)
        colm = np.repeat(gdof[:, None, :], ndir, axis=1)
        return sp.csr_matrix((Jl.ravel(), (rows.ravel(), colm.ravel())), shape=(4 * self.n, 4 * self.n))

    def lumped_mass(self):
        """integral of each basis function (the mass-weighted mean uses it)."""
        det, _ = cell_geometry(self.xyz[self.cells])
        ml = np.einsum("nq,qk->nk", GAUSS_W * det, PHI)
        out = np.zeros(self.n)
        np.add.at(out, self.cells.ravel(), ml.ravel())
        return out
