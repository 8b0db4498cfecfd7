"""Manufactured solution for the oracle's discretisation pins (test helper).

A divergence-free velocity and a mean-zero pressure on the unit cube:
  u =  sin(pi x) cos(pi y) cos(pi z)
  v =  cos(pi x) sin(pi y) cos(pi z)
  w = -2 cos(pi x) cos(pi y) sin(pi z)
  p =  cos(pi x) cos(pi y) cos(pi z)
and the force f = (v.grad) v - nu Lap v + grad p that makes it a steady
solution of the Navier-Stokes equations (Sec. 3.1, strong form); each
component is a product of sines and cosines of pi x, pi y, pi z, so
Lap = -3 pi^2 on every velocity component.
"""
import numpy as np

PI = np.pi


def exact(xyz):
    x, y, z = (PI * xyz[:, i] for i in range(3))
    sx, cx, sy, cy, sz, cz = np.sin(x), np.cos(x), np.sin(y), np.cos(y), np.sin(z), np.cos(z)
    v = np.stack([sx * cy * cz, cx * sy * cz, -2 * cx * cy * sz], axis=1)
    p = cx * cy * cz
    return v, p


def grad_v(xyz):
    """G[n, c, d] = d v_c / d x_d."""
    x, y, z = (PI * xyz[:, i] for i in range(3))
    sx, cx, sy, cy, sz, cz = np.sin(x), np.cos(x), np.sin(y), np.cos(y), np.sin(z), np.cos(z)
    G = np.empty((xyz.shape[0], 3, 3))
    G[:, 0] = PI * np.stack([cx * cy * cz, -sx * sy * cz, -sx * cy * sz], axis=1)
    G[:, 1] = PI * np.stack([-sx * sy * cz, cx * cy * cz, -cx * sy * sz], axis=1)
    G[:, 2] = -2 * PI * np.stack([-sx * cy * sz, -cx * sy * sz, cx * cy * cz], axis=1)
    return G


def grad_p(xyz):
    x, y, z = (PI * xyz[:, i] for i in range(3))
    sx, cx, sy, cy, sz, cz = np.sin(x), np.cos(x), np.sin(y), np.cos(y), np.sin(z), np.cos(z)
    return -PI * np.stack([sx * cy * cz, cx * sy * cz, cx * cy * sz], axis=1)


def force(xyz, nu):
    v, _ = exact(xyz)
    G = grad_v(xyz)
    conv = np.einsum("nd,ncd->nc", v, G)
    return conv + nu * 3 * PI ** 2 * v + grad_p(xyz)


def errors(level, x):
    """(velocity L2, velocity H1-seminorm, pressure L2) errors of the nodal
    solution x [n, 4] on ``level`` (3x3x3 Gauss on every cell)."""
    from oracle import fem
    pts, ws = fem.gauss_points(3)
    PHI = np.array([fem.q1_basis(p)[0] for p in pts])
    DPHI = np.array([fem.q1_basis(p)[1] for p in pts])
    X = level.xyz[level.cells]
    U = x[level.cells]
    det, G = fem.cell_geometry(X, DPHI)
    ev = eg = ep = 0.0
    for q in range(len(pts)):
        xq = np.einsum("k,nkd->nd", PHI[q], X)
        v, p = exact(xq)
        vh = np.einsum("k,nkc->nc", PHI[q], U[:, :, 0:3])
        ph = np.einsum("k,nk->n", PHI[q], U[:, :, 3])
        Gh = np.einsum("nkc,nkd->ncd", U[:, :, 0:3], G[:, q])
        w = ws[q] * det[:, q]
        ev += np.sum(w * np.sum((vh - v) ** 2, axis=1))
        eg += np.sum(w * np.sum((Gh - grad_v(xq)) ** 2, axis=(1, 2)))
        ep += np.sum(w * (ph - p) ** 2)
    return np.sqrt(ev), np.sqrt(eg), np.sqrt(ep)
