"""Grid transfer between level L and level L+1 (oracle).

Prolongation P (the prolongation step of Alg. 1): the Q1 interpolant of the coarse field at
the fine nodes.  With nested refinement every fine node is the midpoint of
a coarse edge, the centre of a coarse face or cell, or a coarse vertex, so
its value is the mean of that entity's vertex values (weights 1, 1/2, 1/4,
1/8).  Restriction R = P^T (the restriction step of Alg. 1), applied to right-hand sides.

Pinned by: exact reproduction of trilinear fields on dyadic meshes,
adjointness <P x, y> = <x, P^T y>, and the Galerkin identity
P^T M_{L+1} P = M_L on affine cells.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def prolongation_matrix(h) -> sp.csr_matrix:
    rows, cols, vals = [], [], []
    for j, par in enumerate(h.parents):
        for v in par:
            rows.append(j)
            cols.append(v)
            vals.append(1.0 / len(par))
    return sp.csr_matrix((vals, (rows, cols)), shape=(h.n_fine, h.n_coarse_vertices))


def prolongate(h, x_coarse: np.ndarray) -> np.ndarray:
    """x_fine[j] = mean over parents(j) of x_coarse (any trailing shape).
    For patches of two levels (``h.levels``) the product of the two
    one-level prolongations."""
    if hasattr(h, "levels"):
        for lv in h.levels:
            x_coarse = prolongate(lv, x_coarse)
        return x_coarse
    out = np.empty((h.n_fine,) + x_coarse.shape[1:])
    for j, par in enumerate(h.parents):
        s = np.zeros(x_coarse.shape[1:])
        for v in par:
            s = s + x_coarse[v]
        out[j] = s / len(par)
    return out


def restrict(h, b_fine: np.ndarray) -> np.ndarray:
    """(P^T b)[v] = sum over fine nodes j with parent v of b[j] / |parents(j)|;
    velocity rows at coarse Dirichlet vertices are then set to zero.  For
    patches of two levels the two one-level restrictions in turn (the
    intermediate zeroing changes nothing: a Dirichlet node of level L+1 has
    only Dirichlet parents)."""
    if hasattr(h, "levels"):
        for lv in reversed(h.levels):
            b_fine = restrict(lv, b_fine)
        return b_fine
    out = np.zeros((h.n_coarse_vertices,) + b_fine.shape[1:])
    for j, par in enumerate(h.parents):
        for v in par:
            out[v] = out[v] + b_fine[j] / len(par)
    out[h.dirichlet_coarse(), 0:3] = 0.0
    return out
