"""One DNN-MG time step on the patch path (oracle), the steps Alg. 1 adds
to a plain Newton-multigrid time step:

  x~  = P x^L                                    (prolongation)
  r   = F - A_{L+1}(x~), zero at Dirichlet rows  (fine residual, Eq. (9))
  X   = Q(x~) | Q(r) | h^c                       (Eqs. (13)-(14), Sec. 5.2)
  Y   = N(X)                                     (Sec. 4)
  d   = L(Y) = mu . sum_P L(Y[P], P)             (Eq. (15))
  b   = Rhs(v~ + d) on level L+1                 (right-hand side, Eq. (6))
  b^L = R b                                      (restriction of the rhs)

Input row layout of X (the paper gives only the order x~, r, geometry):
columns 0..107 are x~ at the 27 patch nodes, node-major (u, v, w, p);
columns 108..215 the residual in the same order; 216.. the geometry features
of the coarse cell: its 12 edge lengths (228 inputs), or with 24 features also
its 4 diagonals and 8 mean face angles (240 inputs, Table 2).  Output row Y[P]: 27 x (u, v, w) in the same node order;
the pressure outputs are absent (Table 2: N_out = 81).
Dirichlet velocity nodes receive no correction.

Pinned by: the zero-network identity (with W_L = 0 the step reproduces the
plain coarse scheme), constant and linear fields through the extension, and
brute-force gather indices; see tests/test_oracle_dnnmg.py.
"""
from __future__ import annotations

import numpy as np

from . import mlp, transfer
from .fem import Level

N_IN = 228
N_OUT = 81


def fine_level(h) -> Level:
    return Level(h.xyz_f, h.cells_f, h.bc_f, patch_groups=True)


def local_restriction(h, field: np.ndarray) -> np.ndarray:
    """Q of Eqs. (13)-(14): row P holds field[dof(P, iota)] for the patch's
    nodes iota (27, or 125 for J = 2), flattened node-major.
    field [n_fine, c] -> [N_c, nodes c]."""
    nc, npn = h.patch_map.shape
    out = np.empty((nc, npn * field.shape[1]))
    for P in range(nc):
        for iota in range(npn):
            out[P, iota * field.shape[1]:(iota + 1) * field.shape[1]] = field[h.patch_map[P, iota]]
    return out


def gather(h, x_fine, r_fine, features: int = 12) -> np.ndarray:
    """Network input rows [N_c, 216 + features]."""
    return np.concatenate([local_restriction(h, x_fine), local_restriction(h, r_fine),
                           h.geometry(features)], axis=1)


def extend(h, Y) -> np.ndarray:
    """L of Eq. (15): d = mu . sum_P L(Y[P], P), mu = 1 / valence; summed in
    patch order; zero at Dirichlet velocity nodes.  Y [N_c, 3 nodes] -> [n_fine, 3]."""
    acc = np.zeros((h.n_fine, 3))
    npn = h.patch_map.shape[1]
    for P in range(h.n_patches):
        for iota in range(npn):
            j = h.patch_map[P, iota]
            acc[j] = acc[j] + Y[P, 3 * iota:3 * iota + 3]
    d = acc * (1.0 / h.mult)[:, None]
    d[h.dirichlet_fine()] = 0.0
    return d


def hot_path_step(h, net, x_coarse, F, prm, level=None, features: int = 12):
    """The patch-correction steps of Alg. 1 for one time step.  ``net`` = (Ws, scales,
    shifts, skip); ``features`` = geometry features per patch (12 or 24).
    Returns every intermediate as a dict."""
    lev = level if level is not None else fine_level(h)
    x_f = transfer.prolongate(h, x_coarse)
    r = lev.residual(x_f, F, prm)
    X = gather(h, x_f, r, features)
    Ws, ss, ts, skip = net
    Y = mlp.forward(X, Ws, ss, ts, skip=skip)
    d = extend(h, Y)
    v_hat = x_f[:, 0:3] + d
    b_f = lev.rhs(v_hat, prm)
    b_c = transfer.restrict(h, b_f)
    return dict(x_fine=x_f, r=r, X=X, Y=Y, d=d, b_fine=b_f, b_coarse=b_c)


def run(h, coarse, net, x0, n_steps, prm, bc_values, newton_tol=1e-13, features=12):
    """DNN-MG time stepping (Alg. 1) on the coarse level ``coarse`` (a
    fem.Level on the cells of h) with the patch correction on level L+1.

    x0 [n_coarse, 4]: initial state.  bc_values(t) -> [n_coarse, 3]
    Dirichlet velocities at time t.  The first right-hand side is the fine
    Rhs of the prolongated initial state, restricted.  Returns the list of
    coarse states x_1..x_n and the last step's intermediates."""
    from .solve import newton
    lev = fine_level(h)
    x = np.array(x0, dtype=np.float64)
    F = lev.rhs(transfer.prolongate(h, x[:, 0:3]), prm)
    b = transfer.restrict(h, F)
    states, last = [], None
    for n in range(1, n_steps + 1):
        t = n / prm["m"] if prm["m"] > 0 else float(n)
        xi = x.copy()
        xi[coarse.dirichlet, 0:3] = bc_values(t)[coarse.dirichlet]
        x, _ = newton(coarse, xi, b, prm, tol=newton_tol)
        states.append(x.copy())
        last = hot_path_step(h, net, x, F, prm, level=lev, features=features)
        F, b = last["b_fine"], last["b_coarse"]
    return states, last


def run_plain(coarse, x0, n_steps, prm, bc_values, newton_tol=1e-13):
    """The classical scheme on level L alone: rhs b_L(v_{n-1}) each step."""
    from .solve import newton
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
