"""Newton solve of A_h(x) = F on one level (oracle), Sec. 3.4.

The paper solves each time step's nonlinear system with Newton's method
(stabilisation parameters frozen in the Jacobian) and GMRES preconditioned
by geometric multigrid.  The oracle replaces the linear solver by a sparse
direct solve (scipy's SuperLU), which gives the same Newton iterates up to
rounding; the Jacobian is the exact derivative of A_h with frozen
parameters, obtained by complex-step differentiation of the local
contributions.

Dirichlet velocity unknowns hold their prescribed values; where the whole
boundary is Dirichlet the pressure is fixed up to a constant and is
normalised to zero mean (Sec. 3.1, space L) after every update.

Pinned by the manufactured-solution convergence rates and the zero-network
identity of the DNN-MG step.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def newton(level, x0, F, prm, tol=1e-11, max_iter=25, rtol=1e-12):
    """Solve A_h(x) = F (velocity rows at Dirichlet nodes replaced by the
    values already in x0).  Returns (x, info) with the residual history."""
    x = np.array(x0, dtype=np.float64)
    n = level.n
    fixed = np.zeros((n, 4), dtype=bool)
    fixed[level.dirichlet, 0:3] = True
    pin = None
    if level.pressure_mean_zero:
        pin = 4 * int(np.flatnonzero(~level.dirichlet)[0] if np.any(~level.dirichlet) else 0) + 3
    mass = level.lumped_mass()
    hist = []
    r0 = None
    for it in range(max_iter + 1):
        r = level.residual(x, F, prm)          # F - A(x), Dirichlet rows 0
        rv = r.ravel().copy()
        if pin is not None:
            rv[pin] = 0.0
        nr = float(np.linalg.norm(rv))
        hist.append(nr)
        if r0 is None:
            r0 = max(nr, 1e-300)
        if nr <= tol or nr <= rtol * r0 or it == max_iter:
            break
        J = level.jacobian(x, prm).tolil()
        fix = np.flatnonzero(fixed.ravel())
        if pin is not None:
            fix = np.append(fix, pin)
        for i in fix:
            J.rows[i] = [int(i)]
            J.data[i] = [1.0]
        dx = spla.spsolve(sp.csc_matrix(J), rv)
        x = x + dx.reshape(n, 4)
        if level.pressure_mean_zero:
            x[:, 3] -= np.dot(mass, x[:, 3]) / np.sum(mass)
    return x, dict(residuals=hist, iterations=len(hist) - 1)
