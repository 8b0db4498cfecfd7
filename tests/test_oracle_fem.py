"""Pins of the oracle's Q1/Q1-LPS operator, right-hand side and transfer
against closed forms, a manufactured solution, finite differences and the
Galerkin identities of nested spaces."""
import math

import numpy as np
import pytest

import mms
from paper_2307_14837_gb300 import inputs as I
from oracle import dnnmg, fem, mesh, solve, transfer


def _fine(n, jitter=0.0, seed=0):
    m = I.cavity_mesh(n, jitter=jitter, seed=seed)
    h = mesh.Hierarchy(m["xyz"], m["cells"], m["vertex_bc"])
    return m, h, dnnmg.fine_level(h)


PRM0 = dict(m=0.0, theta=1.0, nu=0.0, alpha0=0.02, delta0=0.1, lps=False)


def _op(lev, x, **kw):
    return lev.operator(x, dict(PRM0, **kw))


def _interior(lev):
    x = lev.xyz
    return ~np.any((np.abs(x) < 1e-12) | (np.abs(x - 1) < 1e-12), axis=1)


@pytest.mark.parametrize("jitter", [0.0, 0.25])
def test_mass_rows_sum_to_volume(jitter):
    _, _, lev = _fine(2, jitter, seed=5)
    x = np.zeros((lev.n, 4))
    x[:, 0] = 1.0
    R = _op(lev, x, m=1.0)
    assert abs(R[:, 0].sum() - 1.0) < 1e-13          # unit cube
    assert np.allclose(R[:, 0], lev.lumped_mass(), rtol=0, atol=1e-15)
    assert np.abs(R[:, 1:]).max() < 1e-15


@pytest.mark.parametrize("jitter", [0.0, 0.25])
def test_divergence_of_linear_fields(jitter):
    _, _, lev = _fine(2, jitter, seed=6)
    A = np.array([[1.0, 2.0, -1.0], [0.5, -3.0, 2.0], [1.5, 0.25, 2.0]])   # trace 0
    x = np.zeros((lev.n, 4))
    x[:, 0:3] = lev.xyz @ A.T
    R = _op(lev, x)
    assert np.abs(R[:, 3]).max() < 1e-14
    x[:, 0:3] = lev.xyz @ np.diag([1.0, 0.0, 0.0]).T     # div = 1
    R = _op(lev, x)
    assert np.allclose(R[:, 3], lev.lumped_mass(), rtol=0, atol=1e-15)


def test_viscous_and_pressure_terms_on_linear_fields():
    _, _, lev = _fine(2)
    inner = _interior(lev)
    A = np.array([[1.0, 2.0, -1.0], [0.5, -3.0, 2.0], [1.5, 0.25, 2.0]])
    x = np.zeros((lev.n, 4))
    x[:, 0:3] = lev.xyz @ A.T
    R = _op(lev, x, nu=0.7) - _op(lev, x, nu=0.0)     # the viscous term alone
    assert np.abs(R[inner, 0:3]).max() < 1e-14         # -nu Lap(linear) = 0
    assert np.abs(R[~inner, 0:3]).max() > 1e-3
    g = np.array([0.3, -1.2, 2.0])
    x = np.zeros((lev.n, 4))
    x[:, 3] = lev.xyz @ g + 0.7
    R = _op(lev, x)
    # -(p, d_c phi_j) = (d_c p, phi_j) for interior j
    assert np.allclose(R[inner, 0:3], lev.lumped_mass()[inner, None] * g[None, :], rtol=0, atol=1e-14)
    # constant pressure: no force on interior nodes; all rows sum to zero
    x[:, 3] = 2.5
    R = _op(lev, x)
    assert np.abs(R[inner, 0:3]).max() < 1e-14
    assert np.abs(R[:, 0:3].sum(axis=0)).max() < 1e-13


def test_convection_equals_mass_of_advected_field():
    # v = A x  =>  (v.grad) v = A A x, linear, so (conv, phi_j) = (A A x, phi_j)
    _, _, lev = _fine(2)
    A = np.array([[0.4, -1.0, 0.3], [0.7, 0.2, -0.5], [-0.2, 0.9, 0.1]])
    x = np.zeros((lev.n, 4))
    x[:, 0:3] = lev.xyz @ A.T
    Rc = _op(lev, x)
    y = np.zeros((lev.n, 4))
    y[:, 0:3] = lev.xyz @ (A @ A).T
    Rm = _op(lev, y, m=1.0) - _op(lev, y, m=0.0)      # the mass term alone
    assert np.allclose(Rc[:, 0:3], Rm[:, 0:3], rtol=0, atol=1e-15)
    assert np.allclose(Rc[:, 0:3].sum(axis=0), A @ A @ np.full(3, 0.5), rtol=0, atol=1e-14)


@pytest.mark.parametrize("theta", [1.0, 0.5])
def test_restriction_of_fine_rhs_equals_coarse_rhs(theta):
    # nested spaces + exact quadrature on affine cells: P^T b_{L+1}(P v) = b_L(v)
    m, h, lev = _fine(4)
    coarse = fem.Level(m["xyz"], m["cells"], m["vertex_bc"], True)
    prm = dict(m=100.0, theta=theta, nu=0.01)
    v = I.coarse_state(m, 1)[:, 0:3]
    bc = coarse.rhs(v, prm)
    bc[h.dirichlet_coarse(), 0:3] = 0.0
    br = transfer.restrict(h, lev.rhs(transfer.prolongate(h, v), prm))
    assert np.abs(br - bc).max() <= 1e-13 * np.abs(bc).max()


def test_prolongation_exact_for_trilinear_and_adjoint():
    m, h, _ = _fine(4, jitter=0.2, seed=2)
    X = m["xyz"][m["cells"]]
    g = I.coarse_state(m, 4)
    xf = transfer.prolongate(h, g)
    for iota in range(27):
        expect = np.einsum("k,nkc->nc", mesh.corner_weights(iota), g[m["cells"]])
        assert np.allclose(xf[h.patch_map[:, iota]], expect, rtol=0, atol=1e-14)
    # on a dyadic mesh a trilinear field is reproduced bit for bit
    m2, h2, _ = _fine(4)
    f = lambda p: 1.0 + 2.0 * p[:, 0] - 0.5 * p[:, 1] + 0.25 * p[:, 2] + p[:, 0] * p[:, 1] * p[:, 2]
    assert np.array_equal(transfer.prolongate(h2, f(m2["xyz"])), f(h2.xyz_f))
    # adjointness
    rng = np.random.default_rng(0)
    a = rng.standard_normal(h.n_coarse_vertices)
    b = rng.standard_normal(h.n_fine)
    P = transfer.prolongation_matrix(h)
    assert abs(np.dot(transfer.prolongate(h, a), b) - np.dot(a, P.T @ b)) < 1e-12


def test_lps_vanishes_on_prolongated_fields_only():
    m, h, lev = _fine(4, jitter=0.2, seed=7)
    xf = transfer.prolongate(h, I.coarse_state(m, 0))
    Xg, Ug = lev.xyz[lev.groups], xf[lev.groups]
    L = fem.group_lps(Xg, Ug, 100.0, 0.01, 0.02, 0.1)
    assert np.abs(L).max() == 0.0
    rng = np.random.default_rng(1)
    Ur = Ug + 0.1 * rng.standard_normal(Ug.shape)
    assert np.abs(fem.group_lps(Xg, Ur, 100.0, 0.01, 0.02, 0.1)).max() > 1e-6


def test_complex_step_jacobian_matches_finite_differences():
    m, h, lev = _fine(2, jitter=0.2, seed=9)
    prm = dict(m=20.0, theta=0.5, nu=0.05, alpha0=0.02, delta0=0.1)
    rng = np.random.default_rng(3)
    x = I.coarse_state(dict(m, xyz=lev.xyz, vertex_bc=lev.bc), 2) + 0.05 * rng.standard_normal((lev.n, 4))
    J = lev.jacobian(x, prm).toarray()
    frozen = dict(prm, vref=x)            # parameters frozen, as in the Jacobian
    eps = 1e-6
    Jfd = np.empty_like(J)
    for k in range(4 * lev.n):
        dx = np.zeros(4 * lev.n)
        dx[k] = eps
        Jfd[:, k] = (lev.operator(x + dx.reshape(-1, 4), frozen).ravel()
                     - lev.operator(x - dx.reshape(-1, 4), frozen).ravel()) / (2 * eps)
    assert np.abs(J - Jfd).max() <= 1e-7 * np.abs(J).max()


def test_manufactured_solution_convergence():
    nu = 0.1
    errs = []
    for n in (2, 4):
        m, h, lev = _fine(n)
        prm = dict(m=10.0, theta=0.5, nu=nu, alpha0=0.02, delta0=0.1)
        v, _ = mms.exact(lev.xyz)
        f = mms.force(lev.xyz, nu)
        F = lev.rhs(v, prm, f_new=f, f_old=f)
        x0 = np.zeros((lev.n, 4))
        x0[lev.dirichlet, 0:3] = v[lev.dirichlet]
        x, info = solve.newton(lev, x0, F, prm)
        assert info["residuals"][-1] < 1e-10
        errs.append(mms.errors(lev, x))
    rates = np.log2(np.array(errs[0]) / np.array(errs[1]))
    assert rates[0] > 1.8, rates      # velocity L2 ~ h^2
    assert rates[1] > 0.95, rates     # velocity H1 ~ h
    assert rates[2] > 1.5, rates      # pressure L2 (LPS: at least h)


def _brute_force_jacobian(xyz, cells, v0, m, th, nu):
    """The linearised Q1/Q1 operator (without stabilisation) at velocity v0,
    assembled cell by cell from explicit basis functions and a 3-point Gauss
    rule per axis: unknown 4 j + c, rows
      momentum (k, c):  m (v_c, N_k) + th [nu (grad v_c, grad N_k)
                        + ((dv . grad) v0_c + (v0 . grad) dv_c, N_k)] - (p, d_c N_k)
      continuity (k):   (div v, N_k)."""
    g, w = np.polynomial.legendre.leggauss(3)
    g, w = 0.5 * (g + 1.0), 0.5 * w
    n = xyz.shape[0]
    J = np.zeros((4 * n, 4 * n))
    for cell in cells:
        X = xyz[cell]                                       # [8, 3]
        for a in range(3):
            for b in range(3):
                for c in range(3):
                    xi = (g[a], g[b], g[c])
                    wq = w[a] * w[b] * w[c]
                    N = np.empty(8)
                    dN = np.empty((8, 3))                   # reference derivatives
                    for k in range(8):
                        f = [xi[d] if (k >> d) & 1 else 1.0 - xi[d] for d in range(3)]
                        s = [1.0 if (k >> d) & 1 else -1.0 for d in range(3)]
                        N[k] = f[0] * f[1] * f[2]
                        dN[k] = [s[0] * f[1] * f[2], f[0] * s[1] * f[2], f[0] * f[1] * s[2]]
                    Jm = X.T @ dN                           # dx_d / dxi_e
                    det = np.linalg.det(Jm)
                    G = dN @ np.linalg.inv(Jm)              # physical gradients [8, 3]
                    dv = wq * det
                    V0 = v0[cell]                           # [8, 3]
                    vq = N @ V0                             # v0 at the point
                    Dv0 = V0.T @ G                          # d v0_c / d x_e
                    for k in range(8):
                        rk = 4 * cell[k]
                        for l in range(8):
                            cl = 4 * cell[l]
                            adv = vq @ G[l]                 # (v0 . grad) N_l
                            for cc in range(3):
                                J[rk + cc, cl + cc] += dv * (m * N[l] * N[k] + th * nu * (G[l] @ G[k])
                                                             + th * adv * N[k])
                                for e in range(3):
                                    J[rk + cc, cl + e] += dv * th * N[l] * Dv0[cc, e] * N[k]
                                J[rk + cc, cl + 3] += -dv * N[l] * G[k, cc]
                                J[rk + 3, cl + cc] += dv * G[l, cc] * N[k]
    return J


def test_brute_force_assembled_matrix_matches_matrix_free_operator():
    # the 2^3 cavity under a shear: parallelepiped cells, on which both Gauss
    # rules integrate every term exactly; the oracle's matrix-free operator,
    # linearised at a non-zero velocity (exact complex-step derivative),
    # against the matrix assembled by brute force
    m_ = I.cavity_mesh(2)
    S = np.array([[1.0, 0.3, -0.2], [0.1, 0.9, 0.25], [0.0, -0.15, 1.1]])
    xyz = m_["xyz"] @ S.T
    lev = fem.Level(xyz, m_["cells"], m_["vertex_bc"], True)
    rng = np.random.default_rng(3)
    x0 = np.zeros((lev.n, 4))
    x0[:, 0:3] = rng.standard_normal((lev.n, 3))
    x0[:, 3] = rng.standard_normal(lev.n)
    prm = dict(m=37.0, theta=0.5, nu=0.3, alpha0=0.02, delta0=0.1, lps=False)
    Jo = lev.jacobian(x0, prm).toarray()
    Jb = _brute_force_jacobian(xyz, np.asarray(m_["cells"]), x0[:, 0:3], 37.0, 0.5, 0.3)
    assert np.abs(Jo - Jb).max() <= 1e-12 * np.abs(Jb).max()
    # and the operator itself at a state with zero velocity (where it is linear in p)
    xp = np.zeros((lev.n, 4))
    xp[:, 3] = rng.standard_normal(lev.n)
    Ao = lev.operator(xp, prm).ravel()
    assert np.abs(Ao - Jb @ xp.ravel()).max() <= 1e-12 * np.abs(Ao).max()


# ---- closed-form values of the local projection terms (Eqs. (5), (8)) ------
# One group: the unit cube split into 8 children of side 1/2; group node
# iota = a + 3b + 9c sits at (a, b, c) / 2.  Every child has diameter
# h_T = sqrt(3)/2, so nu / h_T^2 = 4 nu / 3.  The fields below are piecewise
# linear in each child with integrands of degree <= 3 per direction, so the
# 2 x 2 x 2 Gauss rule integrates them exactly and the values follow by hand.
_NU, _M, _A0, _D0 = 0.3, 2.0, 0.02, 0.1
_HT = math.sqrt(3.0) / 2.0


def _unit_group():
    a, b, c = np.meshgrid(np.arange(3), np.arange(3), np.arange(3), indexing="ij")
    pos = np.stack([a.T.ravel(), b.T.ravel(), c.T.ravel()], axis=1) / 2.0   # iota = a + 3b + 9c
    return pos[None]


def test_lps_pressure_term_closed_form():
    # v = 0, p = 1 at the centre node (iota 13), 0 elsewhere: pi p = 0, so
    # p - pi p is the centre's fine hat function.  With v = 0 every child has
    # alpha_T = alpha0 / (nu / h_T^2 + m).  Rows of the pressure test
    # functions xi_i - pi xi_i (Q1 stiffness on a cube of side s: diagonal
    # s/3, face diagonal -s/12, edge neighbour 0; the parent-trilinear part
    # of a corner's test function is orthogonal to the centre hat):
    #   centre        8 children x (1/2)/3            =  4/3  alpha_T
    #   face centre   edge neighbours in 4 children    =  0
    #   edge midpoint face diagonals in 2 children     = -1/12 alpha_T
    #   corner        space diagonal in 1 child        = -1/24 alpha_T
    X = _unit_group()
    U = np.zeros((1, 27, 4))
    U[0, 13, 3] = 1.0
    R = fem.group_lps(X, U, _M, _NU, _A0, _D0)[0]
    aT = _A0 / (_NU / _HT ** 2 + _M)
    want = np.zeros(27)
    for i in range(27):
        ones = sum(1 for v in (i % 3, (i // 3) % 3, i // 9) if v == 1)   # coordinates at 1/2
        want[i] = {3: 4.0 / 3.0, 2: 0.0, 1: -1.0 / 12.0, 0: -1.0 / 24.0}[ones] * aT
    np.testing.assert_allclose(R[:, 3], want, rtol=1e-13, atol=1e-16)
    np.testing.assert_array_equal(R[:, 0:3], 0.0)
    assert abs(R[:, 3].sum()) < 1e-15          # test functions xi - pi xi sum to 0


def test_lps_convection_term_closed_form():
    # v = (f(x), 0, 0), f piecewise linear with nodal values f(0) = 0,
    # f(1/2) = 3/2, f(1) = 1, i.e. f = x + 2 psi(x) with psi the hat at 1/2;
    # p = 0.  Then pi v = (x, 0, 0) and
    #   g = v.grad v - pi v.grad pi v = (f f' - x) e_x = 8x e_x (x < 1/2),
    #                                                   -2 e_x (x > 1/2).
    # |v|_inf = 3/2 in every child, so delta_T = delta0 / (nu/h^2 + 1.5/h + m).
    # The velocity rows tested against a nodal vector q give
    # delta_T (g, v.grad q - pi v.grad pi q):
    #   q = f: (g, g)                          = 64/24 + 2   = 14/3
    #   q = x: (g, f - x) = (g, 2 psi)         = 2/3 - 1/2   = 1/6
    # and the v, w rows vanish.
    X = _unit_group()
    x = X[0, :, 0]
    f = np.where(x == 0.5, 1.5, np.where(x == 1.0, 1.0, 0.0))
    U = np.zeros((1, 27, 4))
    U[0, :, 0] = f
    R = fem.group_lps(X, U, _M, _NU, _A0, _D0)[0]
    dT = _D0 / (_NU / _HT ** 2 + 1.5 / _HT + _M)
    assert f @ R[:, 0] == pytest.approx(dT * 14.0 / 3.0, rel=1e-13)
    assert x @ R[:, 0] == pytest.approx(dT / 6.0, rel=1e-12)
    np.testing.assert_allclose(R[:, 1:4], 0.0, atol=1e-16)


def test_lps_parameters_scale_as_eq8():
    # alpha_T and delta_T of Eq. (8) as functions of nu, m and |v|: the term
    # is linear in alpha0 / delta0 and every other factor is fixed by the
    # fields, so the ratio of two evaluations is the ratio of the
    # denominators nu / h_T^2 + |v|_inf / h_T + m
    X = _unit_group()
    x = X[0, :, 0]
    U = np.zeros((1, 27, 4))
    U[0, :, 0] = np.where(x == 0.5, 1.5, np.where(x == 1.0, 1.0, 0.0))
    U[0, 13, 3] = 1.0
    for (nu1, m1), (nu2, m2) in [((0.3, 2.0), (0.03, 2.0)), ((0.3, 2.0), (0.3, 50.0))]:
        R1 = fem.group_lps(X, U, m1, nu1, _A0, _D0)[0]
        R2 = fem.group_lps(X, U, m2, nu2, _A0, _D0)[0]
        den = lambda nu, m: nu / _HT ** 2 + 1.5 / _HT + m   # noqa: E731
        ratio = den(nu2, m2) / den(nu1, m1)
        np.testing.assert_allclose(R2[:, 0] * ratio, R1[:, 0], rtol=1e-12, atol=1e-18)
        np.testing.assert_allclose(R2[:, 3] * ratio, R1[:, 3], rtol=1e-12, atol=1e-18)
