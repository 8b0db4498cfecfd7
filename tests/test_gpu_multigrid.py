"""Geometric multigrid in the GPU Newton solver (Sec. 3.4): the Newton
solution with a V-cycle preconditioner (group-Vanka smoothing, dense FP64 LU
on the coarsest level) against the FP64 oracle's Newton solution, the
hierarchy the device builds against the host's, and GMRES iterations per
Newton step that stay flat under refinement."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2307_14837_gb300 import build, capi, inputs as I  # noqa: E402
from paper_2307_14837_gb300.path import PatchPath  # noqa: E402
from oracle import dnnmg as odnnmg, fem, mesh as omesh, solve as osolve  # noqa: E402

NU, DT = 0.01, 0.01
PRM = dict(m=1.0 / DT, nu=NU, alpha0=0.02, delta0=0.1)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    capi.load()


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def _start(m, xyz, kind):
    d = (kind == 1) | (kind == 2)
    x = np.zeros((xyz.shape[0], 4))
    x[d, 0:3] = I.dirichlet_values(m, xyz, kind)[d]
    return x


@pytest.mark.parametrize("theta", [1.0, 0.5])
def test_multigrid_newton_matches_oracle(theta):
    m = I.cavity_mesh(8, levels=2, jitter=0.1, seed=1)
    lev = fem.Level(m["xyz"], m["cells"], m["vertex_bc"], True)
    prm = dict(PRM, theta=theta)
    x_old = _start(m, m["xyz"], m["vertex_bc"])
    b = lev.rhs(x_old[:, 0:3], prm)
    # the oracle's Newton (direct solves) run to round-off as well
    ref, _ = osolve.newton(lev, x_old, b, prm, tol=1e-14, rtol=1e-15)
    p = PatchPath(m, NU, DT, theta, "fp64")
    # Newton run to 1e-13 (the oracle solves each Newton step directly)
    sp = capi.dnnmg_solver_defaults(mg_levels=2, newton_atol=1e-13, newton_rtol=1e-13, gmres_rtol=1e-10)
    assert capi.dnnmg_level_mg(p.ctx, capi.LEVEL_COARSE, sp) == [729, 125]
    x = _dev(x_old)
    st = capi.dnnmg_solve(p.ctx, capi.LEVEL_COARSE, _dev(b), x, sp)
    assert st["converged"] == 1
    xg = x.cpu().numpy()
    assert np.abs(xg - ref).max() <= 1e-9 * np.abs(ref).max()
    p.close()


def test_fine_level_multigrid_solve_matches_oracle():
    # level L+1 (17^3 nodes) over L = 8^3 and 4^3
    m = I.cavity_mesh(8, levels=2)
    h = omesh.Hierarchy(m["xyz"], m["cells"], m["vertex_bc"])
    lev = odnnmg.fine_level(h)
    prm = dict(PRM, theta=1.0)
    p = PatchPath(m, NU, DT, 1.0, "fp64")
    sp = capi.dnnmg_solver_defaults(mg_levels=4, newton_atol=1e-13, newton_rtol=1e-13, gmres_rtol=1e-10)
    assert capi.dnnmg_level_mg(p.ctx, capi.LEVEL_FINE, sp) == [4913, 729, 125]
    x_old = _start(m, p.mesh_data(capi.FINE_XYZ), p.mesh_data(capi.FINE_KIND))
    b = lev.rhs(x_old[:, 0:3], prm)
    ref, _ = osolve.newton(lev, x_old, b, prm, tol=1e-14, rtol=1e-15)
    x = _dev(x_old)
    st = capi.dnnmg_solve(p.ctx, capi.LEVEL_FINE, _dev(b), x, sp)
    assert st["converged"] == 1
    assert np.abs(x.cpu().numpy() - ref).max() <= 1e-9 * np.abs(ref).max()
    p.close()


def test_device_hierarchy_equals_host_hierarchy():
    m = I.channel_mesh(8, seed=2, levels=2)
    p = PatchPath(m, m["meta"]["nu_re200"], 0.005, 0.5, "fp32")
    h = capi.HostHierarchy(m)
    for level in (capi.LEVEL_COARSE, capi.LEVEL_FINE):
        sp = capi.dnnmg_solver_defaults(mg_levels=8)
        assert capi.dnnmg_level_mg(p.ctx, level, sp) == h.mg_nodes(level, 8)
    h.close()
    p.close()


def _gmres_per_newton(m, mg):
    p = PatchPath(m, NU, DT, 1.0, "fp64")
    sp = capi.dnnmg_solver_defaults(mg_levels=mg, newton_rtol=1e-10, newton_atol=1e-12, gmres_rtol=1e-8)
    x = _dev(_start(m, m["xyz"], m["vertex_bc"]))
    per = []
    for _ in range(2):
        st = capi.dnnmg_plain_step(p.ctx, capi.LEVEL_COARSE, 1, x, sp)
        assert st["converged"] == 1
        per.append(st["gmres_iterations"] / max(st["newton_iterations"], 1))
    p.close()
    return float(np.mean(per))


def test_gmres_iterations_stay_flat_under_refinement():
    # the cavity on 8^3, 16^3 and 32^3 with the V-cycle down to 4^3: GMRES
    # iterations per Newton step within +-20% of their mean (the one-level
    # preconditioner's grow with the mesh)
    its = [_gmres_per_newton(I.cavity_mesh(n, levels=k), k - 1) for n, k in [(8, 2), (16, 3), (32, 4)]]
    mean = np.mean(its)
    assert max(its) <= 1.2 * mean and min(its) >= 0.8 * mean, its
    one = _gmres_per_newton(I.cavity_mesh(16, levels=3), 0)
    assert its[1] < 0.5 * one, (its, one)


@pytest.mark.parametrize("theta", [1.0, 0.5])
def test_bf16_smoother_newton_matches_oracle(theta):
    # the additive smoother on bf16 copies of the matrices and inverses: a
    # cheaper preconditioner, the same Newton solution (FP64 residual)
    m = I.cavity_mesh(8, levels=2, jitter=0.1, seed=1)
    lev = fem.Level(m["xyz"], m["cells"], m["vertex_bc"], True)
    prm = dict(PRM, theta=theta)
    x_old = _start(m, m["xyz"], m["vertex_bc"])
    b = lev.rhs(x_old[:, 0:3], prm)
    ref, _ = osolve.newton(lev, x_old, b, prm, tol=1e-14, rtol=1e-15)
    its = {}
    for bf16 in (0, 1):
        p = PatchPath(m, NU, DT, theta, "fp64")
        sp = capi.dnnmg_solver_defaults(mg_levels=2, newton_atol=1e-13, newton_rtol=1e-13, gmres_rtol=1e-10,
                                        mg_bf16=bf16)
        x = _dev(x_old)
        st = capi.dnnmg_solve(p.ctx, capi.LEVEL_COARSE, _dev(b), x, sp)
        assert st["converged"] == 1
        assert np.abs(x.cpu().numpy() - ref).max() <= 1e-9 * np.abs(ref).max()
        its[bf16] = st["gmres_iterations"] / max(1, st["newton_iterations"])
        p.close()
    assert its[1] <= 1.3 * its[0] + 1
    p = PatchPath(m, NU, DT, theta, "fp64")
    try:
        with pytest.raises(capi.DnnmgError):
            capi.dnnmg_solve(p.ctx, capi.LEVEL_COARSE, _dev(b), _dev(x_old), capi.dnnmg_solver_defaults(mg_bf16=2))
    finally:
        p.close()
