"""The Q2/Q2 patch path (the paper's element, Sec. 3.2) on the GPU against
the FP64 oracle (oracle/q2.py), stage by stage with the oracle's inputs:
prolongation x~ = P x^L of the coarse Q2 field, the fine residual with the
one-level projection terms, the network input rows of the 125-node patches,
the network, the extension, the corrected rhs and its restriction.
Tolerances as for Q1: FP64 1e-12, FP32 1e-5 (relative to the size of the
terms), BF16 rows within bf16 rounding and outputs per patch 2e-2."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2307_14837_gb300 import build, capi, inputs as I  # noqa: E402
from paper_2307_14837_gb300.path import PatchPath  # noqa: E402
from oracle import mesh as omesh, mlp as omlp, q2 as oq2  # noqa: E402
from parity_util import patch_output_err  # noqa: E402

TOL = {"fp64": 1e-12, "fp32": 1e-5}
CASES = {
    "cavity2_jitter": dict(mesh=lambda: I.cavity_mesh(2, jitter=0.2, seed=3), nu=0.01, dt=0.01, theta=0.5,
                           widths=(1012, 32, 32, 375), features=12),
    "cavity3": dict(mesh=lambda: I.cavity_mesh(3, grouped=False), nu=0.01, dt=0.01, theta=1.0,
                    widths=(1024, 48, 48, 375), features=24),
    "channel2": dict(mesh=lambda: I.channel_mesh(2, seed=1), nu=5e-4, dt=0.005, theta=0.5,
                     widths=(1012, 32, 32, 375), features=12),
}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    capi.load()


def _case(name):
    c = CASES[name]
    m = c["mesh"]()
    h = omesh.Hierarchy(m["xyz"], m["cells"], m["vertex_bc"])
    h2 = omesh.Hierarchy2(m["xyz"], m["cells"], m["vertex_bc"])
    coarse = oq2.coarse_level(h)
    xc = I.smooth_field(h.xyz_f, 7)
    xc[:, 0:3] *= 0.5
    dirc = coarse.dirichlet
    xc[dirc, 0:3] = I.dirichlet_values(m, h.xyz_f, h.bc_f)[dirc]
    F = I.fine_rhs(h2.n_fine, 3, scale=1e-2)
    Ws, ss, ts = I.network_weights(c["widths"], seed=2, scale_shift=True)
    prm = dict(m=1.0 / c["dt"], theta=c["theta"], nu=c["nu"], alpha0=0.02, delta0=0.1)
    ref = oq2.hot_path_step(h, h2, (Ws, ss, ts, True), xc, F, prm, features=c["features"])
    return c, m, h, h2, xc, F, (Ws, ss, ts), ref


def _rel(a, b, scale):
    return float(np.abs(np.asarray(a, dtype=np.float64) - b).max() / scale)


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
def test_q2_patch_path_matches_oracle(name, precision):
    c, m, h, h2, xc, F, (Ws, ss, ts), ref = _case(name)
    p = PatchPath(m, c["nu"], c["dt"], c["theta"], precision, features=c["features"], patch_levels=2, element=2)
    assert p.n_coarse == h.n_fine and p.n_fine == h2.n_fine and p.sizes["element"] == 2
    assert np.array_equal(p.mesh_data(capi.PATCH_MAP), h2.patch_map)
    p.set_network(c["widths"], Ws, ss, ts)
    tol = TOL.get(precision, 1e-5)          # fields are FP32 in the BF16 form
    dev = lambda a: p.to_device(a)           # noqa: E731
    xf = p.prolongate(dev(xc)).double().cpu().numpy()
    assert _rel(xf, ref["x_fine"], np.abs(ref["x_fine"]).max()) <= tol
    r = p.residual(dev(xc), dev(F)).double().cpu().numpy()
    A = F - ref["r"]                          # A(x~) at the free rows
    assert _rel(r, ref["r"], np.abs(F).max() + np.abs(A).max()) <= tol
    X = p.local_restrict(dev(xc), dev(ref["r"])).double().cpu().numpy()
    n_in = c["widths"][0]
    Xr = ref["X"]
    if precision == "bf16":
        # rows within one bf16 rounding of the oracle's values
        assert np.all(np.abs(X[:, :n_in] - Xr) <= np.abs(Xr) * 2.0 ** -7 + 1e-30)
    else:
        assert _rel(X[:, :n_in], Xr, np.abs(Xr).max()) <= tol
    assert np.all(X[:, n_in:] == 0)
    Xin = torch.as_tensor(Xr, dtype=torch.float64)
    Xin = torch.nn.functional.pad(Xin, (0, p.sizes["n_in_padded"] - n_in)).to(p.device, p.x_dtype).contiguous()
    Y = p.network(Xin).double().cpu().numpy()
    Yr = omlp.forward(Xin.double().cpu().numpy()[:, :n_in], Ws, ss, ts, skip=True)
    if precision == "bf16":
        worst, _ = patch_output_err(Y, Yr)
        assert worst <= 2e-2
    else:
        assert _rel(Y, Yr, np.abs(Yr).max()) <= tol
    d = p.extend(dev(ref["Y"])).double().cpu().numpy()
    assert _rel(d, ref["d"], np.abs(ref["d"]).max()) <= tol
    bf, bc = p.rhs_restrict(dev(xc), dev(ref["d"]))
    bf, bc = bf.double().cpu().numpy(), bc.double().cpu().numpy()
    assert _rel(bf, ref["b_fine"], np.abs(ref["b_fine"]).max()) <= tol
    assert _rel(bc, ref["b_coarse"], np.abs(ref["b_coarse"]).max()) <= tol
    p.close()


def test_q2_restricted_fine_rhs_equals_coarse_rhs_on_the_gpu():
    # nested Q2 spaces: R b_{L+1}(P v) = b_L(v) on a parallelepiped mesh at
    # theta = 1 (the 3-point rule integrates the mass term exactly); the coarse
    # Q2 rhs is the oracle's, the fine one and R are the GPU's
    m = I.cavity_mesh(2)
    h = omesh.Hierarchy(m["xyz"], m["cells"], m["vertex_bc"])
    coarse = oq2.coarse_level(h)
    rng = np.random.default_rng(6)
    v = np.zeros((h.n_fine, 4))
    v[:, 0:3] = rng.standard_normal((h.n_fine, 3))
    p = PatchPath(m, 0.01, 1.0 / 7.0, 1.0, "fp64", patch_levels=2, element=2)
    zero_d = torch.zeros((p.n_fine, 3), dtype=torch.float64, device="cuda")
    _, bc = p.rhs_restrict(p.to_device(v), zero_d)
    ref = coarse.rhs(v[:, 0:3], dict(m=7.0, theta=1.0, nu=0.01))
    assert _rel(bc.cpu().numpy(), ref, np.abs(ref).max()) <= 1e-12
    p.close()


def _q2_start(m, h):
    coarse = oq2.coarse_level(h)
    x0 = np.zeros((coarse.n, 4))
    x0[coarse.dirichlet, 0:3] = I.dirichlet_values(m, coarse.xyz, coarse.bc)[coarse.dirichlet]
    return coarse, x0


def test_q2_exact_jacobian_matches_complex_step():
    m = I.cavity_mesh(2, jitter=0.15, seed=4)
    h = omesh.Hierarchy(m["xyz"], m["cells"], m["vertex_bc"])
    coarse = oq2.coarse_level(h)
    prm = dict(m=100.0, theta=0.5, nu=0.01, alpha0=0.02, delta0=0.1)
    x = I.smooth_field(coarse.xyz, 6)
    x[:, 0:3] *= 0.3
    p = PatchPath(m, 0.01, 0.01, 0.5, "fp64", patch_levels=2, element=2)
    J = capi.dnnmg_level_jacobian(p.ctx, capi.LEVEL_COARSE, torch.as_tensor(x, device="cuda"))
    ref = coarse.jacobian(x, prm).toarray()
    fixed = [4 * j + c for j in np.flatnonzero(coarse.dirichlet) for c in range(3)]
    pin = 4 * int(np.flatnonzero(~coarse.dirichlet)[0]) + 3
    for r in fixed + [pin]:
        ref[r, :] = 0.0
        ref[r, r] = 1.0
    assert np.abs(J - ref).max() <= 1e-11 * np.abs(ref).max()
    p.close()


@pytest.mark.parametrize("theta", [1.0, 0.5])
def test_q2_newton_matches_oracle(theta):
    from oracle import solve as osolve
    m = I.cavity_mesh(4)
    h = omesh.Hierarchy(m["xyz"], m["cells"], m["vertex_bc"])
    coarse, x0 = _q2_start(m, h)
    prm = dict(m=100.0, theta=theta, nu=0.01, alpha0=0.02, delta0=0.1)
    b = coarse.rhs(x0[:, 0:3], prm)
    ref, _ = osolve.newton(coarse, x0, b, prm, tol=1e-14, rtol=1e-15)
    p = PatchPath(m, 0.01, 0.01, theta, "fp64", patch_levels=2, element=2)
    sp = capi.dnnmg_solver_defaults(newton_atol=1e-13, newton_rtol=1e-13, gmres_rtol=1e-10)
    x = torch.as_tensor(x0, device="cuda")
    st = capi.dnnmg_solve(p.ctx, capi.LEVEL_COARSE, torch.as_tensor(b, device="cuda"), x, sp)
    assert st["converged"] == 1
    assert np.abs(x.cpu().numpy() - ref).max() <= 1e-9 * np.abs(ref).max()
    p.close()


def test_q2_time_loop_matches_oracle_and_zero_network_is_plain_scheme():
    m = I.cavity_mesh(2)
    h = omesh.Hierarchy(m["xyz"], m["cells"], m["vertex_bc"])
    h2 = omesh.Hierarchy2(m["xyz"], m["cells"], m["vertex_bc"])
    coarse, x0 = _q2_start(m, h)
    prm = dict(m=100.0, theta=1.0, nu=0.01, alpha0=0.02, delta0=0.1)
    bcv = lambda t: I.dirichlet_values(m, coarse.xyz, coarse.bc)     # noqa: E731
    widths = (1012, 16, 375)
    Ws, ss, ts = I.network_weights(widths, seed=0)
    Ws[-1] = 0.05 * Ws[-1]
    ref = oq2.run(h, h2, (Ws, ss, ts, True), x0, 3, prm, bcv)
    sp = capi.dnnmg_solver_defaults(newton_atol=1e-13, newton_rtol=1e-13, gmres_rtol=1e-10)
    p = PatchPath(m, 0.01, 0.01, 1.0, "fp64", patch_levels=2, element=2)
    p.set_network(widths, Ws, ss, ts)
    x = torch.as_tensor(x0, device="cuda")
    bf, bc = p.rhs_restrict(x, torch.zeros((p.n_fine, 3), dtype=torch.float64, device="cuda"))
    for k in range(3):
        capi.dnnmg_time_step(p.ctx, 1, x, bc, bf, sp)
        err = np.abs(x.cpu().numpy() - ref[k]).max() / np.abs(ref[k]).max()
        assert err <= 1e-9, (k, err)
    p.close()
    # with W_L = 0 the DNN-MG loop is the plain coarse Q2 scheme (nested spaces)
    Ws[-1] = np.zeros_like(Ws[-1])
    p = PatchPath(m, 0.01, 0.01, 1.0, "fp64", patch_levels=2, element=2)
    p.set_network(widths, Ws, ss, ts)
    xa, xb = torch.as_tensor(x0, device="cuda"), torch.as_tensor(x0, device="cuda")
    bf, bc = p.rhs_restrict(xa, torch.zeros((p.n_fine, 3), dtype=torch.float64, device="cuda"))
    capi.dnnmg_time_step(p.ctx, 3, xa, bc, bf, sp)
    capi.dnnmg_plain_step(p.ctx, capi.LEVEL_COARSE, 3, xb, sp)
    a, b = xa.cpu().numpy(), xb.cpu().numpy()
    assert np.abs(a - b).max() <= 1e-10 * np.abs(b).max()
    assert np.abs(b[:, 0:3]).max() > 0.1
    p.close()
