"""Training data in the library (Sec. 5.2, Sec. 6.4): the level-(L+2)
reference solve of a J = 2 context against the oracle's Newton on the twice
refined mesh, the patch targets Q(v - P x^L) against the oracle's
prolongation and patch maps, and the column statistics, standardisation and
row gather against their definitions."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2307_14837_gb300 import build, capi, inputs as I  # noqa: E402
from paper_2307_14837_gb300.path import PatchPath  # noqa: E402
from oracle import dnnmg as odnnmg, mesh as omesh, solve as osolve, transfer  # noqa: E402

NU, DT = 0.01, 0.01


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    capi.load()


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda").to(dtype)


def _start(m, xyz, kind):
    d = (kind == 1) | (kind == 2)
    x = np.zeros((xyz.shape[0], 4))
    x[d, 0:3] = I.dirichlet_values(m, xyz, kind)[d]
    return x


def test_level_l2_newton_matches_oracle():
    # J = 2 over L = 4^3: the fine level is the 16^3 mesh (level L+2), its
    # multigrid runs through 8^3 and 4^3
    m = I.cavity_mesh(4, levels=1, jitter=0.1, seed=4)
    h2 = omesh.Hierarchy2(m["xyz"], m["cells"], m["vertex_bc"])
    lev = odnnmg.fine_level(h2)
    prm = dict(m=1.0 / DT, nu=NU, alpha0=0.02, delta0=0.1, theta=1.0)
    p = PatchPath(m, NU, DT, 1.0, "fp64", patch_levels=2)
    sp = capi.dnnmg_solver_defaults(mg_levels=4, newton_atol=1e-13, newton_rtol=1e-13, gmres_rtol=1e-10)
    assert capi.dnnmg_level_mg(p.ctx, capi.LEVEL_FINE, sp) == [17 ** 3, 9 ** 3, 5 ** 3]
    xyz, kind = p.mesh_data(capi.FINE_XYZ), p.mesh_data(capi.FINE_KIND)
    assert np.allclose(xyz, h2.xyz_f, rtol=0, atol=1e-15)
    x_old = _start(m, xyz, kind)
    b = lev.rhs(x_old[:, 0:3], prm)
    ref, _ = osolve.newton(lev, x_old, b, prm, tol=1e-14, rtol=1e-15)
    x = _dev(x_old)
    st = capi.dnnmg_solve(p.ctx, capi.LEVEL_FINE, _dev(b), x, sp)
    assert st["converged"] == 1
    assert np.abs(x.cpu().numpy() - ref).max() <= 1e-9 * np.abs(ref).max()
    # the level rhs of the context is the oracle's
    F = torch.empty_like(x)
    capi.dnnmg_level_rhs(p.ctx, capi.LEVEL_FINE, _dev(x_old), F)
    assert np.abs(F.cpu().numpy() - b).max() <= 1e-12 * np.abs(b).max()
    p.close()


@pytest.mark.parametrize("J", [1, 2])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_patch_targets_match_oracle(J, precision):
    m = I.cavity_mesh(4, jitter=0.15, seed=2)
    h = omesh.Hierarchy(m["xyz"], m["cells"], m["vertex_bc"]) if J == 1 else \
        omesh.Hierarchy2(m["xyz"], m["cells"], m["vertex_bc"])
    p = PatchPath(m, NU, DT, 1.0, precision, patch_levels=J)
    xc = I.coarse_state(m, seed=3)
    vf = I.smooth_field(h.xyz_f, seed=10)
    n_out = 3 * h.patch_map.shape[1]
    ref = (vf - transfer.prolongate(h, xc))[:, 0:3][h.patch_map].reshape(-1, n_out)
    # row stride above n_out: the padding stays untouched
    Tt = torch.full((h.n_patches, n_out + 7), 7.0, dtype=torch.float32, device="cuda")
    capi.dnnmg_patch_targets(p.ctx, p.to_device(xc), p.to_device(vf), Tt, ldt=n_out + 7)
    got = Tt.cpu().numpy()
    assert np.all(got[:, n_out:] == 7.0)
    tol = 1e-6 if precision == "fp64" else 1e-5   # fp32 output / fp32 fields
    assert np.abs(got[:, :n_out] - ref).max() <= tol * np.abs(ref).max()
    # the same as the library's own prolongation, gathered (bit for bit)
    xt = torch.empty((p.n_fine, 4), dtype=p.dtype, device="cuda")
    capi.dnnmg_prolongate(p.ctx, p.to_device(xc), xt)
    pm = torch.as_tensor(p.mesh_data(capi.PATCH_MAP).astype(np.int64), device="cuda")
    own = (p.to_device(vf) - xt)[:, 0:3][pm].reshape(-1, n_out).float()
    assert torch.equal(Tt[:, :n_out], own)
    with pytest.raises(capi.DnnmgError):
        capi.dnnmg_patch_targets(p.ctx, p.to_device(xc), p.to_device(vf), Tt, ldt=n_out - 1)
    p.close()


def _matrix(rows, cols, ld, seed, dtype):
    a = I.splitmix_normal(700 + seed, rows * ld).reshape(rows, ld) * 3.0 + np.arange(ld)[None, :] * 0.25
    return torch.as_tensor(a, device="cuda").to(dtype)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
def test_column_stats_definition(dtype):
    rows, cols, ld = 5003, 229, 256      # a ragged row count, cols < ld
    A = _matrix(rows, cols, ld, 1, dtype)
    mean = torch.empty(cols, dtype=torch.float64, device="cuda")
    sd = torch.empty(cols, dtype=torch.float64, device="cuda")
    capi.dnnmg_column_stats(A, mean, sd, cols=cols)
    a = A[:, :cols].double().cpu().numpy()
    mu = a.sum(axis=0) / rows
    sig = np.sqrt(((a - mu) ** 2).sum(axis=0) / (rows - 1))
    assert np.allclose(mean.cpu().numpy(), mu, rtol=1e-12, atol=1e-13)
    assert np.allclose(sd.cpu().numpy(), sig, rtol=1e-12, atol=0)
    # fixed summation order: the same bits on a second call
    m2, s2 = torch.empty_like(mean), torch.empty_like(sd)
    capi.dnnmg_column_stats(A, m2, s2, cols=cols)
    assert torch.equal(m2, mean) and torch.equal(s2, sd)
    # fewer rows than partition blocks
    B = A[:3]
    capi.dnnmg_column_stats(B, m2, s2, cols=cols)
    b = a[:3]
    assert np.allclose(m2.cpu().numpy(), b.mean(axis=0), rtol=1e-12, atol=1e-13)
    assert np.allclose(s2.cpu().numpy(), b.std(axis=0, ddof=1), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
def test_standardize_definition(dtype):
    rows, cols, ld = 777, 228, 256
    A = _matrix(rows, cols, ld, 2, dtype)
    shift = _dev(np.linspace(-1.0, 1.0, cols))
    scale = _dev(np.linspace(0.5, 3.0, cols))
    B = torch.full_like(A, 9.0)
    capi.dnnmg_standardize(A, shift, scale, B, cols=cols)
    acc = torch.float64 if dtype == torch.float64 else torch.float32
    ref = ((A[:, :cols].to(acc) - shift.to(acc)) / scale.to(acc)).to(dtype)
    assert torch.equal(B[:, :cols], ref)
    assert torch.all(B[:, cols:] == 9.0)
    # in place
    C = A.clone()
    capi.dnnmg_standardize(C, shift, scale, C, cols=cols)
    assert torch.equal(C[:, :cols], ref) and torch.equal(C[:, cols:], A[:, cols:])


@pytest.mark.parametrize("shape,dtype", [((1000, 256), torch.bfloat16), ((1000, 81), torch.float32),
                                         ((1000, 3), torch.int16)])
def test_gather_rows_definition(shape, dtype):
    src = torch.arange(shape[0] * shape[1], device="cuda").reshape(shape).to(dtype)
    g = torch.Generator(device="cpu").manual_seed(5)
    idx = torch.randint(0, shape[0], (613,), generator=g)
    idx[7] = -1
    idx[100] = shape[0]        # outside the source: zero rows
    idx = idx.to("cuda")
    dst = torch.full((613, shape[1]), 5, dtype=dtype, device="cuda")
    capi.dnnmg_gather_rows(src, idx, dst)
    ok = (idx >= 0) & (idx < shape[0])
    assert torch.equal(dst[ok], src[idx[ok]])
    assert torch.all(dst[~ok] == 0)


def test_normalization_pipeline_on_the_device():
    # fit_normalization (library column statistics + host floors) and
    # normalize (library standardisation) on bf16 rows and fp32 targets
    from paper_2307_14837_gb300 import train as T
    n = 4096
    a = np.zeros((n, 256))
    a[:, :228] = 3.0 + I.splitmix_normal(0, n * 228).reshape(n, 228) * (1.0 + np.arange(228) % 7)
    X = torch.as_tensor(a, device="cuda").to(torch.bfloat16)
    Tg = torch.as_tensor(0.5 * I.splitmix_normal(1, n * 81).reshape(n, 81), device="cuda", dtype=torch.float32)
    mu, sig, ts = T.fit_normalization(X, Tg)
    xd = X.double().cpu().numpy()
    assert np.allclose(mu[:228], xd[:, :228].mean(0), rtol=1e-12, atol=1e-12)
    assert np.allclose(sig[:228], xd[:, :228].std(0, ddof=1), rtol=1e-12)
    assert abs(ts - float(torch.sqrt((Tg.double() ** 2).mean()))) < 1e-10 * ts
    Xn, Tn = T.normalize(X, (mu, sig, ts), Tg)
    assert Xn.dtype == torch.bfloat16 and Tn.dtype == torch.float32
    assert torch.allclose(Xn[:, :228].double().mean(0), torch.zeros(228, dtype=torch.float64, device="cuda"),
                          atol=2e-3)
    assert torch.allclose(Xn[:, :228].double().std(0), torch.ones(228, dtype=torch.float64, device="cuda"),
                          atol=5e-3)
    assert torch.equal(Xn[:, 228:], X[:, 228:])          # padding stays zero
    assert abs(float((Tn.double() ** 2).mean()) - 1.0) < 1e-5


def test_refined_reference_samples_match_oracle():
    # make_samples with the level-(L+2) reference: each step's L+2 solve,
    # the level-(L+1) rhs of the injected previous state, the coarse solve
    # with its restriction, and the targets, against the oracle doing the
    # same steps (two backward-Euler steps on 4^3 -> 16^3)
    from paper_2307_14837_gb300 import train as T
    from oracle import fem
    m = I.cavity_mesh(4, levels=1, jitter=0.1, seed=6)
    n_steps = 2
    tight = lambda mg: capi.dnnmg_solver_defaults(mg_levels=mg, newton_atol=1e-13, newton_rtol=1e-13,  # noqa: E731
                                                  gmres_rtol=1e-10)
    X, Tg, st = T.make_samples(m, NU, DT, 1.0, n_steps, ref_levels=2, solver=tight(2), ref_solver=tight(4))
    h1 = omesh.Hierarchy(m["xyz"], m["cells"], m["vertex_bc"])
    h2 = omesh.Hierarchy2(m["xyz"], m["cells"], m["vertex_bc"])
    lev1, lev2 = odnnmg.fine_level(h1), odnnmg.fine_level(h2)
    coarse = fem.Level(m["xyz"], m["cells"], m["vertex_bc"], True)
    prm = dict(m=1.0 / DT, nu=NU, alpha0=0.02, delta0=0.1, theta=1.0)
    v2 = _start(m, h2.xyz_f, h2.bc_f)
    xc = _start(m, m["xyz"], m["vertex_bc"])
    nf, nc = h1.n_fine, h1.n_patches
    assert X.shape == (n_steps * nc, 256) and Tg.shape == (n_steps * nc, 81)
    for n in range(n_steps):
        F1 = lev1.rhs(v2[:nf, 0:3], prm)
        v2, _ = osolve.newton(lev2, v2, lev2.rhs(v2[:, 0:3], prm), prm, tol=1e-14, rtol=1e-15)
        xc, _ = osolve.newton(coarse, xc, transfer.restrict(h1, F1), prm, tol=1e-14, rtol=1e-15)
        s = st[n]
        for got, ref in ((s["v_fine"], v2[:nf]), (s["F"], F1), (s["x_coarse"], xc)):
            ref = np.asarray(ref)
            assert np.abs(got.cpu().numpy() - ref).max() <= 1e-9 * np.abs(ref).max()
        t_ref = (v2[:nf] - transfer.prolongate(h1, xc))[:, 0:3][h1.patch_map].reshape(nc, 81)
        t_got = Tg[n * nc:(n + 1) * nc].double().cpu().numpy()
        assert np.abs(t_got - t_ref).max() <= 1e-6 * np.abs(t_ref).max()


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_add_noise_statistics_and_determinism(dtype):
    rows, ld, c0, c1, sigma = 20000, 256, 108, 216, 0.25
    A = torch.zeros((rows, ld), dtype=dtype, device="cuda")
    capi.dnnmg_add_noise(A, c0, c1, sigma, seed=7)
    z = A[:, c0:c1].double()
    assert torch.all(A[:, :c0] == 0) and torch.all(A[:, c1:] == 0)
    n = z.numel()
    assert abs(float(z.mean())) < 5 * sigma / n ** 0.5
    assert abs(float(z.std()) / sigma - 1.0) < 0.01
    # a standard normal's fourth moment is 3 (the Box-Muller output, not a uniform)
    assert abs(float(((z / sigma) ** 4).mean()) - 3.0) < 0.05
    B = torch.zeros_like(A)
    capi.dnnmg_add_noise(B, c0, c1, sigma, seed=7)
    assert torch.equal(A, B)
    capi.dnnmg_add_noise(B, c0, c1, sigma, seed=8)
    assert not torch.equal(A, B)
    # the draws of different entries are uncorrelated
    cc = float((z[:, 0] * z[:, 1]).mean() / sigma ** 2)
    assert abs(cc) < 5 / rows ** 0.5


def test_prolongated_fine_boundary_gives_zero_targets_on_dirichlet_nodes():
    # with the reference's Dirichlet values taken from the prolongated
    # coarse data, the targets vanish on the fine Dirichlet nodes (where the
    # DNN-MG correction is zero), and the interior still carries a correction
    from paper_2307_14837_gb300 import train as T
    m = I.cavity_mesh(4, levels=1, jitter=0.1, seed=6)
    X, Tg, st = T.make_samples(m, NU, DT, 1.0, 2, ref_levels=2, fine_boundary="prolongated")
    p = PatchPath(m, NU, DT, 1.0, "fp64")
    kind = p.mesh_data(capi.FINE_KIND)
    pm = p.mesh_data(capi.PATCH_MAP)
    p.close()
    dir_pn = ((kind == 1) | (kind == 2))[pm]                 # [nc][27] Dirichlet patch nodes
    t = Tg.reshape(2, -1, 27, 3).double().cpu().numpy()
    scale = np.abs(t).max()
    assert scale > 0
    assert np.abs(t[:, dir_pn]).max() <= 1e-6 * scale
    assert np.abs(t[:, ~dir_pn]).max() > 1e-3 * scale
