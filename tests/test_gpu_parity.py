"""Parity of the CUDA patch path (through the C ABI) with the FP64 oracle,
stage by stage and composed, in the three precision forms.  Tolerances are
stated in parity_util."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from parity_util import CASES, TOL, case_data, patch_output_err, rel_max, residual_err  # noqa: E402
from paper_2307_14837_gb300 import build, capi  # noqa: E402
from paper_2307_14837_gb300.path import PatchPath  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    capi.load()


def _path(d, precision):
    c = d["case"]
    p = PatchPath(d["mesh"], c["nu"], c["dt"], c["theta"], precision, features=c.get("features", 12),
                  patch_levels=c.get("patch_levels", 1))
    Ws, ss, ts = d["net"]
    p.set_network(c["widths"], Ws, ss, ts, skip=True)
    return p


def _np(t):
    return t.detach().float().cpu().numpy() if t.dtype == torch.bfloat16 else t.detach().cpu().numpy()


@pytest.mark.parametrize("name", list(CASES))
def test_mesh_data_bit_exact(name):
    d = case_data(name)
    h = d["h"]
    nf = d["case"].get("features", 12)
    J = d["case"].get("patch_levels", 1)
    p = PatchPath(d["mesh"], 0.01, 0.01, 1.0, "fp64", features=nf, patch_levels=J)
    assert p.n_fine == h.n_fine and p.n_patches == h.n_patches
    npn = h.patch_map.shape[1]
    assert p.sizes["n_in"] == 8 * npn + nf and p.sizes["n_out"] == 3 * npn
    assert np.array_equal(p.mesh_data(capi.PATCH_MAP), h.patch_map)
    assert np.array_equal(p.mesh_data(capi.VALENCE), h.mult)
    assert np.array_equal(p.mesh_data(capi.FINE_KIND), h.bc_f)
    assert np.allclose(p.mesh_data(capi.FINE_XYZ), h.xyz_f, rtol=0, atol=1e-15)
    assert np.allclose(p.mesh_data(capi.EDGE_LENGTHS), h.edge_lengths(), rtol=1e-15, atol=0)
    # the geometry features in double: lengths to rounding, angles through acos
    assert np.allclose(p.mesh_data(capi.GEOMETRY), h.geometry(nf), rtol=1e-13, atol=1e-13)
    p.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("name", list(CASES))
def test_stagewise_parity(name, precision):
    d = case_data(name)
    o = d["out"]
    tol = TOL[precision]
    p = _path(d, precision)
    xc = p.to_device(d["xc"])
    F = p.to_device(d["F"])
    xf = p.prolongate(xc)
    r = p.residual(xc, F)
    X = p.local_restrict(xc, r)
    Y = p.network(X)
    dd = p.extend(Y)
    bf, bc = p.rhs_restrict(xc, dd)
    torch.cuda.synchronize()
    ftol = 1e-12 if precision == "fp64" else 1e-5
    assert rel_max(_np(xf), o["x_fine"]) <= ftol
    assert residual_err(_np(r), d) <= ftol
    n_in = p.sizes["n_in"]
    Xn = _np(X)[:, :n_in]
    if precision == "bf16":
        assert np.all(np.abs(Xn - o["X"]) <= 2.0 ** -8 * np.abs(o["X"]) + 1e-5 * np.abs(o["X"]).max())
    else:
        assert rel_max(Xn, o["X"]) <= ftol
    assert np.all(_np(X)[:, n_in:] == 0)
    emax, ep99 = patch_output_err(_np(Y), o["Y"])
    assert emax <= tol, (emax, ep99)
    assert rel_max(_np(dd), o["d"]) <= tol
    assert rel_max(_np(bf), o["b_fine"]) <= tol
    assert rel_max(_np(bc), o["b_coarse"]) <= tol
    # the composed step gives exactly the stage-by-stage result
    bf2, bc2 = p.step(xc, F)
    torch.cuda.synchronize()
    assert torch.equal(bf2, bf) and torch.equal(bc2, bc)
    p.close()


@pytest.mark.parametrize("precision", ["fp64", "bf16"])
def test_deterministic_and_host_entry_point(precision):
    d = case_data("channel4")
    p = _path(d, precision)
    xc, F = p.to_device(d["xc"]), p.to_device(d["F"])
    a = p.step(xc, F)
    b = p.step(xc, F)
    torch.cuda.synchronize()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    # host buffers, copies inside the call
    ht = np.float64 if precision == "fp64" else np.float32
    xh = np.ascontiguousarray(d["xc"].astype(ht))
    Fh = np.ascontiguousarray(d["F"].astype(ht))
    bfh = np.empty_like(Fh)
    bch = np.empty_like(xh)
    capi.dnnmg_patch_step_host(p.ctx, xh, Fh, bfh, bch)
    assert np.array_equal(bfh, _np(a[0])) and np.array_equal(bch, _np(a[1]))
    p.close()


def test_b_fine_may_alias_F():
    d = case_data("cavity8")
    p = _path(d, "fp64")
    xc, F = p.to_device(d["xc"]), p.to_device(d["F"])
    ref_f, ref_c = p.step(xc, F)
    Fa = F.clone()
    p.step(xc, Fa, b_fine=Fa)
    torch.cuda.synchronize()
    assert torch.equal(Fa, ref_f)
    p.close()


def test_errors_and_empty_batch():
    d = case_data("cavity3_ragged")
    c = d["case"]
    p = PatchPath(d["mesh"], c["nu"], c["dt"], c["theta"], "fp32")
    X = torch.zeros((p.n_patches, 256), device="cuda")
    Y = torch.zeros((p.n_patches, 81), device="cuda")
    with pytest.raises(capi.DnnmgError) as e:
        capi.dnnmg_network(p.ctx, X, Y, p.n_patches)
    assert e.value.status == -7                        # ESTATE: no network yet
    Ws, ss, ts = d["net"]
    p.set_network(c["widths"], Ws, ss, ts)
    capi.dnnmg_network(p.ctx, X, Y, 0)                 # empty batch is a no-op
    with pytest.raises(capi.DnnmgError) as e:
        capi.dnnmg_network(p.ctx, X, Y, p.n_patches + 1)
    assert e.value.status == -1
    with pytest.raises(capi.DnnmgError):
        p.set_network((228, 5000, 81), [np.zeros((5000, 228)), np.zeros((81, 5000))])   # width > 4096
    with pytest.raises(capi.DnnmgError):
        p.set_network((240, 20, 81), [np.zeros((20, 240)), np.zeros((81, 20))])   # input width of the other form
    capi.dnnmg_sync(p.ctx, 10_000_000)
    p.close()
