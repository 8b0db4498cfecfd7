"""Checkpoint / resume and failure reporting:
* a DNN-MG run saved after some steps and resumed in a new context gives
  the uninterrupted run's next steps bit for bit (every stage is
  deterministic);
* a Newton iteration cap ends the solve with converged = 0 and the stats
  filled (DNNMG_ENOCONV is a result, not an error);
* a non-finite right-hand side is reported as DNNMG_ENAN;
* a serving request whose context cannot be built fails alone while the
  others are served."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2307_14837_gb300 import build, capi, inputs as I  # noqa: E402
from paper_2307_14837_gb300.checkpoint import TimeLoop  # noqa: E402
from paper_2307_14837_gb300.path import PatchPath  # noqa: E402
from paper_2307_14837_gb300.serve import Request, Server  # noqa: E402

WIDTHS = (228, 64, 64, 81)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    capi.load()


def _net():
    Ws, ss, ts = I.network_weights(WIDTHS, seed=5, scale_shift=True)
    Ws[-1] = 0.05 * Ws[-1]
    return Ws, ss, ts


@pytest.mark.parametrize("precision", ["fp64", "bf16"])
def test_resume_reproduces_the_next_steps_bit_exactly(precision, tmp_path):
    m = I.cavity_mesh(4, jitter=0.1, seed=2)
    Ws, ss, ts = _net()
    a = TimeLoop(m, 0.01, 0.01, 0.5, precision, WIDTHS, Ws, ss, ts).start().advance(4)
    b = TimeLoop(m, 0.01, 0.01, 0.5, precision, WIDTHS, Ws, ss, ts).start().advance(2)
    ck = tmp_path / "run.npz"
    b.save(ck)
    b.close()
    c = TimeLoop.load(ck).advance(2)
    torch.cuda.synchronize()
    assert c.step_count == 4
    assert torch.equal(a.x, c.x) and torch.equal(a.b, c.b) and torch.equal(a.F, c.F)
    assert np.abs(a.x.cpu().numpy()[:, 0:3]).max() > 0.1
    a.close()
    c.close()


def test_iteration_cap_and_non_finite_input():
    m = I.cavity_mesh(4)
    p = PatchPath(m, 0.01, 0.01, 1.0, "fp64")
    bc = I.dirichlet_values(m, m["xyz"], m["vertex_bc"])
    dirc = (m["vertex_bc"] == 1) | (m["vertex_bc"] == 2)
    x0 = np.zeros((p.n_coarse, 4))
    x0[dirc, 0:3] = bc[dirc]
    x = torch.as_tensor(x0, device="cuda")
    b = torch.zeros_like(x)
    capi.dnnmg_level_rhs(p.ctx, capi.LEVEL_COARSE, x, b)
    prm = capi.dnnmg_solver_defaults(newton_max=1, newton_rtol=1e-15, newton_atol=1e-30)
    st = capi.dnnmg_solve(p.ctx, capi.LEVEL_COARSE, b, x.clone(), prm=prm)
    assert st["converged"] == 0 and st["newton_iterations"] == 1 and st["residual"] < st["residual0"]
    bad = b.clone()
    bad[int(np.flatnonzero(~dirc)[0]), 0] = float("nan")   # an interior row (Dirichlet rows are overwritten)
    with pytest.raises(capi.DnnmgError) as e:
        capi.dnnmg_solve(p.ctx, capi.LEVEL_COARSE, bad, x.clone())
    assert e.value.status == -5
    # the context stays usable
    st = capi.dnnmg_solve(p.ctx, capi.LEVEL_COARSE, b, x)
    assert st["converged"] == 1
    p.close()


@pytest.mark.parametrize("workers", [0, 2])
def test_server_survives_a_request_that_cannot_be_built(workers):
    Ws, ss, ts = _net()
    bad_mesh = I.cavity_mesh(2)
    bad_cells = np.array(bad_mesh["cells"]).copy()
    bad_cells[0, 0] = 10 ** 6                   # vertex index out of range
    bad = dict(xyz=bad_mesh["xyz"], cells=bad_cells, vertex_bc=bad_mesh["vertex_bc"])
    reqs = [Request("a", I.cavity_mesh(4), 0.01, 0.01, 1.0, 2),
            Request("bad", bad, 0.01, 0.01, 1.0, 2),
            Request("c", I.cavity_mesh(2), 0.01, 0.01, 1.0, 3)]
    srv = Server(WIDTHS, Ws, ss, ts, memory_budget=1 << 33, max_rows=4096, precision="bf16", prepare_workers=workers)
    for r in reqs:
        srv.submit(r)
    while srv.live or srv.queue:
        srv.step()
    srv.close()
    assert set(srv.results) == {"a", "c"} and "bad" in srv.failures
    assert ("failed", "bad") in [(e, n) for e, n, _ in srv.log]
    assert srv.results["c"]["steps"] == 3


def test_tensor_core_wait_expiry_is_reported_and_recovered():
    # the first operand stage of the first layer is armed but never filled:
    # the kernel's bounded waits run out, it returns, dnnmg_sync reports
    # DNNMG_ETIMEOUT, and the context then computes the network normally
    m = I.cavity_mesh(4)
    widths = (228, 256, 256, 81)
    Ws, ss, ts = I.network_weights(widths, seed=1)
    p = PatchPath(m, 0.01, 0.01, 1.0, "bf16")
    p.set_network(widths, Ws, ss, ts)
    X = torch.zeros((p.n_patches, 256), dtype=torch.bfloat16, device="cuda")
    X[:, :228] = torch.as_tensor(I.splitmix_normal(4, p.n_patches * 228).reshape(p.n_patches, 228),
                                 device="cuda").to(torch.bfloat16)
    ref = p.network(X)
    capi.dnnmg_sync(p.ctx, 10_000_000)
    Y = torch.zeros_like(ref)
    capi.dnnmg_network_wait_test(p.ctx, X, Y, p.n_patches)
    with pytest.raises(capi.DnnmgError) as e:
        capi.dnnmg_sync(p.ctx, 30_000_000)
    assert e.value.status == -6
    again = p.network(X)
    capi.dnnmg_sync(p.ctx, 10_000_000)                  # the error was cleared
    assert torch.equal(again, ref)
    p.close()


def test_wait_expiry_in_a_whole_time_step_is_reported_by_that_step_only():
    # an expiry inside dnnmg_time_step is returned by that call (its
    # correction feeds the next coarse solve), and recorded in the context's
    # own error word: a second simulation on the same device that runs its
    # network meanwhile reports nothing and computes what it computes alone
    m = I.cavity_mesh(4)
    widths = (228, 256, 256, 81)
    Ws, ss, ts = I.network_weights(widths, seed=1)
    Ws[-1] = 0.05 * Ws[-1]
    prm = capi.dnnmg_solver_defaults(newton_rtol=1e-9, newton_atol=1e-10)
    ref = TimeLoop(m, 0.01, 0.01, 1.0, "bf16", widths, Ws, ss, ts, solver=prm).start().advance(2)
    a = TimeLoop(m, 0.01, 0.01, 1.0, "bf16", widths, Ws, ss, ts, solver=prm).start()
    b = TimeLoop(m, 0.01, 0.01, 1.0, "bf16", widths, Ws, ss, ts, solver=prm).start()
    a.advance(1)
    capi.dnnmg_arm_wait_test(a.path.ctx)
    with pytest.raises(capi.DnnmgError) as e:
        a.advance(1)
    assert e.value.status == -6
    b.advance(2)
    capi.dnnmg_sync(b.path.ctx, 10_000_000)
    assert torch.equal(b.x, ref.x) and torch.equal(b.F, ref.F)
    # the failed context still works: restart it and repeat the reference
    a.start().advance(2)
    assert torch.equal(a.x, ref.x) and torch.equal(a.F, ref.F)
    for t in (ref, a, b):
        t.close()


def test_host_step_reports_a_wait_expiry():
    m = I.cavity_mesh(4)
    widths = (228, 256, 256, 81)
    Ws, ss, ts = I.network_weights(widths, seed=1)
    p = PatchPath(m, 0.01, 0.01, 1.0, "bf16")
    p.set_network(widths, Ws, ss, ts)
    xc = torch.as_tensor(I.coarse_state(m, seed=1), dtype=torch.float32).pin_memory()
    F = torch.zeros((p.n_fine, 4), dtype=torch.float32).pin_memory()
    bf = torch.zeros_like(F)
    bc = torch.zeros((p.n_coarse, 4), dtype=torch.float32).pin_memory()
    capi.dnnmg_patch_step_host(p.ctx, xc, F, bf, bc)
    ok_bf = bf.clone()
    capi.dnnmg_arm_wait_test(p.ctx)
    with pytest.raises(capi.DnnmgError) as e:
        capi.dnnmg_patch_step_host(p.ctx, xc, F, bf, bc)
    assert e.value.status == -6
    capi.dnnmg_patch_step_host(p.ctx, xc, F, bf, bc)
    assert torch.equal(bf, ok_bf)
    p.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_misaligned_fields_are_refused_and_element_aligned_slices_read_alike(precision):
    # [n][4] fields move 4 values at a time and X rows in 16-byte pieces: a
    # view starting inside a row is refused with DNNMG_EINVAL before any
    # launch.  Y and d need only element alignment (serving hands over row
    # slices of one Y): the extension of a slice that starts one element into
    # an array equals that of an aligned copy bit for bit.
    m = I.cavity_mesh(4, jitter=0.1, seed=4)
    p = PatchPath(m, 0.01, 0.01, 1.0, precision)
    es = 8 if precision == "fp64" else 4
    xc = torch.zeros((p.n_coarse + 1, 4), dtype=p.dtype, device="cuda")
    F = torch.zeros((p.n_fine + 1, 4), dtype=p.dtype, device="cuda")
    r = p.field(p.n_fine, 4)
    X = torch.zeros((p.n_patches + 1) * p.sizes["n_in_padded"], dtype=p.x_dtype, device="cuda")
    d = p.field(p.n_fine, 3)
    n0 = p.launches()
    refused = [
        lambda: capi.dnnmg_prolongate(p.ctx, xc.data_ptr() + es, F),
        lambda: capi.dnnmg_residual(p.ctx, xc.data_ptr() + es, F, r),
        lambda: capi.dnnmg_residual(p.ctx, xc, F.data_ptr() + 2 * es, r),
        lambda: capi.dnnmg_local_restrict(p.ctx, xc, r, X.data_ptr() + 8),
        lambda: capi.dnnmg_rhs_restrict(p.ctx, xc, d, F.data_ptr() + es, None),
        lambda: capi.dnnmg_extend(p.ctx, p.field(p.n_patches * 81 + 1, 1).data_ptr() + 2, d),
    ]
    for call in refused:
        with pytest.raises(capi.DnnmgError) as e:
            call()
        assert e.value.status == -1
    assert p.launches() == n0
    rng = np.random.default_rng(7)
    Y_big = torch.as_tensor(rng.standard_normal(p.n_patches * 81 + 1), device="cuda").to(p.dtype)
    d_copy = p.extend(Y_big[1:].clone().reshape(p.n_patches, 81))
    d_slice = p.field(p.n_fine, 3)
    capi.dnnmg_extend(p.ctx, Y_big.data_ptr() + es, d_slice)
    torch.cuda.synchronize()
    assert torch.equal(d_slice, d_copy)
    p.close()
