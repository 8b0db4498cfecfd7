"""Serving several DNN-MG simulations with one shared network launch per
step: each simulation's result is the same alone (its own time loop) and in
any mix of others, agrees with the FP64 oracle, admission respects the
memory budget and the row capacity, and a Poisson request stream reports
its throughput and latency."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2307_14837_gb300 import build, capi, inputs as I  # noqa: E402
from paper_2307_14837_gb300.path import PatchPath  # noqa: E402
from paper_2307_14837_gb300.serve import Request, Server, memory_estimate, poisson_requests  # noqa: E402

NU, DT = 0.01, 0.01
WIDTHS = (228, 64, 64, 81)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    capi.load()


def _net():
    Ws, ss, ts = I.network_weights(WIDTHS, seed=3)
    Ws[-1] = 0.05 * Ws[-1]
    return Ws, ss, ts


def _requests():
    return [Request("a", I.cavity_mesh(4), NU, DT, 1.0, 3),
            Request("b", I.cavity_mesh(6, jitter=0.15, seed=2), 2 * NU, DT, 1.0, 2),
            Request("c", I.cavity_mesh(2), NU, 2 * DT, 0.5, 4),
            Request("d", I.cavity_mesh(4, jitter=0.1, seed=5), NU, DT, 1.0, 2, solve=False)]


def _alone(req, precision, Ws, ss, ts):
    """The request on its own context through the single-simulation API."""
    p = PatchPath(req.mesh, req.nu, req.dt, req.theta, precision)
    p.set_network(WIDTHS, Ws, ss, ts)
    m = req.mesh
    dirc = (np.asarray(m["vertex_bc"]) == 1) | (np.asarray(m["vertex_bc"]) == 2)
    x0 = np.zeros((p.n_coarse, 4))
    x0[dirc, 0:3] = I.dirichlet_values(m, m["xyz"], m["vertex_bc"])[dirc]
    x = torch.as_tensor(x0, device="cuda")
    F, bcf = p.rhs_restrict(x.to(p.dtype), torch.zeros((p.n_fine, 3), dtype=p.dtype, device="cuda"))
    b = bcf.double().contiguous()
    X = torch.zeros((p.n_patches, 256), dtype=p.x_dtype, device="cuda")
    for _ in range(req.n_steps):
        if req.solve:
            capi.dnnmg_time_step(p.ctx, 1, x, b, F)
        else:
            capi.dnnmg_step_begin(p.ctx, x, b, F, X, solve=False)
            Y = p.network(X, p.n_patches)
            capi.dnnmg_step_end(p.ctx, Y, F, b)
    torch.cuda.synchronize()
    out = x.cpu().numpy(), F.double().cpu().numpy()
    p.close()
    return out


@pytest.mark.parametrize("precision,workers", [("fp64", 0), ("bf16", 0), ("bf16", 2)])
def test_mixed_equals_alone(precision, workers):
    Ws, ss, ts = _net()
    reqs = _requests()
    srv = Server(WIDTHS, Ws, ss, ts, memory_budget=1 << 33, max_rows=4096, precision=precision,
                 prepare_workers=workers)
    for r in reqs[:3]:
        srv.submit(r)
    while len(srv.live) + len(srv.results) < 3:
        srv.step()                              # a, b, c admitted (prepared in the background with workers)
    srv.submit(reqs[3])                         # d joins at a later step
    while srv.live or srv.queue:
        srv.step()
    srv.close()
    if workers == 0:
        assert len(srv.step_latencies) == 4     # c has 4 steps; d joined at step 2 and ran 2
    for r in reqs:
        xa, Fa = _alone(r, precision, Ws, ss, ts)
        got = srv.results[r.name]
        assert got["steps"] == r.n_steps
        np.testing.assert_array_equal(got["x"], xa, err_msg=r.name)
        np.testing.assert_array_equal(got["F"], Fa, err_msg=r.name)
        if r.solve:
            assert np.abs(xa[:, 0:3]).max() > 0.1


def test_whole_steps_with_multigrid_mixed_equal_alone():
    # whole DNN-MG steps (the coarse Newton-GMRES-multigrid solve on) for
    # nested meshes of different sizes served together: every result is the
    # one the simulation gets on its own, bit for bit
    Ws, ss, ts = _net()
    prm = capi.dnnmg_solver_defaults(mg_levels=3)
    reqs = [Request("m8", I.cavity_mesh(8, levels=2), NU, DT, 1.0, 3),
            Request("m8j", I.cavity_mesh(8, levels=2, jitter=0.1, seed=4), 2 * NU, DT, 1.0, 2),
            Request("m16", I.cavity_mesh(16, levels=3), NU, DT, 1.0, 2)]
    srv = Server(WIDTHS, Ws, ss, ts, memory_budget=1 << 33, max_rows=8192, precision="bf16", solver=prm)
    for r in reqs:
        srv.submit(r)
    while srv.live or srv.queue:
        srv.step()
    srv.close()
    for r in reqs:
        p = PatchPath(r.mesh, r.nu, r.dt, r.theta, "bf16")
        p.set_network(WIDTHS, Ws, ss, ts)
        m = r.mesh
        dirc = (np.asarray(m["vertex_bc"]) == 1) | (np.asarray(m["vertex_bc"]) == 2)
        x0 = np.zeros((p.n_coarse, 4))
        x0[dirc, 0:3] = I.dirichlet_values(m, m["xyz"], m["vertex_bc"])[dirc]
        x = torch.as_tensor(x0, device="cuda")
        F, bcf = p.rhs_restrict(x.to(p.dtype), torch.zeros((p.n_fine, 3), dtype=p.dtype, device="cuda"))
        b = bcf.double().contiguous()
        for _ in range(r.n_steps):
            st = capi.dnnmg_time_step(p.ctx, 1, x, b, F, prm)
            assert st["converged"] == 1
        torch.cuda.synchronize()
        assert capi.dnnmg_level_mg(p.ctx, capi.LEVEL_COARSE, prm)[-1] == 125   # down to 4^3
        np.testing.assert_array_equal(srv.results[r.name]["x"], x.cpu().numpy(), err_msg=r.name)
        np.testing.assert_array_equal(srv.results[r.name]["F"], F.double().cpu().numpy(), err_msg=r.name)
        p.close()


def test_served_fp64_matches_oracle():
    from oracle import dnnmg as odnnmg, fem, mesh as omesh
    Ws, ss, ts = _net()
    m = I.cavity_mesh(4)
    h = omesh.Hierarchy(m["xyz"], m["cells"], m["vertex_bc"])
    coarse = fem.Level(m["xyz"], m["cells"], m["vertex_bc"], True)
    prm = dict(m=1.0 / DT, nu=NU, alpha0=0.02, delta0=0.1, theta=1.0)
    bcv = I.dirichlet_values(m, m["xyz"], m["vertex_bc"])
    x0 = np.zeros((coarse.n, 4))
    x0[coarse.dirichlet, 0:3] = bcv[coarse.dirichlet]
    ref, _ = odnnmg.run(h, coarse, (Ws, ss, ts, True), x0, 3, prm, lambda t: bcv)
    srv = Server(WIDTHS, Ws, ss, ts, memory_budget=1 << 33, max_rows=4096, precision="fp64")
    srv.submit(Request("a", m, NU, DT, 1.0, 3))
    srv.submit(Request("other", I.cavity_mesh(6, jitter=0.1, seed=9), NU, DT, 1.0, 3))
    while srv.live or srv.queue:
        srv.step()
    srv.close()
    x = srv.results["a"]["x"]
    assert np.abs(x - ref[-1]).max() <= 1e-9 * np.abs(ref[-1]).max()


def test_admission_by_memory_and_rows():
    Ws, ss, ts = _net()
    big = Request("big", I.cavity_mesh(6), NU, DT, 1.0, 2)
    small = [Request(f"s{i}", I.cavity_mesh(4), NU, DT, 1.0, 2) for i in range(3)]
    huge = Request("huge", I.cavity_mesh(8), NU, DT, 1.0, 1)
    mb, ms = memory_estimate(big.mesh, "bf16"), memory_estimate(small[0].mesh, "bf16")
    budget = mb + ms // 2                       # the big one alone, or a few small ones
    assert memory_estimate(huge.mesh, "bf16") > budget and mb > 2 * ms
    srv = Server(WIDTHS, Ws, ss, ts, memory_budget=budget, max_rows=4096, precision="bf16")
    for r in [big] + small + [huge]:
        srv.submit(r)
    while srv.live or srv.queue:
        srv.step()
        assert srv.used <= srv.budget
    srv.close()
    events = [(e, n) for e, n, _ in srv.log]
    assert ("rejected", "huge") in events and "huge" not in srv.results
    # FIFO: the small ones wait until the big one has finished
    assert events.index(("admitted", "s0")) > events.index(("finished", "big"))
    assert set(srv.results) == {"big", "s0", "s1", "s2"}
    # row capacity: rows for one 64-patch mesh at a time, so they run one after another
    srv = Server(WIDTHS, Ws, ss, ts, memory_budget=1 << 33, max_rows=100, precision="bf16")
    for r in small:
        srv.submit(Request(r.name, r.mesh, r.nu, r.dt, r.theta, r.n_steps))
    while srv.live or srv.queue:
        srv.step()
        assert len(srv.live) <= 1
    srv.close()
    assert len(srv.step_latencies) == 6
    with pytest.raises(Exception):
        Server(WIDTHS, Ws, ss, ts, memory_budget=1 << 30, max_rows=0, precision="bf16")


def test_poisson_stream_reports_latency_and_throughput():
    Ws, ss, ts = _net()

    def make(i, u):
        # 4, 6 or 8 coarse cells per side (a jittered 2^3 cavity has one interior
        # vertex and leaves the pressure undetermined)
        n = 4 + 2 * int(u * 3)
        return Request(f"r{i}", I.cavity_mesh(n, jitter=0.1, seed=i), NU, DT, 1.0, 2 + i % 3)

    reqs = poisson_requests(8, rate=200.0, seed=1, make_request=make)
    assert all(b.arrival >= a.arrival for a, b in zip(reqs, reqs[1:]))
    srv = Server(WIDTHS, Ws, ss, ts, memory_budget=1 << 33, max_rows=8192, precision="bf16")
    stats = srv.run(reqs, timeout=120.0)
    srv.close()
    assert stats["simulations"] == 8
    assert stats["patches_per_s"] > 0
    assert 0 < stats["p50_step_latency_ms"] <= stats["p99_step_latency_ms"]
    for r in reqs:
        assert srv.results[r.name]["steps"] == r.n_steps
