"""Patches of J = 2 (125 nodes, level L+2) through the DNN-MG time loop on
the GPU: several steps against the FP64 oracle, the zero-network identity,
and the fine-level solver's refusal for J = 2.  Stage-wise parity of J = 2
patches is in test_gpu_parity.py."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2307_14837_gb300 import build, capi, inputs as I  # noqa: E402
from paper_2307_14837_gb300.path import PatchPath  # noqa: E402
from oracle import dnnmg as odnnmg, fem, mesh as omesh  # noqa: E402

NU, DT = 0.01, 0.01
PRM = dict(m=1.0 / DT, nu=NU, alpha0=0.02, delta0=0.1)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    capi.load()


def _setup(m, widths, precision="fp64", zero_last=False):
    Ws, ss, ts = I.network_weights(widths, seed=0)
    if zero_last:
        Ws[-1] = np.zeros_like(Ws[-1])
    p = PatchPath(m, NU, DT, 1.0, precision, features=widths[0] - 1000, patch_levels=2)
    p.set_network(widths, Ws, ss, ts)
    coarse = fem.Level(m["xyz"], m["cells"], m["vertex_bc"], True)
    bcv = I.dirichlet_values(m, m["xyz"], m["vertex_bc"])
    x0 = np.zeros((coarse.n, 4))
    x0[coarse.dirichlet, 0:3] = bcv[coarse.dirichlet]
    return p, (Ws, ss, ts), coarse, bcv, x0


def test_j2_time_loop_matches_oracle():
    # a 4^3 cavity with non-affine cells (the jittered 2^3 cavity has a single
    # interior vertex and no control of the pressure: singular for both sides)
    m = I.cavity_mesh(4, jitter=0.1, seed=4)
    widths = (1024, 32, 32, 375)
    p, net, coarse, bcv, x0 = _setup(m, widths)
    h = omesh.Hierarchy2(m["xyz"], m["cells"], m["vertex_bc"])
    ref, _ = odnnmg.run(h, coarse, net + (True,), x0, 2, dict(PRM, theta=1.0), lambda t: bcv, features=24)
    x = torch.as_tensor(x0, device="cuda")
    bf, bc = p.rhs_restrict(x, torch.zeros((p.n_fine, 3), dtype=torch.float64, device="cuda"))
    for k in range(2):
        capi.dnnmg_time_step(p.ctx, 1, x, bc, bf)
        err = np.abs(x.cpu().numpy() - ref[k]).max() / np.abs(ref[k]).max()
        assert err <= 1e-9, (k, err)
    p.close()


def test_j2_zero_network_equals_plain_scheme():
    m = I.cavity_mesh(4)
    p, _, coarse, bcv, x0 = _setup(m, (1012, 32, 375), zero_last=True)
    xa, xb = torch.as_tensor(x0, device="cuda"), torch.as_tensor(x0, device="cuda")
    bf, bc = p.rhs_restrict(xa, torch.zeros((p.n_fine, 3), dtype=torch.float64, device="cuda"))
    capi.dnnmg_time_step(p.ctx, 3, xa, bc, bf)
    capi.dnnmg_plain_step(p.ctx, capi.LEVEL_COARSE, 3, xb)
    a, b = xa.cpu().numpy(), xb.cpu().numpy()
    assert np.abs(a - b).max() <= 1e-10 * np.abs(b).max()
    assert np.abs(b[:, 0:3]).max() > 0.1
    # the fine level of a J = 2 context is level L+2 (16^3 cells), grouped
    # by the level-(L+1) cells
    assert capi.dnnmg_level_info(p.ctx, capi.LEVEL_FINE) == (17 ** 3, True)
    p.close()
