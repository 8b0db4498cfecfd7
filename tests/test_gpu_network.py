"""The patch network on many rows (several output tiles per SM, pipeline
stages wrapping around, both TMEM accumulators reused) against the FP64
oracle, per row; and the tensor-core kernel's error flag stays clear."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from parity_util import patch_output_err  # noqa: E402
from paper_2307_14837_gb300 import build, capi, inputs as I  # noqa: E402
from paper_2307_14837_gb300.path import PatchPath  # noqa: E402
from oracle import mlp as omlp  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


@pytest.fixture(scope="module")
def mesh():
    # any mesh works for network-only calls; rows come from the caller
    return I.cavity_mesh(2)


def _rows(M, seed, n_in=228):
    X = np.zeros((M, 256))
    X[:, :n_in] = I.splitmix_normal(900 + seed, M * n_in).reshape(M, n_in)
    return X


@pytest.mark.parametrize("precision,widths,M,bn", [
    ("bf16", (228, 512, 512, 512, 81), 40000 + 77, True),   # 4-5 tiles per SM, ragged last tile
    ("bf16", (228, 1024, 1024, 81), 9000 + 5, False),
    ("bf16", (228, 192, 192, 81), 1000, True),              # N not a multiple of the tile
    ("fp32", (228, 512, 512, 81), 5000 + 3, True),
    # the paper's networks (Table 2): 240 inputs, 8 hidden layers of width
    # 750 or 512 with batch normalisation and skips; 750 is not a multiple
    # of the 256-column tile or of the 64-column K block
    ("bf16", (240,) + (750,) * 8 + (81,), 20000 + 19, True),
    ("bf16", (240,) + (512,) * 8 + (81,), 3000 + 1, True),
    ("fp32", (240,) + (750,) * 8 + (81,), 2000 + 3, True),
])
def test_network_rows_against_oracle(mesh, precision, widths, M, bn):
    feats = widths[0] - 216
    p = PatchPath(mesh, 0.01, 0.01, 1.0, precision, features=feats)
    Ws, ss, ts = I.network_weights(widths, seed=7, scale_shift=bn)
    # capacity of the context's activation buffers is its patch count, so
    # use a context whose mesh has at least M patches
    if p.n_patches < M:
        p.close()
        n = int(np.ceil(M ** (1 / 3)))
        p = PatchPath(I.cavity_mesh(n + (n % 2)), 0.01, 0.01, 1.0, precision, features=feats)
    p.set_network(widths, Ws, ss, ts, skip=True)
    X = _rows(M, 1, widths[0])
    Xd = torch.as_tensor(X, device="cuda").to(p.x_dtype)
    Y = p.network(Xd, M)
    torch.cuda.synchronize()
    capi.dnnmg_sync(p.ctx, 10_000_000)                # raises if a bounded wait expired
    Xo = Xd.double().cpu().numpy()[:, :widths[0]]     # the oracle sees the same (rounded) inputs
    ref = omlp.forward(Xo, Ws, ss, ts, skip=True)
    emax, ep99 = patch_output_err(Y.double().cpu().numpy(), ref)
    tol = 2e-2 if precision == "bf16" else 1e-5
    assert emax <= tol, (emax, ep99)
    p.close()


def test_fma_probe_measures_a_plausible_simt_peak():
    # the ALU roof of the element kernels is measured, not derived: FP32
    # between 10 and 200 TFLOP/s on this part (152 SMs x 128 lanes x 2 flop
    # x ~2 GHz = 80), FP64 far below FP32
    f32 = capi.dnnmg_probe_fma(capi.FP32, iters=16384)
    f64 = capi.dnnmg_probe_fma(capi.FP64, iters=512)
    assert 10.0 < f32 < 200.0, f32
    assert 0.0 < f64 < 0.5 * f32, (f32, f64)
