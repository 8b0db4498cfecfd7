"""The learned part: forward/backward kernels of the patch network behind
torch.autograd against the FP64 oracle (analytic gradients and finite
differences), the loss and AdamW kernels against their formulas, and what a
network trained on the GPU solver's corrections gains over no network."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2307_14837_gb300 import build, capi, inputs as I  # noqa: E402
from paper_2307_14837_gb300 import train as T  # noqa: E402
from oracle import mlp as omlp  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    capi.load()


def _batch(B, seed, dtype):
    X = np.zeros((B, 256))
    X[:, :228] = I.splitmix_normal(300 + seed, B * 228).reshape(B, 228)
    Xd = torch.as_tensor(X, device="cuda").to(dtype)
    Tg = 0.3 * I.splitmix_normal(400 + seed, B * 81).reshape(B, 81)
    return Xd, torch.as_tensor(Tg, device="cuda", dtype=torch.float32), Tg


def _grads(net, X, Tt):
    Y = net(X)
    loss = T.mse_loss(Y, Tt)
    for p in net.params():
        p.grad = None
    loss.backward()
    return float(loss.detach()), [p.grad.double().cpu().numpy() for p in net.params()]


@pytest.mark.parametrize("precision,tol", [("fp32", 2e-4), ("bf16", 3e-2)])
def test_gradients_match_oracle(precision, tol):
    widths = (228, 64, 64, 64, 81)
    net = T.PatchNet(widths, precision=precision, max_batch=256, seed=3)
    with torch.no_grad():
        for b in net.b:
            b.copy_(0.05 * torch.randn(b.shape, generator=torch.Generator().manual_seed(b.numel())).cuda())
    X, Tt, Tg = _batch(192, 1, torch.bfloat16 if precision == "bf16" else torch.float32)
    loss, g = _grads(net, X, Tt)
    Ws = [w.detach().double().cpu().numpy() for w in net.W]
    bs = [b.detach().double().cpu().numpy() for b in net.b]
    Xo = X.double().cpu().numpy()[:, :228]
    ref_loss, dWs, dbs = omlp.loss_and_grads(Xo, Ws, bs, Tg, skip=True)
    assert abs(loss - ref_loss) <= tol * ref_loss
    for got, want in zip(g, dWs + dbs):
        assert np.linalg.norm(got - want) <= tol * np.linalg.norm(want)
    if precision == "fp32":
        # direct central differences of the loss for a few weights
        eps = 1e-5
        for li, (r, c) in [(0, (3, 7)), (1, (10, 20)), (3, (80, 63))]:
            Wp = [w.copy() for w in Ws]
            Wm = [w.copy() for w in Ws]
            Wp[li][r, c] += eps
            Wm[li][r, c] -= eps
            fd = (omlp.loss_and_grads(Xo, Wp, bs, Tg)[0] - omlp.loss_and_grads(Xo, Wm, bs, Tg)[0]) / (2 * eps)
            assert abs(g[li][r, c] - fd) <= 1e-3 * max(abs(fd), 1e-3 * np.abs(g[li]).max())
    net.close()


def test_loss_and_adamw_kernels():
    B = 128
    Y = torch.randn(B, 81, device="cuda")
    Tt = torch.randn(B, 81, device="cuda")
    loss = T.mse_loss(Y, Tt)
    ref = ((Y - Tt) ** 2).sum().item() / B
    assert abs(loss.item() - ref) <= 1e-5 * ref
    w = torch.randn(1000, device="cuda")
    g = torch.randn(1000, device="cuda")
    m = 0.1 * torch.randn(1000, device="cuda")
    v = torch.rand(1000, device="cuda")
    w0, m0, v0 = w.clone(), m.clone(), v.clone()
    lr, b1, b2, eps, wd, t = 1e-3, 0.9, 0.999, 1e-8, 1e-5, 3
    capi.dnnmg_adamw(w, g, m, v, lr, b1, b2, eps, wd, t, torch.cuda.current_stream())
    m1 = b1 * m0 + (1 - b1) * g
    v1 = b2 * v0 + (1 - b2) * g * g
    w1 = w0 - lr * ((m1 / (1 - b1 ** t)) / (torch.sqrt(v1 / (1 - b2 ** t)) + eps) + wd * w0)
    assert torch.allclose(m, m1, rtol=1e-6, atol=1e-7) and torch.allclose(v, v1, rtol=1e-6, atol=1e-7)
    assert torch.allclose(w, w1, rtol=1e-5, atol=1e-7)


def test_trained_network_gains_over_the_method_without_it():
    """Trained (BF16 kernels, AdamW) on GPU-solver corrections of the cavity at
    two viscosities, evaluated at a third: (1) the predicted correction
    removes most of the gap between the prolongated coarse solution and the
    fine solution, where the method without the network adds nothing;
    (2) in the DNN-MG time loop the velocity error against the fine-mesh
    solution is below the plain coarse scheme's at every step."""
    m = I.cavity_mesh(8)
    dt, steps = 0.01, 8
    Xs, Ts = [], []
    for nu in (0.008, 0.0125):
        X, Tg, _ = T.make_samples(m, nu, dt, 1.0, steps)
        Xs.append(X)
        Ts.append(Tg)
    X, Tg = torch.cat(Xs), torch.cat(Ts)
    Xh, Th, held = T.make_samples(m, 0.01, dt, 1.0, steps)
    norm = T.fit_normalization(X, Tg)
    Xn, Tn = T.normalize(X, norm, Tg)
    widths = (228, 256, 256, 81)
    net = T.PatchNet(widths, precision="bf16", max_batch=4096, seed=0)
    hist = T.train(net, Xn, Tn, epochs=300, batch=1024, lr=1e-3)
    assert hist[-1] < 0.01 * hist[0]
    Y = net.predict(T.normalize(Xh, norm)) * norm[2]
    gap = torch.linalg.norm(Th).item()                  # no network: correction 0
    err = torch.linalg.norm(Th - Y).item()
    assert err < 0.2 * gap, (err, gap)
    e_net = T.trajectory_errors(m, 0.01, dt, 1.0, held, network=(widths, *net.export(norm)))
    e_plain = T.trajectory_errors(m, 0.01, dt, 1.0, held)
    assert all(a < b for a, b in zip(e_net, e_plain)), (e_net, e_plain)
    assert sum(e_net) < 0.85 * sum(e_plain), (e_net, e_plain)
    net.close()
