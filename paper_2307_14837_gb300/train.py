"""Training of the patch network on corrections generated by the GPU solver.

* ``PatchNetFunction`` (torch.autograd.Function): forward and backward run
  libdnnmg's trainer kernels (tensor-core GEMMs in BF16, or FP32); the
  parameters are fp32 torch tensors owned by ``PatchNet``.
* ``AdamW``: the optimiser of Sec. 6.4 through libdnnmg's AdamW kernel
  (weight decay 1e-5 stands for the paper's Tikhonov term).
* ``make_samples``: training pairs from a fine-level simulation (Sec. 5.2):
  for each time step n the fine solution v_n (level L+1) and its right-hand
  side F_n = Rhs(v_{n-1}); the coarse state x^L_n solves the coarse system
  with the restricted rhs R F_n (what the DNN-MG coarse solve computes after
  exact corrections); the network input is the row X of x^L_n and of the
  residual F_n - A(P x^L_n), the target T = Q(v_n - P x^L_n), velocity only.
"""
from __future__ import annotations

import numpy as np
import torch

from . import capi, inputs as I
from .path import PatchPath

N_IN_PAD = 256


class PatchNetFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, trainer, n_layers, *params):
        Ws, bs = list(params[:n_layers]), list(params[n_layers:])
        B = X.shape[0]
        Y = torch.empty((B, capi.N_OUT), dtype=torch.float32, device=X.device)
        capi.dnnmg_trainer_forward(trainer, X, Ws, bs, Y, B)
        # the trainer reads X again in the backward pass: keep it alive
        ctx.x_keep = X
        ctx.trainer, ctx.n_layers = trainer, n_layers
        ctx.shapes = [p.shape for p in params]
        return Y

    @staticmethod
    def backward(ctx, dY):
        dY = dY.contiguous().float()
        grads = [torch.empty(s, dtype=torch.float32, device=dY.device) for s in ctx.shapes]
        capi.dnnmg_trainer_backward(ctx.trainer, dY, grads[:ctx.n_layers], grads[ctx.n_layers:])
        return (None, None, None, *grads)


class PatchNet:
    """fp32 parameters of the training form (W_i, b_i) and a trainer."""

    def __init__(self, widths, precision="bf16", max_batch=65536, seed=0, skip=True, device="cuda"):
        self.widths = tuple(widths)
        self.precision = capi.BF16 if precision == "bf16" else capi.FP32
        self.skip = skip
        Ws, _, _ = I.network_weights(widths, seed=seed)
        self.W = [torch.tensor(w, dtype=torch.float32, device=device, requires_grad=True) for w in Ws]
        self.b = [torch.zeros(w, dtype=torch.float32, device=device, requires_grad=True) for w in widths[1:-1]]
        self.max_batch = max_batch
        self.trainer = capi.dnnmg_trainer_create(widths, self.precision, max_batch,
                                                 torch.cuda.current_stream(), skip=skip)

    def params(self):
        return self.W + self.b

    def __call__(self, X):
        return PatchNetFunction.apply(X, self.trainer, len(self.W), *self.params())

    @torch.no_grad()
    def predict(self, X):
        """N(X) for any number of rows (chunks of at most max_batch, the last
        one padded with zero rows to a multiple of 64)."""
        out = []
        for i in range(0, X.shape[0], self.max_batch):
            x = X[i:i + self.max_batch]
            n = x.shape[0]
            if n % 64:
                x = torch.cat([x, torch.zeros((64 - n % 64, x.shape[1]), dtype=x.dtype, device=x.device)])
            out.append(self(x.contiguous())[:n])
        return torch.cat(out)

    def export(self, norm=None):
        """(Ws, scales, shifts) for dnnmg_set_network: scale 1, shift = bias.
        With ``norm`` (from fit_normalization) the input standardisation is
        folded into the first layer (W_1 / sigma, b_1 - W_1 mu / sigma) and the
        target scale into the last (t_scale W_L), so the exported network
        takes raw input rows."""
        Ws = [w.detach().double().cpu().numpy() for w in self.W]
        bs = [b.detach().double().cpu().numpy() for b in self.b]
        if norm is not None:
            n_in = self.widths[0]
            mu = torch.as_tensor(norm[0]).double().cpu().numpy()[:n_in]
            sig = torch.as_tensor(norm[1]).double().cpu().numpy()[:n_in]
            ts = float(norm[2])
            W1 = Ws[0] / sig[None, :]
            bs[0] = bs[0] - W1 @ mu
            Ws[0] = W1
            Ws[-1] = ts * Ws[-1]
        ss = [np.ones(w) for w in self.widths[1:]]
        shifts = bs + [np.zeros(self.widths[-1])]
        return Ws, ss, shifts

    def close(self):
        if self.trainer:
            capi.dnnmg_trainer_destroy(self.trainer)
            self.trainer = None


class AdamW:
    def __init__(self, params, lr=1e-3, betas=(0.9, 0.999), eps=1e-8, weight_decay=1e-5):
        self.params = list(params)
        self.lr, self.betas, self.eps, self.wd = lr, betas, eps, weight_decay
        self.m = [torch.zeros_like(p) for p in self.params]
        self.v = [torch.zeros_like(p) for p in self.params]
        self.t = 0

    def step(self):
        self.t += 1
        with torch.no_grad():
            for p, m, v in zip(self.params, self.m, self.v):
                capi.dnnmg_adamw(p, p.grad, m, v, self.lr, self.betas[0], self.betas[1], self.eps, self.wd, self.t,
                                 torch.cuda.current_stream())

    def zero_grad(self):
        for p in self.params:
            p.grad = None


def mse_loss(Y, T):
    """l2 loss of Sec. 6.4 with its gradient, through libdnnmg's kernel."""
    return _MSE.apply(Y, T)


class _MSE(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Y, T):
        loss = torch.empty(1, dtype=torch.float32, device=Y.device)
        dY = torch.empty_like(Y)
        capi.dnnmg_mse_loss(Y.shape[0], Y.contiguous(), T.contiguous(), loss, dY, torch.cuda.current_stream())
        ctx.save_for_backward(dY)
        return loss[0]

    @staticmethod
    def backward(ctx, g):
        (dY,) = ctx.saved_tensors
        return dY * g, None


def make_samples(mesh, nu, dt, theta, n_steps, x_dtype=torch.bfloat16, solver=None, features=12):
    """(X, T) training pairs from a fine-level simulation started at rest
    with the mesh's Dirichlet data.  X [n_steps * N_c][256] in x_dtype (216 +
    features used columns), T [n_steps * N_c][81] fp32.  Also returns the
    per-step arrays for evaluation."""
    prec = "bf16" if x_dtype == torch.bfloat16 else "fp32"
    f64 = PatchPath(mesh, nu, dt, theta, "fp64")          # fine solves, restriction
    low = PatchPath(mesh, nu, dt, theta, prec, features=features)   # network inputs as at inference
    dev = f64.device
    nv, nf, nc = f64.n_coarse, f64.n_fine, f64.n_patches
    kind = f64.mesh_data(capi.FINE_KIND)
    fxyz = f64.mesh_data(capi.FINE_XYZ)
    dirf = (kind == 1) | (kind == 2)
    pm = torch.as_tensor(f64.mesh_data(capi.PATCH_MAP).astype(np.int64), device=dev)
    dirc = (mesh["vertex_bc"] == 1) | (mesh["vertex_bc"] == 2)
    xc = np.zeros((nv, 4))
    xc[dirc, 0:3] = I.dirichlet_values(mesh, mesh["xyz"], mesh["vertex_bc"])[dirc]
    vf = np.zeros((nf, 4))
    vf[dirf, 0:3] = I.dirichlet_values(mesh, fxyz, kind)[dirf]
    xc, vf = torch.as_tensor(xc, device=dev), torch.as_tensor(vf, device=dev)
    F = torch.empty((nf, 4), dtype=torch.float64, device=dev)
    bL = torch.empty((nv, 4), dtype=torch.float64, device=dev)
    Xs, Ts, steps = [], [], []
    for n in range(n_steps):
        capi.dnnmg_level_rhs(f64.ctx, capi.LEVEL_FINE, vf, F)            # F_n = Rhs(v_{n-1})
        capi.dnnmg_solve(f64.ctx, capi.LEVEL_FINE, F, vf, solver)        # v_n
        capi.dnnmg_restrict(f64.ctx, F, bL)                              # R F_n
        capi.dnnmg_solve(f64.ctx, capi.LEVEL_COARSE, bL, xc, solver)     # x^L_n
        xt = f64.prolongate(xc)
        xcl, Fl = xc.to(low.dtype), F.to(low.dtype)
        r = low.residual(xcl, Fl)
        X = low.local_restrict(xcl, r)
        D = (vf - xt)[:, 0:3].float()
        T = D[pm].reshape(nc, 81)
        Xs.append(X.clone())
        Ts.append(T)
        steps.append(dict(x_coarse=xc.clone(), v_fine=vf.clone(), F=F.clone()))
    f64.close()
    low.close()
    return torch.cat(Xs), torch.cat(Ts), steps


def trajectory_errors(mesh, nu, dt, theta, steps, network=None, solver=None):
    """l2 velocity error against a fine trajectory (``steps`` from
    make_samples) of DNN-MG with ``network`` = (widths, Ws, scales, shifts)
    on the FP64 path, or of the plain coarse scheme when network is None;
    one value per time step (the corrected fine velocity P x^L + d for
    DNN-MG, P x^L for the plain scheme)."""
    p = PatchPath(mesh, nu, dt, theta, "fp64")
    dirc = (mesh["vertex_bc"] == 1) | (mesh["vertex_bc"] == 2)
    x0 = np.zeros((p.n_coarse, 4))
    x0[dirc, 0:3] = I.dirichlet_values(mesh, mesh["xyz"], mesh["vertex_bc"])[dirc]
    x = torch.as_tensor(x0, device=p.device)
    errs = []
    if network is not None:
        widths, Ws, ss, ts = network
        p.set_network(widths, Ws, ss, ts)
        bf, bc = p.rhs_restrict(x, torch.zeros((p.n_fine, 3), dtype=torch.float64, device=p.device))
    for s in steps:
        if network is not None:
            capi.dnnmg_time_step(p.ctx, 1, x, bc, bf, solver)
            d = torch.empty((p.n_fine, 3), dtype=torch.float64, device=p.device)
            capi.dnnmg_extend(p.ctx, capi.dnnmg_get_buffer(p.ctx, capi.BUF_Y), d)
            v = p.prolongate(x)[:, 0:3] + d
        else:
            capi.dnnmg_plain_step(p.ctx, capi.LEVEL_COARSE, 1, x, solver)
            v = p.prolongate(x)[:, 0:3]
        errs.append(float(torch.linalg.norm(v - s["v_fine"][:, 0:3])))
    p.close()
    return errs


def fit_normalization(X, T, n_in=228):
    """Per-column mean and standard deviation of the input rows (padding
    columns and constant columns get mean 0 / sigma 1) and one scale for the
    targets (their root mean square).  n_in = 228 (edge lengths) or 240
    (edge lengths, diagonals, angles)."""
    Xf = X.float()
    mu = Xf.mean(dim=0)
    sig = Xf.std(dim=0)
    # a column whose spread is far below that of its kind (the same unknown
    # of x~ or of r at the other patch nodes, or the edge lengths) would be
    # amplified without bound: floor sigma at 5% of the kind's median
    groups = [list(range(c, 108, 4)) for c in range(4)] + [list(range(108 + c, 216, 4)) for c in range(4)]
    groups.append(list(range(216, 228)))
    if n_in > 228:
        groups += [list(range(228, 232)), list(range(232, n_in))]   # diagonals, angles
    for g in groups:
        floor = 0.05 * float(sig[g].median())
        if floor <= 0.0:
            floor = 1.0
        sig[g] = torch.clamp(sig[g], min=floor)
    mu[n_in:] = 0.0
    sig[n_in:] = 1.0
    ts = float(torch.sqrt((T.float() ** 2).mean()))
    return mu, sig, (ts if ts > 0 else 1.0)


def normalize(X, norm, T=None):
    """Standardised input rows in X's dtype (and targets divided by the scale)."""
    mu, sig, ts = norm
    Xn = ((X.float() - mu[None, :]) / sig[None, :]).to(X.dtype)
    return (Xn, T / ts) if T is not None else Xn


def train(net, X, T, epochs=100, batch=4096, lr=1e-3, weight_decay=1e-5, seed=0, log=None):
    """AdamW on the l2 loss; batches are multiples of 64 (the tail of an epoch
    is dropped).  Returns the loss history (one value per epoch, mean over
    its batches)."""
    opt = AdamW(net.params(), lr=lr, weight_decay=weight_decay)
    n = X.shape[0]
    batch = min(batch, n) // 64 * 64
    g = torch.Generator(device="cpu").manual_seed(seed)
    hist = []
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).to(X.device)
        tot, cnt = 0.0, 0
        for i in range(0, n - batch + 1, batch):
            idx = perm[i:i + batch]
            Y = net(X[idx].contiguous())
            loss = mse_loss(Y, T[idx].contiguous())
            opt.zero_grad()
            loss.backward()
            opt.step()
            tot += float(loss.detach())
            cnt += 1
        hist.append(tot / max(cnt, 1))
        if log:
            log(ep, hist[-1])
    return hist
