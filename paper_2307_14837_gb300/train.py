"""Training of the patch network on corrections generated by the GPU solver.

* ``PatchNetFunction`` (torch.autograd.Function): forward and backward run
  libdnnmg's trainer kernels (tensor-core GEMMs in BF16, or FP32); the
  parameters are fp32 torch tensors owned by ``PatchNet``.
* ``AdamW``: the optimiser of Sec. 6.4 through libdnnmg's AdamW kernel
  (weight decay 1e-5 stands for the paper's Tikhonov term).
* ``make_samples``: training pairs from a fine simulation (Sec. 5.2): for
  each time step n the reference velocity v_n (the solve on level L+1, or on
  level L+2 injected onto level L+1) and the fine right-hand side
  F_n = Rhs_{L+1}(v_{n-1}); the coarse state x^L_n solves the coarse system
  with the restricted rhs R F_n (what the DNN-MG coarse solve computes after
  exact corrections); the network input is the row X of x^L_n and of the
  residual F_n - A(P x^L_n), the target T = Q(v_n - P x^L_n), velocity only.
* Standardisation, batch assembly and targets run in libdnnmg
  (dnnmg_column_stats, dnnmg_standardize, dnnmg_gather_rows,
  dnnmg_patch_targets); PyTorch holds the memory and the autograd wrapper.
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


def _rest_state(p, mesh, fine, prolongated_from=None):
    """Field at rest with the Dirichlet data of the fine (or coarse) nodes;
    with ``prolongated_from`` (a coarse field), the fine Dirichlet values
    are its prolongation instead of the boundary data."""
    if fine and prolongated_from is not None:
        xf = torch.empty((p.n_fine, 4), dtype=torch.float64, device=p.device)
        capi.dnnmg_prolongate(p.ctx, prolongated_from, xf)
        kind = p.mesh_data(capi.FINE_KIND)
        mask = torch.as_tensor((kind == 1) | (kind == 2), device=p.device)
        x = torch.zeros_like(xf)
        x[mask, 0:3] = xf[mask, 0:3]
        return x
    if fine:
        kind, xyz = p.mesh_data(capi.FINE_KIND), p.mesh_data(capi.FINE_XYZ)
    else:
        kind, xyz = mesh["vertex_bc"], mesh["xyz"]
    d = (kind == 1) | (kind == 2)
    x = np.zeros((xyz.shape[0], 4))
    x[d, 0:3] = I.dirichlet_values(mesh, xyz, kind)[d]
    return torch.as_tensor(x, device=p.device)


def make_samples(mesh, nu, dt, theta, n_steps, x_dtype=torch.bfloat16, solver=None, features=12, ref_levels=1,
                 ref_solver=None, keep_steps=True, fine_boundary="exact"):
    """(X, T) training pairs from a fine simulation started at rest with the
    mesh's Dirichlet data.  X [n_steps * N_c][256] in x_dtype (216 +
    features used columns), T [n_steps * N_c][81] fp32, both written by
    libdnnmg (dnnmg_local_restrict, dnnmg_patch_targets).  Also returns the
    per-step states (x^L_n, the reference velocity on level L+1, F_n) when
    keep_steps.

    ref_levels = 1: the reference v_n is the solve on level L+1 with
    F_n = Rhs_{L+1}(v_{n-1}).  ref_levels = 2 (the twofold refinement of
    Sec. 6.4): v_n is the solve on level L+2 (the fine level of a J = 2
    context, its own right-hand side from its previous state), injected
    onto level L+1 (its first n_fine(L+1) nodes), and F_n =
    Rhs_{L+1}(injected v_{n-1}).

    fine_boundary = "prolongated": the reference's Dirichlet values are the
    prolongation of the coarse Dirichlet data (the values the DNN-MG loop
    has there, where its correction is zero) instead of the boundary data
    evaluated at the fine nodes."""
    if ref_levels not in (1, 2):
        raise ValueError("ref_levels must be 1 or 2")
    prec = "bf16" if x_dtype == torch.bfloat16 else "fp32"
    f64 = PatchPath(mesh, nu, dt, theta, "fp64")          # level L+1 rhs, restriction, coarse solve, targets
    low = PatchPath(mesh, nu, dt, theta, prec, features=features)   # network inputs as at inference
    ref = f64 if ref_levels == 1 else PatchPath(mesh, nu, dt, theta, "fp64", patch_levels=2)
    dev = f64.device
    nv, nf, nc = f64.n_coarse, f64.n_fine, f64.n_patches
    xc = _rest_state(f64, mesh, fine=False)
    vr = _rest_state(ref, mesh, fine=True,                # reference state on its own level
                     prolongated_from=xc if fine_boundary == "prolongated" else None)
    F = torch.empty((nf, 4), dtype=torch.float64, device=dev)
    Fr = F if ref_levels == 1 else torch.empty((ref.n_fine, 4), dtype=torch.float64, device=dev)
    bL = torch.empty((nv, 4), dtype=torch.float64, device=dev)
    X = torch.empty((n_steps * nc, low.sizes["n_in_padded"]), dtype=low.x_dtype, device=dev)
    T = torch.empty((n_steps * nc, 81), dtype=torch.float32, device=dev)
    steps = []
    for n in range(n_steps):
        if ref_levels == 2:
            capi.dnnmg_level_rhs(f64.ctx, capi.LEVEL_FINE, vr[:nf], F)     # F_n = Rhs_{L+1}(inj v_{n-1})
        capi.dnnmg_level_rhs(ref.ctx, capi.LEVEL_FINE, vr, Fr)             # the reference level's rhs
        capi.dnnmg_solve(ref.ctx, capi.LEVEL_FINE, Fr, vr, ref_solver if ref_levels == 2 else solver)
        capi.dnnmg_restrict(f64.ctx, F, bL)                                # R F_n
        capi.dnnmg_solve(f64.ctx, capi.LEVEL_COARSE, bL, xc, solver)       # x^L_n
        v = vr[:nf]                                                        # v_n on level L+1
        xcl, Fl = xc.to(low.dtype), F.to(low.dtype)
        r = low.residual(xcl, Fl)
        capi.dnnmg_local_restrict(low.ctx, xcl, r, X[n * nc:(n + 1) * nc])
        capi.dnnmg_patch_targets(f64.ctx, xc, v, T[n * nc:(n + 1) * nc])
        if keep_steps:
            steps.append(dict(x_coarse=xc.clone(), v_fine=v.clone(), F=F.clone()))
    if ref is not f64:
        ref.close()
    f64.close()
    low.close()
    return X, T, steps


def rollout_samples(mesh, nu, dt, theta, steps, network, horizon=8, solver=None, precision="bf16", features=12):
    """Training pairs from the states the DNN-MG loop itself visits (the
    dataset aggregation of Ross, Gordon and Bagnell, 2011): from the
    reference state of every `horizon`-th step of ``steps`` (from
    make_samples) the loop runs `horizon` steps with ``network``; each
    step's input rows are the loop's own (its coarse state and the residual
    of its right-hand side), its targets the correction that takes the
    loop's prolongated coarse state to the reference velocity,
    Q(v_ref,n - P x_n).  Returns (X, T) as make_samples does."""
    p = PatchPath(mesh, nu, dt, theta, precision, features=features)    # the loop and its input rows
    f64 = PatchPath(mesh, nu, dt, theta, "fp64")                          # reference rhs and targets
    widths, Ws, ss, ts = network
    p.set_network(widths, Ws, ss, ts)
    dev, nv, nc = p.device, p.n_coarse, p.n_patches
    Xs, Ts = [], []
    bL = torch.empty((nv, 4), dtype=torch.float64, device=dev)
    try:
        for s0 in range(0, len(steps) - 1, horizon):
            x = steps[s0]["x_coarse"].clone()
            Fd = torch.empty_like(steps[s0]["v_fine"])
            capi.dnnmg_level_rhs(f64.ctx, capi.LEVEL_FINE, steps[s0]["v_fine"], Fd)   # Rhs_{L+1}(v_ref)
            capi.dnnmg_restrict(f64.ctx, Fd, bL)
            bf = Fd.to(p.dtype).contiguous()
            bc = bL.clone()
            for n in range(s0 + 1, min(s0 + 1 + horizon, len(steps))):
                Fn = bf.clone()                                  # the rhs this step solves with
                try:
                    capi.dnnmg_time_step(p.ctx, 1, x, bc, bf, solver)
                except capi.DnnmgError:
                    break                                        # a diverged rollout ends its samples
                xl = x.to(p.dtype)
                X = torch.empty((nc, p.sizes["n_in_padded"]), dtype=p.x_dtype, device=dev)
                capi.dnnmg_local_restrict(p.ctx, xl, p.residual(xl, Fn), X)
                T = torch.empty((nc, 81), dtype=torch.float32, device=dev)
                capi.dnnmg_patch_targets(f64.ctx, x, steps[n]["v_fine"], T)
                Xs.append(X)
                Ts.append(T)
    finally:
        p.close()
        f64.close()
    return torch.cat(Xs), torch.cat(Ts)


def velocity_errors(vel, ref):
    """The error measures of Sec. 6.5-6.6 of velocity snapshots ``vel``
    against ``ref`` (lists of [n][3] arrays, one per time step):
    e_v(n) = |v_n - v_ref,n| / |v_ref,n| and the time-integrated
    E_v = (sum_n |v_n - v_ref,n|^2 / sum_n |v_ref,n|^2)^(1/2) (equal steps)."""
    err = [float(np.linalg.norm(v - r)) for v, r in zip(vel, ref)]
    nrm = [float(np.linalg.norm(r)) for r in ref]
    return {"e_v": [e / n for e, n in zip(err, nrm)],
            "E_v": (sum(e * e for e in err) / sum(n * n for n in nrm)) ** 0.5}


def trajectory_errors(mesh, nu, dt, theta, steps, network=None, solver=None, precision="fp64", velocities=None):
    """l2 velocity errors |v_n - v_ref,n| per time step against the
    reference velocities of ``steps`` (from make_samples), for DNN-MG with
    ``network`` = (widths, Ws, scales, shifts) in the given precision form
    (the corrected fine velocity P x^L + d) or for the plain coarse scheme
    when network is None (P x^L).  The coarse state and the coarse
    right-hand side stay FP64 in every form.  With a list ``velocities``,
    the corrected velocities are appended to it (numpy [n][3])."""
    p = PatchPath(mesh, nu, dt, theta, precision if network is not None else "fp64")
    x = _rest_state(p, mesh, fine=False)
    errs = []
    try:
        if network is not None:
            widths, Ws, ss, ts = network
            p.set_network(widths, Ws, ss, ts)
            bf, bcf = p.rhs_restrict(x.to(p.dtype), torch.zeros((p.n_fine, 3), dtype=p.dtype, device=p.device))
            bc = bcf.double().contiguous()
        for s in steps:
            if network is not None:
                capi.dnnmg_time_step(p.ctx, 1, x, bc, bf, solver)
                d = torch.empty((p.n_fine, 3), dtype=p.dtype, device=p.device)
                capi.dnnmg_extend(p.ctx, capi.dnnmg_get_buffer(p.ctx, capi.BUF_Y), d)
                v = (p.prolongate(x.to(p.dtype))[:, 0:3] + d).double()
            else:
                capi.dnnmg_plain_step(p.ctx, capi.LEVEL_COARSE, 1, x, solver)
                v = p.prolongate(x)[:, 0:3]
            errs.append(float(torch.linalg.norm(v - s["v_fine"][:, 0:3])))
            if velocities is not None:
                velocities.append(v.cpu().numpy())
    finally:
        p.close()
    return errs


def column_groups(n_in=228):
    """Input columns by kind: each unknown of x~ and of r over the patch
    nodes, the edge lengths, and (n_in = 240) the diagonals and the angles."""
    groups = [list(range(c, 108, 4)) for c in range(4)] + [list(range(108 + c, 216, 4)) for c in range(4)]
    groups.append(list(range(216, 228)))
    if n_in > 228:
        groups += [list(range(228, 232)), list(range(232, n_in))]
    return groups


def normalization_from_stats(x_mean, x_sd, t_mean, t_sd, n_rows, n_in=228):
    """The standardisation from column statistics (numpy float64 arrays):
    input shift = column mean and scale = column deviation, the deviation
    floored at 5% of the lower median deviation of the columns of the same
    kind (a column whose spread is far below its kind's would be amplified
    without bound), shift 0 / scale 1 on the padding columns; one target
    scale, the root mean square of all target entries, from the target
    columns' means and sample deviations over n_rows rows.  Returns
    (mu, sigma, t_scale)."""
    mu = np.array(x_mean, dtype=np.float64)
    sig = np.array(x_sd, dtype=np.float64)
    for g in column_groups(n_in):
        floor = 0.05 * float(np.sort(sig[g])[(len(g) - 1) // 2])
        if floor <= 0.0:
            floor = 1.0
        sig[g] = np.maximum(sig[g], floor)
    mu[n_in:] = 0.0
    sig[n_in:] = 1.0
    tm, tsd = np.asarray(t_mean, dtype=np.float64), np.asarray(t_sd, dtype=np.float64)
    ms = float(np.mean(tsd ** 2 * (n_rows - 1) / n_rows + tm ** 2))
    ts = ms ** 0.5
    return mu, sig, (ts if ts > 0 else 1.0)


def fit_normalization(X, T, n_in=228):
    """Per-column mean and deviation of the input rows and the target scale
    (normalization_from_stats), the statistics computed by libdnnmg
    (dnnmg_column_stats) on the device tensors X and T."""
    def stats(A):
        mean = torch.empty(A.shape[1], dtype=torch.float64, device=A.device)
        sd = torch.empty_like(mean)
        capi.dnnmg_column_stats(A, mean, sd, stream=torch.cuda.current_stream(A.device))
        return mean.cpu().numpy(), sd.cpu().numpy()
    xm, xs = stats(X)
    tm, tsd = stats(T)
    return normalization_from_stats(xm, xs, tm, tsd, X.shape[0], n_in=n_in)


def normalize(X, norm, T=None):
    """Standardised input rows in X's dtype (and targets divided by the
    scale), written by libdnnmg (dnnmg_standardize) into new tensors."""
    mu, sig, ts = norm
    dev = X.device
    st = torch.cuda.current_stream(dev)
    Xn = torch.empty_like(X)
    capi.dnnmg_standardize(X, torch.as_tensor(mu, dtype=torch.float64, device=dev),
                           torch.as_tensor(sig, dtype=torch.float64, device=dev), Xn, stream=st)
    if T is None:
        return Xn
    Tn = torch.empty_like(T)
    capi.dnnmg_standardize(T, torch.zeros(T.shape[1], dtype=torch.float64, device=dev),
                           torch.full((T.shape[1],), float(ts), dtype=torch.float64, device=dev), Tn, stream=st)
    return Xn, Tn


def train(net, X, T, epochs=100, batch=4096, lr=1e-3, weight_decay=1e-5, seed=0, log=None, val=None,
          val_hist=None, noise=None):
    """AdamW on the l2 loss; batches are multiples of 64 (the tail of an epoch
    is dropped), gathered from X and T by libdnnmg (dnnmg_gather_rows) in a
    seeded random order.  Returns the loss history (one value per epoch,
    mean over its batches).  With ``val`` = (Xv, Tv) the validation loss is
    taken after every epoch (appended to ``val_hist`` when given) and the
    parameters of the epoch with the lowest one are kept (Sec. 6.4).  With
    ``noise`` = (c0, c1, sigma), every batch's input columns c0..c1-1 get
    seeded Gaussian noise of deviation sigma (dnnmg_add_noise) while its
    targets stay the reference's."""
    opt = AdamW(net.params(), lr=lr, weight_decay=weight_decay)
    n = X.shape[0]
    batch = min(batch, n) // 64 * 64
    st = torch.cuda.current_stream(X.device)
    Xb = torch.empty((batch, X.shape[1]), dtype=X.dtype, device=X.device)
    Tb = torch.empty((batch, T.shape[1]), dtype=T.dtype, device=T.device)
    g = torch.Generator(device="cpu").manual_seed(seed)
    hist = []
    best, best_params = None, None
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).to(X.device)
        tot, cnt = 0.0, 0
        for i in range(0, n - batch + 1, batch):
            idx = perm[i:i + batch]
            capi.dnnmg_gather_rows(X, idx, Xb, stream=st)
            capi.dnnmg_gather_rows(T, idx, Tb, stream=st)
            if noise is not None:
                capi.dnnmg_add_noise(Xb, noise[0], noise[1], noise[2], seed=(seed << 32) + ep * 65536 + i // batch,
                                     stream=st)
            Y = net(Xb)
            loss = mse_loss(Y, Tb)
            opt.zero_grad()
            loss.backward()
            opt.step()
            tot += float(loss.detach())
            cnt += 1
        hist.append(tot / max(cnt, 1))
        if val is not None:
            vl = validation_loss(net, *val)
            if val_hist is not None:
                val_hist.append(vl)
            if best is None or vl < best:
                best = vl
                best_params = [p.detach().clone() for p in net.params()]
        if log:
            log(ep, hist[-1])
    if best_params is not None:
        with torch.no_grad():
            for p, q in zip(net.params(), best_params):
                p.copy_(q)
    return hist


@torch.no_grad()
def validation_loss(net, Xv, Tv):
    """(1/rows) sum_P |N(X_P) - T_P|^2 over all validation rows."""
    Y = net.predict(Xv)
    loss = torch.empty(1, dtype=torch.float32, device=Y.device)
    capi.dnnmg_mse_loss(Y.shape[0], Y, Tv.contiguous(), loss, stream=torch.cuda.current_stream(Y.device))
    return float(loss)
