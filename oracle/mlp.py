"""The patch network N of Sec. 4 (oracle, float64).

Layers f_1(x) = sigma(N_1(W_1 x)), f_i(x) = sigma(N_i(W_i x)) + x for
i = 2..L-1 where input and output widths match, f_L(x) = W_L x.  No linear
biases (Table 2's parameter counts hold only without them).  At inference
the batch normalisation N_i(z) = (z - mu_i) / s_i * gamma_i + beta_i is the
per-feature affine map z -> scale_i * z + shift_i with
scale = gamma / s and shift = beta - mu * gamma / s.  sigma is ReLU.

Pinned by: Table 2's parameter counts (integer exact), an explicit
triple-loop evaluation on small inputs, and folded vs unfolded normalisation.
"""
from __future__ import annotations

import numpy as np


def relu(z):
    return np.maximum(z, 0.0)


def forward(X, Ws, scales, shifts, skip=True, return_hidden=False):
    """Y = N(X) row by row.  X [n, widths[0]], Ws[i] [widths[i+1], widths[i]]."""
    h = np.asarray(X, dtype=np.float64)
    hidden = []
    L = len(Ws)
    for i in range(L):
        z = h @ np.asarray(Ws[i], dtype=np.float64).T
        z = z * scales[i][None, :] + shifts[i][None, :]
        if i < L - 1:
            out = relu(z)
            if skip and i > 0 and out.shape[1] == h.shape[1]:
                out = out + h
            h = out
            hidden.append(h)
        else:
            h = z
    return (h, hidden) if return_hidden else h


def loss_and_grads(X, Ws, bs, T, skip=True):
    """Training loss of Sec. 6.4 for one batch and its gradients (float64).

    The network is trained with the normalisation replaced by a per-feature
    bias b_i on hidden layers (scale 1): f_i(h) = relu(W_i h + b_i) (+ h).
    loss = (1 / B) sum_P ||Y_P - T_P||^2 (l2 over a patch's outputs, averaged
    over the B patches of the batch).  Returns (loss, dWs, dbs) by reverse-mode
    differentiation of that composition."""
    h = np.asarray(X, dtype=np.float64)
    B = h.shape[0]
    L = len(Ws)
    hs, zs, sk = [h], [], []
    for i in range(L - 1):
        z = h @ Ws[i].T + bs[i][None, :]
        a = relu(z)
        s = skip and i > 0 and a.shape[1] == h.shape[1]
        h = a + h if s else a
        zs.append(z)
        sk.append(s)
        hs.append(h)
    Y = h @ Ws[L - 1].T
    diff = Y - T
    loss = float(np.sum(diff * diff) / B)
    dWs = [None] * L
    dbs = [None] * (L - 1)
    dz = 2.0 * diff / B
    dWs[L - 1] = dz.T @ hs[L - 1]
    dh = dz @ Ws[L - 1]
    for i in range(L - 2, -1, -1):
        dzi = dh * (zs[i] > 0)
        dWs[i] = dzi.T @ hs[i]
        dbs[i] = dzi.sum(axis=0)
        dprev = dzi @ Ws[i]
        if sk[i]:
            dprev = dprev + dh
        dh = dprev
    return loss, dWs, dbs


def fold_batchnorm(gamma, beta, mu, s):
    """(scale, shift) equivalent to (z - mu) / s * gamma + beta."""
    scale = gamma / s
    return scale, beta - mu * scale


def trainable_parameters(n_in, n_hidden, n_out, n_hidden_layers=8, batchnorm=True):
    """Trainable parameters of the paper's feedforward net: weight matrices
    n_in x h, (n_hidden_layers - 1) x (h x h), h x n_out, plus gamma and beta
    of the normalisation after each hidden layer."""
    n = n_in * n_hidden + (n_hidden_layers - 1) * n_hidden * n_hidden + n_hidden * n_out
    if batchnorm:
        n += 2 * n_hidden * n_hidden_layers
    return n
