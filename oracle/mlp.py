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
