"""A context of the patch-correction path with torch-owned device buffers.

``PatchPath`` holds one libdnnmg context and allocates the caller-side
buffers (coarse state, fine right-hand side, outputs) as torch CUDA tensors;
every computation is a call into libdnnmg.
"""
from __future__ import annotations

import numpy as np
import torch

from . import capi

_FIELD_DTYPE = {capi.FP64: torch.float64, capi.FP32: torch.float32, capi.BF16: torch.float32}
_X_DTYPE = {capi.FP64: torch.float64, capi.FP32: torch.float32, capi.BF16: torch.bfloat16}
PRECISIONS = {"fp64": capi.FP64, "fp32": capi.FP32, "bf16": capi.BF16}


class PatchPath:
    def __init__(self, mesh, nu, dt, theta, precision, device="cuda", stream=None, features=12, patch_levels=1,
                 element=1):
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        self.device = torch.device(device)
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        torch.cuda.set_device(self.device)
        self.precision = precision
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.ctx = capi.dnnmg_create(mesh, nu, dt, theta, precision, self.stream, features=features,
                                     patch_levels=patch_levels, element=element)
        self.sizes = capi.dnnmg_get_sizes(self.ctx)
        self.dtype = _FIELD_DTYPE[precision]
        self.x_dtype = _X_DTYPE[precision]
        self.widths = None

    # -- allocation helpers ---------------------------------------------------
    @property
    def n_coarse(self):
        """Rows of the coarse fields: coarse vertices (Q1) or the nodes of the
        mesh refined once (Q2)."""
        return self.sizes["n_coarse_nodes"]

    @property
    def n_fine(self):
        return self.sizes["n_fine_nodes"]

    @property
    def n_patches(self):
        return self.sizes["n_patches"]

    def field(self, rows, cols, dtype=None):
        return torch.empty((rows, cols), dtype=dtype or self.dtype, device=self.device)

    def to_device(self, a: np.ndarray):
        return torch.as_tensor(np.ascontiguousarray(a), device=self.device).to(self.dtype)

    def mesh_data(self, item):
        return capi.dnnmg_get_mesh_data(self.ctx, item)

    # -- the path ---------------------------------------------------------------
    def set_network(self, widths, Ws, scales=None, shifts=None, skip=True):
        capi.dnnmg_set_network(self.ctx, widths, Ws, scales, shifts, skip)
        self.widths = tuple(widths)

    def prolongate(self, xc):
        out = self.field(self.n_fine, 4)
        capi.dnnmg_prolongate(self.ctx, xc, out)
        return out

    def residual(self, xc, F):
        r = self.field(self.n_fine, 4)
        capi.dnnmg_residual(self.ctx, xc, F, r)
        return r

    def local_restrict(self, xc, r):
        X = self.field(self.n_patches, self.sizes["n_in_padded"], self.x_dtype)
        capi.dnnmg_local_restrict(self.ctx, xc, r, X)
        return X

    def network(self, X, n_rows=None):
        n = X.shape[0] if n_rows is None else n_rows
        Y = self.field(n, self.sizes["n_out"])
        capi.dnnmg_network(self.ctx, X, Y, n)
        return Y

    def extend(self, Y):
        d = self.field(self.n_fine, 3)
        capi.dnnmg_extend(self.ctx, Y, d)
        return d

    def rhs_restrict(self, xc, d):
        bf = self.field(self.n_fine, 4)
        bc = self.field(self.n_coarse, 4)
        capi.dnnmg_rhs_restrict(self.ctx, xc, d, bf, bc)
        return bf, bc

    def step(self, xc, F, b_fine=None, b_coarse=None):
        bf = self.field(self.n_fine, 4) if b_fine is None else b_fine
        bc = self.field(self.n_coarse, 4) if b_coarse is None else b_coarse
        capi.dnnmg_patch_step(self.ctx, xc, F, bf, bc)
        return bf, bc

    def launches(self):
        return capi.dnnmg_launch_count(self.ctx)

    def close(self):
        if self.ctx:
            capi.dnnmg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
