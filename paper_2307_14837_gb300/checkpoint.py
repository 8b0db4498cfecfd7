"""A DNN-MG time loop (Alg. 1) with checkpoint and resume.

``TimeLoop`` holds one simulation: its mesh and parameters, the patch
network, and the state the next step needs, which is the coarse solution
x^L_n, the coarse right-hand side b^L_{n+1} and the fine right-hand side
F = b^{L+J}_{n+1} left by the previous patch correction, plus the step
count.  ``save`` writes all of it to one .npz file (arrays in their own
dtypes); ``TimeLoop.load`` rebuilds the context and continues.  Every
stage is deterministic, so a resumed run reproduces the uninterrupted one
bit for bit.
"""
from __future__ import annotations

import json

import numpy as np
import torch

from . import capi
from . import inputs as I
from .path import PatchPath


class TimeLoop:
    def __init__(self, mesh, nu, dt, theta, precision, widths, Ws, scales=None, shifts=None, skip=True,
                 features=12, patch_levels=1, device="cuda", solver=None):
        self.mesh = {k: np.asarray(mesh[k]) for k in ("xyz", "cells", "vertex_bc")}
        self.mesh["meta"] = dict(mesh["meta"]) if "meta" in mesh else {}     # boundary data (kind, inflow)
        self.params = dict(nu=float(nu), dt=float(dt), theta=float(theta), precision=precision,
                           features=int(features), patch_levels=int(patch_levels), skip=bool(skip))
        self.net = (tuple(int(w) for w in widths), [np.asarray(W, dtype=np.float64) for W in Ws],
                    None if scales is None else [np.asarray(s, dtype=np.float64) for s in scales],
                    None if shifts is None else [np.asarray(t, dtype=np.float64) for t in shifts])
        self.path = PatchPath(self.mesh, nu, dt, theta, precision, device=device, features=features,
                              patch_levels=patch_levels)
        self.path.set_network(self.net[0], self.net[1], self.net[2], self.net[3], skip=skip)
        self.solver = solver
        self.step_count = 0
        self.x = self.b = self.F = None
        self.stats = []

    def start(self, x0=None):
        """Initial state: x0 [nv][4] (default: zero with the mesh's Dirichlet
        values); the first right-hand sides are the fine Rhs of the
        prolongated state and its restriction."""
        p = self.path
        if x0 is None:
            bc = self.mesh["vertex_bc"]
            dirc = (bc == 1) | (bc == 2)
            x0 = np.zeros((p.n_coarse, 4))
            x0[dirc, 0:3] = I.dirichlet_values(self.mesh, self.mesh["xyz"], bc)[dirc]
        self.x = torch.as_tensor(np.asarray(x0, dtype=np.float64), device=p.device).contiguous()
        F, bcf = p.rhs_restrict(self.x.to(p.dtype), torch.zeros((p.n_fine, 3), dtype=p.dtype, device=p.device))
        self.F = F
        self.b = bcf.double().contiguous()
        self.step_count = 0
        return self

    def advance(self, n_steps=1):
        """n_steps DNN-MG time steps (coarse Newton solve, then the patch
        correction that leaves the next right-hand sides)."""
        for _ in range(n_steps):
            self.stats.append(capi.dnnmg_time_step(self.path.ctx, 1, self.x, self.b, self.F, prm=self.solver))
            self.step_count += 1
        return self

    # -- checkpoint / resume -------------------------------------------------
    def save(self, path):
        torch.cuda.synchronize(self.path.device)
        widths, Ws, ss, ts = self.net
        arrays = dict(xyz=self.mesh["xyz"], cells=self.mesh["cells"], vertex_bc=self.mesh["vertex_bc"],
                      widths=np.asarray(widths, dtype=np.int64),
                      x=self.x.cpu().numpy(), b=self.b.cpu().numpy(), F=self.F.cpu().numpy(),
                      step=np.asarray(self.step_count, dtype=np.int64),
                      meta=np.asarray(json.dumps(self.mesh["meta"])),
                      params=np.asarray(json.dumps(self.params)))
        for i, W in enumerate(Ws):
            arrays[f"W{i}"] = W
            if ss is not None:
                arrays[f"scale{i}"] = ss[i]
            if ts is not None:
                arrays[f"shift{i}"] = ts[i]
        np.savez(path, **arrays)

    @classmethod
    def load(cls, path, device="cuda", solver=None):
        z = np.load(path, allow_pickle=False)
        prm = json.loads(str(z["params"]))
        widths = tuple(int(w) for w in z["widths"])
        L = len(widths) - 1
        Ws = [z[f"W{i}"] for i in range(L)]
        ss = [z[f"scale{i}"] for i in range(L)] if "scale0" in z else None
        ts = [z[f"shift{i}"] for i in range(L)] if "shift0" in z else None
        mesh = dict(xyz=z["xyz"], cells=z["cells"], vertex_bc=z["vertex_bc"], meta=json.loads(str(z["meta"])))
        run = cls(mesh, prm["nu"], prm["dt"], prm["theta"], prm["precision"], widths, Ws, ss, ts, skip=prm["skip"],
                  features=prm["features"], patch_levels=prm["patch_levels"], device=device, solver=solver)
        dev = run.path.device
        run.x = torch.as_tensor(z["x"], device=dev).contiguous()
        run.b = torch.as_tensor(z["b"], device=dev).contiguous()
        run.F = torch.as_tensor(z["F"], device=dev).contiguous()
        run.step_count = int(z["step"])
        return run

    def close(self):
        self.path.close()
