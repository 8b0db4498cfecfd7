"""Shared helpers of the GPU parity tests: cases, the oracle run, tolerances.

Tolerances (stated with the precision forms of the path):
  FP64: 1e-12 relative (max norm; the residual relative to max|F| + max|A|)
  FP32: 1e-5 relative, same norms
  BF16: network input within bf16 rounding; network output per patch
        ||dY_P||_2 <= 2e-2 max(||Y_P||_2, 0.1 median_P ||Y_P||_2);
        quantities downstream of the network 2e-2 relative.
Integer data (patch map, valences, boundary kinds) must match exactly.
"""
import functools

import numpy as np

from paper_2307_14837_gb300 import inputs as I
from oracle import dnnmg as odnnmg
from oracle import mesh as omesh

CASES = {
    # the cavity workload: 8^3 -> 16^3, Re 100, backward Euler, 228-256-256-81
    "cavity8": dict(mesh=("cavity", 8, 0.0), nu=0.01, dt=0.01, theta=1.0, widths=(228, 256, 256, 81), bn=False),
    # non-affine cells, Crank-Nicolson, folded normalisation, 3 hidden layers
    "cavity6_jitter": dict(mesh=("cavity", 6, 0.2), nu=0.01, dt=0.01, theta=0.5,
                           widths=(228, 64, 64, 64, 81), bn=True),
    # unstructured channel with a cylinder, do-nothing outflow
    "channel4": dict(mesh=("channel", 4, 0.0), nu=5e-4, dt=0.005, theta=0.5, widths=(228, 128, 128, 81), bn=True),
    # 27 patches: not a multiple of any block size
    "cavity3_ragged": dict(mesh=("cavity_plain", 3, 0.0), nu=0.01, dt=0.01, theta=0.5,
                           widths=(228, 32, 32, 81), bn=False),
    # a single patch: every node has valence 1
    "single_cell": dict(mesh=("cavity_plain", 1, 0.0), nu=0.01, dt=0.01, theta=1.0,
                        widths=(228, 16, 81), bn=False),
    # the paper's 24 geometry features (240 inputs, Table 2) on non-affine cells
    "cavity6_jitter_geo24": dict(mesh=("cavity", 6, 0.2), nu=0.01, dt=0.01, theta=0.5,
                                 widths=(240, 64, 64, 64, 81), bn=True, features=24),
    "channel4_geo24": dict(mesh=("channel", 4, 0.0), nu=5e-4, dt=0.005, theta=0.5,
                           widths=(240, 128, 128, 81), bn=True, features=24),
    # J = 2 patches (125 nodes, 1024 / 1012 inputs, 375 outputs, Table 2)
    "cavity4_j2": dict(mesh=("cavity", 4, 0.0), nu=0.01, dt=0.01, theta=1.0,
                       widths=(1024, 128, 128, 375), bn=False, features=24, patch_levels=2),
    "cavity2_jitter_j2": dict(mesh=("cavity", 2, 0.2), nu=0.01, dt=0.01, theta=0.5,
                              widths=(1012, 64, 64, 64, 375), bn=True, features=12, patch_levels=2),
}

TOL = {"fp64": 1e-12, "fp32": 1e-5, "bf16": 2e-2}


def make_mesh(spec, seed=0):
    kind, n, jit = spec
    if kind == "cavity":
        return I.cavity_mesh(n, jitter=jit, seed=seed + 11)
    if kind == "cavity_plain":
        return I.cavity_mesh(n, grouped=False)
    return I.channel_mesh(n, seed=seed)


@functools.lru_cache(maxsize=None)
def case_data(name, seed=0):
    """Inputs and the oracle's intermediates of one hot-path step."""
    c = CASES[name]
    m = make_mesh(c["mesh"], seed)
    hier = omesh.Hierarchy2 if c.get("patch_levels", 1) == 2 else omesh.Hierarchy
    h = hier(m["xyz"], m["cells"], m["vertex_bc"])
    xc = I.coarse_state(m, seed)
    # F stands in for the previous step's rhs: magnitude (1/dt) |v| |cell|
    ext = m["xyz"].max(axis=0) - m["xyz"].min(axis=0)
    F = I.fine_rhs(h.n_fine, seed, scale=(1.0 / c["dt"]) * float(np.prod(ext)) / (8 * h.n_patches))
    Ws, ss, ts = I.network_weights(c["widths"], seed=0, scale_shift=c["bn"])
    prm = dict(m=1.0 / c["dt"], theta=c["theta"], nu=c["nu"], alpha0=0.02, delta0=0.1)
    lev = odnnmg.fine_level(h)
    out = odnnmg.hot_path_step(h, (Ws, ss, ts, True), xc, F, prm, level=lev, features=c.get("features", 12))
    from oracle import transfer
    A = lev.operator(transfer.prolongate(h, xc), prm)
    return dict(case=c, mesh=m, h=h, xc=xc, F=F, net=(Ws, ss, ts), prm=prm, out=out, A=A)


def rel_max(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / (den if den > 0 else 1.0))


def residual_err(r_gpu, d):
    scale = np.abs(d["F"]).max() + np.abs(d["A"]).max()
    return float(np.abs(np.asarray(r_gpu, dtype=np.float64) - d["out"]["r"]).max() / scale)


def patch_output_err(Y_gpu, Y_ref):
    """max over patches of ||dY_P|| / max(||Y_P||, 0.1 median ||Y||) and its p99."""
    Y_gpu, Y_ref = np.asarray(Y_gpu, dtype=np.float64), np.asarray(Y_ref, dtype=np.float64)
    nrm = np.linalg.norm(Y_ref, axis=1)
    den = np.maximum(nrm, 0.1 * np.median(nrm))
    e = np.linalg.norm(Y_gpu - Y_ref, axis=1) / np.where(den > 0, den, 1.0)
    return float(e.max()), float(np.percentile(e, 99))
