"""Benchmark of the DNN-MG patch-correction step on GB300.

A step is one pass of the whole patch path (prolongation, fine residual,
local restriction, patch network, extension, corrected rhs and restriction)
over one coarse solution of the channel workload: ~314k coarse hexahedra
(channel 2.5 x 0.41 x 0.41 with a seeded cylinder, nz = 37), ~2.5M fine cells,
one patch per coarse cell, BF16 network 228-1024x4-81 with FP32 accumulation,
FP32 fields, Crank-Nicolson dt = 0.005, Re = 200.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank runs an independent replica (weak scaling;
the path has no data exchange between simulations); the time is the max over
ranks.  --impl reference times the FP64 CPU oracle on a bounded sample of the
same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DNN-MG time steps/sec and patches/sec (BF16 batched vs plain FP64, same GPU, equal error)"
UNIT = "steps/s"
WIDTHS = (228, 1024, 1024, 1024, 1024, 81)
NZ = 37
DT, THETA = 0.005, 0.5
STAGES = ("residual", "local_restrict", "network", "extend", "rhs_restrict")
FP32_LANES_PER_SM = 128          # FP32 FMA lanes per SM (sm_100 family)
# Work per patch of each stage (FP32 fields, BF16 network input), counted
# from the kernels' arithmetic and the unique data they must move:
#   residual: element integrals 64 Gauss points x ~274 FMA-pipe operations
#     (monomial form) = 17.5k ops = 35.1 kflop, plus the gather of the
#     per-patch partials (27 x 16 B written and read, CSR 27 x 4 B, F and r
#     at ~8 unique fine nodes x 16 B each)
#   local_restrict: x^L (~1 unique coarse node x 16 B), r (~8 x 16 B), edge
#     lengths 48 B read; X row 256 x 2 B written
#   extend: Y 81 x 4 B and the CSR 27 x 4 B read, d (~8 x 12 B) written
#   rhs_restrict: element integrals 64 x ~253 ops = 32.4 kflop, gathers of
#     the partials (27 x 16 B) and corner partials (8 x 16 B), b (~8 x 16 B)
#     and b^L (~1 x 16 B) written
# On a patch whose cell is a parallelepiped the Jacobian is constant: its ~59
# operations per Gauss point (J, cofactors, det, inverse, weight) are done
# once per fine cell, not at each of the 8 points.
STAGE_WORK = {
    "residual": {"bound": "alu", "flop": 64 * 274 * 2, "bytes": 16 + 27 * 16 * 2 + 27 * 4 + 8 * 16 * 2},
    "local_restrict": {"bound": "hbm", "bytes": 16 + 8 * 16 + 48 + 256 * 2},
    "extend": {"bound": "hbm", "bytes": 81 * 4 + 27 * 4 + 8 * 12},
    "rhs_restrict": {"bound": "alu", "flop": 64 * 253 * 2, "bytes": 16 + 8 * 12 + 27 * 16 * 2 + 8 * 16 * 2 + 8 * 16 + 16},
}
JACOBIAN_OPS = 59                # per Gauss point, saved 7 times in 8 on parallelepiped cells


def parallelepiped_fraction(mesh):
    """Share of coarse cells that are parallelepipeds to 16 float rounding
    units of their edges (corners relative to corner 0): the cells whose
    element integrals form the Jacobian once per fine cell."""
    import numpy as np
    X = mesh["xyz"].astype(np.float32)[mesh["cells"]]
    X = X - X[:, 0:1, :]
    c3 = X[:, 3] - X[:, 2] - X[:, 1]
    c5 = X[:, 5] - X[:, 4] - X[:, 1]
    c6 = X[:, 6] - X[:, 4] - X[:, 2]
    c7 = X[:, 7] - X[:, 6] - X[:, 5] + X[:, 4] - c3
    edge = np.abs(X[:, [1, 2, 4]]).max(axis=(1, 2))
    bend = np.abs(np.stack([c3, c5, c6, c7], 1)).max(axis=(1, 2))
    return float(np.mean(bend <= 16 * np.finfo(np.float32).eps * edge))


def element_flop(name, affine_frac):
    """Element-integral flop per patch of an ALU-bound stage for a mesh with
    the given share of parallelepiped cells."""
    saved = JACOBIAN_OPS * 7 * 64 * 2 // 8
    return STAGE_WORK[name]["flop"] - affine_frac * saved


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def max_over_ranks(x, world, device):
    """Largest value of x over the ranks of the default process group (the
    slowest replica bounds the whole job)."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(steps, elapsed_ms, world):
    """Steps per second of the whole job: every replica runs `steps` steps in
    at most elapsed_ms (weak scaling, one simulation per rank)."""
    return world * steps / (elapsed_ms / 1000.0)


def network_traffic(n_patches):
    """DRAM bytes of one network stage from the committed ncu record
    (profiles/network_traffic.json: dram read + write of the 5 layer launches
    on a smaller channel case, per patch), scaled to n_patches; None when the
    GEMM source has changed since the counters were taken."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "network_traffic.json")))
        src = open(os.path.join(ROOT, rec["source_file"]), "rb").read()
    except (OSError, KeyError, ValueError):
        return None
    if hashlib.sha256(src).hexdigest()[:16] != rec.get("source_sha256_16"):
        return None
    return rec["bytes_per_patch"] * n_patches


def stage_rooflines(stage_ms, n_patches, peaks, peak_src, clocks, affine_frac=0.0, fp32_tflops=None):
    """Per-stage time and the fraction of the roof that binds it: FP32 ALU
    for the element-integral stages (their work counted for the mesh's share
    of parallelepiped cells) against the FMA throughput measured by
    dnnmg_probe_fma (else 152 SMs x 128 lanes x 2 flop x the median SM clock
    under load), HBM (measured copy bandwidth) for the gathers, BF16 tensor
    (measured sustained) for the network."""
    if fp32_tflops:
        alu_tflops, alu_src = fp32_tflops, "FP32 ALU measured by the FMA probe"
    else:
        sm_ghz = (clocks.get("sm_mhz") or 2070.0) / 1000.0
        alu_tflops = 152 * FP32_LANES_PER_SM * 2 * sm_ghz / 1000.0
        alu_src = "FP32 ALU from unit counts x median SM clock"
    out = {}
    for name in STAGES:
        ms = stage_ms[name]
        e = {"ms": round(ms, 4)}
        if name == "network":
            tf = network_flops_per_patch() * n_patches / (ms / 1000.0) / 1e12
            pk = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
            e.update(bound="tensor", achieved=round(tf, 1), peak=pk, unit="TFLOP/s", frac=round(tf / pk, 3))
        else:
            w = STAGE_WORK[name]
            gbs = w["bytes"] * n_patches / (ms / 1000.0) / 1e9
            if w["bound"] == "alu":
                tf = element_flop(name, affine_frac) * n_patches / (ms / 1000.0) / 1e12
                e.update(bound="alu", achieved=round(tf, 2), peak=round(alu_tflops, 1), unit="TFLOP/s",
                         frac=round(tf / alu_tflops, 3), hbm_gbs=round(gbs, 1))
            else:
                e.update(bound="hbm", achieved=round(gbs, 1), peak=peaks["hbm_gbs"], unit="GB/s",
                         frac=round(gbs / peaks["hbm_gbs"], 3))
        out[name] = e
    out["peak_source"] = f"{peak_src} (HBM copy, BF16 sustained); {alu_src}"
    out["parallelepiped_cells"] = round(affine_frac, 4)
    return out


def network_flops_per_patch(widths=WIDTHS):
    return sum(2 * widths[i] * widths[i + 1] for i in range(len(widths) - 1))


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "20"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def build_workload(seed=0, nz=NZ):
    from paper_2307_14837_gb300 import inputs as I
    m = I.channel_mesh(nz, seed=seed)
    nu = m["meta"]["D"] / 200.0          # Re = mean inflow * D / nu = 200
    return m, nu


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_2307_14837_gb300 import capi, inputs as I
    from paper_2307_14837_gb300.path import PatchPath

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    m, nu = build_workload(seed=rank, nz=args.nz)
    stream = torch.cuda.Stream(dev)
    p = PatchPath(m, nu, DT, THETA, "bf16", device=dev, stream=stream)
    Ws, ss, ts = I.network_weights(WIDTHS, seed=0)
    p.set_network(WIDTHS, Ws, ss, ts, skip=True)
    nc, nf, nv = p.n_patches, p.n_fine, p.n_coarse
    xc_h = I.coarse_state(m, seed=rank).astype(np.float32)
    F_h = I.fine_rhs(nf, seed=rank, scale=(1 / DT) * 0.42 / (8 * nc)).astype(np.float32)
    xc = p.to_device(xc_h)
    Fa = p.to_device(F_h)
    Fb = torch.empty_like(Fa)
    bc = p.field(nv, 4)
    r = p.field(nf, 4)
    X = p.field(nc, 256, torch.bfloat16)
    Y = p.field(nc, 81)
    d = p.field(nf, 3)
    ctx = p.ctx

    def step(F_in, F_out, ev=None):
        # the stages of dnnmg_patch_step, called one by one so that each
        # stage can be timed on its own (same kernels, same order); ev[i]
        # is recorded before stage i and ev[5] after the last
        def mark(i):
            if ev:
                ev[i].record(stream)
        mark(0)
        capi.dnnmg_residual(ctx, xc, F_in, r)
        mark(1)
        capi.dnnmg_local_restrict(ctx, xc, r, X)
        mark(2)
        capi.dnnmg_network(ctx, X, Y, nc)
        mark(3)
        capi.dnnmg_extend(ctx, Y, d)
        mark(4)
        capi.dnnmg_rhs_restrict(ctx, xc, d, F_out, bc)
        mark(5)

    with torch.cuda.stream(stream):
        for i in range(args.warmup):
            step(Fa, Fb)
            Fa, Fb = Fb, Fa
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        n0 = capi.dnnmg_launch_count(ctx)
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(args.steps)]
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        with Clocks(local_rank) as clk:
            t0.record(stream)
            for i in range(args.steps):
                step(Fa, Fb, evs[i])
                Fa, Fb = Fb, Fa
            t1.record(stream)
            torch.cuda.synchronize(dev)
        launches = capi.dnnmg_launch_count(ctx) - n0
        if world > 1:
            torch.distributed.barrier()
        elapsed_ms = t0.elapsed_time(t1)
        stage_ms = {name: statistics.mean(e[i].elapsed_time(e[i + 1]) for e in evs) for i, name in enumerate(STAGES)}
        net_ms = [e[2].elapsed_time(e[3]) for e in evs]

    # end to end through the C ABI with host buffers (pinned)
    xc_p = torch.from_numpy(xc_h).pin_memory()
    F_p = torch.from_numpy(F_h).pin_memory()
    bf_p = torch.empty((nf, 4), dtype=torch.float32).pin_memory()
    bc_p = torch.empty((nv, 4), dtype=torch.float32).pin_memory()
    capi.dnnmg_set_stream(ctx, stream)
    for _ in range(max(1, args.warmup // 2)):
        capi.dnnmg_patch_step_host(ctx, xc_p, F_p, bf_p, bc_p)
    torch.cuda.synchronize(dev)
    te0 = time.perf_counter()
    for _ in range(args.steps):
        capi.dnnmg_patch_step_host(ctx, xc_p, F_p, bf_p, bc_p)
    e2e_s = time.perf_counter() - te0

    # the plain FP64 form of the same step on the same GPU
    fp64 = None
    if not args.no_fp64 and rank == 0:
        q = PatchPath(m, nu, DT, THETA, "fp64", device=dev, stream=stream)
        q.set_network(WIDTHS, Ws, ss, ts, skip=True)
        xq, Fq = q.to_device(xc_h.astype(np.float64)), q.to_device(F_h.astype(np.float64))
        bfq, bcq = q.field(nf, 4), q.field(nv, 4)
        with torch.cuda.stream(stream):
            q.step(xq, Fq, bfq, bcq)
            torch.cuda.synchronize(dev)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(3):
                q.step(xq, Fq, bfq, bcq)
            b.record(stream)
            torch.cuda.synchronize(dev)
        ms = a.elapsed_time(b) / 3
        fp64 = {"ms_per_step": round(ms, 3), "steps_per_s": round(1000.0 / ms, 4),
                "patches_per_s": round(nc * 1000.0 / ms, 1), "timed_steps": 3}
        q.close()

    # the FP32 form (FP32 fields, FP32 SIMT network) of the same step
    fp32 = None
    if not args.no_fp64 and rank == 0:
        q = PatchPath(m, nu, DT, THETA, "fp32", device=dev, stream=stream)
        q.set_network(WIDTHS, Ws, ss, ts, skip=True)
        xq, Fq = q.to_device(xc_h), q.to_device(F_h)
        bfq, bcq = q.field(nf, 4), q.field(nv, 4)
        with torch.cuda.stream(stream):
            q.step(xq, Fq, bfq, bcq)
            torch.cuda.synchronize(dev)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(3):
                q.step(xq, Fq, bfq, bcq)
            b.record(stream)
            torch.cuda.synchronize(dev)
        ms = a.elapsed_time(b) / 3
        fp32 = {"ms_per_step": round(ms, 3), "steps_per_s": round(1000.0 / ms, 3),
                "patches_per_s": round(nc * 1000.0 / ms, 1), "timed_steps": 3}
        q.close()

    # the paper's forms (Sec. 5.2, Table 2): 24 geometry features and 8 hidden
    # layers of width 750 with skips, for J = 1 on this workload and for
    # J = 2 (125-node patches on level L+2) on a coarser channel with about
    # as many fine cells
    paper = None
    if not args.no_fp64 and rank == 0:
        paper = {}
        # the channel at ~40k coarse hex with the FP32 network 228-512x3-81
        mc, nuc = build_workload(seed=rank, nz=19)
        q = PatchPath(mc, nuc, DT, THETA, "fp32", device=dev, stream=stream)
        wd = (228, 512, 512, 512, 81)
        Wp, sp, tp = I.network_weights(wd, seed=0)
        q.set_network(wd, Wp, sp, tp, skip=True)
        xq = q.to_device(I.coarse_state(mc, seed=rank).astype(np.float32))
        Fq = q.to_device(I.fine_rhs(q.n_fine, seed=rank, scale=(1 / DT) * 0.42 / (8 * q.n_patches)).astype(np.float32))
        bfq, bcq = q.field(q.n_fine, 4), q.field(q.n_coarse, 4)
        with torch.cuda.stream(stream):
            for _ in range(2):
                q.step(xq, Fq, bfq, bcq)
            torch.cuda.synchronize(dev)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(10):
                q.step(xq, Fq, bfq, bcq)
            b.record(stream)
            torch.cuda.synchronize(dev)
        ms = a.elapsed_time(b) / 10
        paper["channel_40k_fp32_228_512x3_81"] = {
            "workload": f"channel nz=19: {q.n_patches} patches, {q.n_fine} fine nodes, FP32 fields and network",
            "ms_per_step": round(ms, 3), "steps_per_s": round(1000.0 / ms, 2),
            "patches_per_s": round(q.n_patches * 1000.0 / ms, 1), "timed_steps": 10}
        q.close()
        for name, J, el, nz_p in (("j1_240_750x8_81", 1, 1, args.nz), ("j2_1024_750x8_375", 2, 1, max(4, args.nz // 2)),
                                  ("q2_1024_750x8_375", 2, 2, max(4, args.nz // 2))):
            mp, nup = build_workload(seed=rank, nz=nz_p)
            q = PatchPath(mp, nup, DT, THETA, "bf16", device=dev, stream=stream, features=24, patch_levels=J,
                          element=el)
            wd = (q.sizes["n_in"],) + (750,) * 8 + (q.sizes["n_out"],)
            Wp, sp, tp = I.network_weights(wd, seed=0, scale_shift=True)
            q.set_network(wd, Wp, sp, tp, skip=True)
            if el == 2:   # a smooth field at the coarse Q2 nodes (level L+1)
                xm = I.smooth_field(q.mesh_data(capi.COARSE_XYZ), rank)
                xq = q.to_device(xm.astype(np.float32))
            else:
                xq = q.to_device(I.coarse_state(mp, seed=rank).astype(np.float32))
            Fq = q.to_device(I.fine_rhs(q.n_fine, seed=rank, scale=(1 / DT) * 0.42 / (8 * q.n_patches)).astype(np.float32))
            bfq, bcq = q.field(q.n_fine, 4), q.field(q.n_coarse, 4)
            with torch.cuda.stream(stream):
                for _ in range(2):
                    q.step(xq, Fq, bfq, bcq)
                torch.cuda.synchronize(dev)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                for _ in range(5):
                    q.step(xq, Fq, bfq, bcq)
                b.record(stream)
                torch.cuda.synchronize(dev)
            ms = a.elapsed_time(b) / 5
            elem = "Q2/Q2 elements (coarse Q2 nodes at level L+1, fine at L+2), " if el == 2 else ""
            paper[name] = {"workload": f"channel nz={nz_p}: {elem}{q.n_patches} patches, {q.n_fine} fine nodes "
                                       f"(level L+{J}), BF16 network {wd[0]}-750x8-{wd[-1]}",
                           "ms_per_step": round(ms, 3), "steps_per_s": round(1000.0 / ms, 2),
                           "patches_per_s": round(q.n_patches * 1000.0 / ms, 1), "timed_steps": 5}
            q.close()

    # measured SIMT FMA peaks (the ALU roofs of the element-integral stages)
    simt = {"fp32_tflops": round(capi.dnnmg_probe_fma(capi.FP32, iters=65536, blocks_per_sm=8), 2),
            "fp64_tflops": round(capi.dnnmg_probe_fma(capi.FP64, iters=2048, blocks_per_sm=8), 3),
            "how": "dnnmg_probe_fma: 8 x SMs blocks of 256 threads, 8 independent FMA chains each, "
                   "best of 3 timed launches after a warm-up"}
    res = dict(elapsed_ms=elapsed_ms, net_ms=net_ms, stage_ms=stage_ms, launches=launches, clocks=clk.summary(),
               e2e_s=e2e_s, nc=nc, nf=nf, nv=nv, fp64=fp64, fp32=fp32, paper=paper,
               affine_frac=parallelepiped_fraction(m), simt=simt)
    p.close()
    return res


SERVING_SIMS = 64


def serving_requests(n=SERVING_SIMS, seed=5, rate=12.0, steps=(50, 500), cells=(4000, 300000)):
    """The serving stream: n simulations arriving as a Poisson process (rate
    per second), each a channel or a cavity (even odds) whose coarse mesh
    size is log-uniform in `cells` and whose step count is uniform in
    `steps`; each starts from a seeded smooth coarse state.  Draws are
    SplitMix64."""
    import numpy as np
    from paper_2307_14837_gb300 import inputs as I
    from paper_2307_14837_gb300.serve import Request, poisson_requests
    u = I.splitmix_uniform(seed * 104729 + 3, 3 * n).reshape(n, 3)
    chan_cells = {}

    def channel_for(target):
        # channel cell counts grow ~ nz^3; take the nz with the nearest count
        best = None
        for nz in range(6, 40):
            if nz not in chan_cells:
                chan_cells[nz] = len(I.channel_mesh(nz, seed=0)["cells"])
            if best is None or abs(math.log(chan_cells[nz] / target)) < abs(math.log(chan_cells[best] / target)):
                best = nz
        return best

    def make(i, _):
        target = cells[0] * (cells[1] / cells[0]) ** u[i, 0]
        n_steps = int(steps[0] + (steps[1] - steps[0]) * u[i, 1])
        if u[i, 2] < 0.5:
            m = I.channel_mesh(channel_for(target), seed=i)
            nu = m["meta"]["D"] / 200.0
            dt, theta = DT, THETA
        else:
            k = max(16, 2 * int(round(target ** (1.0 / 3.0) / 2)))
            m = I.cavity_mesh(k, jitter=0.1, seed=i)
            nu, dt, theta = 0.01, 0.01, 1.0
        return Request(f"sim{i}", m, nu, dt, theta, n_steps, solve=False, x0=I.coarse_state(m, seed=i))

    return poisson_requests(n, rate, seed, make)


# nested meshes for whole-step serving (multigrid coarse solve): (nz, levels)
# of the channel and (n, levels) of the cavity, 4k-135k coarse hex
NESTED_CHANNELS = ((8, 2), (12, 2), (16, 3), (24, 3))
NESTED_CAVITIES = ((16, 2), (24, 3), (32, 4), (40, 3))


def serving_requests_solve(n=16, seed=7, rate=4.0, steps=(10, 40), cells=(4000, 65536)):
    """The whole-step serving stream: n simulations arriving as a Poisson
    process, each a nested channel or cavity (even odds) whose coarse size
    is the nested mesh nearest to a log-uniform draw in `cells`, with a step
    count uniform in `steps`, started from rest with its Dirichlet data;
    every step runs the coarse Newton-GMRES-multigrid solve.  Draws are
    SplitMix64."""
    from paper_2307_14837_gb300 import inputs as I
    from paper_2307_14837_gb300.serve import Request, poisson_requests
    u = I.splitmix_uniform(seed * 104729 + 11, 3 * n).reshape(n, 3)
    sizes = {}

    def nearest(options, build, target):
        best = None
        for o in options:
            if o not in sizes:
                sizes[o] = len(build(o)["cells"])
            if best is None or abs(math.log(sizes[o] / target)) < abs(math.log(sizes[best] / target)):
                best = o
        return best

    def make(i, _):
        target = cells[0] * (cells[1] / cells[0]) ** u[i, 0]
        n_steps = int(steps[0] + (steps[1] - steps[0]) * u[i, 1])
        if u[i, 2] < 0.5:
            nz, lv = nearest(NESTED_CHANNELS, lambda o: I.channel_mesh(o[0], seed=0, levels=o[1]), target)
            m = I.channel_mesh(nz, seed=i, levels=lv)
            nu, dt, theta = m["meta"]["D"] / 200.0, DT, THETA
        else:
            k, lv = nearest(NESTED_CAVITIES, lambda o: I.cavity_mesh(o[0], levels=o[1]), target)
            m = I.cavity_mesh(k, levels=lv)
            nu, dt, theta = 0.01, 0.01, 1.0
        return Request(f"sim{i}", m, nu, dt, theta, n_steps, solve=True)

    return poisson_requests(n, rate, seed, make)


def run_serving(args):
    """Serve the stream with one BF16 network launch per server step over all
    live patches.  Default: each simulation's coarse state is held fixed
    (the patch correction alone, as in the step benchmark).  With
    --serving-solve: whole DNN-MG time steps (the coarse multigrid solve,
    then the patch correction) on nested meshes."""
    import torch
    from paper_2307_14837_gb300 import capi, inputs as I
    from paper_2307_14837_gb300.serve import Server
    torch.cuda.set_device(0)
    solve = bool(args.serving_solve)
    reqs = serving_requests_solve() if solve else serving_requests(n=args.serving_sims)
    Ws, ss, ts = I.network_weights(WIDTHS, seed=0)
    if solve:
        # random-init weights with a small last layer (as in the whole-step
        # leg): with the coarse solve on, the correction feeds back into
        # the next step, and a full-size random correction blows up
        Ws[-1] = 0.05 * Ws[-1]
    budget = int(args.serving_budget_gb * (1 << 30))
    prm = capi.dnnmg_solver_defaults(mg_levels=16, mg_pre=4, mg_post=4, mg_omega=0.8, newton_rtol=1e-9,
                                     newton_atol=1e-10, gmres_rtol=GMRES_FORCING, mg_bf16=1) if solve else None
    srv = Server(WIDTHS, Ws, ss, ts, memory_budget=budget, max_rows=args.serving_rows, precision="bf16",
                 solver=prm)
    with Clocks(0) as clk:
        stats = srv.run(reqs, timeout=1800.0)
    srv.close()
    cells = [len(r.mesh["cells"]) for r in reqs]
    line = {"metric": "serving: aggregate patches/s over a Poisson stream of simulations, one BF16 network "
                      "launch per server step", "value": stats["patches_per_s"], "unit": "patches/s",
            "n_gpus": 1, "higher_is_better": True, "dtype": "bf16", "data": "synthetic",
            "p50_step_latency_ms": stats["p50_step_latency_ms"], "p99_step_latency_ms": stats["p99_step_latency_ms"],
            "server_steps": stats["server_steps"], "network_launches": stats["network_launches"],
            "wall_s": stats["wall_s"], "simulations": stats["simulations"], "failed": len(srv.failures),
            "failures": {k: v[:160] for k, v in srv.failures.items()},
            "config": {"workload": (f"{len(reqs)} simulations, nested channel/cavity mix, coarse meshes "
                                    f"{min(cells)}-{max(cells)} hex (nearest to log-uniform 4k-65k), 10-40 "
                                    f"steps each, Poisson arrivals 4/s; network {'-'.join(map(str, WIDTHS))}; "
                                    "whole DNN-MG time steps (coarse Newton-GMRES-multigrid solve + patch "
                                    "correction), from rest") if solve else
                                   (f"{len(reqs)} simulations, channel/cavity mix, coarse meshes "
                                    f"{min(cells)}-{max(cells)} hex (log-uniform 4k-300k), 50-500 steps each, "
                                    f"Poisson arrivals 12/s; network {'-'.join(map(str, WIDTHS))}; "
                                    "patch correction only (coarse state held)"),
                       "memory_budget_gb": args.serving_budget_gb, "max_rows": args.serving_rows,
                       "total_patch_steps": int(sum(c * r.n_steps for c, r in zip(cells, reqs)))},
            "clocks": clk.summary()}
    print(json.dumps(line))


def _fine_initial(p, m):
    """The fine-level initial state: at rest with the fine Dirichlet data (the
    start of the training trajectories)."""
    import numpy as np
    import torch
    from paper_2307_14837_gb300 import capi, inputs as I
    kind = p.mesh_data(capi.FINE_KIND)
    dirf = (kind == 1) | (kind == 2)
    xr = np.zeros((p.n_fine, 4))
    xr[dirf, 0:3] = I.dirichlet_values(m, p.mesh_data(capi.FINE_XYZ), kind)[dirf]
    return torch.as_tensor(xr, device="cuda")


def equal_error(steps=20, train_steps=60, epochs=100, train_nus=(0.007, 0.0085, 0.0115, 0.013)):
    """Velocity error against the fine-mesh solution of the plain coarse
    scheme and of DNN-MG in the FP64 and BF16 forms, with a network trained
    on the project's own fine solves (the learned part, Sec. 6.4), on the
    cavity workload: 8^3 -> 16^3, Re 100 (nu = 0.01), backward Euler
    dt = 0.01, 20 steps, network 228-256-256-81.

    Training: fine-level (L+1) trajectories at nu = 0.007, 0.0085, 0.0115
    and 0.013 (train_steps steps each, past the evaluation window: the
    DNN-MG loop feeds its corrections back through the coarse right-hand
    side, and states beyond the training horizon drift) by the GPU
    Newton-GMRES-multigrid solver, BF16 training kernels, AdamW (lr 1e-3,
    weight decay 1e-5), `epochs` epochs of batches of 1024.  Evaluation at
    the held-out nu = 0.01.

    Errors (Sec. 6.5-6.6): e_v(n) = |v~_n + d_n - v_n| / |v_n| over the fine
    nodes' velocities (d = 0 for the plain scheme) and the time-integrated
    E_v = (sum_n |v~_n + d_n - v_n|^2 dt / sum_n |v_n|^2 dt)^(1/2).
    Rates: whole time steps (coarse Newton-GMRES-multigrid solve + patch
    correction), steps 2..steps timed with CUDA events."""
    import numpy as np
    import torch

    from paper_2307_14837_gb300 import capi, inputs as I
    from paper_2307_14837_gb300 import train as T
    from paper_2307_14837_gb300.path import PatchPath

    t0 = time.perf_counter()
    m = I.cavity_mesh(8, levels=2)
    dt, nu = 0.01, 0.01
    widths = (228, 256, 256, 81)
    solver = lambda: capi.dnnmg_solver_defaults(mg_levels=3, gmres_rtol=GMRES_FORCING)   # noqa: E731
    Xs, Ts = [], []
    for nu_t in train_nus:
        X, Tg, _ = T.make_samples(m, nu_t, dt, 1.0, train_steps, solver=solver())
        Xs.append(X)
        Ts.append(Tg)
    X, Tg = torch.cat(Xs), torch.cat(Ts)
    norm = T.fit_normalization(X, Tg)
    Xn, Tn = T.normalize(X, norm, Tg)
    net = T.PatchNet(widths, precision="bf16", max_batch=4096, seed=0)
    hist = T.train(net, Xn, Tn, epochs=epochs, batch=1024, lr=1e-3, weight_decay=1e-5)
    Ws, ss, ts = net.export(norm)
    net.close()
    t_train = time.perf_counter() - t0

    dirc = (m["vertex_bc"] == 1) | (m["vertex_bc"] == 2)
    x0 = np.zeros((m.n_vertices, 4))
    x0[dirc, 0:3] = I.dirichlet_values(m, m["xyz"], m["vertex_bc"])[dirc]
    ev = torch.cuda.Event

    def timed_steps(step):
        """run `steps` steps, record the fine velocity after each; time 2.."""
        out, ms = [], 0.0
        for k in range(steps):
            a, b = ev(enable_timing=True), ev(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            v = step()
            b.record()
            torch.cuda.synchronize()
            if k > 0:
                ms += a.elapsed_time(b)
            out.append(v().double().cpu().numpy())
        return out, round(1000.0 * (steps - 1) / ms, 2)

    vel, rate, stats = {}, {}, {}
    # fine reference: the plain scheme on level L+1
    p = PatchPath(m, nu, dt, 1.0, "fp64")
    xr = _fine_initial(p, m)
    prm = solver()

    def fine_step():
        stats.setdefault("fine", []).append(capi.dnnmg_plain_step(p.ctx, capi.LEVEL_FINE, 1, xr, prm))
        return lambda: xr[:, 0:3]

    vel["fine"], rate["plain_fine_fp64"] = timed_steps(fine_step)
    xp = torch.as_tensor(x0, device="cuda")

    def coarse_step():
        stats.setdefault("plain_coarse", []).append(capi.dnnmg_plain_step(p.ctx, capi.LEVEL_COARSE, 1, xp, prm))
        return lambda: p.prolongate(xp)[:, 0:3]

    vel["plain_coarse"], rate["plain_coarse_fp64"] = timed_steps(coarse_step)
    p.close()
    for prec in ("fp64", "bf16"):
        p = PatchPath(m, nu, dt, 1.0, prec)
        p.set_network(widths, Ws, ss, ts)
        x = torch.as_tensor(x0, device="cuda")
        bf, bcf = p.rhs_restrict(x.to(p.dtype), torch.zeros((p.n_fine, 3), dtype=p.dtype, device="cuda"))
        bc = bcf.double().contiguous()
        prm = solver()

        def dnnmg_step():
            stats.setdefault(f"dnnmg_{prec}", []).append(capi.dnnmg_time_step(p.ctx, 1, x, bc, bf, prm))

            def corrected():          # P x^L + d, evaluated after the timed step
                d = p.field(p.n_fine, 3)
                capi.dnnmg_extend(p.ctx, capi.dnnmg_get_buffer(p.ctx, capi.BUF_Y), d)
                return p.prolongate(x.to(p.dtype))[:, 0:3] + d
            return corrected

        vel[f"dnnmg_{prec}"], rate[f"dnnmg_{prec}"] = timed_steps(dnnmg_step)
        p.close()
    ref = vel["fine"]
    out = {"workload": "cavity 8^3->16^3 (nested: multigrid 8^3, 4^3, 2^3), Re 100, BE dt 0.01, "
                       f"{steps} steps; network 228-256-256-81 trained on the GPU (BF16 kernels, AdamW) on "
                       f"fine-level solves at nu {', '.join(map(str, train_nus))} ({train_steps} steps each, "
                       f"{X.shape[0]} samples, {epochs} epochs), evaluated at nu 0.01",
           "reference": "plain scheme on level L+1 (GPU Newton-GMRES-multigrid, FP64)",
           "train_loss_first_last": [hist[0], hist[-1]], "train_seconds": round(t_train, 2)}
    den = sum(float(np.sum(r ** 2)) for r in ref)
    for k in ("plain_coarse", "dnnmg_fp64", "dnnmg_bf16"):
        err = [float(np.linalg.norm(v - r)) for v, r in zip(vel[k], ref)]
        out[k] = {"e_v_last": err[-1] / float(np.linalg.norm(ref[-1])),
                  "e_v": [round(e / float(np.linalg.norm(r)), 6) for e, r in zip(err, ref)],
                  "E_v": (sum(e * e for e in err) / den) ** 0.5,
                  "newton_gmres_per_step": [round(sum(s["newton_iterations"] for s in stats[k]) / steps, 2),
                                            round(sum(s["gmres_iterations"] for s in stats[k]) / steps, 2)]}
    e64, e16, epl = out["dnnmg_fp64"]["E_v"], out["dnnmg_bf16"]["E_v"], out["plain_coarse"]["E_v"]
    out["E_v_bf16_vs_fp64_relative_difference"] = abs(e16 - e64) / e64
    out["E_v_dnnmg_over_plain_coarse"] = {"fp64": e64 / epl, "bf16": e16 / epl}
    out["time_steps_per_s"] = rate
    out["seconds"] = round(time.perf_counter() - t0, 2)
    return out


WHOLE_NZ, WHOLE_LEVELS = 16, 3
# GMRES stops each Newton step at this relative residual (inexact Newton):
# Newton's own tolerance decides convergence, and on the 65,536-cell channel
# a whole step takes 111 ms at 1e-2 against 298 ms at 1e-8 (93 ms with the
# bf16 smoother storage the whole-step legs use)
GMRES_FORCING = 1e-2


def whole_steps(steps=100, nz=WHOLE_NZ, levels=WHOLE_LEVELS):
    """Whole DNN-MG time steps (Alg. 1: the coarse Newton-GMRES-multigrid
    solve, then the patch correction) on the nested channel: nz = 16 layers
    as the 3rd refinement of the nz = 2 channel, 65,536 coarse hex (level L)
    and 524,288 fine hex (level L+1), seeded cylinder, Re 200, Crank-Nicolson
    dt = 0.005, an impulsive start from rest with the full inflow.  Forms: FP32
    fields with the FP32 SIMT network 228-512x3-81, and FP32 fields with the
    BF16 tensor-core network 228-1024x4-81; random-init weights of those
    architectures (seed 0, last layer x 0.05).  Beside them the plain coarse
    scheme (the same solver, no correction).  The multigrid V-cycle runs
    over levels L, L-1, L-2 and the base (nz = 2, 128 hex) with 4 + 4 Vanka
    sweeps damped by 0.8 on bf16 copies of the matrices and inverses, GMRES
    to GMRES_FORCING per Newton step, Newton to 1e-9; the first step (which
    builds the solver) is not timed; `steps` steps are timed with CUDA
    events."""
    import numpy as np
    import torch

    from paper_2307_14837_gb300 import capi, inputs as I
    from paper_2307_14837_gb300.path import PatchPath

    t_start = time.perf_counter()
    m = I.channel_mesh(nz, seed=0, levels=levels)
    nu = m["meta"]["nu_re200"]
    dirc = (m["vertex_bc"] == 1) | (m["vertex_bc"] == 2)

    def initial(t):
        x0 = np.zeros((m.n_vertices, 4))
        x0[dirc, 0:3] = I.dirichlet_values(m, m["xyz"], m["vertex_bc"], t)[dirc]
        return x0

    prm = lambda: capi.dnnmg_solver_defaults(mg_levels=levels, mg_pre=4, mg_post=4, mg_omega=0.8,  # noqa: E731
                                             newton_rtol=1e-9, newton_atol=1e-10, gmres_rtol=GMRES_FORCING,
                                             mg_bf16=1)
    out = {"workload": f"channel nz={nz} nested ({levels} refinements of nz={nz >> levels}): "
                       f"{m.n_cells} coarse hex, {8 * m.n_cells} fine hex; Re 200, CN dt={DT}; "
                       f"{steps} timed whole time steps after 1 untimed",
           "forms": {}}
    for name, prec, widths in (("fp32_228_512x3_81", "fp32", (228, 512, 512, 512, 81)),
                               ("bf16_228_1024x4_81", "bf16", WIDTHS), ("plain_coarse", "fp32", None)):
        p = PatchPath(m, nu, DT, THETA, prec)
        x = torch.as_tensor(initial(1.0), device="cuda")
        sp = prm()
        stats = []
        if widths is not None:
            Ws, ss, ts = I.network_weights(widths, seed=0)
            Ws[-1] = 0.05 * Ws[-1]
            p.set_network(widths, Ws, ss, ts, skip=True)
            bf, bcf = p.rhs_restrict(x.to(p.dtype), torch.zeros((p.n_fine, 3), dtype=p.dtype, device="cuda"))
            bc = bcf.double().contiguous()
            step = lambda: stats.append(capi.dnnmg_time_step(p.ctx, 1, x, bc, bf, sp))   # noqa: E731
        else:
            step = lambda: stats.append(capi.dnnmg_plain_step(p.ctx, capi.LEVEL_COARSE, 1, x, sp))  # noqa: E731
        step()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            step()
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        timed = stats[1:]
        out["forms"][name] = {
            "ms_per_step": round(ms, 2), "steps_per_s": round(1000.0 / ms, 3),
            "patches_per_s": round(m.n_cells * 1000.0 / ms, 1) if widths is not None else None,
            "newton_per_step": round(sum(s_["newton_iterations"] for s_ in timed) / steps, 2),
            "gmres_per_newton": round(sum(s_["gmres_iterations"] for s_ in timed) /
                                      max(1, sum(s_["newton_iterations"] for s_ in timed)), 2),
            "jacobians_per_step": round(sum(s_["jacobian_assemblies"] for s_ in timed) / steps, 2),
            "converged": all(s_["converged"] for s_ in timed)}
        out["multigrid_nodes"] = capi.dnnmg_level_mg(p.ctx, capi.LEVEL_COARSE, sp)
        p.close()
    out["seconds"] = round(time.perf_counter() - t_start, 2)
    return out


class OracleSample:
    """The FP64 oracle's patch step on a sample of the channel workload: the
    same channel family, time step and network at a smaller nz (nz = 10 has
    ~6.3k patches).  Building the hierarchy is set-up and is not timed; each
    timed step is one call of the oracle's patch step."""

    def __init__(self, nz=10):
        from paper_2307_14837_gb300 import inputs as I
        from oracle import dnnmg as odnnmg, mesh as omesh
        self.odnnmg = odnnmg
        m = I.channel_mesh(nz, seed=0)
        nu = m["meta"]["D"] / 200.0
        self.h = omesh.Hierarchy(m["xyz"], m["cells"], m["vertex_bc"])
        self.lev = odnnmg.fine_level(self.h)
        self.xc = I.coarse_state(m, 0)
        self.F = I.fine_rhs(self.h.n_fine, 0, scale=(1 / DT) * 0.42 / (8 * self.h.n_patches))
        Ws, ss, ts = I.network_weights(WIDTHS, seed=0)
        self.net = (Ws, ss, ts, True)
        self.prm = dict(m=1 / DT, theta=THETA, nu=nu, alpha0=0.02, delta0=0.1)
        self.desc = (f"oracle patch step (FP64 numpy) on the channel family at nz={nz}: "
                     f"{self.h.n_patches} patches, {self.h.n_fine} fine nodes, network "
                     f"{'-'.join(map(str, WIDTHS))}; patches/s divided by the full workload's patches")

    def step(self):
        t = time.perf_counter()
        self.odnnmg.hot_path_step(self.h, self.net, self.xc, self.F, self.prm, level=self.lev)
        return time.perf_counter() - t

    @staticmethod
    def threads():
        n = os.cpu_count()
        try:
            import threadpoolctl
            info = threadpoolctl.threadpool_info()
            n = max((i.get("num_threads", 1) for i in info), default=n)
        except Exception:
            pass
        return n


TRAIN_NZ, TRAIN_LEVELS = 4, 1


def train_at_scale(n_geometries=8, steps=96, eval_steps=64, epochs=150, batch=65536, nz=TRAIN_NZ,
                   levels=TRAIN_LEVELS, dt=0.01, theta=1.0, widths=(228, 1024, 1024, 1024, 1024, 81),
                   horizons=(4, 8, 16), val_fraction=0.05, seed0=100, ref_gmres_rtol=None, save_net=None):
    """The learned part at scale (Sec. 6.4): training data from the
    project's own solver on n_geometries seeded channel obstacles (cylinder
    diameter and centre from the seed) at Re ~ U[100, 300] (nu = D / Re,
    mean inflow 1), a coarse mesh of nz layers nested `levels` times
    (nz = 4: 1,024 coarse hex, level L+1 8,192, level L+2 65,536), the
    reference two refinements up (level L+2, Newton-GMRES-multigrid over
    L+2, L+1, L and L-1, its Dirichlet values the prolongated coarse data)
    injected onto level L+1, backward Euler dt = 0.01 from rest with the
    full inflow, `steps` steps per geometry.  BF16 training (AdamW lr 1e-3,
    weight decay 1e-5, batch 65,536, `epochs` epochs; the parameters of the
    epoch with the lowest loss on a held-back random val_fraction of the
    samples kept) in rounds: round 0 on the reference pairs; after round r,
    DNN-MG with its network, restarted from the reference every
    horizons[r] steps on every training geometry, adds pairs from the
    loop's own states (train.rollout_samples) to the set, and round r + 1
    trains a fresh network on the whole set.  On an unseen geometry (seed
    seed0 + n_geometries, its own Re draw): each round's network's relative
    error on that geometry's reference pairs, and e_v and E_v of the plain
    coarse scheme and of DNN-MG (BF16; FP64 too for the last round) against
    the level-(L+2) reference over eval_steps steps; a run whose solve
    fails reports the step.  save_net: a path for the last network (.npz)."""
    import numpy as np
    import torch

    from paper_2307_14837_gb300 import capi, inputs as I
    from paper_2307_14837_gb300 import train as T

    t0 = time.perf_counter()
    ref_solver = lambda: capi.dnnmg_solver_defaults(  # noqa: E731
        mg_levels=levels + 2, mg_pre=4, mg_post=4, mg_omega=0.8, newton_rtol=1e-9, newton_atol=1e-10,
        gmres_rtol=ref_gmres_rtol or GMRES_FORCING, mg_bf16=1)
    coarse_solver = lambda: capi.dnnmg_solver_defaults(  # noqa: E731
        mg_levels=levels, newton_rtol=1e-9, newton_atol=1e-10, gmres_rtol=GMRES_FORCING)
    re = 100.0 + 200.0 * I.splitmix_uniform(9000 + seed0, n_geometries + 1)
    log = lambda msg: print(f"[train-scale] {msg}, {time.perf_counter() - t0:.1f} s",  # noqa: E731
                            file=sys.stderr, flush=True)
    geos, runs = [], []
    Xs, Ts = [], []
    for k in range(n_geometries):
        seed = seed0 + k
        m = I.channel_mesh(nz, seed=seed, levels=levels)
        D = I.channel_geometry(seed)[0]
        nu = D / re[k]
        X, Tg, st = T.make_samples(m, nu, dt, theta, steps, solver=coarse_solver(), ref_levels=2,
                                   ref_solver=ref_solver(), fine_boundary="prolongated")
        Xs.append(X)
        Ts.append(Tg)
        runs.append((m, nu, st))
        geos.append({"seed": seed, "D": round(float(D), 5), "Re": round(float(re[k]), 2), "nu": float(nu),
                     "patches": int(m["cells"].shape[0])})
        log(f"geometry {k}: Re {re[k]:.1f}, {X.shape[0]} samples")
    X, Tg = torch.cat(Xs), torch.cat(Ts)
    n_ref = int(X.shape[0])
    del Xs, Ts
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    norm = T.fit_normalization(X, Tg)

    def split(X, Tg, seed):
        """standardised training and validation rows (a seeded random subset)"""
        n = X.shape[0]
        perm = torch.randperm(n, generator=torch.Generator(device="cpu").manual_seed(seed)).to(X.device)
        n_val = int(val_fraction * n)
        out = []
        for idx in (perm[n_val:], perm[:n_val]):
            Xa = torch.empty((idx.shape[0], X.shape[1]), dtype=X.dtype, device=X.device)
            Ta = torch.empty((idx.shape[0], 81), dtype=Tg.dtype, device=X.device)
            capi.dnnmg_gather_rows(X, idx, Xa, stream=torch.cuda.current_stream())
            capi.dnnmg_gather_rows(Tg, idx, Ta, stream=torch.cuda.current_stream())
            out.append(T.normalize(Xa, norm, Ta))
        return out

    # the unseen geometry: its reference trajectory and pairs
    seed = seed0 + n_geometries
    mh = I.channel_mesh(nz, seed=seed, levels=levels)
    Dh = I.channel_geometry(seed)[0]
    nuh = Dh / re[n_geometries]
    Xh, Th, held = T.make_samples(mh, nuh, dt, theta, eval_steps, solver=coarse_solver(), ref_levels=2,
                                  ref_solver=ref_solver(), fine_boundary="prolongated")
    Xhn = T.normalize(Xh, norm)
    ref = [s_["v_fine"][:, 0:3].cpu().numpy() for s_ in held]
    log("held-out reference")

    def run_loop(netw, prec):
        vel = []
        try:
            T.trajectory_errors(mh, nuh, dt, theta, held, network=netw, solver=coarse_solver(), precision=prec,
                                velocities=vel)
            failed = None
        except capi.DnnmgError as e:
            failed = {"step": len(vel) + 1, "status": e.status}
        e = T.velocity_errors(vel, ref[:len(vel)]) if vel else {"e_v": [], "E_v": None}
        return {"E_v": e["E_v"], "e_v_last": e["e_v"][-1] if vel else None,
                "e_v": [round(v, 6) for v in e["e_v"]], "failed": failed}

    plain = run_loop(None, "fp64")
    log(f"plain coarse E_v {plain['E_v']}")
    t_train = 0.0

    def fit(parts, name):
        nonlocal t_train
        (Xn, Tn), (Xvn, Tvn) = parts
        net = T.PatchNet(widths, precision="bf16", max_batch=batch, seed=0)
        vh = []
        t1 = time.perf_counter()
        hist = T.train(net, Xn, Tn, epochs=epochs, batch=batch, lr=1e-3, weight_decay=1e-5, val=(Xvn, Tvn),
                       val_hist=vh)
        torch.cuda.synchronize()
        t_train += time.perf_counter() - t1
        network = (widths, *net.export(norm))
        Yh = net.predict(Xhn) * norm[2]
        net.close()
        prior = float(torch.linalg.norm(Yh - Th) / torch.linalg.norm(Th))
        res = {"train_samples": int(Xn.shape[0]), "validation_samples": int(Xvn.shape[0]),
               "train_loss_first_last": [hist[0], hist[-1]], "validation_loss_best": min(vh),
               "validation_best_epoch": int(np.argmin(vh)), "network_relative_error_exact_inputs": prior}
        log(f"{name}: trained, prior {prior:.4f}")
        return network, res

    rounds = []
    Xall, Tall = [X], [Tg]
    del X, Tg
    n_roll = 0
    for r in range(len(horizons) + 1):
        Xc, Tc = torch.cat(Xall), torch.cat(Tall)
        net_r, res = fit(split(Xc, Tc, seed0 + r), f"round {r}")
        del Xc, Tc
        res["dnnmg_bf16"] = run_loop(net_r, "bf16")
        if r == len(horizons):
            res["dnnmg_fp64"] = run_loop(net_r, "fp64")
        for k in ("dnnmg_bf16", "dnnmg_fp64"):
            if k in res and res[k]["failed"] is None:
                res[k]["E_v_over_plain_coarse"] = res[k]["E_v"] / plain["E_v"]
        e = res["dnnmg_bf16"]["e_v"]
        below = next((i for i, v in enumerate(e) if v >= plain["e_v"][i]), len(e))
        res["dnnmg_bf16"]["steps_below_plain_coarse"] = below
        log(f"round {r}: BF16 E_v {res['dnnmg_bf16']['E_v']}, failed {res['dnnmg_bf16']['failed']}, "
            f"below plain for {below} steps")
        rounds.append(res)
        if r < len(horizons):
            for m, nu, st in runs:
                a, b = T.rollout_samples(m, nu, dt, theta, st, net_r, horizon=horizons[r], solver=coarse_solver())
                Xall.append(a)
                Tall.append(b)
                n_roll += int(a.shape[0])
            log(f"rollouts after round {r}: {n_roll} samples in all")
    del runs, Xall, Tall
    if save_net:
        np.savez(save_net, widths=np.array(widths), norm_mu=norm[0], norm_sigma=norm[1], t_scale=norm[2],
                 **{f"W{i}": w.astype(np.float32) for i, w in enumerate(net_r[1])},
                 **{f"shift{i}": b for i, b in enumerate(net_r[3])})
    return {"workload": f"channel nz={nz} nested ({levels} refinement of nz={nz >> levels}) with a seeded "
                        f"cylinder: {geos[0]['patches']} coarse hex, targets from level L+2 "
                        f"({64 * geos[0]['patches']} hex, Dirichlet values the prolongated coarse data) "
                        f"injected onto L+1; backward Euler dt={dt}, {steps} steps per geometry from rest; "
                        f"BF16 network {'-'.join(map(str, widths))}",
            "geometries": geos, "reference_samples": n_ref,
            "rollout_samples": n_roll, "rollout_horizons": list(horizons), "batch": batch, "epochs": epochs,
            "optimizer": "AdamW lr 1e-3, weight decay 1e-5",
            "seconds": {"data": round(t_data, 1), "train": round(t_train, 1),
                        "total": round(time.perf_counter() - t0, 1)},
            "held_out": {"seed": seed, "D": round(float(Dh), 5), "Re": round(float(re[n_geometries]), 2),
                         "steps": eval_steps, "plain_coarse": plain, "rounds": rounds}}


def eval_saved_network(path, seeds, eval_steps=64, nz=TRAIN_NZ, levels=TRAIN_LEVELS, dt=0.01, theta=1.0):
    """A network saved by --train-scale --save-net on further unseen
    geometries: for each seed, the channel of that seed with Re drawn from
    U[100, 300] (its own SplitMix64 stream), the level-(L+2) reference with
    prolongated Dirichlet data, and e_v / E_v of the plain coarse scheme and
    of DNN-MG (BF16) over eval_steps steps, as in train_at_scale."""
    import numpy as np

    from paper_2307_14837_gb300 import capi, inputs as I
    from paper_2307_14837_gb300 import train as T

    z = np.load(path)
    widths = tuple(int(w) for w in z["widths"])
    L = len(widths) - 1
    network = (widths, [z[f"W{i}"].astype(np.float64) for i in range(L)], [np.ones(w) for w in widths[1:]],
               [z[f"shift{i}"] for i in range(L)])
    ref_solver = lambda: capi.dnnmg_solver_defaults(  # noqa: E731
        mg_levels=levels + 2, mg_pre=4, mg_post=4, mg_omega=0.8, newton_rtol=1e-9, newton_atol=1e-10,
        gmres_rtol=GMRES_FORCING, mg_bf16=1)
    coarse_solver = lambda: capi.dnnmg_solver_defaults(  # noqa: E731
        mg_levels=levels, newton_rtol=1e-9, newton_atol=1e-10, gmres_rtol=GMRES_FORCING)
    out = {"network": "-".join(map(str, widths)), "steps": eval_steps, "geometries": []}
    for seed in seeds:
        m = I.channel_mesh(nz, seed=seed, levels=levels)
        D = I.channel_geometry(seed)[0]
        re = float(100.0 + 200.0 * I.splitmix_uniform(9100 + seed, 1)[0])
        nu = D / re
        _, _, held = T.make_samples(m, nu, dt, theta, eval_steps, solver=coarse_solver(), ref_levels=2,
                                    ref_solver=ref_solver(), keep_steps=True, fine_boundary="prolongated")
        ref = [s_["v_fine"][:, 0:3].cpu().numpy() for s_ in held]
        res = {"seed": seed, "D": round(float(D), 5), "Re": round(re, 2)}
        for name, netw in (("plain_coarse", None), ("dnnmg_bf16", network)):
            vel = []
            try:
                T.trajectory_errors(m, nu, dt, theta, held, network=netw, solver=coarse_solver(),
                                    precision="bf16" if netw else "fp64", velocities=vel)
                failed = None
            except capi.DnnmgError as e:
                failed = {"step": len(vel) + 1, "status": e.status}
            e = T.velocity_errors(vel, ref[:len(vel)]) if vel else {"e_v": [], "E_v": None}
            res[name] = {"E_v": e["E_v"], "e_v_first_last": [e["e_v"][0], e["e_v"][-1]] if vel else None,
                         "failed": failed}
        if res["dnnmg_bf16"]["failed"] is None:
            res["E_v_dnnmg_over_plain_coarse"] = res["dnnmg_bf16"]["E_v"] / res["plain_coarse"]["E_v"]
        out["geometries"].append(res)
        print(f"[eval-net] seed {seed}: {res}", file=sys.stderr, flush=True)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving", action="store_true",
                    help="serve a Poisson stream of simulations instead of the step benchmark")
    ap.add_argument("--serving-sims", type=int, default=SERVING_SIMS)
    ap.add_argument("--serving-budget-gb", type=float, default=96.0)
    ap.add_argument("--serving-rows", type=int, default=6_000_000)
    ap.add_argument("--gmres-forcing", type=float, default=None,
                    help="GMRES tolerance per Newton step in the whole-step legs (default 1e-2)")
    ap.add_argument("--serving-solve", action="store_true",
                    help="serve whole time steps (coarse multigrid solve on) on a stream of nested meshes")
    ap.add_argument("--train-scale", action="store_true",
                    help="run only the learned part at scale (8 seeded channel obstacles, level L+2 targets, "
                         "held-out geometry) and print its JSON line")
    ap.add_argument("--train-steps", type=int, default=96, help="time steps per training geometry")
    ap.add_argument("--train-epochs", type=int, default=150)
    ap.add_argument("--train-ref-gmres-rtol", type=float, default=None,
                    help="GMRES tolerance per Newton step of the level-(L+2) reference solves")
    ap.add_argument("--save-net", default=None, help="write the trained network (.npz) to this path")
    ap.add_argument("--eval-net", default=None,
                    help="evaluate a network saved by --save-net on the geometries of --eval-seeds")
    ap.add_argument("--eval-seeds", default="109,110")
    ap.add_argument("--whole-steps-only", type=int, default=0, metavar="K",
                    help="print only the whole-time-step measurement (K timed steps) as one JSON line")
    ap.add_argument("--nz", type=int, default=NZ,
                    help="channel resolution (cells across the height); the measured workload is nz=37")
    args = ap.parse_args()
    if args.gmres_forcing is not None:
        global GMRES_FORCING
        GMRES_FORCING = args.gmres_forcing
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    n_patches_full = 314389

    if args.impl == "reference":
        if rank != 0:
            return
        t0 = time.perf_counter()
        o = OracleSample(nz=6)
        for _ in range(args.warmup):
            o.step()
        secs = sum(o.step() for _ in range(args.steps))
        pps = o.h.n_patches * args.steps / secs
        desc, threads = o.desc, o.threads()
        v = pps / n_patches_full
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / v,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": "channel nz=37 (314389 patches), CN dt=0.005, Re=200, "
                                       "network 228-1024x4-81; oracle timed on a sample", "sample": desc},
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                "patches_per_s": pps, "wall_s": time.perf_counter() - t0}
        print(json.dumps(line))
        return

    if args.serving:
        if rank == 0:
            run_serving(args)
        return

    if args.eval_net:
        if rank == 0:
            import torch
            torch.cuda.set_device(0)
            seeds = [int(v) for v in args.eval_seeds.split(",")]
            print(json.dumps({"eval_saved_network": eval_saved_network(args.eval_net, seeds)}))
        return

    if args.train_scale:
        if rank == 0:
            import torch
            torch.cuda.set_device(0)
            print(json.dumps({"train_at_scale": train_at_scale(steps=args.train_steps, epochs=args.train_epochs,
                                                               ref_gmres_rtol=args.train_ref_gmres_rtol,
                                                               save_net=args.save_net)}))
        return

    if args.whole_steps_only:
        if rank == 0:
            import torch
            torch.cuda.set_device(0)
            print(json.dumps({"whole_time_steps": whole_steps(steps=args.whole_steps_only)}))
        return

    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    res = run_ours(args, rank, world, local_rank)
    el = max_over_ranks(res["elapsed_ms"], world, "cuda")
    if rank != 0:
        torch.distributed.destroy_process_group()
        return
    line = result_line(res, args, world, el)
    if not args.no_fp64:
        line["equal_error"] = equal_error()
        line["whole_time_steps"] = whole_steps()
    if not args.no_cpu_baseline:
        o = OracleSample(nz=10)
        secs, n = 0.0, 0
        while n < 2 or (secs < 10.0 and n < 5):
            secs += o.step()
            n += 1
        pps = o.h.n_patches * n / secs
        line["cpu_baseline"] = {"value": pps / res["nc"], "unit": UNIT, "cores": o.threads(), "kind": "oracle",
                                "sample": f"{o.desc}; {n} timed steps", "patches_per_s": pps}
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def result_line(res, args, world, el):
    """The JSON line of the device arm from run_ours' result ``res`` and the
    slowest rank's elapsed time ``el`` (ms for args.steps steps)."""
    K = args.steps
    ms = el / K
    value = whole_job_rate(K, el, world)
    nc, nf, nv = res["nc"], res["nf"], res["nv"]
    peaks, peak_src = _peaks()
    net_ms = statistics.mean(res["net_ms"])
    flops = network_flops_per_patch() * nc
    achieved = flops / (net_ms / 1000.0) / 1e12
    peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic",
        "config": {"workload": f"channel 2.5x0.41x0.41 with seeded cylinder, nz={args.nz}: {nc} patches "
                               f"(coarse hex), {nf} fine nodes; BF16 network {'-'.join(map(str, WIDTHS))}, "
                               f"FP32 fields, CN dt={DT}, Re=200",
                   "patches_per_step": nc, "l2": "working set > L2 (activations 644 MB per layer)",
                   "parallelism": f"replicas x{world}"},
        "patches_per_s": value * nc,
        "roofline": {"bound": "tensor", "kernel": "network layers (BF16 GEMM chain)",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "peak_source": f"{peak_src} bf16 sustained", "traffic": network_traffic(nc),
                     "traffic_unit": "bytes per network stage (ncu dram read+write, scaled from nz=25)",
                     "network_ms_per_step": net_ms, "network_share": net_ms / ms},
        "e2e": {"value": world * K / res["e2e_s"] if res["e2e_s"] > 0 else None, "unit": UNIT,
                "h2d_bytes_per_step": (nv + nf) * 16, "d2h_bytes_per_step": (nf + nv) * 16},
        "stages": stage_rooflines(res["stage_ms"], nc, peaks, peak_src, res["clocks"], res["affine_frac"],
                                  (res.get("simt") or {}).get("fp32_tflops")),
        "simt_peaks": res.get("simt"),
        "fp32_form": res["fp32"],
        "paper_forms": res["paper"],
        "gpu_launches": res["launches"],
        "clocks": res["clocks"],
        "fp64_plain": res["fp64"],
    }
    return line


if __name__ == "__main__":
    main()
