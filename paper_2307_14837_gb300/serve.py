"""Serving many DNN-MG simulations with one network launch per step.

A ``Server`` owns one network-only libdnnmg context (``dnnmg_net_create``)
and shared input/output row buffers.  Requests (a mesh, viscosity, time step
and a number of steps) wait in a FIFO queue and are admitted while their
device-memory estimate fits the budget and their patches fit the shared
buffers; an admitted simulation keeps its whole state resident (its own
context: mesh hierarchy, coarse state, fine rhs, solver) on its own CUDA
stream.  One server step advances every live simulation by one DNN-MG step:

  1. per simulation, on its stream: coarse solve (optional), fine residual
     and network input rows written into its slice of the shared rows
     (``dnnmg_step_begin``);
  2. one network launch over all live rows on the server stream, after the
     simulations' events;
  3. per simulation, on its stream after the network's event: extension of
     its slice of the outputs, next fine rhs and its restriction
     (``dnnmg_step_end``).

Finished simulations release their memory at the end of the step, and
waiting requests are admitted at the start of the next one, so requests that
arrive while others run join as slots and memory free up (continuous
batching).  Building a context (the host hierarchy, uploads, the first
right-hand side) takes up to a second for the largest meshes, so by default
worker threads prepare queued requests while the server steps: memory and
rows are reserved when preparation starts, and requests are still admitted
in FIFO order as soon as the head of the queue is ready.  Every stage is deterministic and network rows are independent,
so a simulation's result does not depend on which others share its steps.
"""
from __future__ import annotations

import collections
import time
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np
import torch

from . import capi, inputs as I
from .path import PatchPath

N_IN_PAD = 256


@dataclass
class Request:
    name: str
    mesh: dict
    nu: float
    dt: float
    theta: float
    n_steps: int
    arrival: float = 0.0          # seconds after the start of Server.run
    solve: bool = True            # coarse solve each step (False: patch correction only)
    x0: object = None             # initial coarse state [nv][4] (default: 0 with Dirichlet values)


@dataclass
class Simulation:
    req: Request
    path: PatchPath
    stream: torch.cuda.Stream
    x: torch.Tensor               # coarse state, double [nv][4]
    b: torch.Tensor               # coarse rhs, double [nv][4]
    F: torch.Tensor               # fine rhs, field type [nf][4]
    mem: int
    admitted: float
    steps_done: int = 0
    latencies: list = field(default_factory=list)
    ev_begin: torch.cuda.Event = None
    ev_end: torch.cuda.Event = None


def memory_estimate(mesh, precision="bf16", solve=True):
    """Device bytes one simulation holds (a bound from its sizes): context
    buffers per patch and per fine node, the coarse state, and the Newton
    solver's level (block matrix, group factors) when it solves."""
    nc = int(np.asarray(mesh["cells"]).shape[0])
    nv = int(np.asarray(mesh["xyz"]).shape[0])
    nf = nv + 8 * nc                      # fine nodes <= vertices + edges + faces + cells
    fe = 8 if precision == "fp64" else 4
    xe = 8 if precision == "fp64" else (2 if precision == "bf16" else 4)
    per_patch = 27 * 4 * fe + 8 * 4 * fe + N_IN_PAD * xe + 81 * fe + 27 * 4 * 2 + 32 + 8 * 4 * 2
    per_node = 4 * fe * 3 + 3 * fe + 4 + 4 + 1
    per_vertex = 4 * 8 * 3 + 4 * fe * 2 + 24 + 8
    b = nc * per_patch + nf * per_node + nv * per_vertex
    if solve:
        ng = max(nc // 8, 1)
        b += ng * 108 * 108 * 8 * 2 + nv * 27 * 16 * 8 + nv * 4 * 8 * 48
    return int(1.25 * b) + (1 << 20)


class Server:
    def __init__(self, widths, Ws, scales, shifts, memory_budget, max_rows, precision="bf16", device="cuda",
                 solver=None, prepare_workers=2):
        self.device = torch.device(device)
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        torch.cuda.set_device(self.device)
        self.precision = precision
        self.prec = {"fp64": capi.FP64, "fp32": capi.FP32, "bf16": capi.BF16}[precision]
        self.stream = torch.cuda.Stream(self.device)
        self.net = capi.dnnmg_net_create(widths, Ws, scales, shifts, self.prec, max_rows, self.stream)
        self.widths = tuple(widths)
        self.max_rows = int(max_rows)
        xdt = {"fp64": torch.float64, "fp32": torch.float32, "bf16": torch.bfloat16}[precision]
        ydt = torch.float64 if precision == "fp64" else torch.float32
        self.X = torch.zeros((self.max_rows, N_IN_PAD), dtype=xdt, device=self.device)
        self.Y = torch.zeros((self.max_rows, capi.N_OUT), dtype=ydt, device=self.device)
        self.budget = int(memory_budget)
        self.used = 0
        self.queue = collections.deque()
        self.live: list[Simulation] = []
        self.results = {}
        self.log = []
        self.solver = solver
        self.ev_net = torch.cuda.Event()
        self.step_latencies = []
        self.patches = 0
        # background preparation of queued requests (0 workers: inside the step)
        self.pool = ThreadPoolExecutor(max_workers=prepare_workers) if prepare_workers > 0 else None
        self.preparing = {}          # id(request) -> (future, memory, rows)
        self.reserved = 0
        self.rows_reserved = 0
        self.admission_s = 0.0       # host time the step loop spent admitting
        self.failures = {}           # request name -> why it failed (context build, network wait)

    # -- admission -----------------------------------------------------------
    def submit(self, req: Request):
        self.queue.append(req)

    def _rows(self):
        return sum(s.path.n_patches for s in self.live)

    def _needs(self, req):
        return memory_estimate(req.mesh, self.precision, req.solve), int(np.asarray(req.mesh["cells"]).shape[0])

    def _prepare(self, now):
        """Start preparing queued requests, in FIFO order, while their memory
        and rows fit beside the live and already reserved ones."""
        for req in self.queue:
            if id(req) in self.preparing:
                continue
            mem, nc = self._needs(req)
            if mem > self.budget or nc > self.max_rows:
                continue                                        # rejected when it reaches the head
            if (self.used + self.reserved + mem > self.budget or
                    self._rows() + self.rows_reserved + nc > self.max_rows):
                break
            self.preparing[id(req)] = (self.pool.submit(self._start, req, mem, now), mem, nc)
            self.reserved += mem
            self.rows_reserved += nc

    def _admit(self, now):
        t0 = time.perf_counter()
        if self.pool is not None:
            self._prepare(now)
        while self.queue:
            req = self.queue[0]
            mem, nc = self._needs(req)
            if mem > self.budget or nc > self.max_rows:
                self.queue.popleft()
                self.log.append(("rejected", req.name, now))
                continue
            try:
                if self.pool is not None:
                    entry = self.preparing.get(id(req))
                    if entry is None or not entry[0].done():
                        break                                   # FIFO: the head is not ready yet
                    self.queue.popleft()
                    del self.preparing[id(req)]
                    self.reserved -= mem
                    self.rows_reserved -= nc
                    sim = entry[0].result()
                else:
                    if self.used + mem > self.budget or self._rows() + nc > self.max_rows:
                        break                                   # FIFO: wait for memory / rows
                    self.queue.popleft()
                    sim = self._start(req, mem, now)
            except (capi.DnnmgError, ValueError) as e:
                # a request whose context cannot be built (an invalid mesh,
                # no device memory) fails alone; the others go on
                self.log.append(("failed", req.name, now))
                self.failures[req.name] = str(e)
                continue
            self.live.append(sim)
            self.used += mem
            self.log.append(("admitted", req.name, now))
        self.admission_s += time.perf_counter() - t0

    def _start(self, req, mem, now):
        stream = torch.cuda.Stream(self.device)
        p = PatchPath(req.mesh, req.nu, req.dt, req.theta, self.precision, device=self.device, stream=stream)
        with torch.cuda.stream(stream):
            m = req.mesh
            if req.x0 is not None:
                x0 = np.array(req.x0, dtype=np.float64).reshape(p.n_coarse, 4)
            else:
                dirc = (np.asarray(m["vertex_bc"]) == 1) | (np.asarray(m["vertex_bc"]) == 2)
                x0 = np.zeros((p.n_coarse, 4))
                x0[dirc, 0:3] = I.dirichlet_values(m, m["xyz"], m["vertex_bc"])[dirc]
            x = torch.as_tensor(x0, device=self.device)
            # first right-hand sides: the fine Rhs of the prolongated state, restricted
            F, bcf = p.rhs_restrict(x.to(p.dtype), torch.zeros((p.n_fine, 3), dtype=p.dtype, device=self.device))
            b = bcf.double().contiguous() if p.dtype != torch.float64 else bcf
            if req.solve:
                # the solver's level (multigrid hierarchy, matrix and factor
                # storage) is built here, on the preparing thread, rather
                # than inside the simulation's first server step
                capi.dnnmg_level_mg(p.ctx, capi.LEVEL_COARSE, self.solver)
        sim = Simulation(req=req, path=p, stream=stream, x=x, b=b, F=F, mem=mem, admitted=now)
        sim.ev_begin = torch.cuda.Event()
        sim.ev_end = torch.cuda.Event()
        return sim

    # -- one server step -----------------------------------------------------
    def step(self, now=0.0):
        self._admit(now)
        if not self.live:
            if self.preparing:
                time.sleep(0.0005)                      # leave the preparing threads the interpreter
            return 0
        t0 = time.perf_counter()
        xb = self.X.element_size() * N_IN_PAD
        yb = self.Y.element_size() * capi.N_OUT
        off = 0
        offsets = []
        for s in list(self.live):
            try:
                with torch.cuda.stream(s.stream):
                    capi.dnnmg_step_begin(s.path.ctx, s.x, s.b, s.F, self.X.data_ptr() + off * xb,
                                          solve=s.req.solve, prm=self.solver)
                    s.ev_begin.record(s.stream)
            except capi.DnnmgError as e:
                # this simulation's solve failed (no convergence, a non-finite
                # rhs): it leaves the batch before the network launch
                s.stream.synchronize()
                self.live.remove(s)
                self.used -= s.mem
                s.path.close()
                self.log.append(("failed", s.req.name, now))
                self.failures[s.req.name] = str(e)
                continue
            offsets.append(off)
            off += s.path.n_patches
        if not self.live:
            return 0
        for s in self.live:
            self.stream.wait_event(s.ev_begin)
        capi.dnnmg_network(self.net, self.X, self.Y, off)
        self.ev_net.record(self.stream)
        for s, o in zip(self.live, offsets):
            s.stream.wait_event(self.ev_net)
            with torch.cuda.stream(s.stream):
                capi.dnnmg_step_end(s.path.ctx, self.Y.data_ptr() + o * yb, s.F, s.b)
                s.ev_end.record(s.stream)
        for s in self.live:
            s.ev_end.synchronize()
        try:
            capi.dnnmg_sync(self.net)               # the shared network's bounded waits (stream done)
        except capi.DnnmgError as e:
            if e.status != -6:
                raise
            # an expired wait left Y invalid: every simulation of this step
            # took a wrong correction, so all of them fail
            for s in list(self.live):
                self.live.remove(s)
                self.used -= s.mem
                s.path.close()
                self.log.append(("failed", s.req.name, now))
                self.failures[s.req.name] = str(e)
            return 0
        dt = time.perf_counter() - t0
        self.step_latencies.append(dt)
        self.patches += off
        finished = []
        for s in self.live:
            s.steps_done += 1
            s.latencies.append(dt)
            if s.steps_done >= s.req.n_steps:
                finished.append(s)
        for s in finished:
            self.results[s.req.name] = dict(x=s.x.cpu().numpy(), F=s.F.double().cpu().numpy(),
                                            steps=s.steps_done, latencies=list(s.latencies))
            self.live.remove(s)
            self.used -= s.mem
            s.path.close()
            self.log.append(("finished", s.req.name, now))
        return off

    # -- a stream of requests --------------------------------------------------
    def run(self, requests, timeout=600.0):
        """Serve requests arriving at their `arrival` times (seconds after the
        start); returns throughput and latency statistics."""
        pending = sorted(requests, key=lambda r: r.arrival)
        t_start = time.perf_counter()
        i = 0
        while i < len(pending) or self.queue or self.live:
            now = time.perf_counter() - t_start
            while i < len(pending) and pending[i].arrival <= now:
                self.submit(pending[i])
                i += 1
            if not self.live and not self.queue and i < len(pending):
                time.sleep(max(0.0, min(pending[i].arrival - now, 0.05)))
                continue
            self.step(now)
            if now > timeout:
                raise TimeoutError("serving did not finish")
        wall = time.perf_counter() - t_start
        lat = np.array([l for r in self.results.values() for l in r["latencies"]])
        return dict(simulations=len(self.results), wall_s=wall, server_steps=len(self.step_latencies),
                    patches_per_s=self.patches / wall if wall > 0 else 0.0,
                    p50_step_latency_ms=float(np.percentile(lat, 50) * 1e3) if lat.size else None,
                    p99_step_latency_ms=float(np.percentile(lat, 99) * 1e3) if lat.size else None,
                    network_launches=len(self.step_latencies), admission_s=self.admission_s)

    def close(self):
        if self.pool is not None:
            self.pool.shutdown(wait=True)
            for fut, _, _ in self.preparing.values():
                try:
                    fut.result().path.close()
                except (capi.DnnmgError, ValueError):
                    pass
            self.preparing = {}
        for s in self.live:
            s.path.close()
        self.live = []
        if self.net:
            capi.dnnmg_destroy(self.net)
            self.net = None


def poisson_requests(n, rate, seed, make_request):
    """n requests with exponential inter-arrival times (mean 1 / rate seconds,
    SplitMix64 draws); make_request(i, u) builds request i from a uniform u."""
    u = I.splitmix_uniform(seed * 7919 + 17, 2 * n)
    t = np.cumsum(-np.log(1.0 - u[:n]) / rate)
    reqs = []
    for i in range(n):
        r = make_request(i, float(u[n + i]))
        r.arrival = float(t[i])
        reqs.append(r)
    return reqs
