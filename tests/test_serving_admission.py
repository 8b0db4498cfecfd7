"""The serving admission policy on the host, with the GPU parts faked:
FIFO order under the memory budget and the row capacity, rejection of
requests that can never fit, and host-side fault injection (a context whose
build runs out of memory fails alone and releases its reservation), with
and without background preparation."""
import collections
import time
from concurrent.futures import ThreadPoolExecutor
from types import SimpleNamespace

import pytest

from paper_2307_14837_gb300 import capi, serve


def _req(name, mem, nc):
    return SimpleNamespace(name=name, mem=mem, nc=nc)


def _server(budget, max_rows, workers):
    """A Server without its device parts: only the admission state."""
    s = serve.Server.__new__(serve.Server)
    s.budget, s.max_rows, s.used = budget, max_rows, 0
    s.queue, s.live, s.results, s.log, s.failures = collections.deque(), [], {}, [], {}
    s.admission_s, s.preparing, s.reserved, s.rows_reserved = 0.0, {}, 0, 0
    s.pool = ThreadPoolExecutor(max_workers=workers) if workers else None
    s._needs = lambda req: (req.mem, req.nc)

    def start(req, mem, now):
        if req.name.startswith("oom"):            # the injected fault: no device memory
            raise capi.DnnmgError(-2, "out of memory (injected)")
        return SimpleNamespace(req=req, mem=mem, path=SimpleNamespace(n_patches=req.nc))
    s._start = start
    return s


def _admit(s, rounds=50):
    """Admission until nothing changes (background builds get time)."""
    for _ in range(rounds):
        before = (len(s.queue), len(s.live), len(s.log))
        s._admit(0.0)
        if s.pool is None or (before == (len(s.queue), len(s.live), len(s.log)) and not s.preparing):
            break
        time.sleep(0.01)


def _finish(s, name):
    sim = next(x for x in s.live if x.req.name == name)
    s.live.remove(sim)
    s.used -= sim.mem


@pytest.mark.parametrize("workers", [0, 2])
def test_fifo_under_the_memory_budget(workers):
    s = _server(budget=10, max_rows=100, workers=workers)
    for r in (_req("a", 6, 1), _req("b", 6, 1), _req("c", 3, 1)):
        s.queue.append(r)
    _admit(s)
    assert [x.req.name for x in s.live] == ["a"] and [r.name for r in s.queue] == ["b", "c"]
    _finish(s, "a")                                  # a's memory comes back
    _admit(s)
    assert [x.req.name for x in s.live] == ["b", "c"] and s.used == 9 and not s.queue
    assert s.reserved == 0 and s.rows_reserved == 0
    if s.pool:
        s.pool.shutdown()


@pytest.mark.parametrize("workers", [0, 2])
def test_row_capacity_and_never_fitting_requests(workers):
    s = _server(budget=100, max_rows=10, workers=workers)
    for r in (_req("big", 200, 1), _req("wide", 1, 11), _req("a", 1, 6), _req("b", 1, 6)):
        s.queue.append(r)
    _admit(s)
    rejected = [n for e, n, _ in s.log if e == "rejected"]
    assert rejected == ["big", "wide"]              # more memory or rows than the server has
    assert [x.req.name for x in s.live] == ["a"] and [r.name for r in s.queue] == ["b"]
    _finish(s, "a")
    _admit(s)
    assert [x.req.name for x in s.live] == ["b"]
    if s.pool:
        s.pool.shutdown()


@pytest.mark.parametrize("workers", [0, 2])
def test_injected_allocation_failure_fails_one_request(workers):
    s = _server(budget=10, max_rows=100, workers=workers)
    for r in (_req("a", 3, 1), _req("oom", 5, 1), _req("c", 5, 1)):
        s.queue.append(r)
    _admit(s)
    assert [x.req.name for x in s.live] == ["a", "c"] and s.used == 8
    assert "oom" in s.failures and "injected" in s.failures["oom"]
    assert [(e, n) for e, n, _ in s.log] == [("admitted", "a"), ("failed", "oom"), ("admitted", "c")]
    assert s.reserved == 0 and s.rows_reserved == 0 and not s.preparing
    if s.pool:
        s.pool.shutdown()


def test_a_failed_coarse_solve_fails_its_simulation_alone(monkeypatch):
    # one server step with the device calls faked: the solve of "bad" fails
    # (no convergence); it leaves before the network launch, its memory
    # comes back, and the others are batched and finished as usual
    import contextlib
    s = _server(budget=100, max_rows=100, workers=0)
    closed, calls = [], {}

    class Ev:
        def record(self, stream=None):
            pass

        def synchronize(self):
            pass

    class St:
        def synchronize(self):
            pass

        def wait_event(self, e):
            pass

    def sim(name):
        return SimpleNamespace(req=SimpleNamespace(name=name, solve=True, n_steps=5),
                               path=SimpleNamespace(ctx=name, n_patches=4, close=lambda: closed.append(name)),
                               stream=St(), x=None, b=None, F=None, mem=1, ev_begin=Ev(), ev_end=Ev(),
                               steps_done=0, latencies=[])

    s.live = [sim("a"), sim("bad"), sim("c")]
    s.used = 3
    s.X = SimpleNamespace(element_size=lambda: 2, data_ptr=lambda: 0)
    s.Y = SimpleNamespace(element_size=lambda: 4, data_ptr=lambda: 0)
    s.stream, s.ev_net, s.net, s.solver = St(), Ev(), "net", None
    s.patches, s.step_latencies = 0, []
    s._admit = lambda now: None

    def begin(ctx, x, b, F, X, solve, prm):
        if ctx == "bad":
            raise capi.DnnmgError(-4, "Newton did not converge (injected)")
        calls.setdefault("begin", []).append((ctx, X))

    monkeypatch.setattr(serve.torch.cuda, "stream", lambda st: contextlib.nullcontext())
    monkeypatch.setattr(capi, "dnnmg_step_begin", begin)
    monkeypatch.setattr(capi, "dnnmg_network", lambda net, X, Y, rows: calls.setdefault("rows", []).append(rows))
    monkeypatch.setattr(capi, "dnnmg_step_end", lambda ctx, Y, F, b: calls.setdefault("end", []).append((ctx, Y)))
    monkeypatch.setattr(capi, "dnnmg_sync", lambda net: None)
    s.step(0.0)
    assert list(s.failures) == ["bad"] and closed == ["bad"] and s.used == 2
    assert [x.req.name for x in s.live] == ["a", "c"]
    assert calls["begin"] == [("a", 0), ("c", 4 * 256 * 2)]      # rows packed without the failed one
    assert calls["rows"] == [8] and calls["end"] == [("a", 0), ("c", 4 * 81 * 4)]
    assert [x.steps_done for x in s.live] == [1, 1]
