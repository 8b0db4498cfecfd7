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
