"""Serving policy on the CPU: admission by footprint, grouping, continuous admission.

The dispatcher is exercised against a fake backend (sleeps instead of GPU
work), so these tests run without a GPU.
"""
import time

from paper_1701_01170_gb300.serve import (OP_BFS, OP_SSSP, Dispatcher, GraphInfo, Request,
                                          Unit, serve_trace)


def infos(multi=("a",)):
    return {
        "a": GraphInfo("a", 1000, 100, 200, 500, "a" in multi, max_group=4),
        "b": GraphInfo("b", 5000, 300, 600, 900, "b" in multi, max_group=2),
    }


def req(i, g, op, t=0.0):
    return Request(i, g, op, i, t)


def test_bfs_requests_on_low_diameter_graph_are_grouped():
    d = Dispatcher(infos(), lanes=2, budget=10_000)
    d.pending.extend([req(0, "a", OP_BFS), req(1, "b", OP_BFS), req(2, "a", OP_BFS),
                      req(3, "a", OP_SSSP), req(4, "a", OP_BFS), req(5, "a", OP_BFS),
                      req(6, "a", OP_BFS)])
    u, ev = d.admit(0)
    assert u.multi and u.graph == "a" and [r.rid for r in u.requests] == [0, 2, 4, 5]
    assert [r.rid for r in d.pending] == [1, 3, 6]          # order of the rest is kept
    u2, _ = d.admit(1)                                       # "a" is busy with MS-BFS
    assert not u2.multi and u2.requests[0].rid == 1
    d.release(u)
    u3, _ = d.admit(0)
    assert not u3.multi and u3.requests[0].rid == 3          # FIFO: the SSSP comes next


def test_admission_respects_the_memory_budget_and_evicts_lru():
    d = Dispatcher(infos(multi=()), lanes=1, budget=700)
    d.pending.extend([req(0, "a", OP_BFS), req(1, "a", OP_SSSP), req(2, "b", OP_SSSP)])
    u, ev = d.admit(0)
    assert u.requests[0].rid == 0 and d.used == 100 and not ev
    u, ev = d.admit(0)
    assert u.requests[0].rid == 1 and d.used == 300 and not ev
    u, ev = d.admit(0)                    # needs 600: evicts a/BFS then a/SSSP
    assert u.requests[0].rid == 2 and ev == [(0, ("a", OP_BFS)), (0, ("a", OP_SSSP))]
    assert d.used == 600 and d.evictions == 2


def test_idle_lanes_workspaces_are_evicted_too():
    # the budget is held by two lanes; a request that needs both lanes' memory is
    # admitted only when the other lane is idle, and evicts the own lane's first
    d = Dispatcher(infos(multi=()), lanes=2, budget=650)
    d.pending.extend([req(0, "a", OP_SSSP), req(1, "b", OP_BFS), req(2, "b", OP_SSSP)])
    u, _ = d.admit(0)
    assert u.requests[0].rid == 0                 # lane 0 holds a/SSSP (200)
    u, _ = d.admit(1)
    assert u.requests[0].rid == 1                 # lane 1 holds b/BFS (300)
    u, ev = d.admit(0, idle=[0])                  # lane 1 busy: 600 does not fit
    assert u is None and d.used == 500
    u, ev = d.admit(0, idle=[0, 1])
    assert u.requests[0].rid == 2
    assert ev == [(0, ("a", OP_SSSP)), (1, ("b", OP_BFS))]
    assert d.used == 600 and not d.lane_ws[1]


def test_request_that_cannot_fit_waits_while_others_proceed():
    d = Dispatcher(infos(multi=()), lanes=2, budget=350)
    d.pending.extend([req(0, "a", OP_SSSP), req(1, "b", OP_SSSP), req(2, "a", OP_BFS)])
    u, _ = d.admit(0)
    assert u.requests[0].rid == 0                 # 200 used
    u, _ = d.admit(1)                             # b/SSSP (600) does not fit anywhere
    assert u.requests[0].rid == 2                 # the later BFS (100) is admitted instead
    assert [r.rid for r in d.pending] == [1]


class FakeBackend:
    """Runs units by sleeping 1 ms per request (2 ms for a group); records overlap."""

    def __init__(self):
        self.active = 0
        self.max_active = 0

    def graph_infos(self, multi):
        return infos(multi=tuple(multi))

    def evict(self, lane, keys):
        pass

    def run(self, lane, unit: Unit, t0):
        self.active += 1
        self.max_active = max(self.max_active, self.active)
        for r in unit.requests:
            r.t_start = time.perf_counter() - t0
        time.sleep(0.002 if unit.multi else 0.001)
        done = time.perf_counter() - t0
        for r in unit.requests:
            r.t_done = done
            r.result = (unit.graph, r.src)
        self.active -= 1


def test_trace_completes_when_the_budget_is_spread_over_idle_lanes():
    # two lanes end up holding one workspace each; the next request needs the
    # memory of both (a dispatcher that lets a lane evict only its own
    # workspaces waits for ever here, with every lane idle)
    trace = [Request(0, "a", OP_SSSP, 0, 0.0), Request(1, "b", OP_BFS, 1, 0.0),
             Request(2, "b", OP_SSSP, 2, 0.05)]
    be = FakeBackend()
    stats = serve_trace(be, trace, lanes=2, budget=650)
    assert stats["completed"] == 3 and stats["errors"] == 0
    assert all(r.result == (r.graph, r.src) for r in trace)


def test_request_beyond_the_budget_is_an_error():
    import pytest
    trace = [Request(0, "b", OP_SSSP, 0, 0.0)]
    with pytest.raises(RuntimeError):
        serve_trace(FakeBackend(), trace, lanes=2, budget=500)


def test_trace_completes_with_overlap_and_grouping():
    trace = [Request(i, "a" if i % 3 else "b", OP_BFS if i % 2 else OP_SSSP, i, 0.0005 * i)
             for i in range(60)]
    be = FakeBackend()
    stats = serve_trace(be, trace, lanes=3, budget=10_000, multi_names=("a",))
    assert stats["completed"] == 60 and stats["errors"] == 0
    assert all(r.result == (r.graph, r.src) for r in trace)
    assert all(r.t_done >= r.t_arrival for r in trace)
    assert be.max_active >= 2                                   # lanes overlapped
    assert stats["p99_ms"] >= stats["p50_ms"] > 0
