"""Host logic of the continuous-batching server, with fake device operations
(no GPU): budgeted FIFO and shortest-work-first admission with an age bound,
release on completion, rejection of requests larger than the whole budget,
and per-request step accounting."""
from dataclasses import dataclass

import numpy as np

from paper_2301_10041_gb300.serve import Ops, Request, Server


@dataclass
class FakeCase:
    N: int


@dataclass
class FakeInfo:
    status: int = 0


class FakeDevice:
    def __init__(self):
        self.rng = np.random.default_rng(1)
        self.live = {}
        self.next = 0
        self.peak_used = 0

    def ops(self, server_ref):
        def footprint(case):
            return case.N * 1000

        def create(case):
            h = self.next
            self.next += 1
            self.live[h] = {"N": case.N, "steps": 0}
            self.peak_used = max(self.peak_used, server_ref[0].used + footprint(case))
            return h

        def step_async(h):
            self.live[h]["steps"] += 1
            self.live[h]["polls"] = int(self.rng.integers(0, 3))   # still running for a few polls

        def poll(h):
            if self.live[h]["polls"] > 0:
                self.live[h]["polls"] -= 1
                return None
            return FakeInfo()

        def finish(h):
            return {"N": self.live[h]["N"], "steps": self.live[h]["steps"]}

        def close(h):
            del self.live[h]

        return Ops(footprint, create, step_async, poll, finish, close)


def test_budgeted_fifo_admission_and_release():
    dev = FakeDevice()
    ref = [None]
    srv = Server(dev.ops(ref), budget_bytes=100_000, max_resident=8, admit_per_tick=2,
                 clock=iter(np.arange(0, 1e6, 1e-3)).__next__, policy="fifo")
    ref[0] = srv
    rng = np.random.default_rng(0)
    reqs = [Request(rid=i, arrival=0.0, case=FakeCase(int(rng.choice([16, 32, 64]))), steps=int(rng.integers(1, 6)))
            for i in range(40)]
    reqs.append(Request(rid=99, arrival=0.0, case=FakeCase(1000), steps=3))   # larger than the whole budget
    wall = srv.run(reqs, realtime=False)
    assert wall > 0
    assert len(srv.finished) == 40 and [r.rid for r in srv.rejected] == [99]
    assert not dev.live                                   # every instance was closed
    assert dev.peak_used <= 100_000                       # never above the budget
    for r in srv.finished:
        assert r.result["steps"] == r.steps == r.done == len(r.step_ms)
    # FIFO: admission order is submission order
    order = sorted(srv.finished, key=lambda r: r.admit_seq)
    assert [r.rid for r in order] == sorted(r.rid for r in order)
    rep = srv.report(wall)
    assert rep["steps"] == sum(r.steps for r in reqs if r.rid != 99)
    assert rep["requests_rejected"] == 1


def test_admission_footprint_follows_the_solid_element():
    """The server's footprint (host logic of the library, no device call)
    takes the element type from the mesh: Q1 quadrilaterals (9 rule points
    per element) need more coupling storage than the same counts as P1, and
    P1 and Q1 sizes are cached apart."""
    import pytest
    import fsi_inputs as fi
    from paper_2301_10041_gb300 import build
    from paper_2301_10041_gb300.serve import gpu_ops
    try:
        build.build()
    except RuntimeError as e:
        pytest.skip(str(e))
    ops = gpu_ops(precision=1)
    q1 = fi.annulus_case(16, quads=True)
    p1_same_counts = fi.FsiCase(N=q1.N, rho_f=q1.rho_f, nu=q1.nu, kappa=q1.kappa, dt=q1.dt, lid_u=0.0,
                                ref_xy=q1.ref_xy, tris=np.zeros((q1.tris.shape[0], 3), dtype=np.int32),
                                u0=q1.u0, X0=q1.X0, rtol=q1.rtol)
    f_q1 = ops.footprint(q1)
    f_p1 = ops.footprint(p1_same_counts)
    assert f_q1 > 0 and f_p1 > 0 and f_q1 != f_p1
    assert ops.footprint(q1) == f_q1    # cached per (N, nodes, elements, element type)


def _sjf_run(max_wait_s, budget=100_000):
    dev = FakeDevice()
    ref = [None]
    srv = Server(dev.ops(ref), budget_bytes=budget, max_resident=2, admit_per_tick=1,
                 clock=iter(np.arange(0, 1e6, 1e-3)).__next__, policy="sjf", max_wait_s=max_wait_s,
                 cost=lambda case: case.N ** 2)
    ref[0] = srv
    # one large request first in the queue, then many small ones, all at t = 0
    reqs = [Request(rid=0, arrival=0.0, case=FakeCase(90), steps=5)]
    reqs += [Request(rid=i, arrival=0.0, case=FakeCase(8), steps=2) for i in range(1, 30)]
    wall = srv.run(reqs, realtime=False)
    return srv, dev, wall


def test_shortest_work_first_admits_small_requests_past_a_large_head():
    """With a large age bound the small requests are admitted before the
    large one at the head of the queue (which FIFO would take first)."""
    srv, dev, wall = _sjf_run(max_wait_s=1e9)
    assert len(srv.finished) == 30 and not dev.live and dev.peak_used <= 100_000
    order = [r.rid for r in sorted(srv.finished, key=lambda r: r.admit_seq)]
    assert order[-1] == 0                        # the large request went last
    for r in srv.finished:
        assert r.result["steps"] == r.steps == r.done


def test_age_bound_lets_a_waiting_request_through():
    """The server's clock advances 1 ms per reading; once the large request
    has waited longer than the bound it is admitted before the remaining small
    ones, so it cannot starve."""
    srv, dev, wall = _sjf_run(max_wait_s=0.05)
    assert len(srv.finished) == 30 and not dev.live
    order = [r.rid for r in sorted(srv.finished, key=lambda r: r.admit_seq)]
    assert 0 < order.index(0) < len(order) - 1   # past some small ones, not after all of them


def test_aged_request_that_does_not_fit_holds_the_queue():
    """While the oldest aged request does not fit in the free budget, nothing
    younger is admitted: the budget frees up for it."""
    srv, dev, wall = _sjf_run(max_wait_s=0.0, budget=91_000)   # the large one needs 90 000
    order = [r.rid for r in sorted(srv.finished, key=lambda r: r.admit_seq)]
    assert order[0] == 0                         # aged at once, first in, alone in the budget
    assert dev.peak_used <= 91_000
