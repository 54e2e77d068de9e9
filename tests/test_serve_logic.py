"""Host logic of the continuous-batching server, with fake device operations
(no GPU): budgeted FIFO admission, release on completion, rejection of
requests larger than the whole budget, and per-request step accounting."""
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
                 clock=iter(np.arange(0, 1e6, 1e-3)).__next__)
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
