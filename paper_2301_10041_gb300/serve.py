"""Continuous-batching server for FSI instances on one GPU.

Requests (an FSI case and a number of time steps) arrive over time.  The
server admits waiting requests while their device footprint
(``fsi_footprint_bytes``) fits in the free part of the memory budget, keeps
every admitted instance resident on the device (meshes, coupling matrices,
multipliers, Krylov state), and keeps every resident instance busy: each has
its own stream, a step is queued with ``fsi_step_async`` as soon as the
previous one of that instance has finished (``fsi_step_poll``), so the steps
of different instances overlap on the GPU and a slow instance never holds the
others back.  An instance that has done its steps leaves at once and frees its
budget for the next waiting request.

Admission order (``policy``): "fifo" takes the head of the queue and waits
until it fits; "sjf" (the default) takes, among the waiting requests that fit,
the one with the least predicted work (steps x predicted cost of one step, by
default proportional to the fluid unknowns), so that a large, slow request at
the head no longer holds back the small ones behind it.  A request that has
waited longer than ``max_wait_s`` is aged: aged requests go first, oldest
first, and while the oldest one does not fit nothing younger is admitted, so
no request waits forever.

The scheduling logic (``Server``) takes its device operations as callables so
that it can be exercised on the CPU with fakes; ``gpu_ops()`` binds them to the
CUDA library.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the run
    case: object            # fsi_inputs.FsiCase
    steps: int
    footprint: int = 0
    admitted_at: float | None = None
    admit_seq: int = -1
    finished_at: float | None = None
    done: int = 0
    step_ms: list = field(default_factory=list)
    handle: object = None
    started: float | None = None      # clock at which the running step was queued
    result: object = None
    error: str | None = None


@dataclass
class Ops:
    """Device operations the server needs (the CUDA library, or fakes)."""
    footprint: callable      # case -> bytes
    create: callable         # case -> handle
    step_async: callable     # handle -> None (queue one time step)
    poll: callable           # handle -> None while running, else an info with .status
    finish: callable         # handle -> result (host copy of the final state)
    close: callable          # handle -> None


def unknowns_cost(case) -> float:
    """Predicted cost of one time step: the fluid unknowns, 2 (2N-1)^2 + 3 N^2."""
    return 2.0 * (2 * case.N - 1) ** 2 + 3.0 * case.N ** 2


class Server:
    def __init__(self, ops: Ops, budget_bytes: int, max_resident: int = 16, admit_per_tick: int = 1,
                 clock=time.perf_counter, policy: str = "sjf", max_wait_s: float = 2.0, cost=unknowns_cost):
        if policy not in ("fifo", "sjf"):
            raise ValueError("policy")
        self.ops = ops
        self.budget = int(budget_bytes)
        self.max_resident = max_resident
        self.admit_per_tick = admit_per_tick   # creation is host work: bound it per tick
        self.clock = clock
        self.policy = policy
        self.max_wait_s = max_wait_s
        self.cost = cost
        self.waiting: deque[Request] = deque()
        self.resident: list[Request] = []
        self.finished: list[Request] = []
        self.rejected: list[Request] = []
        self.used = 0
        self.ticks = 0
        self.steps_done = 0
        self.admissions = 0

    def submit(self, req: Request):
        req.footprint = int(self.ops.footprint(req.case))
        if req.footprint > self.budget:
            req.error = "footprint above the whole budget"
            self.rejected.append(req)
            return
        self.waiting.append(req)

    def _next(self, now: float):
        """The waiting request to admit next, or None (nothing fits, or an
        aged request that does not fit yet holds the queue)."""
        if self.policy == "fifo":
            r = self.waiting[0]
            return r if self.used + r.footprint <= self.budget else None
        oldest = self.waiting[0]           # arrival order is queue order
        if now - oldest.arrival > self.max_wait_s:
            return oldest if self.used + oldest.footprint <= self.budget else None
        best = None
        for r in self.waiting:
            if self.used + r.footprint > self.budget:
                continue
            if best is None or r.steps * self.cost(r.case) < best.steps * self.cost(best.case):
                best = r
        return best

    def _admit(self, now: float):
        admitted = 0
        while self.waiting and len(self.resident) < self.max_resident and admitted < self.admit_per_tick:
            r = self._next(now)
            if r is None:
                break
            self.waiting.remove(r)
            r.handle = self.ops.create(r.case)
            r.admitted_at = now
            r.admit_seq = self.admissions
            self.admissions += 1
            self.used += r.footprint
            self.resident.append(r)
            admitted += 1

    def tick(self, now: float):
        """Admit what fits, queue a step on every idle resident instance, and
        collect the steps that have finished."""
        self._admit(now)
        for r in self.resident:
            if r.started is None:
                r.started = self.clock()
                self.ops.step_async(r.handle)
        keep = []
        progressed = 0
        for r in self.resident:
            inf = self.ops.poll(r.handle)
            if inf is None:
                keep.append(r)
                continue
            progressed += 1
            r.step_ms.append((self.clock() - r.started) * 1e3)
            r.started = None
            r.done += 1
            self.steps_done += 1
            failed = getattr(inf, "status", 0) != 0
            if failed:
                r.error = f"status {inf.status}"
            if r.done >= r.steps or failed:
                r.result = self.ops.finish(r.handle)
                self.ops.close(r.handle)
                r.handle = None
                r.finished_at = self.clock()
                self.used -= r.footprint
                self.finished.append(r)
            else:
                keep.append(r)
        self.resident = keep
        self.ticks += 1
        return progressed

    def run(self, requests: list[Request], realtime: bool = True, max_wall: float | None = None):
        """Replay the arrival trace (in wall time when realtime) until every
        request has finished or been rejected."""
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        start = self.clock()
        while pending or self.waiting or self.resident:
            now = self.clock() - start
            # without realtime every request is there from the start
            while pending and (pending[0].arrival <= now or not realtime):
                self.submit(pending.popleft())
            if not self.resident and not self.waiting and pending and realtime:
                time.sleep(max(0.0, min(0.01, pending[0].arrival - now)))
                continue
            if self.tick(now) == 0 and self.resident and realtime:
                time.sleep(50e-6)   # nothing finished yet: do not spin on the driver
            if max_wall is not None and self.clock() - start > max_wall:
                break
        return self.clock() - start

    def report(self, wall_s: float) -> dict:
        lat = [ms for r in self.finished for ms in r.step_ms]
        waits = [r.admitted_at - r.arrival for r in self.finished
                 if r.admitted_at is not None and np.isfinite(r.admitted_at)]
        return {
            "requests_finished": len(self.finished),
            "requests_rejected": len(self.rejected),
            "requests_unfinished": len(self.waiting) + len(self.resident),
            "steps": self.steps_done,
            "steps_per_s": self.steps_done / wall_s if wall_s > 0 else None,
            "step_latency_ms": {"p50": float(np.percentile(lat, 50)) if lat else None,
                                "p99": float(np.percentile(lat, 99)) if lat else None},
            "queue_wait_s": {"p50": float(np.percentile(waits, 50)) if waits else None,
                             "p99": float(np.percentile(waits, 99)) if waits else None},
            "ticks": self.ticks,
            "wall_s": wall_s,
        }


def gpu_ops(precision: int = 1, restart: int = 60, stokes_its: int = 8, precond: int = 2,
            max_solid_nodes=None) -> Ops:
    """Bind the server to the CUDA library (instances own their streams).

    ``max_solid_nodes(N) -> (n_nodes, n_tris)``, when given, makes the
    admission footprint a per-N upper bound computed once per grid size (the
    fluid part dominates); otherwise it is computed per distinct mesh size."""
    from . import fsi

    cache: dict = {}

    def params(case):
        # a mesh of quadrilaterals takes the Q1 solid
        return fsi.make_params(case.N, case.rho_f, case.nu, case.kappa, case.dt, case.lid_u,
                               precond=precond, precision=precision, rtol=case.rtol, restart=restart,
                               max_it=6000, stokes_its=stokes_its, solid_elem=int(case.tris.shape[1] == 4))

    def footprint(case):
        if max_solid_nodes is not None:
            key = (case.N,) + tuple(max_solid_nodes(case.N)) + (case.tris.shape[1],)
        else:
            key = (case.N, case.ref_xy.shape[0], case.tris.shape[0], case.tris.shape[1])
        if key not in cache:
            cache[key] = fsi.footprint_bytes(params(case), key[1], key[2])
        return cache[key]

    def create(case):
        return fsi.Problem(params(case), case.ref_xy, case.tris, u0=case.u0, X0=case.X0)

    def step_async(h):
        h.step_async()

    def poll(h):
        return h.step_poll()

    def finish(h):
        return h.get_state()

    def close(h):
        h.close()

    return Ops(footprint, create, step_async, poll, finish, close)
