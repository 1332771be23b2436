"""Served stream of MD requests on one GPU: continuous batching over one gbmd batch.

A request asks for `steps` velocity-Verlet steps of an LJ system it supplies
(positions, velocities, types, box, pair table).  The server

* admits waiting requests strictly in arrival order while the summed
  ``gbmd_footprint_bytes`` of the resident systems stays within an HBM budget (a
  request larger than the whole budget is rejected at arrival);
* steps every resident system together through one gbmd batch -- one launch per
  kernel per step for all of them, captured in CUDA graphs -- in quanta of at most
  ``max_quantum`` steps, the quantum ending when the resident request closest to
  completion finishes;
* stops each system at exactly its own step count (``gbmd_set_step_limit``: a
  system past its limit is skipped inside the shared launches), then reads its
  final thermodynamic state, removes it from the batch and frees it.

Completion latency is retirement time minus arrival time.  The policy (``Scheduler``)
is independent of the device: it drives a backend with four operations, so the
host logic is tested on the CPU with a simulated backend and clock, and runs on the
GPU with ``GpuBackend``.
"""
from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass
from typing import Callable, Optional


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the trace
    steps: int
    n: int
    payload: object = None  # what the backend needs to build the system (a Workload)


@dataclass
class Record:
    rid: int
    n: int
    steps: int
    arrival: float
    admitted: Optional[float] = None
    finished: Optional[float] = None
    footprint: int = 0
    rejected: bool = False
    result: Optional[dict] = None

    @property
    def latency(self) -> Optional[float]:
        return None if self.finished is None else self.finished - self.arrival


@dataclass
class Summary:
    records: list
    makespan: float
    particle_steps: int
    peak_resident_bytes: int
    quanta: int
    p50: float
    p99: float
    mean: float

    @property
    def throughput(self) -> float:
        return self.particle_steps / self.makespan if self.makespan > 0 else 0.0


def percentile(xs, q):
    """Nearest-rank percentile (q in [0, 100]) of a non-empty sequence."""
    s = sorted(xs)
    k = max(0, min(len(s) - 1, math.ceil(q / 100.0 * len(s)) - 1))
    return s[k]


class Scheduler:
    """Continuous batching with FIFO admission under a byte budget.

    backend: object with
      footprint(req) -> int            bytes the system will hold on the device
      start(req) -> handle             create the system, cap it at req.steps, add it
      advance(k)                       run k steps of the batch and wait for them
      done(handle) -> int              steps the system has completed
      finish(handle) -> dict           read the result, remove and free the system
    clock: () -> seconds (monotonic); wait(t): block until clock() >= t.
    """

    def __init__(self, backend, budget_bytes: int, max_quantum: int = 2000,
                 min_quantum: int = 16, clock: Callable[[], float] = time.perf_counter,
                 wait: Optional[Callable[[float], None]] = None):
        if budget_bytes <= 0 or max_quantum < 1 or not 1 <= min_quantum <= max_quantum:
            raise ValueError("need budget > 0 and 1 <= min_quantum <= max_quantum")
        self.backend = backend
        self.budget = int(budget_bytes)
        self.max_quantum = int(max_quantum)
        self.min_quantum = int(min_quantum)
        self.clock = clock
        self.wait = wait or (lambda t: time.sleep(max(0.0, t - self.clock())))

    def run(self, requests) -> Summary:
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        recs = {r.rid: Record(r.rid, r.n, r.steps, r.arrival) for r in reqs}
        pending = deque(reqs)        # not yet arrived
        waiting: deque = deque()     # arrived, not admitted
        active = {}                  # rid -> (request, backend handle)
        used = peak = 0
        quanta = 0
        t0 = self.clock()
        now = lambda: self.clock() - t0
        while pending or waiting or active:
            t = now()
            while pending and pending[0].arrival <= t:
                r = pending.popleft()
                rec = recs[r.rid]
                rec.footprint = int(self.backend.footprint(r))
                if rec.footprint > self.budget:
                    rec.rejected = True
                else:
                    waiting.append(r)
            while waiting and used + recs[waiting[0].rid].footprint <= self.budget:
                r = waiting.popleft()
                rec = recs[r.rid]
                h = self.backend.start(r)
                rec.admitted = now()
                used += rec.footprint
                peak = max(peak, used)
                active[r.rid] = (r, h)
            if not active:
                if pending:
                    self.wait(t0 + pending[0].arrival)
                    continue
                if waiting:   # cannot happen: an empty device admits the head
                    raise RuntimeError("head request does not fit an empty device")
                break
            left = min(r.steps - self.backend.done(h) for r, h in active.values())
            k = max(self.min_quantum, min(self.max_quantum, left))
            self.backend.advance(k)
            quanta += 1
            t = now()
            for rid in [rid for rid, (r, h) in active.items() if self.backend.done(h) >= r.steps]:
                r, h = active.pop(rid)
                rec = recs[rid]
                rec.result = self.backend.finish(h)
                rec.finished = t
                used -= rec.footprint
        makespan = now()
        out = [recs[r.rid] for r in reqs]
        lat = [x.latency for x in out if x.latency is not None]
        ps = sum(x.n * x.steps for x in out if x.finished is not None)
        return Summary(out, makespan, ps, peak, quanta,
                       percentile(lat, 50) if lat else float("nan"),
                       percentile(lat, 99) if lat else float("nan"),
                       sum(lat) / len(lat) if lat else float("nan"))


class GpuBackend:
    """Resident systems in one gbmd batch on the current CUDA device.

    A request's payload is a Workload, or a trace entry (dict with n, rho, T, seed)
    from which the seeded LJ fluid is generated when the request is admitted."""

    def __init__(self, precision: str = "mixed", stream=None, cuda_device: int = -1,
                 tuning: Optional[tuple] = None, keep_state: bool = False,
                 r_buff: float = 0.4, dt: float = 0.005):
        from . import gbmd
        self.gbmd = gbmd
        self.precision = precision
        self.stream = stream
        self.cuda_device = cuda_device
        self.keep_state = keep_state
        self.r_buff, self.dt = r_buff, dt
        self.batch = gbmd.Batch(precision, stream=stream, cuda_device=cuda_device)
        if tuning:
            self.batch.set_tuning(*tuning)
        self.slots = {}

    def _workload(self, payload):
        if isinstance(payload, dict):
            from . import workloads as wl
            return wl.lj_fluid(payload["n"], payload["rho"], payload["T"], payload["seed"],
                               r_buff=self.r_buff, dt=self.dt)
        return payload

    def footprint(self, req: Request) -> int:
        import numpy as np
        w = req.payload
        if isinstance(w, dict):   # geometry only: no positions are needed
            box = (w["n"] / w["rho"]) ** (1.0 / 3.0)
            z = np.zeros((1, 3))
            d, keep = self.gbmd.make_desc(w["n"], box, z, z, None, 1.0, 1.0, 2.5, self.r_buff,
                                          self.dt, 1.0, self.precision)
        else:
            p = w.pairs
            d, keep = self.gbmd.make_desc(w.n, w.box, w.pos, w.vel, w.types, p.eps, p.sigma,
                                          p.rcut, w.r_buff, w.dt, w.mass, self.precision)
        return self.gbmd.gbmd_footprint_bytes(d)

    def start(self, req: Request):
        s = self.gbmd.System.from_workload(self._workload(req.payload), precision=self.precision,
                                           stream=self.stream, cuda_device=self.cuda_device)
        s.set_step_limit(req.steps)
        self.slots[id(s)] = [self.batch.add(s), req.steps, 0]
        return s

    def advance(self, k: int):
        self.batch.step(k)
        self.batch.sync()   # raises on a device error; recovers list overflows
        for v in self.slots.values():   # a system stops at its step limit
            v[2] = min(v[1], v[2] + k)

    def done(self, s) -> int:
        return self.slots[id(s)][2]

    def finish(self, s) -> dict:
        res = dict(s.thermo())
        if res["step"] != self.slots[id(s)][1]:
            raise RuntimeError(f"system stopped at step {res['step']}, "
                               f"not at its limit {self.slots[id(s)][1]}")
        if self.keep_state:
            res["state"] = s.state()
        self.batch.remove(self.slots.pop(id(s))[0])
        s.close()
        return res

    def close(self):
        self.batch.close()


class SimBackend:
    """Device stand-in for testing the policy on the CPU: a simulated clock that a
    step of the batch advances by (resident particles) / rate seconds."""

    def __init__(self, rate: float = 1e9, footprint_per_particle: int = 700):
        self.rate = rate
        self.fpp = footprint_per_particle
        self.t = 0.0
        self.live = {}      # handle -> [request, steps done]
        self.next = 0
        self.log = []       # (event, rid, time, resident bytes)

    def clock(self) -> float:
        return self.t

    def wait(self, t: float):
        self.t = max(self.t, t)

    def footprint(self, req: Request) -> int:
        return self.fpp * req.n

    def start(self, req: Request):
        self.next += 1
        self.live[self.next] = [req, 0]
        self.log.append(("start", req.rid, self.t, self.resident()))
        return self.next

    def resident(self) -> int:
        return sum(self.fpp * r.n for r, _ in self.live.values())

    def advance(self, k: int):
        self.t += k * sum(r.n for r, _ in self.live.values()) / self.rate
        for v in self.live.values():
            v[1] = min(v[0].steps, v[1] + k)   # the step limit stops a system exactly

    def done(self, h) -> int:
        return self.live[h][1]

    def finish(self, h) -> dict:
        r, d = self.live.pop(h)
        self.log.append(("finish", r.rid, self.t, self.resident()))
        return {"step": d}


def requests_from_trace(trace):
    """workloads.request_trace entries -> Requests whose payload is the entry itself
    (the backend generates the system when it admits the request)."""
    return [Request(k, d["arrival"], d["steps"], d["n"], d) for k, d in enumerate(trace)]
