"""Serving loop with continuous batching of independent Euler solves.

Requests (a periodic box of n^3 elements at degree p, a vortex or
Taylor-Green initial state, a number of LSERK45 steps) arrive over time.  The
server admits waiting requests first-come first-served while their device
memory (state, RK register, second state: three float state arrays) fits a
byte budget, keeps every admitted state resident on the GPU, and advances all
active requests together: between steps it gives the batch the new active set when requests joined or
finished, then replays the batch's recorded step graph; while the active set
cannot change it keeps a second step enqueued behind the one in flight, so
the GPU does not idle during the host's bookkeeping.  A
request completes after exactly its number of steps, each with its own CFL
time step, so its result does not depend on what else is in the batch.

The GPU work runs in the C library (dg_batch_*); this module only schedules.
"""
import collections
import dataclasses
import math
import time
from typing import List, Optional

from . import inputs

NF = 5


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the run
    n: int                  # elements per side
    p: int                  # polynomial degree
    kind: str               # "vortex" or "tgv"
    nsteps: int             # LSERK45 steps to take
    L: float = 10.0         # box side
    cfl: float = 0.5
    params: Optional[list] = None

    @property
    def dof(self):
        return self.n ** 3 * (self.p + 1) ** 3

    def state_bytes(self):
        return NF * self.dof * 4

    def device_bytes(self):
        """Device memory the request holds while admitted: Q, dQ, second state."""
        return 3 * self.state_bytes()

    def spec(self):
        return dict(nx=self.n, ny=self.n, nz=self.n, p=self.p, Lx=self.L, Ly=self.L, Lz=self.L)


def make_requests(seed, count, rate, nrange=(8, 48), prange=(2, 6), steps_range=(50, 500),
                  L=2 * math.pi):
    """Poisson arrivals (mean `rate` per second) of `count` requests with
    seeded sizes, degrees, step counts and initial states (vortex or
    Taylor-Green, 50/50).  All draws come from splitmix64(seed)."""
    r = inputs.uniforms(seed, 5 * count)
    t = 0.0
    reqs = []
    for i in range(count):
        u = r[5 * i:5 * i + 5]
        t += -math.log(1.0 - u[0]) / rate
        n = nrange[0] + min(int(u[1] * (nrange[1] - nrange[0] + 1)), nrange[1] - nrange[0])
        p = prange[0] + min(int(u[2] * (prange[1] - prange[0] + 1)), prange[1] - prange[0])
        s0, s1 = steps_range
        nsteps = s0 + min(int(u[3] * (s1 - s0 + 1)), s1 - s0)
        kind = "vortex" if u[4] < 0.5 else "tgv"
        box = (0.0, 0.0, 0.0, L, L, L)
        params = (inputs.vortex_params(seed * 100003 + i, box) if kind == "vortex"
                  else inputs.tgv_params(0.1))
        reqs.append(Request(i, t, n, p, kind, nsteps, L=L, params=params))
    return reqs


@dataclasses.dataclass
class Outcome:
    rid: int
    arrival: float
    admitted: float
    completed: float
    steps: int
    result: object          # executor-defined (final integrals, optionally the state)

    @property
    def latency(self):
        return self.completed - self.arrival


@dataclasses.dataclass
class Report:
    outcomes: List[Outcome]
    wall: float
    dof_stage_total: float
    peak_bytes: int
    peak_active: int
    iterations: int
    rebuilds: int
    rebuild_s: float = 0.0   # host time spent rebuilding the batch
    enqueue_s: float = 0.0   # host time spent enqueueing steps
    wait_s: float = 0.0      # host time spent waiting for steps to finish

    def percentile(self, q):
        lat = sorted(o.latency for o in self.outcomes)
        if not lat:
            return float("nan")
        k = min(len(lat) - 1, max(0, int(math.ceil(q / 100.0 * len(lat))) - 1))
        return lat[k]

    def summary(self):
        return {"requests": len(self.outcomes), "wall_s": self.wall,
                "throughput_dof_stage_per_s": self.dof_stage_total / self.wall if self.wall else None,
                "requests_per_s": len(self.outcomes) / self.wall if self.wall else None,
                "p50_s": self.percentile(50), "p99_s": self.percentile(99),
                "peak_bytes": self.peak_bytes, "peak_active": self.peak_active,
                "iterations": self.iterations, "batch_rebuilds": self.rebuilds,
                "rebuild_s": self.rebuild_s, "enqueue_s": self.enqueue_s, "wait_s": self.wait_s}


class TimeoutError_(RuntimeError):
    pass


class Server:
    """Admission by byte budget, continuous batching between steps."""

    def __init__(self, executor, budget_bytes, clock=time.perf_counter, step_deadline_s=60.0,
                 keep_states=False):
        self.ex = executor
        self.budget = int(budget_bytes)
        self.clock = clock
        self.deadline = step_deadline_s
        self.keep_states = keep_states

    def run(self, requests):
        pending = sorted(requests, key=lambda q: (q.arrival, q.rid))
        for q in pending:
            if q.device_bytes() > self.budget:
                raise ValueError(f"request {q.rid} needs {q.device_bytes()} B, above the budget")
        waiting = []
        # active: [request, steps not yet enqueued, steps not yet completed, admit time]
        active = []
        inflight = collections.deque()   # enqueued steps: (token, k)
        outcomes = []
        used = peak = peak_active = iters = rebuilds = 0
        dof_stage = rebuild_s = enqueue_s = wait_s = 0.0
        t0 = self.clock()
        changed = False
        i = 0

        def arrive(now):
            nonlocal i
            while i < len(pending) and pending[i].arrival <= now:
                waiting.append(pending[i])
                i += 1

        def enqueue():
            nonlocal enqueue_s
            k = 2 if all(a[1] >= 2 for a in active) else 1
            tr = self.clock()
            token = self.ex.step(k)
            enqueue_s += self.clock() - tr
            for a in active:
                a[1] -= k
            inflight.append((token, k))

        while i < len(pending) or waiting or active:
            now = self.clock() - t0
            arrive(now)
            if inflight:
                # one more step before waiting, when it cannot change what
                # is active: nobody's last step is in flight and nobody
                # waiting could be admitted now
                if (len(inflight) < 2 and all(a[1] > 0 for a in active)
                        and not (waiting and used + waiting[0].device_bytes() <= self.budget)):
                    enqueue()
                token, k = inflight.popleft()
                tw = self.clock()
                if not self.ex.wait(self.deadline, token):
                    raise TimeoutError_(f"step did not finish within {self.deadline} s")
                wait_s += self.clock() - tw
                iters += 1
                done_t = self.clock() - t0
                still = []
                for a in active:
                    q = a[0]
                    a[2] -= k
                    dof_stage += 5.0 * k * q.dof
                    if a[2] == 0:
                        res = self.ex.finish(q, keep_state=self.keep_states)
                        used -= q.device_bytes()
                        outcomes.append(Outcome(q.rid, q.arrival, a[3], done_t, q.nsteps, res))
                        changed = True
                    else:
                        still.append(a)
                active = still
                continue
            # nothing in flight: admissions (first come, first served while
            # the head of the queue fits), the batch for the new active set
            while waiting and used + waiting[0].device_bytes() <= self.budget:
                q = waiting.pop(0)
                self.ex.admit(q)
                used += q.device_bytes()
                active.append([q, q.nsteps, q.nsteps, now])
                changed = True
            peak = max(peak, used)
            peak_active = max(peak_active, len(active))
            if not active:
                if i < len(pending):
                    self.ex.idle_until(t0 + pending[i].arrival, self.clock)
                continue
            if changed:
                tr = self.clock()
                self.ex.rebuild([a[0] for a in active])
                rebuild_s += self.clock() - tr
                rebuilds += 1
                changed = False
            enqueue()
        wall = self.clock() - t0
        return Report(sorted(outcomes, key=lambda o: o.rid), wall, dof_stage, peak, peak_active,
                      iters, rebuilds, rebuild_s, enqueue_s, wait_s)


class GpuExecutor:
    """Runs the batch on the current CUDA device through the C library.

    The library steps a batch with one CFL number, so the active requests are
    grouped by their CFL number into one batch per distinct value, stepped
    one after the other on the executor's stream: every request takes its
    own time steps, whatever else is active."""

    def __init__(self, stream=None):
        import torch

        from . import dg
        self.torch, self.dg = torch, dg
        self.stream = stream or torch.cuda.Stream()
        self.handles = {}     # rid -> dict(Q, dQ, Qt, fresh, req)
        self.groups = []      # [(cfl, Batch, [rid, ...])]
        self.where = {}       # rid -> (group index, index in the batch)

    def admit(self, q):
        t = self.torch
        shape = self.dg.state_shape(q.spec())
        with t.cuda.stream(self.stream):
            h = {"Q": t.empty(shape, dtype=t.float32, device="cuda"),
                 "dQ": t.zeros(shape, dtype=t.float32, device="cuda"),
                 "Qt": t.empty(shape, dtype=t.float32, device="cuda"), "fresh": True, "req": q}
        self.handles[q.rid] = h

    def rebuild(self, reqs):
        """The active set changed (between steps, the GPU idle): each CFL
        group's batch takes its new instance list in place (dg_batch_update:
        its device arrays and streams are kept), a new group gets a batch."""
        by_cfl = {}
        for q in reqs:
            by_cfl.setdefault(float(q.cfl), []).append(q)
        old = {cfl: batch for cfl, batch, _ in self.groups}
        with self.torch.cuda.stream(self.stream):
            self.groups = []
            self.where = {}
            for cfl in sorted(by_cfl):
                members = by_cfl[cfl]
                specs = []
                for q in members:
                    h = self.handles[q.rid]
                    s = q.spec()
                    s.update(Q=h["Q"], dQ=h["dQ"], Qt=h["Qt"])
                    specs.append(s)
                batch = old.pop(cfl, None)
                if batch is None:
                    batch = self.dg.Batch(specs)
                else:
                    batch.update(specs)
                for idx, q in enumerate(members):
                    h = self.handles[q.rid]
                    if h["fresh"]:
                        batch.init(idx, q.kind, q.params)
                        h["fresh"] = False
                    self.where[q.rid] = (len(self.groups), idx)
                self.groups.append((cfl, batch, [q.rid for q in members]))

    def step(self, k):
        """Enqueue k steps of every group; returns the event that marks their end."""
        with self.torch.cuda.stream(self.stream):
            for cfl, batch, _ in self.groups:
                batch.step(cfl, nsteps=k, use_graph=True)
            event = self.torch.cuda.Event()
            event.record(self.stream)
        return event

    def wait(self, deadline_s, event):
        """Poll a step's event until it completes or the deadline passes."""
        t_end = time.perf_counter() + deadline_s
        while not event.query():
            if time.perf_counter() > t_end:
                return False
            time.sleep(20e-6)
        return True

    def finish(self, q, keep_state=False):
        h = self.handles.pop(q.rid)
        g, idx = self.where[q.rid]
        with self.torch.cuda.stream(self.stream):
            integrals = self.groups[g][1].norms(idx).cpu().tolist()
            state = h["Q"].cpu() if keep_state else None
        return {"integrals": integrals, "state": state}

    def idle_until(self, t_abs, clock):
        dt = t_abs - clock()
        if dt > 0:
            time.sleep(min(dt, 0.05))


class FakeExecutor:
    """Stand-in for the GPU executor in host-logic tests: a step costs
    `cost_per_dof_step` seconds per DOF of the active set, and a request's
    result is a deterministic function of the request alone."""

    def __init__(self, clock, cost_per_dof_step=1e-9):
        self.clock = clock
        self.cost = cost_per_dof_step
        self.active = []
        self.log = []

    def admit(self, q):
        self.log.append(("admit", q.rid))

    def rebuild(self, reqs):
        self.active = list(reqs)
        self.log.append(("rebuild", tuple(q.rid for q in reqs)))

    def step(self, k):
        self.clock.advance(k * self.cost * sum(q.dof for q in self.active))
        return k

    def wait(self, deadline_s, token):
        return True

    def finish(self, q, keep_state=False):
        self.log.append(("finish", q.rid))
        return {"integrals": [float(q.rid), float(q.nsteps)], "state": None}

    def idle_until(self, t_abs, clock):
        self.clock.advance(max(0.0, t_abs - clock()))


class ManualClock:
    """Deterministic clock for FakeExecutor runs."""

    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def advance(self, dt):
        self.t += dt
