"""Host logic of the serving loop (no GPU): admission by byte budget, first
come first served, continuous batching between steps, exact step counts,
latency accounting, bounded waits."""
import pytest

from paper_2006_15698_gb300 import serve


def _reqs(n=12, rate=50.0, seed=3):
    return serve.make_requests(seed, n, rate, nrange=(4, 10), prange=(1, 4), steps_range=(3, 9))


def test_make_requests_is_seeded_and_poisson_ordered():
    a, b = _reqs(), _reqs()
    assert [(q.arrival, q.n, q.p, q.nsteps, q.kind) for q in a] == \
           [(q.arrival, q.n, q.p, q.nsteps, q.kind) for q in b]
    assert all(a[i].arrival < a[i + 1].arrival for i in range(len(a) - 1))
    assert {q.kind for q in serve.make_requests(1, 200, 10.0)} == {"vortex", "tgv"}


def test_all_requests_complete_within_budget():
    clock = serve.ManualClock()
    ex = serve.FakeExecutor(clock, cost_per_dof_step=2e-8)
    reqs = _reqs(rate=2000.0)
    budget = 3 * max(q.device_bytes() for q in reqs)
    rep = serve.Server(ex, budget, clock=clock).run(reqs)
    assert sorted(o.rid for o in rep.outcomes) == sorted(q.rid for q in reqs)
    for o, q in zip(rep.outcomes, sorted(reqs, key=lambda r: r.rid)):
        assert o.steps == q.nsteps
        assert o.admitted >= o.arrival and o.completed > o.admitted
        assert o.result["integrals"] == [float(q.rid), float(q.nsteps)]
    assert rep.peak_bytes <= budget
    assert rep.peak_active >= 2                   # requests overlap on the device
    assert rep.percentile(50) <= rep.percentile(99)
    # first come, first served admission
    admits = [rid for ev, rid in ex.log if ev == "admit"]
    assert admits == [q.rid for q in sorted(reqs, key=lambda r: r.arrival)]


def test_joins_and_leaves_between_steps():
    clock = serve.ManualClock()
    ex = serve.FakeExecutor(clock, cost_per_dof_step=1e-8)
    reqs = _reqs(8, rate=1000.0)
    rep = serve.Server(ex, 10 ** 12, clock=clock).run(reqs)
    rebuilds = [members for ev, members in ex.log if ev == "rebuild"]
    assert len(rebuilds) == rep.rebuilds >= 2
    # a finished request never reappears in a later batch
    finished = set()
    for ev in ex.log:
        if ev[0] == "finish":
            finished.add(ev[1])
        if ev[0] == "rebuild":
            assert not finished & set(ev[1])


def test_oversize_request_rejected():
    reqs = _reqs(3)
    with pytest.raises(ValueError):
        serve.Server(serve.FakeExecutor(serve.ManualClock()), 100).run(reqs)


def test_step_deadline():
    class Stuck(serve.FakeExecutor):
        def wait(self, deadline_s, token):
            return False

    clock = serve.ManualClock()
    with pytest.raises(serve.TimeoutError_):
        serve.Server(Stuck(clock), 10 ** 12, clock=clock, step_deadline_s=0.01).run(_reqs(2))


class Tracking(serve.FakeExecutor):
    """FakeExecutor that checks the pipelining rules: at most two steps in
    flight, and batch changes (rebuild) and result reads (finish) only with
    nothing in flight; records every request's steps."""

    def __init__(self, clock, cost_per_dof_step=1e-9):
        super().__init__(clock, cost_per_dof_step)
        self.outstanding = 0
        self.max_outstanding = 0
        self.steps_of = {}

    def step(self, k):
        self.outstanding += 1
        assert self.outstanding <= 2
        self.max_outstanding = max(self.max_outstanding, self.outstanding)
        for q in self.active:
            self.steps_of[q.rid] = self.steps_of.get(q.rid, 0) + k
        return super().step(k)

    def wait(self, deadline_s, token):
        self.outstanding -= 1
        return True

    def rebuild(self, reqs):
        assert self.outstanding == 0
        super().rebuild(reqs)

    def finish(self, q, keep_state=False):
        assert self.outstanding == 0
        return super().finish(q, keep_state)


def test_pipelined_steps_keep_exact_step_counts():
    # requests arriving at once under a budget that holds a few: joins and
    # leaves between steps, and a second step enqueued behind the one in
    # flight whenever the active set cannot change
    clock = serve.ManualClock()
    ex = Tracking(clock, cost_per_dof_step=1e-8)
    reqs = _reqs(10, rate=1e6)
    budget = 3 * max(q.device_bytes() for q in reqs)
    rep = serve.Server(ex, budget, clock=clock).run(reqs)
    assert sorted(o.rid for o in rep.outcomes) == sorted(q.rid for q in reqs)
    for q in reqs:
        assert ex.steps_of[q.rid] == q.nsteps, q
    assert ex.max_outstanding == 2
    assert ex.outstanding == 0
