"""The serving loop on the GPU: every request completes under the byte budget,
and a request's result is the same bit for bit whether it ran alone or in the
mix with others (its own CFL time steps, its own tiles; the batch composition
does not enter its arithmetic)."""
import pytest

from gpu_helpers import dg_module
from paper_2006_15698_gb300 import serve

pytestmark = pytest.mark.gpu


def test_alone_equals_in_the_mix():
    dg_module()
    import torch
    reqs = serve.make_requests(5, 10, 200.0, nrange=(3, 7), prange=(1, 6), steps_range=(3, 7),
                               L=10.0)
    # all present at once; the byte budget holds about four, so the others
    # join as earlier ones leave (continuous batching, independent of timing)
    for q in reqs:
        q.arrival = 0.0
    budget = 4 * max(q.device_bytes() for q in reqs)
    mix = serve.Server(serve.GpuExecutor(), budget, keep_states=True).run(reqs)
    assert len(mix.outcomes) == len(reqs) and mix.peak_bytes <= budget
    assert mix.peak_active >= 2 and mix.rebuilds >= 3
    for q in reqs[:4] + reqs[-2:]:
        alone = serve.Server(serve.GpuExecutor(), budget, keep_states=True).run(
            [serve.Request(q.rid, 0.0, q.n, q.p, q.kind, q.nsteps, q.L, q.cfl, q.params)])
        a = alone.outcomes[0].result
        m = mix.outcomes[q.rid].result
        assert torch.equal(a["state"], m["state"]), q
        assert a["integrals"] == m["integrals"]


def test_mixed_cfl_alone_equals_in_the_mix():
    # requests with different CFL numbers share the device: each takes its own
    # time steps (one batch per CFL number), so its result is the one it gets
    # alone, bit for bit
    dg_module()
    import torch
    reqs = serve.make_requests(9, 8, 500.0, nrange=(3, 6), prange=(1, 4), steps_range=(3, 6),
                               L=10.0)
    for i, q in enumerate(reqs):
        q.cfl = (0.3, 0.5, 0.8)[i % 3]
        q.arrival = 0.0  # all present at once: every CFL group active together
    budget = 8 * max(q.device_bytes() for q in reqs)
    mix = serve.Server(serve.GpuExecutor(), budget, keep_states=True).run(reqs)
    assert len(mix.outcomes) == len(reqs) and mix.peak_active >= 3
    for q in reqs:
        alone = serve.Server(serve.GpuExecutor(), budget, keep_states=True).run(
            [serve.Request(q.rid, 0.0, q.n, q.p, q.kind, q.nsteps, q.L, q.cfl, q.params)])
        a = alone.outcomes[0].result
        m = mix.outcomes[q.rid].result
        assert torch.equal(a["state"], m["state"]), q
        assert a["integrals"] == m["integrals"]
    # the CFL number matters: the same request at another CFL ends elsewhere
    q = reqs[0]
    other = serve.Server(serve.GpuExecutor(), budget, keep_states=True).run(
        [serve.Request(q.rid, 0.0, q.n, q.p, q.kind, q.nsteps, q.L, 0.45, q.params)])
    assert not torch.equal(other.outcomes[0].result["state"], mix.outcomes[q.rid].result["state"])
