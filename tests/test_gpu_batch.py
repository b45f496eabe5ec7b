"""Tile variants of the float form's fused stage, and batches of independent
float meshes (the shared instances: one launch per RK stage and degree of the
line kernel over work items (instance, column, z chunk); the others on own
launches on the batch's streams; optional CUDA graph).  The batch tests run
with every instance shared, with the default split and with every instance
on its own launches (dg_set_batch_direct_nodes).  (The tests that compare a
single mesh with a batch bitwise select the line kernel for it, which the
shared launches run.)

* every tile variant of every degree gives the oracle's right-hand side
  (FP32 tolerance), also on meshes that tiles cover raggedly;
* an instance advanced inside a batch equals the same instance advanced
  alone, bitwise (the same line-kernel body, the same arithmetic), and its
  time step equals dg_cfl_dt's;
* graph-replayed steps equal directly launched steps bitwise.
"""
import math

import numpy as np
import pytest

import oracle
from gpu_helpers import dg_module, rhs_scale, to_dev, to_host
from paper_2006_15698_gb300 import inputs

pytestmark = pytest.mark.gpu

BOX = (0.0, 0.0, 0.0, 10.0, 10.0, 10.0)


@pytest.fixture
def dgm():
    dg = dg_module()
    saved = {p: (dg.dg_get_tile_variant(p), dg.dg_get_stage_kernel(p)) for p in range(0, 7)}
    direct = dg.dg_get_batch_direct_nodes()
    yield dg
    for p, (v, k) in saved.items():
        dg.dg_set_tile_variant(p, v)
        dg.dg_set_stage_kernel(p, k)
    dg.dg_set_batch_direct_nodes(direct)


DIRECT = ["never", "default", "all"]


def _set_direct(dg, mode):
    if mode == "never":
        dg.dg_set_batch_direct_nodes(dg.BATCH_NEVER_DIRECT)
    elif mode == "all":
        dg.dg_set_batch_direct_nodes(0)


@pytest.mark.parametrize("p", range(0, 7))
def test_every_tile_variant_matches_oracle(dgm, p):
    dg = dgm
    import torch
    nel = (5, 7, 3)  # ragged against every tile shape
    om = oracle.Mesh(*nel, p, *BOX)
    prm = inputs.vortex_params(p, BOX)
    prm[0] = 1.0 + 0.25 * (prm[0] - 1.0)
    Q = om.init("vortex", prm).astype(np.float32).astype(np.float64)
    R_or = om.rhs(Q)
    dg.dg_set_stage_kernel(p, dg.DG_STAGE_TILE)
    for v in range(dg.dg_tile_variant_count(p)):
        dg.dg_set_tile_variant(p, v)
        m = dg.Mesh(*nel, p, *BOX, precision=dg.DG_FP32)
        R = to_host(m.rhs(to_dev(Q, torch.float32)))
        err = np.linalg.norm(R - R_or) / rhs_scale(om, Q)
        assert err < 2e-6, (v, dg.dg_tile_shape(p, v), err)


def _specs(seed, n):
    r = inputs.uniforms(seed, 2 * n)
    specs = []
    for i in range(n):
        ne = 3 + int(r[2 * i] * 6)      # 3..8 elements per side
        p = 1 + int(r[2 * i + 1] * 5)   # 1..5
        specs.append(dict(nx=ne, ny=ne + 1, nz=ne, p=p, Lx=10.0, Ly=10.0, Lz=10.0))
    return specs


@pytest.mark.parametrize("direct", DIRECT)
@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_matches_single_meshes(dgm, use_graph, direct):
    dg = dgm
    import torch
    _set_direct(dg, direct)
    for p in range(0, 7):  # single meshes on the batch's line kernel: bitwise comparable
        dg.dg_set_stage_kernel(p, dg.DG_STAGE_LINES)
    specs = _specs(11, 7)
    batch = dg.Batch(specs)
    for i, s in enumerate(specs):
        batch.init(i, "vortex", inputs.vortex_params(100 + i, BOX))
    singles = []
    for i, s in enumerate(specs):
        m = dg.Mesh(s["nx"], s["ny"], s["nz"], s["p"], *BOX, precision=dg.DG_FP32)
        Q = batch.Q[i].clone()
        singles.append((m, Q, torch.zeros_like(Q), torch.zeros(1, dtype=torch.float64, device="cuda")))
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for step in range(3):
            batch.step(0.5, use_graph=use_graph)
            for m, Q, dQ, dt in singles:
                m.cfl_dt(Q, 0.5, dt)
                m.rk_step(Q, dQ, dt)
    torch.cuda.synchronize()
    dts = batch.dts()
    for i, (m, Q, dQ, dt) in enumerate(singles):
        assert dts[i] == float(dt.item()), i
        assert torch.equal(batch.Q[i], Q), (i, specs[i])
    assert batch.last_error() == dg.DG_OK


def test_batch_instance_against_oracle(dgm):
    # one instance of a mixed batch after one step, against the FP64 oracle
    dg = dgm
    import torch
    specs = [dict(nx=4, ny=3, nz=2, p=3, Lx=10.0, Ly=10.0, Lz=10.0),
             dict(nx=5, ny=5, nz=5, p=1, Lx=10.0, Ly=10.0, Lz=10.0)]
    om = oracle.Mesh(4, 3, 2, 3, *BOX)
    Q0 = om.init("vortex", inputs.vortex_params(8, BOX)).astype(np.float32).astype(np.float64)
    batch = dg.Batch(specs)
    batch.Q[0].copy_(to_dev(Q0, torch.float32))
    batch.init(1, "tgv", inputs.tgv_params(0.1))
    batch.step(0.5, use_graph=False)
    dt = batch.dts()[0]
    Q1, _ = om.rk_steps(Q0, dt, 1)
    err = np.linalg.norm(to_host(batch.Q[0]) - Q1) / np.linalg.norm(Q1)
    assert err < 2e-7, err
    out = to_host(batch.norms(0))
    assert abs(out[0] - om.norms(Q1)[0]) < 1e-6 * abs(out[0])


@pytest.mark.parametrize("direct", DIRECT)
def test_batch_graph_equals_direct(dgm, direct):
    dg = dgm
    import torch
    _set_direct(dg, direct)
    specs = _specs(5, 5)
    a, b = dg.Batch(specs), dg.Batch(specs)
    for i in range(len(specs)):
        a.init(i, "vortex", inputs.vortex_params(i, BOX))
        b.init(i, "vortex", inputs.vortex_params(i, BOX))
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for _ in range(4):
            a.step(0.4, use_graph=True)
            b.step(0.4, use_graph=False)
    torch.cuda.synchronize()
    for i in range(len(specs)):
        assert torch.equal(a.Q[i], b.Q[i])


@pytest.mark.parametrize("direct", DIRECT)
@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_multi_step_call(dgm, use_graph, direct):
    # nsteps in one call (two-step groups ending in Q without a copy, then a
    # last single step with the copy) equals nsteps single-step calls
    dg = dgm
    import torch
    _set_direct(dg, direct)
    specs = _specs(7, 4)
    a, b = dg.Batch(specs), dg.Batch(specs)
    for i in range(len(specs)):
        a.init(i, "vortex", inputs.vortex_params(50 + i, BOX))
        b.init(i, "vortex", inputs.vortex_params(50 + i, BOX))
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        a.step(0.5, nsteps=5, use_graph=use_graph)
        for _ in range(5):
            b.step(0.5, nsteps=1, use_graph=use_graph)
    torch.cuda.synchronize()
    assert a.dts() == b.dts()
    for i in range(len(specs)):
        assert torch.equal(a.Q[i], b.Q[i])


def test_batch_rejects_bad_specs(dgm):
    dg = dgm
    with pytest.raises(dg.DGError):
        dg.Batch([dict(nx=2, ny=2, nz=2, p=7)])
    with pytest.raises(dg.DGError):
        dg.Batch([dict(nx=0, ny=2, nz=2, p=1)])


@pytest.mark.parametrize("kernel", ["column", "lines", "tile"])
def test_hybrid_batch_large_instances_match_single_meshes(dgm, kernel):
    """Instances of at least 2^19 nodes run the single-mesh stage kernels as
    launches of their own inside the batch's step (and graph); each still
    equals the same mesh stepped alone, bit for bit, next to small instances
    that share the persistent launch."""
    dg = dgm
    import torch
    # the large instances' degrees (3, 4) run the kernel under test; the small
    # instances (degrees 2, 5) share the batched line-kernel launches, so their
    # single meshes use the line kernel
    dg.dg_set_batch_direct_nodes(1 << 19)
    for p in range(0, 7):
        big = p in (3, 4)
        dg.dg_set_stage_kernel(p, dg.STAGE_KINDS[kernel] if big else dg.DG_STAGE_LINES)
    specs = [dict(nx=24, ny=24, nz=24, p=3, Lx=10.0, Ly=10.0, Lz=10.0),   # 884,736 nodes: own launches
             dict(nx=5, ny=6, nz=5, p=2, Lx=10.0, Ly=10.0, Lz=10.0),
             dict(nx=12, ny=10, nz=9, p=5, Lx=10.0, Ly=10.0, Lz=10.0),    # 233,280 nodes: shared
             dict(nx=20, ny=20, nz=12, p=4, Lx=10.0, Ly=10.0, Lz=10.0)]   # 600,000 nodes: own launches
    batch = dg.Batch(specs)
    for i in range(len(specs)):
        batch.init(i, "vortex", inputs.vortex_params(200 + i, BOX))
    singles = []
    for i, sp in enumerate(specs):
        m = dg.Mesh(sp["nx"], sp["ny"], sp["nz"], sp["p"], *BOX, precision=dg.DG_FP32)
        Q = batch.Q[i].clone()
        singles.append((m, Q, torch.zeros_like(Q), torch.zeros(1, dtype=torch.float64, device="cuda")))
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for use_graph in (False, True, True):
            batch.step(0.5, use_graph=use_graph)
            for m, Q, dQ, dt in singles:
                m.cfl_dt(Q, 0.5, dt)
                m.rk_step(Q, dQ, dt)
    torch.cuda.synchronize()
    dts = batch.dts()
    for i, (m, Q, dQ, dt) in enumerate(singles):
        assert dts[i] == float(dt.item()), i
        assert torch.equal(batch.Q[i], Q), (i, specs[i])
    assert batch.last_error() == dg.DG_OK


@pytest.mark.parametrize("use_graph", [False, True])
def test_shared_launch_every_degree_matches_single_meshes(dgm, use_graph):
    # every instance in the shared line-kernel launches, degrees 0..6 (ragged
    # columns, z chunks), each equal to the same mesh stepped alone
    dg = dgm
    import torch
    dg.dg_set_batch_direct_nodes(dg.BATCH_NEVER_DIRECT)
    for p in range(0, 7):
        dg.dg_set_stage_kernel(p, dg.DG_STAGE_LINES)
    specs = [dict(nx=5, ny=4, nz=19, p=0, Lx=10.0, Ly=10.0, Lz=10.0),
             dict(nx=9, ny=3, nz=2, p=1, Lx=10.0, Ly=10.0, Lz=10.0),
             dict(nx=4, ny=5, nz=9, p=2, Lx=10.0, Ly=10.0, Lz=10.0),
             dict(nx=3, ny=5, nz=17, p=3, Lx=10.0, Ly=10.0, Lz=10.0),
             dict(nx=3, ny=2, nz=3, p=4, Lx=10.0, Ly=10.0, Lz=10.0),
             dict(nx=4, ny=1, nz=10, p=5, Lx=10.0, Ly=10.0, Lz=10.0),
             dict(nx=3, ny=2, nz=1, p=6, Lx=10.0, Ly=10.0, Lz=10.0)]
    batch = dg.Batch(specs)
    assert batch.n_items > 0
    for i in range(len(specs)):
        batch.init(i, "vortex", inputs.vortex_params(300 + i, BOX))
    singles = []
    for i, sp in enumerate(specs):
        m = dg.Mesh(sp["nx"], sp["ny"], sp["nz"], sp["p"], *BOX, precision=dg.DG_FP32)
        Q = batch.Q[i].clone()
        singles.append((m, Q, torch.zeros_like(Q), torch.zeros(1, dtype=torch.float64, device="cuda")))
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        batch.step(0.5, nsteps=3, use_graph=use_graph)
        for _ in range(3):
            for m, Q, dQ, dt in singles:
                m.cfl_dt(Q, 0.5, dt)
                m.rk_step(Q, dQ, dt)
    torch.cuda.synchronize()
    dts = batch.dts()
    for i, (m, Q, dQ, dt) in enumerate(singles):
        assert dts[i] == float(dt.item()), i
        assert torch.equal(batch.Q[i], Q), (i, specs[i])
    assert batch.last_error() == dg.DG_OK


@pytest.mark.parametrize("direct", ["never", "default"])
def test_batch_update_equals_single_meshes(dgm, direct):
    """dg_batch_update replaces the instance list in place (requests joining
    and leaving): after updates that shrink, grow (beyond the batch's array
    capacities) and reorder the list, every instance still steps exactly as
    the same mesh alone."""
    dg = dgm
    import torch
    _set_direct(dg, direct)
    for p in range(0, 7):
        dg.dg_set_stage_kernel(p, dg.DG_STAGE_LINES)
    pool = _specs(21, 9) + [dict(nx=12, ny=10, nz=9, p=5, Lx=10.0, Ly=10.0, Lz=10.0)]
    tensors = []
    for i, sp in enumerate(pool):
        N = sp["p"] + 1
        shape = (5, sp["nx"] * sp["ny"] * sp["nz"], N, N, N)
        tensors.append(dict(Q=torch.empty(shape, dtype=torch.float32, device="cuda"),
                            dQ=torch.zeros(shape, dtype=torch.float32, device="cuda"),
                            Qt=torch.empty(shape, dtype=torch.float32, device="cuda")))
    singles = []
    for i, sp in enumerate(pool):
        m = dg.Mesh(sp["nx"], sp["ny"], sp["nz"], sp["p"], *BOX, precision=dg.DG_FP32)
        Q = m.init("vortex", inputs.vortex_params(400 + i, BOX))
        tensors[i]["Q"].copy_(Q)
        singles.append((m, Q, torch.zeros_like(Q), torch.zeros(1, dtype=torch.float64, device="cuda")))
    lists = [[0, 1, 2], [2, 0], [3, 9, 4, 5, 6, 7, 8, 1], [8, 2]]
    stream = torch.cuda.Stream()
    batch = None
    for members in lists:
        specs = [dict(pool[i], **tensors[i]) for i in members]
        if batch is None:
            batch = dg.Batch(specs)
        else:
            batch.update(specs)
        with torch.cuda.stream(stream):
            batch.step(0.5, nsteps=2, use_graph=True)
            for i in members:
                m, Q, dQ, dt = singles[i]
                for _ in range(2):
                    m.cfl_dt(Q, 0.5, dt)
                    m.rk_step(Q, dQ, dt)
        torch.cuda.synchronize()
        dts = batch.dts()
        for k, i in enumerate(members):
            assert dts[k] == float(singles[i][3].item()), (members, i)
            assert torch.equal(tensors[i]["Q"], singles[i][1]), (members, i)
    assert batch.last_error() == dg.DG_OK
