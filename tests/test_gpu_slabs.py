"""z slabs on the GPU: a periodic mesh split into slabs on one device, each a
library mesh whose z boundary reads face traces from halo buffers
(dg_mesh_set_zhalo), refreshed from the neighbours' dg_zhalo_traces before
every stage (dg_rk_stage) -- the paper's partitioned mesh (Sec. III, Sec. IV)
with the exchange as device copies.

* five dg_rk_stage calls are one dg_rk_step, bit for bit (both precisions);
* each slab's right-hand side equals the undivided mesh's on its layers, bit
  for bit (double form and both float column kernels), and the oracle's;
* LSERK45 steps of the slabs (slabs.SlabSolver) equal the undivided mesh's
  steps bit for bit, time steps included;
* calls that cannot honour a slab's halos are refused.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import dg_module, rhs_scale, to_dev, to_host
from paper_2006_15698_gb300 import inputs

pytestmark = pytest.mark.gpu

BOX = (0.0, 0.0, 0.0, 10.0, 10.0, 10.0)


def _state(nel, p, seed, dtype):
    import torch
    om = oracle.Mesh(*nel, p, *BOX)
    prm = inputs.vortex_params(seed, BOX)
    prm[0] = 1.0 + 0.25 * (prm[0] - 1.0)
    Q0 = om.init("vortex", prm)
    if dtype == torch.float32:
        Q0 = Q0.astype(np.float32).astype(np.float64)
    return om, Q0


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("p", [1, 4])
def test_five_stages_are_one_step(prec, p):
    dg = dg_module()
    import torch
    precision = dg.DG_FP64 if prec == "fp64" else dg.DG_FP32
    dtype = torch.float64 if prec == "fp64" else torch.float32
    nel = (4, 3, 5)
    om, Q0 = _state(nel, p, 1, dtype)
    m = dg.Mesh(*nel, p, *BOX, precision=precision)
    Q = to_dev(Q0, dtype)
    dQ = torch.zeros_like(Q)
    dt = m.cfl_dt(Q, 0.5)
    m.rk_step(Q, dQ, dt)
    Qs, dQs = to_dev(Q0, dtype), torch.zeros_like(Q)
    other = torch.empty_like(Qs)
    for s in range(5):
        if prec == "fp64":
            m.rk_stage(Qs, Qs, dQs, dt, s)
        else:
            m.rk_stage(Qs, other, dQs, dt, s)
            Qs, other = other, Qs
    torch.cuda.synchronize()
    assert torch.equal(Qs, Q) and torch.equal(dQs, dQ)


def _slab_meshes(dg, nel, p, precision, Q, ranges):
    from paper_2006_15698_gb300 import slabs
    out = []
    for zb, nzs in ranges:
        bx = slabs.slab_box(BOX, nel[2], zb, nzs)
        out.append(slabs.GpuSlab((nel[0], nel[1], nzs), p, bx, precision,
                                 Q=slabs.slab_of(Q, nel, zb, nzs).contiguous()))
    return out


CASES = [((4, 3, 7), 0, (3, 4)), ((3, 5, 6), 1, (2, 2, 2)), ((5, 4, 5), 3, (1, 4)),
         ((3, 2, 4), 4, (2, 2)), ((2, 3, 3), 6, (1, 1, 1)), ((6, 5, 9), 2, (4, 5))]


@pytest.mark.parametrize("prec", ["fp64", "lines", "column"])
@pytest.mark.parametrize("nel,p,splits", CASES)
def test_slab_rhs_equals_undivided(prec, nel, p, splits):
    dg = dg_module()
    import torch
    from paper_2006_15698_gb300 import slabs
    precision = dg.DG_FP64 if prec == "fp64" else dg.DG_FP32
    dtype = torch.float64 if prec == "fp64" else torch.float32
    saved = dg.dg_get_stage_kernel(p)
    try:
        if prec != "fp64":
            dg.dg_set_stage_kernel(p, dg.STAGE_KINDS[prec])
        om, Q0 = _state(nel, p, 2 + p, dtype)
        Q = to_dev(Q0, dtype)
        R = dg.Mesh(*nel, p, *BOX, precision=precision).rhs(Q)
        ranges, z = [], 0
        for n in splits:
            ranges.append((z, n))
            z += n
        parts = _slab_meshes(dg, nel, p, precision, Q, ranges)
        sends = [s.traces() for s in parts]
        K = len(parts)
        for k, s in enumerate(parts):
            s.halos[0].copy_(sends[(k - 1) % K][1])
            s.halos[1].copy_(sends[(k + 1) % K][0])
        for (zb, nzs), s in zip(ranges, parts):
            Rs = s.mesh.rhs(s.Q)
            assert torch.equal(Rs, slabs.slab_of(R, nel, zb, nzs)), (zb, nzs)
        # and the oracle's right-hand side (the precision's tolerance)
        Rall = torch.cat([s.mesh.rhs(s.Q) for s in parts], dim=1)
        tol = 1e-12 if prec == "fp64" else 2e-6
        assert np.linalg.norm(to_host(Rall) - om.rhs(Q0)) / rhs_scale(om, Q0) < tol
    finally:
        dg.dg_set_stage_kernel(p, saved)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("nel,p,nslab", [((4, 3, 8), 3, 2), ((3, 4, 7), 4, 3), ((5, 2, 4), 1, 4)])
def test_slab_steps_equal_undivided(prec, nel, p, nslab):
    dg = dg_module()
    import torch
    from paper_2006_15698_gb300 import slabs
    precision = dg.DG_FP64 if prec == "fp64" else dg.DG_FP32
    dtype = torch.float64 if prec == "fp64" else torch.float32
    om, Q0 = _state(nel, p, 5, dtype)
    m = dg.Mesh(*nel, p, *BOX, precision=precision)
    Q = to_dev(Q0, dtype)
    dQ = torch.zeros_like(Q)
    ranges = slabs.split_layers(nel[2], nslab)
    solver = slabs.SlabSolver(_slab_meshes(dg, nel, p, precision, Q, ranges))
    for _ in range(3):
        dt = m.cfl_dt(Q, 0.5)
        m.rk_step(Q, dQ, dt)
        dts = solver.step(0.5)
        torch.cuda.synchronize()
        assert torch.equal(dts, dt)
    for (zb, nzs), s in zip(ranges, solver.slabs):
        assert torch.equal(s.Q, slabs.slab_of(Q, nel, zb, nzs))
        assert s.mesh.last_error() == dg.DG_OK
    I = to_host(solver.integrals())
    I_ref = to_host(m.norms(Q))[:6]
    assert np.max(np.abs(I - I_ref) / np.maximum(np.abs(I_ref), 1.0)) < 1e-13


def test_slab_calls_refused():
    dg = dg_module()
    import torch
    nel, p = (3, 3, 4), 2
    m = dg.Mesh(*nel, p, *BOX)
    lo, hi = m.empty_halo(), m.empty_halo()
    m.set_zhalo(lo, hi)
    Q = m.init("uniform", [1.0, 0.1, 0.2, 0.3, 1.0])
    dQ = torch.zeros_like(Q)
    dt = m.cfl_dt(Q, 0.5)
    for call in (lambda: m.rk_step(Q, dQ, dt), lambda: m.advance(Q, dQ, 0.5, 1)):
        with pytest.raises(dg.DGError) as e:
            call()
        assert e.value.status == dg.DG_ERR_UNSUPPORTED
    with pytest.raises(dg.DGError) as e:
        dg.dg_mesh_set_zhalo(m.h, lo, None)
    assert e.value.status == dg.DG_ERR_ARG
    m.set_zhalo(None, None)  # periodic again
    m.rk_step(Q, dQ, dt)
    # the float tile kernel does not read halos
    saved = dg.dg_get_stage_kernel(p)
    try:
        dg.dg_set_stage_kernel(p, dg.DG_STAGE_TILE)
        mf = dg.Mesh(*nel, p, *BOX, precision=dg.DG_FP32)
        with pytest.raises(dg.DGError) as e:
            mf.set_zhalo(mf.empty_halo(), mf.empty_halo())
        assert e.value.status == dg.DG_ERR_UNSUPPORTED
    finally:
        dg.dg_set_stage_kernel(p, saved)
    torch.cuda.synchronize()
