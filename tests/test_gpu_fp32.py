"""The FP32 bulk form (float state and volume/surface arithmetic, double
reductions) against the FP64 oracle after 100 RK steps, and both against the
exactly advected isentropic vortex.

Bar: relative L2 distance of the FP32 state from the FP64 oracle's state
<= 1e-5 after 100 steps; the FP32 state's error against the exact solution
stays within 1e-5 (relative) of the oracle's own discretisation error.
"""
import math

import numpy as np
import pytest

import oracle
from gpu_helpers import dev_scalar, dg_module, rel_l2, to_dev, to_host
from paper_2006_15698_gb300 import inputs

pytestmark = pytest.mark.gpu

BOX16 = (0.0, 0.0, 0.0, 16.0, 16.0, 16.0)


def _run(nel, p, steps, seed=0):
    dg = dg_module()
    import torch
    om = oracle.Mesh(*nel, p, *BOX16)
    prm = inputs.vortex_params(seed, BOX16)
    Q0 = om.init("vortex", prm)
    dt, _ = om.cfl_dt(Q0, 0.5)
    Q_or, _ = om.rk_steps(Q0, dt, steps)
    m = dg.Mesh(*nel, p, *BOX16, precision=dg.DG_FP32)
    Q = to_dev(Q0, torch.float32)
    dQ = torch.empty_like(Q)
    dtd = dev_scalar(dt)
    for _ in range(steps):
        m.rk_step(Q, dQ, dtd)
    Q32 = to_host(Q)
    pe = list(prm)
    pe[6] = dt * steps
    Q_ex = om.init("vortex", pe)
    assert m.last_error() == dg.DG_OK
    return Q32, Q_or, Q_ex


@pytest.mark.parametrize("nel,p", [((8, 8, 8), 3), ((32, 32, 32), 3)])
def test_fp32_100_steps_vs_fp64_oracle_and_exact(nel, p):
    Q32, Q_or, Q_ex = _run(nel, p, 100)
    err_or = rel_l2(Q32, Q_or)
    assert err_or < 1e-5, err_or
    e32 = rel_l2(Q32, Q_ex)
    e64 = rel_l2(Q_or, Q_ex)
    assert abs(e32 - e64) < 1e-5, (e32, e64)
    print(f"FP32 vs FP64 oracle after 100 steps: {err_or:.3e}; vs exact: FP32 {e32:.3e}, FP64 {e64:.3e}")


@pytest.mark.parametrize("p", [1, 4, 6])
def test_fp32_step_and_dt(p):
    # one step from the float-rounded state, and the double-precision time
    # step of the float state, against the oracle on the same rounded input
    dg = dg_module()
    import torch
    om = oracle.Mesh(5, 4, 3, p, *BOX16)
    Q0 = om.init("vortex", inputs.vortex_params(3, BOX16)).astype(np.float32).astype(np.float64)
    dt, _ = om.cfl_dt(Q0, 0.5)
    m = dg.Mesh(5, 4, 3, p, *BOX16, precision=dg.DG_FP32)
    Q = to_dev(Q0, torch.float32)
    assert abs(float(to_host(m.cfl_dt(Q, 0.5))[0]) - dt) <= 1e-6 * dt
    dQ = torch.empty_like(Q)
    m.rk_step(Q, dQ, dev_scalar(dt))
    Q1, _ = om.rk_steps(Q0, dt, 1)
    assert rel_l2(to_host(Q), Q1) < 2e-7
    # integrals of the float state accumulate in double; the five conserved
    # fields' integrands are exact in double, the kinetic-energy density is
    # evaluated in float (the state's precision)
    out = to_host(m.norms(Q))
    ref = om.norms(to_host(Q))
    assert np.max(np.abs(out[:5] - ref[:5]) / np.maximum(np.abs(ref[:5]), 1)) < 1e-13
    assert abs(out[5] - ref[5]) < 1e-6 * abs(ref[5])


# meshes for the column stage kernel: many z chunks per column (short columns
# against the GPU's resident CTA count), ragged cross-sections, nz = 1 and 2
# (the layer above/below is the layer itself or its only neighbour), and a
# single column (the neighbour column is the column itself)
COLUMN_MESHES = [((5, 7, 24), 3), ((3, 2, 1), 2), ((1, 1, 5), 4), ((4, 3, 2), 1),
                 ((2, 3, 9), 5), ((2, 1, 3), 6), ((6, 5, 4), 0)]


@pytest.mark.parametrize("nel,p", COLUMN_MESHES)
def test_column_kernel_rhs_and_step(nel, p):
    """The column stage kernel against the oracle (float tolerance) and
    against the tile kernel (same arithmetic up to float rounding order)."""
    dg = dg_module()
    import torch
    from gpu_helpers import rhs_scale
    om = oracle.Mesh(*nel, p, *BOX16)
    prm = inputs.vortex_params(7 + p, BOX16)
    prm[0] = 1.0 + 0.25 * (prm[0] - 1.0)
    Q0 = om.init("vortex", prm).astype(np.float32).astype(np.float64)
    R_or = om.rhs(Q0)
    saved = dg.dg_get_stage_kernel(p)
    try:
        out = {}
        for kind in (dg.DG_STAGE_COLUMN, dg.DG_STAGE_TILE):
            dg.dg_set_stage_kernel(p, kind)
            m = dg.Mesh(*nel, p, *BOX16, precision=dg.DG_FP32)
            R = to_host(m.rhs(to_dev(Q0, torch.float32)))
            assert np.linalg.norm(R - R_or) / rhs_scale(om, Q0) < 2e-6, kind
            Q = to_dev(Q0, torch.float32)
            dQ = torch.zeros_like(Q)
            dt = m.cfl_dt(Q, 0.5)
            m.rk_step(Q, dQ, dt)
            out[kind] = (R, to_host(Q))
        dtv = float(om.cfl_dt(Q0, 0.5)[0])
        Q1, _ = om.rk_steps(Q0, dtv, 1)
        for kind, (R, Q) in out.items():
            assert rel_l2(Q, Q1) < 2e-7, kind
        assert rel_l2(out[dg.DG_STAGE_COLUMN][1], out[dg.DG_STAGE_TILE][1]) < 2e-7
    finally:
        dg.dg_set_stage_kernel(p, saved)



@pytest.mark.parametrize("nel,p", COLUMN_MESHES + [((9, 10, 7), 3), ((17, 5, 6), 2), ((3, 5, 11), 4)])
def test_line_kernel_equals_column_kernel(nel, p):
    """The column kernel with one thread per z node line performs the same
    float operations in the same order as the one with one thread per node:
    the right-hand side, one LSERK45 step and three steps of dg_advance
    (dQ-only fifth stage, step epilogue, time steps and integrals) agree
    bitwise; the right-hand side also against the oracle."""
    dg = dg_module()
    import torch
    from gpu_helpers import rhs_scale
    om = oracle.Mesh(*nel, p, *BOX16)
    prm = inputs.vortex_params(11 + p, BOX16)
    prm[0] = 1.0 + 0.25 * (prm[0] - 1.0)
    Q0 = om.init("vortex", prm).astype(np.float32).astype(np.float64)
    R_or = om.rhs(Q0)
    saved = dg.dg_get_stage_kernel(p)
    try:
        out = {}
        for kind in (dg.DG_STAGE_COLUMN, dg.DG_STAGE_LINES):
            dg.dg_set_stage_kernel(p, kind)
            m = dg.Mesh(*nel, p, *BOX16, precision=dg.DG_FP32)
            R = to_host(m.rhs(to_dev(Q0, torch.float32)))
            assert np.linalg.norm(R - R_or) / rhs_scale(om, Q0) < 2e-6, kind
            Q = to_dev(Q0, torch.float32)
            dQ = torch.zeros_like(Q)
            dt = m.cfl_dt(Q, 0.5)
            m.rk_step(Q, dQ, dt)
            Q1 = to_host(Q)
            dQ.zero_()
            dts, integ = m.advance(Q, dQ, 0.5, 3)
            torch.cuda.synchronize()
            assert m.last_error() == dg.DG_OK
            out[kind] = (R, Q1, to_host(Q), dts.cpu().numpy(), integ.cpu().numpy())
        for a, b in zip(out[dg.DG_STAGE_COLUMN], out[dg.DG_STAGE_LINES]):
            assert np.array_equal(a, b)
    finally:
        dg.dg_set_stage_kernel(p, saved)
