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
