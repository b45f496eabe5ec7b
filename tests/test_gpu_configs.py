"""The workloads' own checks, through the GPU path (dg_advance, FP64):

* config 1 -- isentropic vortex, [0,10]^3, 8^3 elements, p = 3, ten
  LSERK45 steps at CFL 0.5 with seeded vortex strength, centre and drift:
  against the oracle's ten steps (each step's time step from its own state);
* config 2 downsampled -- Taylor-Green at Mach 0.1 on 16^3 elements, p = 4,
  ten steps: state, kinetic energy and the five conserved integrals against
  the oracle's, conservation to round-off;
* convergence to the exact advected isentropic vortex, p = 1..4, at the
  meshes and bar of the oracle's own convergence pin.
"""
import math

import numpy as np
import pytest

import oracle
from gpu_helpers import dev_scalar, dg_module, rel_l2, to_dev, to_host
from paper_2006_15698_gb300 import inputs

pytestmark = pytest.mark.gpu


def _oracle_run(om, Q, cfl, nsteps):
    dts, kes = [], []
    for _ in range(nsteps):
        dt, _ = om.cfl_dt(Q, cfl)
        Q, _ = om.rk_steps(Q, dt, 1)
        dts.append(dt)
        kes.append(om.norms(Q))
    return Q, np.array(dts), np.array(kes)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_config1_vortex8_p3_ten_steps(seed):
    dg = dg_module()
    import torch
    box = (0.0, 0.0, 0.0, 10.0, 10.0, 10.0)
    om = oracle.Mesh(8, 8, 8, 3, *box)
    Q0 = om.init("vortex", inputs.vortex_params(seed, box))
    Q_or, dts_or, integ_or = _oracle_run(om, Q0, 0.5, 10)
    m = dg.Mesh(8, 8, 8, 3, *box)
    Q = to_dev(Q0)
    dQ = torch.zeros_like(Q)
    dts, integ = m.advance(Q, dQ, 0.5, 10)
    dts, integ = to_host(dts), to_host(integ)
    assert dts[0] == dts_or[0]                       # same state: bitwise
    assert np.max(np.abs(dts - dts_or) / dts_or) < 1e-13
    assert rel_l2(to_host(Q), Q_or) < 1e-11          # 1e-12 per step, ten steps
    absI = om.norms(np.abs(Q0))[:5]
    assert np.max(np.abs(integ[:, :5] - integ_or[:, :5]) / absI) < 1e-13
    assert np.max(np.abs(integ[:, 5] - integ_or[:, 5]) / integ_or[:, 5]) < 1e-12
    assert m.last_error() == dg.DG_OK


def test_config2_tgv16_p4_ten_steps_invariants():
    dg = dg_module()
    import torch
    box = (0.0, 0.0, 0.0, 2 * math.pi, 2 * math.pi, 2 * math.pi)
    om = oracle.Mesh(16, 16, 16, 4, *box)
    Q0 = om.init("tgv", inputs.tgv_params(0.1))
    Q_or, dts_or, integ_or = _oracle_run(om, Q0, 0.5, 10)
    m = dg.Mesh(16, 16, 16, 4, *box)
    Q = to_dev(Q0)
    dQ = torch.zeros_like(Q)
    dts, integ = m.advance(Q, dQ, 0.5, 10)
    Qg, dts, integ = to_host(Q), to_host(dts), to_host(integ)
    assert rel_l2(Qg, Q_or) < 1e-11
    assert np.max(np.abs(dts - dts_or) / dts_or) < 1e-13
    # kinetic energy: equal to the oracle's at every step, and nearly
    # constant over these early steps of the inviscid flow
    ke, ke_or = integ[:, 5], integ_or[:, 5]
    assert np.max(np.abs(ke - ke_or) / ke_or) < 1e-12
    ke0 = om.norms(Q0)[5]
    assert np.max(np.abs(ke - ke0)) / ke0 < 1e-3
    # the five conserved integrals: constant to round-off on the periodic box
    # (against the GPU's own sum of the initial state: the oracle's sequential
    # sum over 512,000 nodes differs from it by summation order, ~4e-13)
    I0 = to_host(m.norms(to_dev(Q0)))[:5]
    absI = om.norms(np.abs(Q0))[:5]
    scale = np.maximum(absI, 1e-3 * absI.max())
    assert np.max(np.abs(integ[:, :5] - I0) / scale) < 1e-13
    assert m.last_error() == dg.DG_OK


@pytest.mark.parametrize("p,ns", [(1, (16, 32, 64)), (2, (16, 32, 64)), (3, (8, 16, 32)),
                                  (4, (8, 16, 32))])
def test_gpu_convergence_to_the_exact_vortex(p, ns):
    """Relative L2 error of the GPU solution against the exactly advected
    vortex at t = 0.5 on a 16 x 16 periodic column (the oracle's convergence
    pin, same meshes and time steps): every rate above (p + 1)/2, the finest
    pair's above p + 0.4 (the DG bound for smooth solutions is p + 1/2)."""
    dg = dg_module()
    import torch
    L = 16.0
    prm = [3.0, 7.3, 8.6, 0.6, -0.4, 0.3, 0.0]
    t_end = 0.5
    errs = []
    for n in ns:
        box = (0.0, 0.0, 0.0, L, L, L / n)  # n x n x 1 elements (the vortex is columnar)
        m = dg.Mesh(n, n, 1, p, *box)
        Q = m.init("vortex", prm)
        dQ = torch.zeros_like(Q)
        dt0 = float(to_host(m.cfl_dt(Q, 0.3))[0])
        nsteps = math.ceil(t_end / dt0)
        dt = dev_scalar(t_end / nsteps)
        for _ in range(nsteps):
            m.rk_step(Q, dQ, dt)
        exact = m.init("vortex", prm[:6] + [t_end])
        errs.append(float(to_host(m.norms(Q, exact))[6]))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(r > 0.5 * (p + 1) for r in rates), (errs, rates)
    assert rates[-1] > p + 0.4, (errs, rates)
