"""dg_advance: nsteps of (time step, LSERK45 step, integrals) in one call
equal the separate dg_cfl_dt / dg_rk_step / dg_norms calls bit for bit --
time steps, states and the integrals (and the RK register in the double
form; the float form leaves it as scratch) -- for both precisions, the three
float stage kernels, ragged meshes, odd and even step counts and the
degenerate one-step call."""
import math

import numpy as np
import pytest

import oracle
from gpu_helpers import dg_module, to_dev
from paper_2006_15698_gb300 import inputs

pytestmark = pytest.mark.gpu

BOX = (0.0, 0.0, 0.0, 10.0, 10.0, 10.0)


def _state(om, seed):
    prm = inputs.vortex_params(seed, BOX)
    prm[0] = 1.0 + 0.25 * (prm[0] - 1.0)
    return om.init("vortex", prm)


def _separate(m, Q, dQ, cfl, n):
    import torch
    dts, integ = [], []
    for _ in range(n):
        dt = m.cfl_dt(Q, cfl)
        m.rk_step(Q, dQ, dt)
        dts.append(dt.clone())
        integ.append(m.norms(Q).clone())
    return torch.cat(dts), torch.stack(integ)


CASES = [("fp64", 2, (5, 3, 2), None), ("fp64", 4, (3, 3, 3), None), ("fp64", 0, (4, 1, 3), None),
         ("fp32", 3, (5, 7, 6), "column"), ("fp32", 3, (5, 7, 6), "tile"),
         ("fp32", 1, (4, 3, 5), "tile"), ("fp32", 5, (2, 3, 4), "column"),
         ("fp32", 6, (1, 2, 3), "tile"), ("fp32", 3, (5, 7, 6), "lines"),
         ("fp32", 2, (9, 4, 3), "lines"), ("fp32", 6, (3, 1, 4), "lines")]


@pytest.mark.parametrize("prec,p,nel,kernel", CASES)
def test_advance_equals_separate_calls(prec, p, nel, kernel):
    dg = dg_module()
    import torch
    fp = dg.DG_FP64 if prec == "fp64" else dg.DG_FP32
    dtype = torch.float64 if prec == "fp64" else torch.float32
    saved = dg.dg_get_stage_kernel(p)
    try:
        if kernel:
            dg.dg_set_stage_kernel(p, dg.STAGE_KINDS[kernel])
        om = oracle.Mesh(*nel, p, *BOX)
        Q0 = to_dev(_state(om, 5 + p), dtype)
        m = dg.Mesh(*nel, p, *BOX, precision=fp)
        Qa, dQa = Q0.clone(), torch.zeros_like(Q0)
        dts_a, integ_a = _separate(m, Qa, dQa, 0.5, 3)
        Qb, dQb = Q0.clone(), torch.zeros_like(Q0)
        dts_b, integ_b = m.advance(Qb, dQb, 0.5, 3)
        torch.cuda.synchronize()
        assert torch.equal(dts_a, dts_b)
        assert torch.equal(Qa, Qb)
        if prec == "fp64":
            # the float form's fifth stage writes only the new state: dQ is
            # scratch on return
            assert torch.equal(dQa, dQb)
        assert torch.equal(integ_a, integ_b)
        assert m.last_error() == dg.DG_OK
        # an even number of steps (the float form's result lands in Q
        # without the final copy)
        Qe, dQe = Q0.clone(), torch.zeros_like(Q0)
        dts_e, integ_e = m.advance(Qe, dQe, 0.5, 2)
        Qf, dQf = Q0.clone(), torch.zeros_like(Q0)
        dts_f, integ_f = _separate(m, Qf, dQf, 0.5, 2)
        assert torch.equal(dts_e, dts_f) and torch.equal(Qe, Qf) and torch.equal(integ_e, integ_f)
        # one step, no integrals requested
        Qc, dQc = Q0.clone(), torch.zeros_like(Q0)
        dts_c, integ_c = m.advance(Qc, dQc, 0.5, 1, with_integrals=False)
        assert integ_c is None
        Qd, dQd = Q0.clone(), torch.zeros_like(Q0)
        dts_d, _ = _separate(m, Qd, dQd, 0.5, 1)
        assert torch.equal(dts_c, dts_d) and torch.equal(Qc, Qd)
    finally:
        dg.dg_set_stage_kernel(p, saved)


def test_advance_flags_nonpositive_pressure_and_rejects_bad_arguments():
    dg = dg_module()
    import torch
    om = oracle.Mesh(3, 2, 2, 2, *BOX)
    Q = _state(om, 1)
    m = dg.Mesh(3, 2, 2, 2, *BOX)
    Qd = to_dev(Q)
    dQ = torch.zeros_like(Qd)
    with pytest.raises(dg.DGError):
        m.advance(Qd, dQ, 0.5, 0)
    with pytest.raises(dg.DGError):
        m.advance(Qd, dQ, -1.0, 2)
    with pytest.raises(dg.DGError):
        m.advance(Qd, Qd, 0.5, 2)
    bad = Q.copy()
    bad[4, 7, 1, 2, 0] = 0.0  # rho E = 0 -> p < 0 at one node (host-side corruption)
    dts, _ = m.advance(to_dev(bad), dQ, 0.5, 1)
    assert math.isnan(float(dts[0].item()))
    assert m.last_error() == dg.DG_ERR_NONFINITE


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_mesh_create_reports_oom_and_the_context_stays_usable(prec):
    """A mesh whose workspace cannot be allocated (10^9 elements at p = 3:
    1.3 TB of float or 1.9 TB of double workspace, beyond any one GPU) is
    refused with DG_ERR_OOM; the failed allocation leaves nothing behind, and
    the next mesh steps as usual (host-side failure, no device fault)."""
    dg = dg_module()
    import torch
    precision = dg.DG_FP64 if prec == "fp64" else dg.DG_FP32
    with pytest.raises(dg.DGError) as ei:
        dg.Mesh(1000, 1000, 1000, 3, precision=precision)
    assert ei.value.status == dg.DG_ERR_OOM
    om = oracle.Mesh(3, 2, 2, 2, *BOX)
    Q = _state(om, 1)
    m = dg.Mesh(3, 2, 2, 2, *BOX, precision=precision)
    Qd = to_dev(Q).to(m.dtype)
    dQ = torch.zeros_like(Qd)
    dts, integ = m.advance(Qd, dQ, 0.5, 2)
    assert torch.isfinite(dts).all() and torch.isfinite(Qd).all()
    assert m.last_error() == dg.DG_OK
