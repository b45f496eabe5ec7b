"""Parity at the full size of the bench workloads (Taylor-Green vortex,
64^3 elements, p = 4, FP64; isentropic vortex, 128^3 elements, p = 3, FP32),
in the launch configuration bench.py times (dg_advance).

The oracle cannot evaluate the whole mesh quickly, so the right-hand side is
compared on a sample of elements (including every kind of periodic wrap),
the time step bitwise on the whole mesh, and one full RK step through the
properties that hold at any size (discrete conservation of the five
integrals; agreement of the step's change with dt * rhs to first order).
"""
import math

import numpy as np
import pytest

import oracle
from gpu_helpers import dev_scalar, dg_module, to_dev, to_host
from paper_2006_15698_gb300 import inputs

pytestmark = pytest.mark.gpu

NEL = (64, 64, 64)
P = 4
BOX = (0.0, 0.0, 0.0, 2 * math.pi, 2 * math.pi, 2 * math.pi)


@pytest.fixture(scope="module")
def full():
    dg = dg_module()
    om = oracle.Mesh(*NEL, P, *BOX)
    Q = om.init("tgv", inputs.tgv_params(0.1))
    m = dg.Mesh(*NEL, P, *BOX)
    return dg, om, m, Q


def _sample(E, nx, ny, nz, k=160, seed=3):
    rng = np.random.Generator(np.random.PCG64(seed))
    corners = [ex + nx * (ey + ny * ez) for ex in (0, nx - 1) for ey in (0, ny - 1) for ez in (0, nz - 1)]
    return np.unique(np.concatenate([corners, rng.integers(0, E, k)]))


def test_rhs_sampled_elements(full):
    dg, om, m, Q = full
    # a perturbed Taylor-Green state, so that every term of the rhs is active
    Qp = Q * (1 + 0.01 * inputs.random_state(Q.shape, 17, rho=(-1, 1), vel=0, eint=(0, 0))[0])
    R = to_host(m.rhs(to_dev(Qp)))
    el = _sample(om.E, *NEL)
    R_or = om.rhs_elements(Qp, el)
    Rg = R[:, el]
    hmin = 2 * math.pi / 64
    _, lam = om.cfl_dt(Qp, 1.0)
    scale = (2 / hmin) * lam * np.linalg.norm(Qp[:, el])
    assert np.linalg.norm(Rg - R_or) / scale < 1e-12


def test_cfl_bitwise_full(full):
    dg, om, m, Q = full
    dt_or, _ = om.cfl_dt(Q, 0.5)
    dt = float(to_host(m.cfl_dt(to_dev(Q), 0.5))[0])
    assert dt == dt_or


def test_rk_step_conserves_and_is_consistent(full):
    dg, om, m, Q = full
    Qd = to_dev(Q)
    dQ = Qd.clone()
    dt = om.cfl_dt(Q, 0.5)[0]
    R = to_host(m.rhs(Qd))
    m.rk_step(Qd, dQ, dev_scalar(dt))
    Q1 = to_host(Qd)
    # quadrature weights J w_i w_j w_k per node, summed pairwise (numpy): a
    # sequential sum over 32.8 M nodes would itself carry ~1e-12 relative
    # rounding noise, larger than the conservation being checked
    _, w = oracle.gl_nodes(P + 1)
    J = (2 * math.pi / 64) ** 3 / 8
    W = J * np.einsum("k,j,i->kji", w, w, w)

    def integrals(A):
        return np.array([(A[n] * W).sum() for n in range(5)])

    I0, I1 = integrals(Q), integrals(Q1)
    absI = integrals(np.abs(Q))
    # the five integrals are conserved to round-off by the periodic scheme
    # (relative to the integral of |Q_n|; the Taylor-Green z-momentum is
    # identically zero, so its scale is taken from the other fields)
    scale = np.maximum(absI, 1e-3 * absI.max())
    assert np.max(np.abs(I1 - I0) / scale) < 1e-13
    # Q1 - Q = dt R + O(dt^2): check the first-order agreement on the whole mesh
    d = Q1 - Q
    rel = np.linalg.norm(d - dt * R) / np.linalg.norm(dt * R)
    assert rel < 0.05, rel
    assert m.last_error() == dg.DG_OK


def test_advance_full_fp64_equals_separate_calls(full):
    """The bench's launch path (dg_advance, two steps) on the full headline
    mesh: bitwise the separate cfl/rk/norms calls; the first time step is the
    oracle's bit for bit; the integrals are conserved across the steps."""
    dg, om, m, Q = full
    import torch
    Qa, Qb = to_dev(Q), to_dev(Q)
    dQa, dQb = torch.zeros_like(Qa), torch.zeros_like(Qb)
    dts_a, integ_a = [], []
    for _ in range(2):
        dt = m.cfl_dt(Qa, 0.5)
        m.rk_step(Qa, dQa, dt)
        dts_a.append(dt.clone())
        integ_a.append(m.norms(Qa).clone())
    dts_b, integ_b = m.advance(Qb, dQb, 0.5, 2)
    torch.cuda.synchronize()
    assert torch.equal(torch.cat(dts_a), dts_b)
    assert torch.equal(torch.stack(integ_a), integ_b)
    assert torch.equal(Qa, Qb)
    assert float(dts_b[0].item()) == om.cfl_dt(Q, 0.5)[0]
    I0 = to_host(m.norms(to_dev(Q)))
    I2 = to_host(integ_b)[1]
    absI = om.norms(np.abs(Q))[:5]
    scale = np.maximum(absI, 1e-3 * absI.max())
    assert np.max(np.abs(I2[:5] - I0[:5]) / scale) < 1e-13
    assert m.last_error() == dg.DG_OK


def test_config2_full_100_steps_invariants(full):
    """The headline configuration's own run (Taylor-Green, 64^3, p = 4, FP64,
    100 LSERK45 steps at CFL 0.5) through dg_advance, checked by what holds
    at any size: the five integrals stay at their initial values to round-off
    at every step (periodic box, conservative scheme), the kinetic energy
    stays within 1e-3 of its initial value over these early steps of the
    inviscid flow (t ~ 0.017), every time step is positive, finite and within
    1 % of the first (the flow barely changes), and no non-physical state is
    flagged."""
    dg, om, m, Q = full
    import torch
    Qd = to_dev(Q)
    dQ = torch.zeros_like(Qd)
    I0 = to_host(m.norms(Qd))
    dts, integ = m.advance(Qd, dQ, 0.5, 100)
    dts, integ = to_host(dts), to_host(integ)
    assert np.all(np.isfinite(dts)) and np.all(dts > 0)
    assert np.max(np.abs(dts - dts[0])) / dts[0] < 1e-2
    absI = om.norms(np.abs(Q))[:5]
    scale = np.maximum(absI, 1e-3 * absI.max())
    drift = np.max(np.abs(integ[:, :5] - I0[:5]) / scale)
    print(f"config 2 (64^3 p=4, 100 steps): integral drift {drift:.2e} of scale, "
          f"KE {integ[-1, 5] / I0[5] - 1:+.2e} relative, t = {dts.sum():.4f}")
    assert drift < 1e-12
    assert np.max(np.abs(integ[:, 5] - I0[5])) / I0[5] < 1e-3
    assert m.last_error() == dg.DG_OK


def test_advance_full_fp32_vortex128():
    """The FP32 bench configuration (isentropic vortex, 128^3 elements, p = 3)
    through dg_advance: bitwise the separate calls (whose last stage and
    copy-back the step epilogue replaces), finite, and the five integrals
    conserved to float rounding."""
    dg = dg_module()
    import torch
    L = 16.0
    box = (0.0, 0.0, 0.0, L, L, L)
    m = dg.Mesh(128, 128, 128, 3, *box, precision=dg.DG_FP32)
    Q0 = m.init("vortex", inputs.vortex_params(0, box))
    Qa, Qb = Q0.clone(), Q0.clone()
    dQa, dQb = torch.zeros_like(Qa), torch.zeros_like(Qb)
    dt = m.cfl_dt(Qa, 0.5)
    m.rk_step(Qa, dQa, dt)
    integ_a = m.norms(Qa)
    dts_b, integ_b = m.advance(Qb, dQb, 0.5, 1)
    torch.cuda.synchronize()
    assert torch.equal(dt, dts_b)
    assert torch.equal(Qa, Qb)
    assert torch.equal(integ_a, integ_b[0])
    assert bool(torch.isfinite(Qb).all())
    I0 = to_host(m.norms(Q0))
    I1 = to_host(integ_b)[0]
    absI = to_host(m.norms(Q0.abs()))
    scale = np.maximum(absI[:5], 1e-3 * absI[:5].max())
    assert np.max(np.abs(I1[:5] - I0[:5]) / scale) < 1e-6
    assert m.last_error() == dg.DG_OK


def _patch_rhs(om_cls, Qdev, nel, p, h, centres):
    """Oracle right-hand side of each listed element of a periodic mesh from
    its 3x3x3 neighbourhood alone: the neighbourhood, gathered from the
    device state, is a periodic 3x3x3 oracle mesh of the same element size
    whose centre element has the same six face neighbours as in the full
    mesh.  Returns (R, Q) of the centres, shape (5, len(centres), N, N, N)."""
    import torch
    nx, ny, nz = nel
    pm = om_cls(3, 3, 3, p, 0.0, 0.0, 0.0, 3 * h[0], 3 * h[1], 3 * h[2])
    R, Qc = [], []
    for e in centres:
        ex, ey, ez = e % nx, (e // nx) % ny, e // (nx * ny)
        idx = [((ex + a - 1) % nx) + nx * (((ey + b - 1) % ny) + ny * ((ez + c - 1) % nz))
               for c in range(3) for b in range(3) for a in range(3)]
        Qp = Qdev[:, torch.tensor(idx, device=Qdev.device)].double().cpu().numpy()
        R.append(pm.rhs(Qp)[:, 13])
        Qc.append(Qp[:, 13])
    return np.stack(R, axis=1), np.stack(Qc, axis=1)


def _fp32_sampled_rhs_check(dg, m, Q, nel, p, L):
    import torch
    h = tuple(L / n for n in nel)
    el = _sample(nel[0] * nel[1] * nel[2], *nel, k=48, seed=5)
    R = m.rhs(Q)
    Rg = R[:, torch.tensor(el, device=R.device)].double().cpu().numpy()
    del R
    R_or, Qc = _patch_rhs(oracle.Mesh, Q, nel, p, h, el)
    lam = max(oracle.Mesh(1, 1, 1, p, 0, 0, 0, *h).cfl_dt(Qc[:, i:i + 1], 1.0)[1]
              for i in range(len(el)))
    scale = (2 / min(h)) * lam * np.linalg.norm(Qc)
    assert np.linalg.norm(Rg - R_or) / scale < 2e-6


def test_fp32_rhs_sampled_vortex128():
    """The FP32 bench configuration's right-hand side (default stage kernel)
    on sampled elements, every kind of periodic wrap included, against the
    oracle's evaluation of each element's neighbourhood."""
    dg = dg_module()
    L = 16.0
    box = (0.0, 0.0, 0.0, L, L, L)
    m = dg.Mesh(128, 128, 128, 3, *box, precision=dg.DG_FP32)
    Q = m.init("vortex", inputs.vortex_params(0, box))
    _fp32_sampled_rhs_check(dg, m, Q, (128, 128, 128), 3, L)
    assert m.last_error() == dg.DG_OK


def test_fp32_64bit_index_path():
    """A float mesh with 5 E N^3 >= 2^31 (201 x 179 x 187 elements, p = 3,
    9 GB per state) runs the kernels' 64-bit index instantiations: the
    right-hand side on sampled elements against the oracle, one RK step of
    the line kernel bitwise equal to the node-per-thread column kernel's and
    to float rounding equal to the tile kernel's, dg_advance bitwise equal
    to the separate calls, integrals conserved."""
    dg = dg_module()
    import torch
    nel, p, L = (201, 179, 187), 3, 16.0
    assert 5 * nel[0] * nel[1] * nel[2] * (p + 1) ** 3 >= 2 ** 31
    box = (0.0, 0.0, 0.0, L, L, L)
    saved = dg.dg_get_stage_kernel(p)
    try:
        dg.dg_set_stage_kernel(p, dg.DG_STAGE_LINES)
        m = dg.Mesh(*nel, p, *box, precision=dg.DG_FP32)
        Q0 = m.init("vortex", inputs.vortex_params(4, box))
        _fp32_sampled_rhs_check(dg, m, Q0, nel, p, L)
        dt = m.cfl_dt(Q0, 0.5)
        Q = Q0.clone()
        dQ = torch.zeros_like(Q)
        m.rk_step(Q, dQ, dt)
        integ_sep = m.norms(Q)
        Qb, dQb = Q0.clone(), torch.zeros_like(Q0)
        dts_b, integ_b = m.advance(Qb, dQb, 0.5, 1)
        torch.cuda.synchronize()
        assert torch.equal(dt, dts_b) and torch.equal(Q, Qb) and torch.equal(integ_sep, integ_b[0])
        del Qb, dQb
        dg.dg_set_stage_kernel(p, dg.DG_STAGE_COLUMN)
        Qc = Q0.clone()
        dQ.zero_()
        m.rk_step(Qc, dQ, dt)
        torch.cuda.synchronize()
        assert torch.equal(Q, Qc)
        # the tile kernel's 64-bit instantiation: same step to float rounding
        dg.dg_set_stage_kernel(p, dg.DG_STAGE_TILE)
        dQ.zero_()
        Qc.copy_(Q0)
        m.rk_step(Qc, dQ, dt)
        torch.cuda.synchronize()
        rel = float(torch.linalg.vector_norm((Qc - Q).double()) / torch.linalg.vector_norm(Q.double()))
        assert rel < 2e-7, rel
        del Qc
        I0 = to_host(m.norms(Q0))
        I1 = to_host(integ_sep)
        absI = to_host(m.norms(Q0.abs()))
        scale = np.maximum(absI[:5], 1e-3 * absI[:5].max())
        assert np.max(np.abs(I1[:5] - I0[:5]) / scale) < 1e-6
        assert m.last_error() == dg.DG_OK
    finally:
        dg.dg_set_stage_kernel(p, saved)
