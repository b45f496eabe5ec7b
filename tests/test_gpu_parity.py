"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.  Inputs are generated on the host (oracle initial states
or the seeded generator) and uploaded; nothing the GPU computes feeds the
oracle.

Bars:
  * one LSERK45 step, FP64: relative L2 of the new state <= 1e-12
  * right-hand side, FP64: ||dR|| <= 1e-12 * rhs_scale (the size of the
    terms being summed; see gpu_helpers.rhs_scale)
  * time step: bitwise equal (explicitly rounded reduction in both)
  * integrals: 1e-13 relative to the integral of |Q|
"""
import math

import numpy as np
import pytest

import oracle
from gpu_helpers import dev_scalar, dg_module, rel_l2, rhs_scale, to_dev, to_host
from paper_2006_15698_gb300 import inputs

pytestmark = pytest.mark.gpu

BOX10 = (0.0, 0.0, 0.0, 10.0, 10.0, 10.0)
TGV_BOX = (0.0, 0.0, 0.0, 2 * math.pi, 2 * math.pi, 2 * math.pi)

# meshes: self-neighbour, thin, ragged against every elements-per-CTA tiling
MESHES = [(1, 1, 1), (3, 2, 2), (5, 3, 2), (2, 1, 7)]


def _state(kind, om, seed):
    if kind == "random":
        return inputs.random_state(om.shape, seed)
    if kind == "vortex":
        # strength reduced to [1, 2]: on the coarsest test meshes (elements
        # up to 10 wide) a stronger vortex makes the degree-p polynomial's
        # face traces non-physical (negative pressure; NaN in the oracle too)
        prm = inputs.vortex_params(seed, om.box)
        prm[0] = 1.0 + 0.25 * (prm[0] - 1.0)
        return om.init("vortex", prm)
    return om.init("tgv", inputs.tgv_params(0.1))


@pytest.mark.parametrize("p", range(0, 7))
@pytest.mark.parametrize("nel", MESHES)
@pytest.mark.parametrize("kind", ["random", "vortex"])
def test_rhs_fp64(p, nel, kind):
    dg = dg_module()
    om = oracle.Mesh(*nel, p, *BOX10)
    Q = _state(kind, om, 7 * p + sum(nel))
    R_or = om.rhs(Q)
    assert np.isfinite(R_or).all(), "test input has non-physical face traces"
    m = dg.Mesh(*nel, p, *BOX10)
    R = to_host(m.rhs(to_dev(Q)))
    err = np.linalg.norm(R - R_or) / rhs_scale(om, Q)
    assert err < 1e-12, err


@pytest.mark.parametrize("p", [1, 3, 4, 6])
def test_rhs_fp64_tgv(p):
    dg = dg_module()
    om = oracle.Mesh(4, 4, 4, p, *TGV_BOX)
    Q = _state("tgv", om, 0)
    R_or = om.rhs(Q)
    m = dg.Mesh(4, 4, 4, p, *TGV_BOX)
    R = to_host(m.rhs(to_dev(Q)))
    assert np.linalg.norm(R - R_or) / rhs_scale(om, Q) < 1e-12


@pytest.mark.parametrize("p", range(0, 7))
@pytest.mark.parametrize("nel", [(3, 2, 2), (5, 3, 2)])
def test_rk_step_fp64_per_step(p, nel):
    # three consecutive steps, each compared after the step from the same input
    dg = dg_module()
    om = oracle.Mesh(*nel, p, *BOX10)
    Q = _state("vortex", om, p)
    m = dg.Mesh(*nel, p, *BOX10)
    for step in range(3):
        dt, _ = om.cfl_dt(Q, 0.5)
        Q1, dQ1 = om.rk_steps(Q, dt, 1)
        Qd = to_dev(Q)
        dQd = torch_empty_like(Qd)
        m.rk_step(Qd, dQd, dev_scalar(dt))
        Qg = to_host(Qd)
        err = rel_l2(Qg, Q1)
        assert err < 1e-12, (step, err)
        assert rel_l2(to_host(dQd), dQ1) < 1e-10
        Q = Q1


def torch_empty_like(t):
    import torch
    return torch.empty_like(t)


@pytest.mark.parametrize("kind", ["random", "vortex", "tgv"])
@pytest.mark.parametrize("p", [0, 2, 5])
def test_cfl_dt_bitwise(kind, p):
    dg = dg_module()
    box = TGV_BOX if kind == "tgv" else BOX10
    om = oracle.Mesh(5, 3, 2, p, *box)
    Q = _state(kind, om, 3 + p)
    dt_or, _ = om.cfl_dt(Q, 0.5)
    m = dg.Mesh(5, 3, 2, p, *box)
    dt = float(to_host(m.cfl_dt(to_dev(Q), 0.5))[0])
    assert dt == dt_or, (dt, dt_or)
    # FP32 state: node speeds in float, maximum and dt in double
    m32 = dg.Mesh(5, 3, 2, p, *box, precision=dg.DG_FP32)
    Q32 = Q.astype(np.float32)
    dt32_or, _ = om.cfl_dt(Q32.astype(np.float64), 0.5)
    import torch
    dt32 = float(to_host(m32.cfl_dt(to_dev(Q32, torch.float32), 0.5))[0])
    assert abs(dt32 - dt32_or) <= 1e-6 * dt32_or


def _uniform(om, rho=1.0, u=(0.3, -0.2, 0.1), p=1.0):
    return om.init("uniform", [rho, *u, p])


@pytest.mark.parametrize("case", ["all_equal", "near_ties", "high_mach", "float_range",
                                  "spike_first", "spike_last", "spike_middle"])
def test_cfl_pruned_reduction_bitwise(case):
    """The FP64 reduction evaluates only the nodes a float estimate cannot
    exclude; the time step stays bitwise equal to the oracle's in the cases
    that stress the estimate: every node tied, ties closer than float can
    resolve, Mach-20 nodes (pressure cancelled in float), magnitudes outside
    the estimate's range, and a single fastest node at either end or in the
    middle of a mesh large enough for several grid-stride sweeps per warp."""
    dg = dg_module()
    big = case.startswith("spike")
    om = oracle.Mesh(40, 40, 40, 2, *BOX10) if big else oracle.Mesh(5, 3, 2, 3, *BOX10)
    Q = _uniform(om)
    flat = Q.reshape(5, -1)
    rng = np.random.default_rng(17)
    nn = flat.shape[1]
    if case == "all_equal":
        pass                         # every node ties: all evaluated exactly
    elif case == "near_ties":
        idx = rng.choice(nn, nn // 3, replace=False)
        flat[1, idx] *= 1.0 + 1e-9 * rng.random(idx.size)
    elif case == "high_mach":
        idx = rng.choice(nn, 7, replace=False)
        flat[1, idx] = 40.0          # |u| = 40 against c = 1.18: p << E/100
        flat[4, idx] = 2.5 + 0.5 * 40.0 ** 2
    elif case == "float_range":
        flat[0, 3] = 1e-12           # density below the estimate's range
        flat[1, 3] = flat[2, 3] = flat[3, 3] = 0.0
        flat[4, 3] = 2.5e-12
        flat[4, 11] = 2e9            # energy above it: the fastest node
    else:
        # spread speeds (the estimate skips most nodes), one fastest node and
        # a twin slower by less than the estimate resolves
        flat = inputs.random_state(om.shape, 23).reshape(5, -1)
        t = {"spike_first": 0, "spike_last": nn - 1, "spike_middle": nn // 2 + 5}[case]
        t2 = (t + 12345) % nn
        for node, f in ((t, 1.0), (t2, 1.0 - 1e-7)):
            flat[:, node] = [1.0, 2.0 * f, 0.1, -0.1, 2.5 + 0.5 * (4.0 * f * f + 0.02)]
    Q = flat.reshape(om.shape)
    dt_or, _ = om.cfl_dt(Q, 0.5)
    m = dg.Mesh(om.nx, om.ny, om.nz, om.p, *BOX10)
    dt = float(to_host(m.cfl_dt(to_dev(Q), 0.5))[0])
    assert m.last_error() == dg.DG_OK
    assert dt == dt_or, (dt, dt_or)


def test_cfl_flags_nonpositive_pressure():
    dg = dg_module()
    om = oracle.Mesh(3, 2, 2, 2, *BOX10)
    Q = _state("random", om, 1)
    Q[4, 7, 1, 2, 0] = 0.0  # rho E = 0 -> p < 0 at one node (host-side corruption)
    m = dg.Mesh(3, 2, 2, 2, *BOX10)
    dt = to_host(m.cfl_dt(to_dev(Q), 0.5))[0]
    assert math.isnan(dt)
    assert m.last_error() == dg.DG_ERR_NONFINITE
    assert m.last_error() == dg.DG_OK  # cleared on read
    Q[4, 7, 1, 2, 0] = 2.5
    dt = to_host(m.cfl_dt(to_dev(Q), 0.5))[0]
    assert dt == om.cfl_dt(Q, 0.5)[0]


@pytest.mark.parametrize("p", [0, 3, 6])
@pytest.mark.parametrize("with_ref", [False, True])
def test_norms(p, with_ref):
    dg = dg_module()
    om = oracle.Mesh(5, 3, 2, p, *BOX10)
    Q = _state("vortex", om, 2)
    Qr = _state("random", om, 9) if with_ref else None
    out_or = om.norms(Q, Qr)
    m = dg.Mesh(5, 3, 2, p, *BOX10)
    out = to_host(m.norms(to_dev(Q), None if Qr is None else to_dev(Qr)))
    absq = om.norms(np.abs(Q))[:5]
    assert np.max(np.abs(out[:5] - out_or[:5]) / absq) < 1e-13
    assert abs(out[5] - out_or[5]) / out_or[5] < 1e-13
    assert abs(out[6] - out_or[6]) <= 1e-13 * max(out_or[6], 1e-300)
    # bitwise reproducible run to run
    out2 = to_host(m.norms(to_dev(Q), None if Qr is None else to_dev(Qr)))
    assert np.array_equal(out, out2)


@pytest.mark.parametrize("kind", ["uniform", "vortex", "tgv"])
@pytest.mark.parametrize("p", [0, 3, 6])
def test_state_init(kind, p):
    dg = dg_module()
    box = TGV_BOX if kind == "tgv" else BOX10
    prm = {"uniform": inputs.uniform_params(1), "vortex": inputs.vortex_params(5, box, t=2.5),
           "tgv": inputs.tgv_params(0.1)}[kind]
    om = oracle.Mesh(4, 3, 2, p, *box)
    Q_or = om.init(kind, prm)
    m = dg.Mesh(4, 3, 2, p, *box)
    Q = to_host(m.init(kind, prm))
    assert np.max(np.abs(Q - Q_or) / np.maximum(np.abs(Q_or), 1)) < 1e-14


def test_free_stream_and_conservation_fp64():
    dg = dg_module()
    om = oracle.Mesh(6, 5, 4, 4, *BOX10)
    m = dg.Mesh(6, 5, 4, 4, *BOX10)
    Q = om.init("uniform", inputs.uniform_params(3))
    R = to_host(m.rhs(to_dev(Q)))
    assert np.max(np.abs(R)) < 1e-12 * rhs_scale(om, Q) / np.sqrt(Q.size)
    Q = _state("random", om, 4)
    R = to_host(m.rhs(to_dev(Q)))
    I = om.norms(R)[:5]
    assert np.max(np.abs(I)) < 1e-12 * om.norms(np.abs(R))[:5].max()


@pytest.mark.parametrize("p", [1, 3, 6])
def test_rhs_fp32(p):
    # FP32 bulk form: float state and arithmetic, against the FP64 oracle on
    # the float-rounded input; error of a few float ulps of the term size
    dg = dg_module()
    import torch
    om = oracle.Mesh(5, 3, 2, p, *BOX10)
    Q = _state("vortex", om, p).astype(np.float32).astype(np.float64)
    R_or = om.rhs(Q)
    m = dg.Mesh(5, 3, 2, p, *BOX10, precision=dg.DG_FP32)
    R = to_host(m.rhs(to_dev(Q, torch.float32)))
    assert np.linalg.norm(R - R_or) / rhs_scale(om, Q) < 2e-6


def test_device_errors_are_host_side():
    dg = dg_module()
    m = dg.Mesh(2, 2, 2, 1, *BOX10)
    Q = m.init("uniform", [1, 0, 0, 0, 1])
    with pytest.raises(dg.DGError):
        dg.dg_rhs(m.h, Q, Q)  # R aliasing Q is rejected
    with pytest.raises(dg.DGError):
        dg.dg_state_init(m.h, 1, [1.0, 2.0], Q)  # too few vortex parameters
    with pytest.raises(dg.DGError):
        dg.dg_cfl_dt(m.h, Q, -1.0, dev_scalar(0))
    assert m.last_error() == dg.DG_OK


def test_sound_speed_root_within_one_ulp():
    """The double face kernel's sound speed sqrt(gamma p / rho) is a refined
    reciprocal-square-root approximation, not the correctly rounded root:
    on a sweep over twelve decades (and the range of the workloads,
    gamma p / rho in [0.5, 200]) it is within one ulp of CUDA's sqrt."""
    dg = dg_module()
    import torch
    g = np.random.Generator(np.random.PCG64(7))
    a = np.concatenate([np.logspace(-6, 6, 400_001), g.uniform(0.5, 200.0, 400_000),
                        np.nextafter(1.0, 2.0) ** np.arange(1, 2001)])
    fast, ieee = dg.dg_selfcheck_sqrt(torch.from_numpy(a).cuda())
    fast, ieee = to_host(fast), to_host(ieee)
    assert np.array_equal(ieee, np.sqrt(a))          # CUDA's sqrt is the correctly rounded one
    ulps = np.abs(fast.view(np.int64) - ieee.view(np.int64))
    assert ulps.max() <= 1, ulps.max()
    print(f"sound-speed root: {np.mean(ulps == 0):.4f} of {a.size} roots exact, max {ulps.max()} ulp")
