"""The workloads' own checks, through the GPU path (dg_advance, FP64):

* config 1 -- isentropic vortex, [0,10]^3, 8^3 elements, p = 3, ten
  LSERK45 steps at CFL 0.5 with seeded vortex strength, centre and drift
  (seeds 0..9): against the oracle's ten steps (each step's time step from
  its own state);
* config 2 downsampled -- Taylor-Green at Mach 0.1 on 16^3 elements, p = 4,
  the config's 100 steps: state, kinetic energy and the five conserved
  integrals against the oracle's, conservation to round-off;
* configs 4 and 5 (FP32 batched form, FP32 serving loop) -- the error of a
  sample of their instances against the FP64 oracle's solve of the same
  instance, at the workloads' own step counts;
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


@pytest.mark.parametrize("seed", range(10))
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


def test_config2_tgv16_p4_100_steps_invariants():
    # the config's 100 LSERK45 steps on its downsampled 16^3 copy
    dg = dg_module()
    import torch
    box = (0.0, 0.0, 0.0, 2 * math.pi, 2 * math.pi, 2 * math.pi)
    om = oracle.Mesh(16, 16, 16, 4, *box)
    Q0 = om.init("tgv", inputs.tgv_params(0.1))
    Q_or, dts_or, integ_or = _oracle_run(om, Q0, 0.5, 100)
    m = dg.Mesh(16, 16, 16, 4, *box)
    Q = to_dev(Q0)
    dQ = torch.zeros_like(Q)
    dts, integ = m.advance(Q, dQ, 0.5, 100)
    Qg, dts, integ = to_host(Q), to_host(dts), to_host(integ)
    err = rel_l2(Qg, Q_or)
    print(f"config 2 (16^3 p=4, 100 steps): FP64 GPU vs oracle rel L2 {err:.2e}")
    assert err < 1e-10                               # 1e-12 per step, 100 steps
    assert np.max(np.abs(dts - dts_or) / dts_or) < 1e-12
    # kinetic energy: equal to the oracle's at every step, and nearly
    # constant over these early steps of the inviscid flow (t ~ 0.25)
    ke, ke_or = integ[:, 5], integ_or[:, 5]
    assert np.max(np.abs(ke - ke_or) / ke_or) < 1e-11
    ke0 = om.norms(Q0)[5]
    assert np.max(np.abs(ke - ke0)) / ke0 < 1e-2
    # the five conserved integrals: constant to round-off on the periodic box
    # (against the GPU's own sum of the initial state: the oracle's sequential
    # sum over 512,000 nodes differs from it by summation order, ~4e-13)
    I0 = to_host(m.norms(to_dev(Q0)))[:5]
    absI = om.norms(np.abs(Q0))[:5]
    scale = np.maximum(absI, 1e-3 * absI.max())
    assert np.max(np.abs(integ[:, :5] - I0) / scale) < 1e-12
    assert m.last_error() == dg.DG_OK


def _oracle_solve(nel, p, box, kind, params, nsteps, cfl=0.5):
    """FP64 oracle solve with the CFL time step of each step's own state."""
    om = oracle.Mesh(*nel, p, *box)
    Q = om.init(kind, params)
    for _ in range(nsteps):
        dt, _ = om.cfl_dt(Q, cfl)
        Q, _ = om.rk_steps(Q, dt, 1)
    return Q


def test_config4_batch_sample_fp32_vs_fp64_oracle():
    """FP32 batched form (config 4): the batch workload's first instances that
    the oracle holds (elements per side <= 10), 100 LSERK45 steps in one
    batch (persistent and own launches, CUDA graph), each instance against
    the oracle's FP64 solve of the same instance (each with the time steps
    of its own state)."""
    dg = dg_module()
    import torch
    import bench
    w = bench.WORKLOADS["batch256_fp32"]
    specs = [dict(s, idx=i) for i, s in enumerate(bench.batch_specs(w))]
    sample = [s for s in specs if s["nx"] <= 10][:5]
    assert {s["p"] for s in sample} and len(sample) == 5
    b = dg.Batch([{k: v for k, v in s.items() if k != "idx"} for s in sample])
    prms = [inputs.vortex_params(1000 + s["idx"], w["box"]) for s in sample]
    for i, prm in enumerate(prms):
        b.init(i, "vortex", prm)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b.step(w["cfl"], nsteps=100, use_graph=True)
    torch.cuda.synchronize()
    assert b.last_error() == dg.DG_OK
    errs = []
    for i, s in enumerate(sample):
        nel = (s["nx"], s["ny"], s["nz"])
        Q_or = _oracle_solve(nel, s["p"], w["box"], "vortex", prms[i], 100, w["cfl"])
        errs.append(rel_l2(to_host(b.Q[i]), Q_or))
    print("config 4 sample (n, p, rel L2 vs FP64 oracle after 100 steps): " +
          ", ".join(f"({s['nx']}, {s['p']}, {e:.2e})" for s, e in zip(sample, errs)))
    assert max(errs) < 1e-5, errs


def test_config5_serving_sample_fp32_vs_fp64_oracle():
    """FP32 serving loop (config 5): the serving workload's first requests
    that the oracle holds (elements per side <= 10), served together by the
    loop for their full step counts (50..500), each final state against the
    oracle's FP64 solve of the same request (vortex or Taylor-Green)."""
    dg_module()
    import bench
    from paper_2006_15698_gb300 import serve
    w = bench.WORKLOADS["serve2000_fp32"]
    reqs = serve.make_requests(w["seed"], 400, 1e6, nrange=w["nrange"], prange=w["prange"],
                               steps_range=w["steps_range"])
    sample = [q for q in reqs if q.n <= 10 and q.dof * q.nsteps <= 2.0e8][:4]
    assert len(sample) == 4 and {q.kind for q in sample} == {"vortex", "tgv"}
    for q in sample:
        q.arrival = 0.0
    rep = serve.Server(serve.GpuExecutor(), w["budget"], keep_states=True).run(sample)
    errs = []
    for q in sample:
        o = [o for o in rep.outcomes if o.rid == q.rid][0]
        box = (0.0, 0.0, 0.0, q.L, q.L, q.L)
        Q_or = _oracle_solve((q.n, q.n, q.n), q.p, box, q.kind, q.params, q.nsteps, q.cfl)
        errs.append(rel_l2(o.result["state"].double().numpy(), Q_or))
    print("config 5 sample (n, p, kind, steps, rel L2 vs FP64 oracle): " +
          ", ".join(f"({q.n}, {q.p}, {q.kind}, {q.nsteps}, {e:.2e})" for q, e in zip(sample, errs)))
    assert max(errs) < 1e-5, errs


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
