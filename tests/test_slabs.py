"""z slabs on the CPU: one periodic mesh split along z into slabs that
exchange one layer of face traces per stage (the paper's partitioned mesh,
Sec. III and Sec. IV), with the oracle as the compute engine.

* the oracle's slab right-hand side (its z neighbours' traces from halo
  buffers) on the slabs of a split mesh equals the undivided mesh's, bit for
  bit, and five of its RK stages equal one LSERK45 step;
* the slab driver (paper_2006_15698_gb300/slabs.py) in one process with 2 to
  4 slabs, exchanging traces by copies, steps the mesh exactly as the
  undivided oracle does (state and time steps bit for bit);
* the same driver over 2 and 3 gloo ranks (1 and 2 slabs each), exchanging
  traces by point-to-point messages and reducing the time step (MIN) and the
  integrals (SUM) across ranks.
"""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2006_15698_gb300 import inputs, slabs

torch = pytest.importorskip("torch")


class OracleSlab:
    """A slab for slabs.SlabSolver computed by the oracle (float64, host)."""

    def __init__(self, nel, p, box, Q):
        self.om = oracle.Mesh(*nel, p, *box)
        self.Qn = np.ascontiguousarray(Q, dtype=np.float64).copy()
        self.dQn = np.zeros_like(self.Qn)
        hs = self.om.halo_shape
        self.sends = (torch.zeros(hs, dtype=torch.float64), torch.zeros(hs, dtype=torch.float64))
        self.halos = (torch.zeros(hs, dtype=torch.float64), torch.zeros(hs, dtype=torch.float64))

    def cfl_dt(self, cfl):
        dt, _ = self.om.cfl_dt(self.Qn, cfl)
        return torch.tensor([dt], dtype=torch.float64)

    def traces(self):
        lo, hi = self.om.ztraces(self.Qn)
        self.sends[0].copy_(torch.from_numpy(lo))
        self.sends[1].copy_(torch.from_numpy(hi))
        return self.sends

    def stage(self, dt, s):
        self.om.rk_stage(self.Qn, self.dQn, float(dt), s, self.halos[0].numpy(),
                         self.halos[1].numpy())

    def integrals(self):
        return torch.from_numpy(self.om.norms(self.Qn)[:6].copy())


def _problem(nel, p, seed):
    box = (0.0, 0.0, 0.0, 10.0, 10.0, 10.0)
    om = oracle.Mesh(*nel, p, *box)
    prm = inputs.vortex_params(seed, box)
    return box, om, om.init("vortex", prm)


def _make_slabs(nel, p, box, Q, ranges):
    out = []
    for zb, nzs in ranges:
        bx = slabs.slab_box(box, nel[2], zb, nzs)
        out.append(OracleSlab((nel[0], nel[1], nzs), p, bx,
                              slabs.slab_of(Q, nel, zb, nzs)))
    return out


def _undivided(om, Q, cfl, nsteps):
    dts = []
    for _ in range(nsteps):
        dt, _ = om.cfl_dt(Q, cfl)
        Q, _ = om.rk_steps(Q, dt, 1)
        dts.append(dt)
    return Q, dts


def test_split_layers_and_slab_box():
    assert slabs.split_layers(7, 3) == [(0, 3), (3, 2), (5, 2)]
    assert slabs.split_layers(4, 4) == [(0, 1), (1, 1), (2, 1), (3, 1)]
    with pytest.raises(ValueError):
        slabs.split_layers(3, 4)
    box = (0.5, -1.0, 2.0, 3.0, 4.0, 2 * np.pi)
    b = slabs.slab_box(box, 64, 16, 16)
    assert b[:2] == box[:2] and b[3:5] == box[3:5]
    assert b[5] / 16 == box[5] / 64 and b[2] == 2.0 + 16 * (box[5] / 64)


@pytest.mark.parametrize("p", [0, 1, 3, 6])
@pytest.mark.parametrize("splits", [(2, 3), (1, 1, 1, 2), (5,)])
def test_oracle_slab_rhs_equals_undivided(p, splits):
    # the halo traces of every slab filled from its neighbours' ztraces: each
    # slab's right-hand side is the undivided mesh's on its layers, bit for bit
    nel = (3, 2, sum(splits))
    box, om, _ = _problem(nel, p, 0)
    Q = inputs.random_state(om.shape, 30 + p)
    R = om.rhs(Q)
    ranges, z = [], 0
    for n in splits:
        ranges.append((z, n))
        z += n
    parts = _make_slabs(nel, p, box, Q, ranges)
    tr = [s.om.ztraces(s.Qn) for s in parts]
    K = len(parts)
    for k, ((zb, nzs), s) in enumerate(zip(ranges, parts)):
        Rs = s.om.rhs_zhalo(s.Qn, tr[(k - 1) % K][1], tr[(k + 1) % K][0])
        assert np.array_equal(Rs, slabs.slab_of(R, nel, zb, nzs))


def test_oracle_five_stages_are_one_step():
    nel, p = (3, 2, 4), 3
    _, om, Q0 = _problem(nel, p, 1)
    Q1, dQ1 = om.rk_steps(Q0, 0.01, 1)
    Q, dQ = Q0.copy(), np.zeros_like(Q0)
    for s in range(5):
        om.rk_stage(Q, dQ, 0.01, s)
    assert np.array_equal(Q, Q1) and np.array_equal(dQ, dQ1)
    # a halo filled with the mesh's own traces is the periodic wrap
    lo, hi = om.ztraces(Q0)
    assert np.array_equal(om.rhs_zhalo(Q0, hi, lo), om.rhs(Q0))


@pytest.mark.parametrize("nslab", [2, 3, 4])
def test_slab_solver_in_one_process_equals_undivided(nslab):
    nel, p, nsteps = (3, 2, 7), 2, 3
    box, om, Q0 = _problem(nel, p, 2)
    Q_ref, dts_ref = _undivided(om, Q0, 0.5, nsteps)
    ranges = slabs.split_layers(nel[2], nslab)
    solver = slabs.SlabSolver(_make_slabs(nel, p, box, Q0, ranges))
    assert solver.ex.nslabs == nslab and not solver.ex.multi
    for k in range(nsteps):
        dt = solver.step(0.5)
        assert float(dt) == dts_ref[k]
    for (zb, nzs), s in zip(ranges, solver.slabs):
        assert np.array_equal(s.Qn, slabs.slab_of(Q_ref, nel, zb, nzs))
    I = solver.integrals().numpy()
    I_ref = om.norms(Q_ref)[:6]
    assert np.max(np.abs(I - I_ref) / np.maximum(np.abs(I_ref), 1.0)) < 1e-13


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_worker(rank, ws, port, K, nel, p, nsteps, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        box, om, Q0 = _problem(nel, p, 3)
        ranges = slabs.split_layers(nel[2], ws * K)[rank * K:(rank + 1) * K]
        solver = slabs.SlabSolver(_make_slabs(nel, p, box, Q0, ranges))
        assert solver.ex.multi and solver.ex.nslabs == ws * K
        dts = [float(solver.step(0.5)) for _ in range(nsteps)]
        I = solver.integrals().numpy()
        q.put((rank, dts, [(zb, nzs, s.Qn) for (zb, nzs), s in zip(ranges, solver.slabs)], I))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws,K", [(2, 1), (3, 2)])
def test_slab_solver_over_gloo_ranks_equals_undivided(ws, K):
    import torch.multiprocessing as mp
    nel, p, nsteps = (2, 3, 7), 3, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_worker, args=(r, ws, port, K, nel, p, nsteps, q))
             for r in range(ws)]
    for pr in procs:
        pr.start()
    res = [q.get(timeout=240) for _ in range(ws)]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    _, om, Q0 = _problem(nel, p, 3)
    Q_ref, dts_ref = _undivided(om, Q0, 0.5, nsteps)
    I_ref = om.norms(Q_ref)[:6]
    for rank, dts, parts, I in res:
        assert dts == dts_ref
        for zb, nzs, Qs in parts:
            assert np.array_equal(Qs, slabs.slab_of(Q_ref, nel, zb, nzs))
        assert np.max(np.abs(I - I_ref) / np.maximum(np.abs(I_ref), 1.0)) < 1e-13
