"""One periodic mesh split along z into slabs, on one or several GPUs.

The paper partitions its mesh over MPI ranks, one GPU per partition, and
neighbouring partitions exchange element face data every Runge-Kutta stage
(Sec. III; Sec. IV; Tables I and III compare host-staged with CUDA-aware
exchange).  Here the partitions are slabs of whole z layers: a slab's only
neighbours are the slab below and the slab above (periodic in z, so the
last slab's upper neighbour is the first), and what crosses a slab boundary
per stage is one layer of face traces each way: 5 x nx ny x N^2 values,
a factor N fewer than the layer itself.

Per LSERK45 step:
  1. each slab's time step (dg_cfl_dt, local); the step's dt is their
     minimum over every slab (a MIN all-reduce across ranks) -- the same
     double as the undivided mesh's, because the time step decreases
     monotonically with the maximum wave speed;
  2. five times: every slab computes the traces its neighbours need
     (dg_zhalo_traces), the traces move to the neighbours' halo buffers
     (a device copy between slabs of one process, a send/receive between
     ranks: NCCL on GPUs, gloo on CPU), and every slab runs the stage
     (dg_rk_stage), reading its halos where the periodic mesh would read
     the layer across the boundary.
The result is the undivided mesh's, bit for bit (tests/test_slabs.py on the
oracle, tests/test_gpu_slabs.py on the GPU).

S = world_size x K slabs: rank r holds slabs r K .. r K + K - 1 (K > 1 in
one process emulates the partitioned mesh on one GPU).  All arithmetic runs
in the library's kernels (GpuSlab) or, in the CPU tests, in the oracle; this
module only moves buffers and schedules.
"""
import torch

NF = 5


def split_layers(nz, nslabs):
    """Contiguous z ranges [(z_begin, nz_slab)] of nslabs slabs covering nz
    layers, as even as possible (the first nz % nslabs slabs one layer more)."""
    if not 1 <= nslabs <= nz:
        raise ValueError(f"cannot split {nz} layers into {nslabs} slabs")
    base, extra = divmod(nz, nslabs)
    out, z = [], 0
    for k in range(nslabs):
        n = base + (1 if k < extra else 0)
        out.append((z, n))
        z += n
    return out


def slab_box(box, nz, z_begin, nz_slab):
    """The box of a slab: (x0, y0, z0 + z_begin hz, Lx, Ly, nz_slab hz) with
    hz = Lz / nz.  The slab's element size Lz_slab / nz_slab must be hz to
    the last bit (its geometric factors then equal the undivided mesh's);
    a split that does not round-trip exactly raises."""
    x0, y0, z0, Lx, Ly, Lz = box
    hz = Lz / nz
    Lzs = hz * nz_slab
    if Lzs / nz_slab != hz:
        raise ValueError(f"a slab of {nz_slab} layers does not keep hz = {hz!r} exactly")
    return (x0, y0, z0 + z_begin * hz, Lx, Ly, Lzs)


def slab_of(Q, nel, z_begin, nz_slab):
    """The part of a state (5, nx ny nz, ...) on layers z_begin .. +nz_slab
    (a view: per field the layers are contiguous)."""
    nx, ny, nz = nel
    plane = nx * ny
    return Q[:, z_begin * plane:(z_begin + nz_slab) * plane]


class Exchange:
    """Moves the slabs' face traces to their neighbours' halos and reduces
    the time step and the integrals over all slabs.

    K slabs in this process; with torch.distributed initialised and more than
    one rank, the neighbours across the process boundary are ranks r - 1 and
    r + 1 (periodic), reached by batched point-to-point operations."""

    def __init__(self, K):
        import torch.distributed as dist
        self.dist = dist
        self.K = K
        self.multi = dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1
        self.rank = dist.get_rank() if self.multi else 0
        self.world = dist.get_world_size() if self.multi else 1

    @property
    def nslabs(self):
        return self.K * self.world

    def halos(self, sends, halos):
        """sends[k] = (lo, hi) of local slab k, halos[k] = (halo_lo, halo_hi)
        to fill: halo_lo of slab g <- hi of slab g - 1, halo_hi <- lo of g + 1."""
        K = self.K
        for k in range(K):
            if k > 0 or not self.multi:
                halos[k][0].copy_(sends[(k - 1) % K][1])
            if k < K - 1 or not self.multi:
                halos[k][1].copy_(sends[(k + 1) % K][0])
        if not self.multi:
            return
        dist = self.dist
        below = (self.rank - 1) % self.world
        above = (self.rank + 1) % self.world
        # canonical order on every rank (NCCL matches a pair's operations in
        # issue order, gloo by tag): send up, send down, receive from below,
        # receive from above
        ops = [dist.P2POp(dist.isend, sends[K - 1][1], above, tag=0),
               dist.P2POp(dist.isend, sends[0][0], below, tag=1),
               dist.P2POp(dist.irecv, halos[0][0], below, tag=0),
               dist.P2POp(dist.irecv, halos[K - 1][1], above, tag=1)]
        for req in dist.batch_isend_irecv(ops):
            req.wait()

    def reduce_min(self, t):
        if self.multi:
            self.dist.all_reduce(t, op=self.dist.ReduceOp.MIN)
        return t

    def reduce_sum(self, t):
        if self.multi:
            self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM)
        return t


class SlabSolver:
    """LSERK45 steps of a mesh split into slabs.  `slabs` are this process's
    slabs (bottom to top), objects with
        cfl_dt(cfl)    -> 1-element float64 tensor, the slab's time step
        traces()       -> (send_lo, send_hi) of the current state
        halos          -> (halo_lo, halo_hi), the buffers its stages read
        stage(dt, s)   -> LSERK45 stage s with those halos
        integrals()    -> float64 tensor of the 5 integrals and the kinetic energy
    (GpuSlab below; an oracle-backed stand-in in the CPU tests)."""

    def __init__(self, slabs, exchange=None):
        self.slabs = list(slabs)
        self.ex = exchange or Exchange(len(self.slabs))

    def time_step(self, cfl):
        dt = self.slabs[0].cfl_dt(cfl)
        for s in self.slabs[1:]:
            dt = torch.minimum(dt, s.cfl_dt(cfl))
        return self.ex.reduce_min(dt)

    def step(self, cfl):
        """One LSERK45 step; returns the time step (a tensor)."""
        dt = self.time_step(cfl)
        for st in range(5):
            sends = [s.traces() for s in self.slabs]
            self.ex.halos(sends, [s.halos for s in self.slabs])
            for s in self.slabs:
                s.stage(dt, st)
        return dt

    def integrals(self):
        tot = self.slabs[0].integrals().clone()
        for s in self.slabs[1:]:
            tot += s.integrals()
        return self.ex.reduce_sum(tot)


class GpuSlab:
    """A slab on the current GPU: a library mesh with its halos set, its
    states (two for the float form's ping-pong) and trace buffers."""

    def __init__(self, nel, p, box, precision, Q=None):
        from . import dg
        self.dg = dg
        nx, ny, nz = nel
        self.mesh = dg.Mesh(nx, ny, nz, p, *box, precision=precision)
        m = self.mesh
        self.Q = m.empty() if Q is None else m._chk(Q)
        self.other = m.empty() if precision == dg.DG_FP32 else None
        self.dQ = torch.zeros_like(self.Q)
        self.sends = (m.empty_halo(), m.empty_halo())
        self.halos = (m.empty_halo(), m.empty_halo())
        m.set_zhalo(*self.halos)
        self.dt = torch.zeros(1, dtype=torch.float64, device=m.device)

    def cfl_dt(self, cfl):
        return self.mesh.cfl_dt(self.Q, cfl, self.dt)

    def traces(self):
        return self.mesh.ztraces(self.Q, *self.sends)

    def stage(self, dt, st):
        if self.other is None:
            self.mesh.rk_stage(self.Q, self.Q, self.dQ, dt, st)
        else:
            self.mesh.rk_stage(self.Q, self.other, self.dQ, dt, st)
            self.Q, self.other = self.other, self.Q

    def integrals(self):
        return self.mesh.norms(self.Q)[:6]
