#!/usr/bin/env python
"""Throughput of the GB300 DG Euler solver in DOF-updates per second per RK stage.

One bench step = one full pass of the hot path on the resident state:
the CFL time-step reduction, one five-stage LSERK45 step (per stage: the
interface-flux kernel and the fused volume/lift/update kernel) and the
quadrature integrals of the new state.  value = DOF x 5 stages x steps x ranks
/ max-over-ranks time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores

The default run (one GPU) also measures, in the same process, the FP32 bulk
form (128^3 p=3, and the headline's 64^3 p=4 for the FP32/FP64 ratio), the
batched form (256 uneven instances) and the serving loop (200 requests):
extra keys of the JSON line (--no-extras skips them).

Multi-GPU: one process per GPU (torchrun).  By default the workload's mesh is
split along z into one slab per rank, the slabs exchanging face traces every
RK stage over NCCL (strong scaling); --replicas runs independent replicas
instead (weak scaling).
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

TWO_PI = 2 * math.pi
WORKLOADS = {
    # the headline: inviscid Taylor-Green vortex, Mach 0.1, 64^3 elements, p = 4, FP64
    "tgv64_p4_fp64": dict(nel=(64, 64, 64), p=4, box=(0, 0, 0, TWO_PI, TWO_PI, TWO_PI),
                          init="tgv", params=[1.0, 1.0, 0.1], prec="fp64", cfl=0.5,
                          desc="inviscid Taylor-Green vortex, Mach 0.1, periodic [0,2pi]^3, "
                               "64^3 hex elements, p=4 (125 nodes/element), FP64 state"),
    # FP32 bulk form: isentropic vortex, 128^3 elements, p = 3
    "vortex128_p3_fp32": dict(nel=(128, 128, 128), p=3, box=(0, 0, 0, 16.0, 16.0, 16.0),
                              init="vortex", params=None, prec="fp32", cfl=0.5,
                              desc="isentropic vortex (seed 0) on a periodic 16^3 box, 128^3 hex "
                                   "elements, p=3, FP32 state and arithmetic, FP64 reductions"),
    # the headline problem in the FP32 bulk form (FP32 / FP64 on equal terms)
    "tgv64_p4_fp32": dict(nel=(64, 64, 64), p=4, box=(0, 0, 0, TWO_PI, TWO_PI, TWO_PI),
                          init="tgv", params=[1.0, 1.0, 0.1], prec="fp32", cfl=0.5,
                          desc="inviscid Taylor-Green vortex, Mach 0.1, periodic [0,2pi]^3, "
                               "64^3 hex elements, p=4, FP32 state and arithmetic, FP64 reductions"),
    # small cases (profiling captures, quick checks)
    "tgv32_p4_fp64": dict(nel=(32, 32, 32), p=4, box=(0, 0, 0, TWO_PI, TWO_PI, TWO_PI),
                          init="tgv", params=[1.0, 1.0, 0.1], prec="fp64", cfl=0.5,
                          desc="Taylor-Green vortex, 32^3 elements, p=4, FP64"),
    "vortex64_p3_fp32": dict(nel=(64, 64, 64), p=3, box=(0, 0, 0, 16.0, 16.0, 16.0),
                             init="vortex", params=None, prec="fp32", cfl=0.5,
                             desc="isentropic vortex (seed 0), 16^3 box, 64^3 elements, p=3, FP32"),
    "tgv32_p4_fp32": dict(nel=(32, 32, 32), p=4, box=(0, 0, 0, TWO_PI, TWO_PI, TWO_PI),
                          init="tgv", params=[1.0, 1.0, 0.1], prec="fp32", cfl=0.5,
                          desc="Taylor-Green vortex, 32^3 elements, p=4, FP32"),
    "vortex48_p4_fp32": dict(nel=(48, 48, 48), p=4, box=(0, 0, 0, 16.0, 16.0, 16.0),
                             init="vortex", params=None, prec="fp32", cfl=0.5,
                             desc="isentropic vortex (seed 0), 16^3 box, 48^3 elements, p=4, FP32"),
    "vortex8_p3_fp64": dict(nel=(8, 8, 8), p=3, box=(0, 0, 0, 10.0, 10.0, 10.0),
                            init="vortex", params=None, prec="fp64", cfl=0.5,
                            desc="isentropic vortex (seed 0), [0,10]^3, 8^3 elements, p=3, FP64"),
}
# roofline curves: Taylor-Green at p = 1..6, about 30 M DOF each, both precisions
for _p, _n in ((1, 155), (2, 104), (3, 78), (4, 62), (5, 52), (6, 44)):
    for _prec in ("fp64", "fp32"):
        WORKLOADS[f"tgv_p{_p}_30m_{_prec}"] = dict(
            nel=(_n, _n, _n), p=_p, box=(0, 0, 0, TWO_PI, TWO_PI, TWO_PI), init="tgv",
            params=[1.0, 1.0, 0.1], prec=_prec, cfl=0.5,
            desc=f"Taylor-Green vortex, Mach 0.1, {_n}^3 elements, p={_p} "
                 f"({_n ** 3 * (_p + 1) ** 3 / 1e6:.1f} M DOF), {_prec.upper()} (roofline curve over p)")
WORKLOADS["batch256_fp32"] = dict(
    kind="batch", count=256, nrange=(4, 32), prange=(1, 5), seed=0, prec="fp32", cfl=0.5,
    box=(0, 0, 0, 10.0, 10.0, 10.0), p=3, nel=(1, 1, 1), init="vortex", params=None,
    desc="256 independent isentropic-vortex instances, elements per side uniform in 4..32 and p "
         "uniform in 1..5 (seed 0), FP32, shared line-kernel launches per RK stage and degree for "
         "the small instances and own launches on four streams for the others, CUDA-graph step")
WORKLOADS["batch64_fp32"] = dict(WORKLOADS["batch256_fp32"], count=64,
                                 desc="64 instances of the batch256_fp32 distribution (profiling)")
WORKLOADS["serve2000_fp32"] = dict(
    kind="serve", count=2000, nrange=(8, 48), prange=(2, 6), steps_range=(50, 500), seed=0,
    budget=150e9, load=0.8, prec="fp32", cfl=0.5, p=3, nel=(1, 1, 1), box=None, init=None,
    params=None,
    desc="serving: Poisson arrivals of 2,000 requests (periodic [0,2pi]^3 box, 8^3..48^3 "
         "elements, p 2..6, 50..500 LSERK45 steps, vortex or Taylor-Green 50/50, FP32 with FP64 "
         "reductions), 150 GB admission budget, offered load 80 % of measured capacity")
WORKLOADS["serve200_fp32"] = dict(
    WORKLOADS["serve2000_fp32"], count=200, nrange=(8, 24), steps_range=(20, 60),
    desc="serving, scaled: 200 requests, 8^3..24^3 elements, p 2..6, 20..60 steps, vortex or "
         "Taylor-Green 50/50, FP32, 150 GB budget, offered load 80 % of measured capacity")
DEFAULT = "tgv64_p4_fp64"


def run_serve(args, w):
    """Serving loop: calibrate the batch's throughput on requests of the
    workload's distribution, then replay Poisson arrivals at `load` x that
    capacity and report time-to-solution percentiles and throughput."""
    import torch
    from paper_2006_15698_gb300 import dg, serve
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dg.load_tuning()
    kw = dict(nrange=w["nrange"], prange=w["prange"], steps_range=w["steps_range"])
    # capacity: the first requests of the distribution, all present at t = 0;
    # measured twice, the first pass warming up the device (module loads,
    # first graph captures, clocks), the second kept
    calib = serve.make_requests(w["seed"] + 7, 24, 1e9, **kw)
    for q in calib:
        q.arrival = 0.0
        q.nsteps = min(q.nsteps, w["steps_range"][0])
    for _ in range(2):
        rep = serve.Server(serve.GpuExecutor(), w["budget"]).run(calib)
    capacity = rep.dof_stage_total / rep.wall
    sample = serve.make_requests(w["seed"], w["count"], 1.0, **kw)
    mean_work = sum(5.0 * q.nsteps * q.dof for q in sample) / len(sample)
    rate = w["load"] * capacity / mean_work
    reqs = serve.make_requests(w["seed"], w["count"], rate, **kw)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    rep = serve.Server(serve.GpuExecutor(), w["budget"]).run(reqs)
    ck = clocks.stop()
    s = rep.summary()
    value, _ = whole_job_rate(rep.wall * 1e3, rep.dof_stage_total, device="cuda")
    if rank != 0:
        return None
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": None,
            "warmup": None, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {w['desc']}", "requests": w["count"],
                       "arrival_rate_per_s": rate, "calibrated_capacity_dof_stage_per_s": capacity,
                       "budget_bytes": w["budget"], "parallelism": f"replicas x{ws}"},
            "serving": {"p50_time_to_solution_s": s["p50_s"], "p99_time_to_solution_s": s["p99_s"],
                        "requests_per_s": s["requests_per_s"], "wall_s": s["wall_s"],
                        "peak_active": s["peak_active"], "peak_bytes": s["peak_bytes"],
                        "batch_rebuilds": s["batch_rebuilds"], "iterations": s["iterations"],
                        "host_rebuild_s": s["rebuild_s"], "host_enqueue_s": s["enqueue_s"],
                        "host_wait_s": s["wait_s"]},
            "clocks": ck}


def batch_specs(w):
    """Seeded instance list of a batch workload: (nx = ny = nz, p) per instance."""
    from paper_2006_15698_gb300 import inputs
    r = inputs.uniforms(w["seed"], 2 * w["count"])
    n0, n1 = w["nrange"]
    p0, p1 = w["prange"]
    specs = []
    for i in range(w["count"]):
        n = n0 + min(int(r[2 * i] * (n1 - n0 + 1)), n1 - n0)
        p = p0 + min(int(r[2 * i + 1] * (p1 - p0 + 1)), p1 - p0)
        L = w["box"][3]
        specs.append(dict(nx=n, ny=n, nz=n, p=p, Lx=L, Ly=L, Lz=L))
    return specs


def run_batch(args, w):
    """The batched form: every instance of the batch advanced one LSERK45 step
    per bench step (graph replay: time steps, five stages, copy back)."""
    import torch
    from paper_2006_15698_gb300 import dg, inputs
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    tuning = dg.load_tuning()
    specs = batch_specs(w)
    b = dg.Batch(specs)
    for i in range(len(specs)):
        b.init(i, "vortex", inputs.vortex_params(1000 + i, w["box"]))
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        # steps go through the two-step graph (the stages alternate between Q
        # and the second states, so a pair of steps ends in Q with no copy)
        b.step(w["cfl"], nsteps=max(args.warmup, 2), use_graph=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        clocks = ClockSampler(torch.cuda.current_device())
        clocks.start()
        e0.record(stream)
        b.step(w["cfl"], nsteps=args.steps, use_graph=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ck = clocks.stop()
        ms = e0.elapsed_time(e1)
        # the same instances stepped one mesh at a time (single-mesh launches,
        # no graph): what batching buys
        meshes = [dg.Mesh(s["nx"], s["ny"], s["nz"], s["p"], *w["box"], precision=dg.DG_FP32)
                  for s in specs]
        dts = [torch.zeros(1, dtype=torch.float64, device="cuda") for _ in specs]
        seq_steps = max(1, min(args.steps, 5))
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for k in range(seq_steps + 1):
            if k == 1:
                s0.record(stream)
            for m, Q, dQ, dt in zip(meshes, b.Q, b.dQ, dts):
                m.cfl_dt(Q, w["cfl"], dt)
                m.rk_step(Q, dQ, dt)
        s1.record(stream)
        torch.cuda.synchronize()
        seq_ms = s0.elapsed_time(s1) / seq_steps
    dof = b.n_dof
    value, ms_max = whole_job_rate(ms, dof * 5 * args.steps, device="cuda")
    err = b.last_error()
    if rank != 0:
        return None
    p_hist = {}
    for s in specs:
        p_hist[s["p"]] = p_hist.get(s["p"], 0) + 1
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {w['desc']}", "instances": len(specs),
                       "dof": dof, "work_items": b.n_items, "p_histogram": p_hist,
                       "tile_table": None if tuning is None else
                       {p: e["tile"] for p, e in tuning["degrees"].items()},
                       "parallelism": f"replicas x{ws}"},
            "sequential_ms_per_step": seq_ms, "batched_speedup": seq_ms / (ms_max / args.steps),
            "clocks": ck, "device_error_flag": err}
METRIC = "DOF-updates/s per RK stage"
UNIT = "DOF-stage/s"


def _sm_clock_mhz(index):
    """(current, maximum) SM clock of GPU `index` in MHz from nvidia-smi, or None."""
    try:
        r = subprocess.run(["nvidia-smi", f"--id={index}", "--query-gpu=clocks.sm,clocks.max.sm",
                            "--format=csv,noheader,nounits"], capture_output=True, text=True,
                           timeout=10)
        cur, mx = (float(x) for x in r.stdout.strip().split(",")[:2])
        return cur, mx
    except Exception:
        return None


def fp64_peak(dg):
    """Roofline denominator of the FP64-pipe-bound kernels, derived from unit
    counts and clocks: FP64 FMA issue slots per SM per clock (the library's
    FMA probe, dg_fma_throughput, divided by SM count x the SM clock seen just
    after it, rounded to whole slots) x 2 flop x SM count (queried) x the
    maximum SM clock.  Also returns the probe's own rate."""
    import torch
    dev = torch.cuda.current_device()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    flops, _ = dg.dg_fma_throughput(dg.DG_FP64)
    clk = _sm_clock_mhz(dev)
    peaks, _ = _peaks()
    cur, mx = clk if clk else (peaks.get("sm_max_mhz", 2070.0),) * 2
    per_clk = flops / (sms * cur * 1e6)
    slots = max(1, round(per_clk / 2.0))
    peak = slots * 2.0 * sms * mx * 1e6 / 1e12
    return {"peak": peak, "probe_tflops": flops / 1e12, "probe_flop_per_clk_per_sm": per_clk,
            "fma_per_clk_per_sm": slots, "sms": sms, "sm_max_mhz": mx,
            "source": f"derived: {slots} FP64 FMA/clk/SM (library FMA probe: {per_clk:.2f} "
                      f"flop/clk/SM at {cur:.0f} MHz) x 2 flop x {sms} SMs x {mx:.0f} MHz"}


def kernel_flops(kind, N, E):
    """Algorithmic flops per launch of the kernels (FMA = 2, div = sqrt = 1),
    counted from the plain formulas per node / face point (the face kernel's
    regrouped Lax-Friedrichs components execute fewer: the count is the
    method's work, not the instructions issued)."""
    if kind == "volume":  # flux 28 + contraction 30N + lift 60 + RK update 25, per node
        return E * N ** 3 * (113 + 30 * N)
    if kind == "face":  # traces 20N + Lax-Friedrichs 69, per unique face point
        return 3 * E * N ** 2 * (69 + 20 * N)
    if kind == "stage":  # fused: volume + lift + update, and every face flux twice
        return kernel_flops("volume", N, E) + 2 * kernel_flops("face", N, E)
    return 0


def kernel_bytes(kind, N, E, esz):
    """Algorithmic HBM bytes per launch (each array element read or written once)."""
    nodes = E * N ** 3
    fpts = 3 * E * N ** 2
    if kind == "volume":  # Q, dQ read; Q, dQ written; interface fluxes read
        return nodes * 5 * esz * 4 + fpts * 5 * esz
    if kind == "face":  # Q read; interface fluxes written
        return nodes * 5 * esz + fpts * 5 * esz
    if kind == "stage":  # fused stage: Q and dQ read, Q' and dQ written
        return nodes * 5 * esz * 4
    if kind == "cfl":
        return nodes * 5 * esz
    if kind == "norms":
        return nodes * 5 * esz
    return 0


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix=f"dg_clocks_{index}_", suffix=".csv")
        os.close(fd)

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def whole_job_rate(ms_local, units_local, device="cpu"):
    """Whole-job throughput over all ranks: the units every rank processed
    divided by the slowest rank's time (max over ranks).  Returns
    (units/s, max ms).  Single process: no collective."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms_local), float(units_local)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        tm = t[:1].clone()
        tu = t[1:].clone()
        dist.all_reduce(tm, op=dist.ReduceOp.MAX)
        dist.all_reduce(tu, op=dist.ReduceOp.SUM)
        t = torch.cat([tm, tu])
    ms_max, units = float(t[0].item()), float(t[1].item())
    return units / (ms_max / 1e3), ms_max


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _kernel_hash():
    """Hash of the kernel sources' code (comments and whitespace removed: the
    compiled kernels do not depend on them), to tell whether committed ncu
    counters were taken on the current kernels."""
    import re
    h = hashlib.sha256()
    for f in ("dg_kernels.cuh", "dg_fused.cuh", "dg_column.cuh", "dg_lines.cuh",
              "dg_line_body.inc"):
        with open(os.path.join(ROOT, "paper_2006_15698_gb300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def _traffic(workload, kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        d = json.load(open(path))
    except Exception:
        return None
    ent = d.get(workload, {}).get(kernel)
    if not ent or ent.get("kernel_source_sha") != _kernel_hash():
        return None
    return ent.get("bytes_per_launch")


# ----------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline leg and the reference arm)
# ----------------------------------------------------------------------------

def oracle_rate(w, nel, steps):
    """DOF-stage/s of the FP64 CPU oracle on `steps` LSERK45 steps of workload w
    on an nel box (CFL reduction + steps + integrals); returns (rate, cores, seconds)."""
    import oracle
    nx, ny, nz = nel
    box = w["box"]
    # keep the element size of the workload: shrink the box with the element count
    sx, sy, sz = (nel[i] / w["nel"][i] for i in range(3))
    b = (box[0], box[1], box[2], box[3] * sx, box[4] * sy, box[5] * sz)
    om = oracle.Mesh(nx, ny, nz, w["p"], *b)
    Q = om.init(w["init"], _params(w))
    cores = oracle.num_threads()
    t0 = time.perf_counter()
    for _ in range(steps):
        dt, _ = om.cfl_dt(Q, w["cfl"])
        Q, _ = om.rk_steps(Q, dt, 1)
        om.norms(Q)
    sec = time.perf_counter() - t0
    dof = nx * ny * nz * (w["p"] + 1) ** 3
    return dof * 5 * steps / sec, cores, sec


def _params(w):
    if w["params"] is not None:
        return w["params"]
    from paper_2006_15698_gb300 import inputs
    return inputs.vortex_params(0, w["box"])


def run_reference(args, w):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    # each step: one LSERK45 step of a 16^3-element box of the same problem
    # (same element size, order and physics; the oracle's cost per DOF does
    # not depend on the element count)
    nel = tuple(min(16, n) for n in w["nel"])
    for _ in range(args.warmup):
        oracle_rate(w, nel, 1)
    rate, cores, sec = oracle_rate(w, nel, args.steps)
    dof = nel[0] * nel[1] * nel[2] * (w["p"] + 1) ** 3
    out = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
           "higher_is_better": True, "scaling": "strong" if _sharded(args, ws) else "weak",
           "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": _config(w, args.workload, ws, _parallelism(args, ws)),
           "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"{args.steps} LSERK45 steps (CFL + 5 stages + integrals) of "
                                      f"the same problem on a {nel[0]}x{nel[1]}x{nel[2]}-element "
                                      f"box ({dof} DOF), plain FP64 C oracle, OpenMP over elements"},
           "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def _sharded(args, ws):
    return (ws > 1 and not getattr(args, "replicas", False)) or getattr(args, "sharded", False)


def _parallelism(args, ws):
    if _sharded(args, ws):
        return f"z slabs x{ws} (one per GPU, NCCL face-trace exchange per stage)"
    return f"replicas x{ws}"


def _config(w, name, ws=1, parallelism=None):
    """The workload's configuration, the same dict in both arms."""
    nx, ny, nz = w["nel"]
    N = w["p"] + 1
    dof = nx * ny * nz * N ** 3
    state_gb = 5 * dof * (8 if w["prec"] == "fp64" else 4) / 1e9
    return {"workload": f"{name}: {w['desc']}; one step = CFL reduction + LSERK45 step + integrals",
            "elements": nx * ny * nz, "p": w["p"], "dof": dof,
            "unknowns": 5 * dof, "cfl": w["cfl"], "precision": w["prec"],
            "parallelism": parallelism or f"replicas x{ws}",
            "l2": f"state arrays {state_gb:.2f} GB each, larger than the 129 MB L2"}


# ----------------------------------------------------------------------------
# GPU run
# ----------------------------------------------------------------------------

def run_native(args, w, with_e2e=True):
    import torch
    import torch.distributed as dist

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl")
    from paper_2006_15698_gb300 import dg

    nx, ny, nz = w["nel"]
    N = w["p"] + 1
    E = nx * ny * nz
    prec = dg.DG_FP64 if w["prec"] == "fp64" else dg.DG_FP32
    esz = 8 if prec == dg.DG_FP64 else 4
    m = dg.Mesh(nx, ny, nz, w["p"], *w["box"], precision=prec)
    stream = torch.cuda.current_stream()
    Q = m.init(w["init"], _params(w))
    dQ = torch.zeros_like(Q)
    nbuf = max(args.steps, args.warmup, 1)
    dts = torch.zeros(nbuf, dtype=torch.float64, device="cuda")
    integ = torch.zeros((nbuf, dg.DG_NORMS_LEN), dtype=torch.float64, device="cuda")

    def steps(n):
        # n x (CFL time step, LSERK45 step, integrals) through the library's
        # multi-step entry point (one pass over the state between steps)
        m.advance(Q, dQ, w["cfl"], n, dts=dts, integ=integ)

    if args.warmup > 0:
        steps(args.warmup)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.25)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    m.profile_begin()
    torch.cuda.synchronize()
    ev0.record(stream)
    steps(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    prof = m.profile_end()
    if ws > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    ck = clocks.stop()
    err = m.last_error()

    dof = E * N ** 3
    value, ms_max = whole_job_rate(ms, dof * 5 * args.steps, device="cuda")

    # ---- end-to-end through host buffers: one dg_advance_host call per step
    # (the state copied in from pinned host memory, the step, the state, the
    # time step and the integrals copied back; the call synchronises)
    e2e_steps = max(1, min(args.steps, 10)) if with_e2e else 0
    Qh = torch.empty(Q.shape if e2e_steps else (1,), dtype=Q.dtype, pin_memory=True)
    if e2e_steps:
        Qh.copy_(Q)
    dts_h = torch.empty(1, dtype=torch.float64, pin_memory=True)
    integ_h = torch.empty((1, dg.DG_NORMS_LEN), dtype=torch.float64, pin_memory=True)
    if e2e_steps:  # the mesh's small time-step / integral buffer, outside the timed region
        m.advance_host(Qh, Q, dQ, w["cfl"], 1, dts=dts_h, integ=integ_h, stream=stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        m.advance_host(Qh, Q, dQ, w["cfl"], 1, dts=dts_h, integ=integ_h, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_val = None
    if e2e_steps:
        e2e_val, _ = whole_job_rate(e0.elapsed_time(e1), dof * 5 * e2e_steps, device="cuda")

    out = None
    if rank == 0:
        peaks, src = _peaks()
        kernels = {k: {"ms_total": v[0], "launches": v[1],
                       "ms_per_launch": (v[0] / v[1] if v[1] else None)}
                   for k, v in prof.items() if v[1]}
        dom = max((k for k in ("face", "volume", "stage") if prof[k][1]), key=lambda k: prof[k][0])
        avg_s = prof[dom][0] / prof[dom][1] / 1e3
        if prec == dg.DG_FP64:
            ach = kernel_flops(dom, N, E) / avg_s / 1e12
            pk = fp64_peak(dg)
            roof = {"bound": "alu", "achieved": ach, "peak": pk["peak"], "unit": "TFLOP/s",
                    "frac": ach / pk["peak"], "peak_source": pk["source"],
                    "probe_tflops": pk["probe_tflops"], "frac_of_probe": ach / pk["probe_tflops"],
                    "kernel": dom}
        else:
            gbs = kernel_bytes(dom, N, E, esz) / avg_s / 1e9
            roof = {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": gbs / peaks["hbm_gbs"], "peak_source": src, "kernel": dom}
        roof["traffic"] = _traffic(args.workload, dom)
        # HBM view of a whole RK stage for context: the minimum state traffic of
        # a stage (Q and dQ read, Q and dQ written) over the time of all stage
        # kernels (and any copy-back), per stage
        n_stages = 5 * args.steps
        stage_s = sum(prof[k][0] for k in ("face", "volume", "stage", "copy")) / 1e3 / n_stages
        roof["stage_hbm_gbs_algorithmic"] = E * N ** 3 * 5 * esz * 4 / stage_s / 1e9
        roof["stage_hbm_frac_of_measured"] = roof["stage_hbm_gbs_algorithmic"] / peaks["hbm_gbs"]
        # our kernel launches: stage kernels; CFL = reduction + finalize;
        # integrals = partial + final; step epilogue = pass + integrals' final
        # + next time step's finalize (none after the last step of the call)
        n_epi = prof["epilogue"][1]
        launches = (prof["face"][1] + prof["volume"][1] + prof["stage"][1]
                    + 2 * prof["cfl"][1] + 2 * prof["norms"][1]
                    + (3 * n_epi - 1 if n_epi else 0))
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None,
               "dtype": "f64" if prec == dg.DG_FP64 else "f32",
               "data": "synthetic",
               "config": _config(w, args.workload, ws),
               "roofline": roof, "gpu_launches": launches, "kernels": kernels,
               "e2e": {"value": e2e_val, "unit": UNIT, "steps": e2e_steps,
                       "api": "dg_advance_host (host state in, host state, dt and integrals out)",
                       "h2d_bytes_per_step": m.state_bytes,
                       "d2h_bytes_per_step": m.state_bytes + 8 + 8 * dg.DG_NORMS_LEN},
               "clocks": ck, "device_error_flag": err}
    if ws > 1:
        dist.barrier()
    del m
    torch.cuda.synchronize()
    return out


def run_extras(args, headline):
    """The other forms of the metric on one GPU, measured in the same run as
    the headline: the FP32 bulk form at its own workload (128^3 p = 3) and at
    the headline's (64^3 p = 4, for the FP32 / FP64 ratio on equal terms), the
    batched form (256 uneven instances) and the serving loop (200 requests).
    Each is timed like the headline (CUDA events, warm-up first, clocks
    sampled); their throughputs are DOF-stage/s like `value`."""
    import argparse as _ap
    extras = {}

    def sub(name, steps=None, warmup=None):
        return _ap.Namespace(**dict(vars(args), workload=name,
                                    steps=steps or args.steps, warmup=warmup or args.warmup))

    keep = ("value", "unit", "ms_per_step", "steps", "warmup", "dtype", "roofline", "clocks",
            "device_error_flag", "gpu_launches")
    r = run_native(sub("vortex128_p3_fp32"), WORKLOADS["vortex128_p3_fp32"], with_e2e=False)
    extras["fp32_vortex128_p3"] = dict({k: r.get(k) for k in keep},
                                       workload=r["config"]["workload"])
    r = run_native(sub("tgv64_p4_fp32"), WORKLOADS["tgv64_p4_fp32"], with_e2e=False)
    extras["fp32_tgv64_p4"] = dict({k: r.get(k) for k in keep}, workload=r["config"]["workload"],
                                   fp32_over_fp64_same_config=r["value"] / headline["value"])
    r = run_batch(sub("batch256_fp32", steps=max(args.steps, 2)), WORKLOADS["batch256_fp32"])
    extras["batch256_fp32"] = {
        "value": r["value"], "unit": r["unit"], "ms_per_step": r["ms_per_step"],
        "steps": r["steps"], "instances": r["config"]["instances"], "dof": r["config"]["dof"],
        "sequential_ms_per_step": r["sequential_ms_per_step"],
        "batched_speedup": r["batched_speedup"], "clocks": r["clocks"],
        "device_error_flag": r["device_error_flag"], "workload": r["config"]["workload"]}
    r = run_serve(sub("serve200_fp32"), WORKLOADS["serve200_fp32"])
    extras["serve200_fp32"] = dict(r["serving"], value=r["value"], unit=r["unit"],
                                   calibrated_capacity_dof_stage_per_s=
                                   r["config"]["calibrated_capacity_dof_stage_per_s"],
                                   arrival_rate_per_s=r["config"]["arrival_rate_per_s"],
                                   clocks=r["clocks"], workload=r["config"]["workload"])
    return extras


def run_sharded(args, w):
    """N > 1 ranks, one GPU each: the workload's single mesh split along z
    into N slabs (one per rank) that exchange face traces every RK stage
    (NCCL point-to-point) and reduce the time step (MIN) and the integrals
    (SUM) -- the paper's partitioned mesh (Sec. III, IV).  Strong scaling:
    value = the whole mesh's DOF x 5 stages x steps / the slowest rank's time."""
    import torch
    import torch.distributed as dist
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl")
    from paper_2006_15698_gb300 import dg, slabs

    def barrier():
        if ws > 1:
            dist.barrier()

    nx, ny, nz = w["nel"]
    N = w["p"] + 1
    prec = dg.DG_FP64 if w["prec"] == "fp64" else dg.DG_FP32
    esz = 8 if prec == dg.DG_FP64 else 4
    zb, nzs = slabs.split_layers(nz, ws)[rank]
    box = slabs.slab_box(w["box"], nz, zb, nzs)
    slab = slabs.GpuSlab((nx, ny, nzs), w["p"], box, prec)
    slab.mesh.init(w["init"], _params(w), Q=slab.Q)
    solver = slabs.SlabSolver([slab])
    stream = torch.cuda.current_stream()
    integ = torch.zeros(6, dtype=torch.float64, device="cuda")

    def steps(n):
        for _ in range(n):
            solver.step(w["cfl"])
            integ.copy_(solver.integrals())

    steps(args.warmup)
    torch.cuda.synchronize()
    barrier()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.25)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    slab.mesh.profile_begin()
    torch.cuda.synchronize()
    barrier()
    ev0.record(stream)
    steps(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    prof = slab.mesh.profile_end()
    barrier()
    ms = ev0.elapsed_time(ev1)
    ck = clocks.stop()
    err = slab.mesh.last_error()
    dof_all = nx * ny * nz * N ** 3
    value, ms_max = whole_job_rate(ms, dof_all * 5 * args.steps / ws, device="cuda")

    # end to end: each rank's slab state from pinned host memory and back, per step
    e2e_steps = max(1, min(args.steps, 10))
    Qh = torch.empty(slab.Q.shape, dtype=slab.Q.dtype, pin_memory=True)
    Qh.copy_(slab.Q)
    integ_h = torch.empty(6, dtype=torch.float64, pin_memory=True)
    torch.cuda.synchronize()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        slab.Q.copy_(Qh, non_blocking=True)
        steps(1)
        Qh.copy_(slab.Q, non_blocking=True)
        integ_h.copy_(integ, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_val, _ = whole_job_rate(e0.elapsed_time(e1), dof_all * 5 * e2e_steps / ws, device="cuda")
    out = None
    if rank == 0:
        E = nx * ny * nzs
        dom = max((k for k in ("face", "volume", "stage") if prof[k][1]), key=lambda k: prof[k][0])
        avg_s = prof[dom][0] / prof[dom][1] / 1e3
        peaks, src = _peaks()
        if prec == dg.DG_FP64:
            ach = kernel_flops(dom, N, E) / avg_s / 1e12
            pk = fp64_peak(dg)
            roof = {"bound": "alu", "achieved": ach, "peak": pk["peak"], "unit": "TFLOP/s",
                    "frac": ach / pk["peak"], "peak_source": pk["source"], "kernel": dom}
        else:
            gbs = kernel_bytes(dom, N, E, esz) / avg_s / 1e9
            roof = {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": gbs / peaks["hbm_gbs"], "peak_source": src, "kernel": dom}
        roof["traffic"] = None
        n_st = prof["face"][1] + prof["volume"][1] + prof["stage"][1]
        launches = n_st + 2 * prof["cfl"][1] + 2 * prof["norms"][1] + 5 * args.steps  # + ztraces
        cfg = _config(w, args.workload, ws, _parallelism(args, ws))
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
               "scaling": "strong", "vs_baseline": None,
               "dtype": "f64" if prec == dg.DG_FP64 else "f32", "data": "synthetic",
               "config": cfg, "roofline": roof, "gpu_launches": launches,
               "e2e": {"value": e2e_val, "unit": UNIT, "steps": e2e_steps,
                       "h2d_bytes_per_step": slab.mesh.state_bytes,
                       "d2h_bytes_per_step": slab.mesh.state_bytes + 8 * 6},
               "clocks": ck, "device_error_flag": err}
    barrier()
    if ws > 1:
        dist.destroy_process_group()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--replicas", action="store_true",
                    help="N > 1: independent replicas of the workload instead of one mesh split "
                         "into N z slabs")
    ap.add_argument("--sharded", action="store_true",
                    help="the z-slab path even on one GPU (one slab, halos from itself)")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload only: skip the float, batched and serving lines")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "native":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    w = WORKLOADS[args.workload]
    if w.get("kind") == "serve":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable":
                              "the serving loop has no oracle arm; use the default workload"}))
            return 0
        out = run_serve(args, w)
        if out is not None:
            print(json.dumps(out))
        return 0
    if w.get("kind") == "batch":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable":
                              "the batched form has no oracle arm; use the default workload"}))
            return 0
        out = run_batch(args, w)
        if out is not None:
            print(json.dumps(out))
        return 0
    if args.impl == "reference":
        return run_reference(args, w)
    ws, rank, _ = _dist()
    if _sharded(args, ws):
        out = run_sharded(args, w)
        if rank == 0 and out is not None:
            print(json.dumps(out))
        return 0
    out = run_native(args, w)
    if ws == 1 and args.workload == DEFAULT and not args.no_extras:
        out.update(run_extras(args, out))
    if rank == 0 and out is not None:
        if ws == 1 and not args.no_cpu_baseline:
            # bounded sample: one LSERK45 step of the full workload if it is
            # small enough for the host, else of a box with the same element size
            dof_full = out["config"]["dof"]
            nel = w["nel"] if dof_full <= 40_000_000 else tuple(min(32, n) for n in w["nel"])
            rate, cores, sec = oracle_rate(w, nel, 1)
            out["cpu_baseline"] = {
                "value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                "sample": f"1 LSERK45 step (CFL + 5 stages + integrals) of the workload on "
                          f"{nel[0]}x{nel[1]}x{nel[2]} elements, {sec:.1f} s, plain FP64 C oracle"}
        print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
