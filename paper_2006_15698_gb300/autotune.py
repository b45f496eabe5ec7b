"""Autotuner of the float form's RK stage: tile shapes and stage kernel.

For every polynomial degree it times one LSERK45 step of a representative
float mesh (isentropic vortex, about `target_dof` nodes) with each tile
variant the library offers (dg_tile_variant_count / dg_tile_shape) and with
the two column kernels (one thread per node, "column"; one thread per z node
line, "lines"), and writes the table that ``dg.load_tuning`` reads: the
fastest tile variant (used by single meshes when "kernel" is "tile") and the
fastest single-mesh kernel (which a batch's own-launch instances use; its
shared instances always run the line kernel):

    {"gpu": ..., "degrees": {"3": {"variant": 1, "tile": [2, 2], "kernel": "lines",
                                   "ms_per_step": {"0": 5.1, "1": 4.8, "column": 4.1,
                                                   "lines": 3.5}}, ...}}

Run on the GPU the library will serve:
    python -m paper_2006_15698_gb300.autotune [--out PATH] [--degrees 1,2,3]
"""
import argparse
import json
import os
import sys

import torch

from . import dg, inputs


def time_variant(p, variant, target_dof=8e6, steps=6, warmup=2):
    """Milliseconds per LSERK45 step (CFL + 5 stages) of a float vortex mesh
    of about target_dof nodes at degree p with the given tile variant, or
    with a column kernel for variant "column" or "lines"."""
    if variant in ("column", "lines"):
        dg.dg_set_stage_kernel(p, dg.STAGE_KINDS[variant])
    else:
        dg.dg_set_stage_kernel(p, dg.DG_STAGE_TILE)
        dg.dg_set_tile_variant(p, variant)
    N = p + 1
    n = max(4, int(round((target_dof / N ** 3) ** (1 / 3))))
    box = (0.0, 0.0, 0.0, 16.0, 16.0, 16.0)
    m = dg.Mesh(n, n, n, p, *box, precision=dg.DG_FP32)
    Q = m.init("vortex", inputs.vortex_params(0, box))
    dQ = torch.zeros_like(Q)
    dt = torch.zeros(1, dtype=torch.float64, device=Q.device)
    for _ in range(warmup):
        m.cfl_dt(Q, 0.5, dt)
        m.rk_step(Q, dQ, dt)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(steps):
        m.cfl_dt(Q, 0.5, dt)
        m.rk_step(Q, dQ, dt)
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def tune(degrees=(1, 2, 3, 4, 5, 6), target_dof=8e6, steps=6):
    table = {"gpu": torch.cuda.get_device_name(), "target_dof": target_dof, "degrees": {}}
    for p in degrees:
        nv = dg.dg_tile_variant_count(p)
        times = {v: time_variant(p, v, target_dof, steps) for v in range(nv)}
        best = min(times, key=times.get)
        ms = {str(v): t for v, t in times.items()}
        for kind in ("column", "lines"):
            ms[kind] = time_variant(p, kind, target_dof, steps)
        kernel = min(("tile", "column", "lines"),
                     key=lambda k: times[best] if k == "tile" else ms[k])
        dg.dg_set_tile_variant(p, best)
        dg.dg_set_stage_kernel(p, dg.STAGE_KINDS[kernel])
        table["degrees"][str(p)] = {"variant": best, "tile": list(dg.dg_tile_shape(p, best)),
                                    "kernel": kernel, "ms_per_step": ms}
    return table


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=dg.TUNING_PATH)
    ap.add_argument("--degrees", default="1,2,3,4,5,6")
    ap.add_argument("--target-dof", type=float, default=8e6)
    args = ap.parse_args(argv)
    table = tune([int(x) for x in args.degrees.split(",")], args.target_dof)
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    with open(args.out, "w") as f:
        json.dump(table, f, indent=1)
    print(json.dumps(table))
    return 0


if __name__ == "__main__":
    sys.exit(main())
