"""Evaluate a synthetic workload with one path for a few steps (timing / profiling driver).

  python -m paper_2304_09409_gb300.run --workload water12288 --path fp32-compressed --steps 5

Workloads: water192 (the 192-atom water frame), water12288 (it tiled 4x4x4), water1536
(tiled 2x2x2), fcc32000 (Cu-like FCC, 20^3 cells), fcc4000 (10^3 cells).  Paths: fp64,
fp32, tf32, bf16 (network GEMMs on the tensor cores), fp32-compressed, fp64-compressed, bf16-compressed.  Inputs live on the device; each step is one full
dp_compute (neighbour list included).  Prints the mean device time per step.
"""
from __future__ import annotations

import argparse
import json
import sys

import numpy as np


def workload(name: str):
    from . import inputs as I
    if name.startswith("water"):
        cfg = I.water_model()
        fr = I.water_frame(0)
        reps = {"water192": 1, "water1536": 2, "water12288": 4, "water98304": 8}[name]
        if reps > 1:
            fr = I.replicate(fr, (reps, reps, reps))
    elif name.startswith("fcc"):
        cfg = I.metal_model()
        n = {"fcc4000": 10, "fcc32000": 20}[name]
        fr = I.fcc_frame((n, n, n), seed=0)
    else:
        raise ValueError(name)
    return cfg, I.make_params(cfg, 0), fr


PATHS = {"fp64": ("fp64", False), "fp32": ("fp32", False), "tf32": ("tf32", False), "bf16": ("bf16", False),
         "fp32-compressed": ("fp32", True), "fp64-compressed": ("fp64", True), "bf16-compressed": ("bf16", True)}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="water12288")
    ap.add_argument("--path", default="fp32-compressed", choices=sorted(PATHS))
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=2)
    args = ap.parse_args(argv)
    import torch
    from . import dpgb
    cfg, p, fr = workload(args.workload)
    prec, comp = PATHS[args.path]
    m = dpgb.Model(cfg, p, precision=prec, compressed=comp)
    c = torch.tensor(fr.coord, device="cuda")
    t = torch.tensor(fr.atype, device="cuda")
    out = m.compute(c, t, fr.box)
    for _ in range(args.warmup):
        m.compute(c, t, fr.box, out=out)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        m.compute(c, t, fr.box, out=out)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / max(args.steps, 1)
    print(json.dumps({"workload": args.workload, "natoms": fr.natoms, "path": args.path, "ms_per_step": ms,
                      "atom_evals_per_s": fr.natoms / (ms * 1e-3), "energy": float(out[0].cpu()[0])}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
