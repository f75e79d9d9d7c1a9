"""Evaluate a synthetic workload with one path for a few steps (timing / profiling driver).

  python -m paper_2304_09409_gb300.run --workload water12288 --path fp32-compressed --steps 5

Workloads: water192 (the 192-atom water frame), water12288 (it tiled 4x4x4), water1536
(tiled 2x2x2), fcc32000 (Cu-like FCC, 20^3 cells), fcc4000 (10^3 cells); a water workload with the
suffix -r, -hybrid, -e3 or -hybrid_e3 takes the se_e2_r, se_e2_a + se_e2_r, se_e3 or
se_e2_a + se_e3 model of the inputs module instead.  Paths: fp64,
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
        base, _, desc = name.partition("-")
        cfg = {"": I.water_model, "r": I.water_model_r, "hybrid": I.water_model_hybrid, "e3": I.water_model_e3,
               "hybrid_e3": I.water_model_hybrid_e3}[desc]()
        fr = I.water_frame(0)
        reps = {"water192": 1, "water1536": 2, "water12288": 4, "water98304": 8}[base]
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


# Kernel scopes of the path (the names dp_profile_read reports) and the kernels and sources of each.
SCOPES = {
    "nlist": (("k_bin", "k_fill_scan", "k_scan_excl", "k_fill", "k_nlist_cell", "k_nlist"), ("nlist.cu", "dp_internal.cuh")),
    "env": (("k_env_mom",), ("mom.cu", "mom.cuh", "tc_ptx.cuh", "env.cuh", "dp_internal.cuh")),
    "mom_fwd": (("k_mom_fwd",), ("mom.cu", "mom.cuh", "tc_ptx.cuh", "env.cuh", "dp_internal.cuh")),
    "mom_gT": (("k_mom_gT",), ("mom.cu", "mom.cuh", "tc_ptx.cuh", "env.cuh", "dp_internal.cuh")),
    "mom_bwd": (("k_mom_bwd",), ("mom.cu", "mom.cuh", "tc_ptx.cuh", "env.cuh", "dp_internal.cuh")),
    "mom_force": (("k_force_mom",), ("mom.cu", "mom.cuh", "tc_ptx.cuh", "env.cuh", "dp_internal.cuh")),
    "fit_split_tc": (("k_fit_split",), ("fit_split.cu", "fit_tc.cuh", "tc_ptx.cuh", "dp_internal.cuh")),
    "fit_fused_tc": (("k_fit_fused",), ("fit_fused.cu", "fit_tc.cuh", "tc_ptx.cuh", "dp_internal.cuh")),
    "frame_sums": (("k_chunk_sums",), ("driver.cu",)),
    "e3_fwd": (("k_e3",), ("path.cu", "path.cuh", "env.cuh", "tabeval.cuh", "dp_internal.cuh")),
    "e3_bwd": (("k_e3",), ("path.cu", "path.cuh", "env.cuh", "tabeval.cuh", "dp_internal.cuh")),
}


def src_hash(names) -> str:
    """Hash of the CUDA sources a kernel scope is built from."""
    import hashlib
    import os
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc")
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(here, n), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _kernel_base(name: str) -> str:
    """Kernel name with its template arguments, without namespaces and parameters."""
    base = name.split("(")[0].strip()
    for pre in ("void ", "unnamed>::", "(anonymous namespace)::", "dpgb::"):
        base = base.replace(pre, "")
    return base.strip()


def ncu_summary(csv_paths, steps: int, command: str):
    """Per-kernel launches, device time and share (and DRAM bytes per launch where the capture has
    them) from ncu --csv logs; returns (markdown table, {scope: traffic record})."""
    import csv
    import io
    times, dram, launches, full = {}, {}, {}, {}
    for path in csv_paths:
        text = open(path).read()
        lines = text.splitlines()
        start = next(k for k, ln in enumerate(lines) if ln.startswith('"ID"'))
        for row in csv.DictReader(io.StringIO("\n".join(lines[start:]))):
            name = row["Kernel Name"]
            base = _kernel_base(name)
            key = (path, row["ID"])
            unit = row.get("Metric Unit", "")
            try:
                val = float(row["Metric Value"].replace(",", ""))
            except ValueError:
                continue
            metric = row["Metric Name"]
            if metric == "gpu__time_duration.sum":
                scale = {"ns": 1e-3, "nsecond": 1e-3, "us": 1.0, "usecond": 1.0, "ms": 1e3, "msecond": 1e3,
                         "s": 1e6, "second": 1e6}.get(unit, 1.0)
                times.setdefault(base, {})[key] = val * scale
                full[base] = name.split("(")[0].replace("void ", "").replace("unnamed>::", "")
            elif metric in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
                scale = {"byte": 1.0, "B": 1.0, "Kbyte": 1e3, "KB": 1e3, "Mbyte": 1e6, "MB": 1e6, "Gbyte": 1e9,
                         "GB": 1e9}.get(unit, 1.0)
                dram.setdefault(base, {}).setdefault(key, 0.0)
                dram[base][key] += val * scale
    total = sum(sum(v.values()) for v in times.values()) or 1.0
    out = ["| kernel | launches | total us | us/launch | share | DRAM MB/launch |", "|---|---:|---:|---:|---:|---:|"]
    for base, v in sorted(times.items(), key=lambda kv: -sum(kv[1].values())):
        t = sum(v.values())
        d = dram.get(base)
        dm = f"{sum(d.values()) / len(d) / 1e6:.2f}" if d else "-"
        out.append(f"| {base} | {len(v)} | {t:.1f} | {t / len(v):.1f} | {100 * t / total:.1f}% | {dm} |")
    out.append(f"\nTotal {total:.1f} us.")
    traffic = {}
    for scope, (kernels, sources) in SCOPES.items():
        names = [b for b in dram if b.split("<")[0] in kernels]
        per = [sum(dram[b].values()) / len(dram[b]) for b in names]
        if per:
            traffic[scope] = {"dram_bytes_per_launch": float(sum(per)), "kernels": " + ".join(names),
                              "sources": list(sources), "src_hash": src_hash(sources), "command": command,
                              "per": "one step (all launches of the scope)"}
    return "\n".join(out), traffic


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="water12288")
    ap.add_argument("--path", default="fp32-compressed", choices=sorted(PATHS))
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--ncu-summary", nargs="+", default=None,
                    help="summarise ncu --csv logs (launch list; DRAM bytes where captured) instead of running")
    ap.add_argument("--md", default=None, help="with --ncu-summary: write the markdown table here")
    ap.add_argument("--traffic", default=None, help="with --ncu-summary: merge DRAM bytes per scope into this JSON")
    ap.add_argument("--command", default="", help="with --ncu-summary: the capture command, recorded with the figures")
    args = ap.parse_args(argv)
    if args.ncu_summary:
        import os
        md, traffic = ncu_summary(args.ncu_summary, args.steps, args.command)
        if args.md:
            with open(args.md, "w") as fh:
                fh.write(md + "\n")
        else:
            print(md)
        if args.traffic:
            old = {}
            if os.path.exists(args.traffic):
                with open(args.traffic) as fh:
                    old = json.load(fh)
            old.update(traffic)
            with open(args.traffic, "w") as fh:
                json.dump(old, fh, indent=1)
        return 0
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
