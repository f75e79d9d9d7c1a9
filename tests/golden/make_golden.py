"""Writes the stored expected values under tests/golden/ from the FP64 oracle alone.

    python tests/golden/make_golden.py

Every value in the fixtures comes from `oracle/` (brute-force neighbour list, per-atom forward of
Sec. II.A.1-2, hand-written reverse pass for the forces and the virial); the frames and weights come
from the seeded generators of `paper_2304_09409_gb300.inputs`, which hold none of the method's
arithmetic.  The paper prints no worked example with numeric outputs, so no fixture holds a value of
the paper's own.

Format (plain text, one fixture per file): lines starting with '#' are comments; `@case NAME` opens a
case; `@array NAME D0 [D1]` is followed by D0 lines of D1 values (FP64 as %.17e, integers as %d);
`@end` closes the case.  `read()` parses it back into {case: {array: ndarray}}.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))


def _write_array(out, name, a):
    a = np.asarray(a)
    if a.ndim == 0:
        a = a.reshape(1)
    rows = a.reshape(a.shape[0], -1) if a.ndim > 1 else a.reshape(-1, 1)
    dims = f"{a.shape[0]}" if a.ndim == 1 else f"{a.shape[0]} {rows.shape[1]}"
    out.append(f"@array {name} {dims}")
    integer = np.issubdtype(a.dtype, np.integer)
    for r in rows:
        out.append(" ".join(("%d" % v) if integer else ("%.17e" % v) for v in r))


def write(path, header, cases):
    """cases: list of (name, {array name: array}); header: comment lines."""
    out = ["# " + h if h else "#" for h in header]
    for name, arrays in cases:
        out.append(f"@case {name}")
        for k, v in arrays.items():
            _write_array(out, k, v)
        out.append("@end")
    with open(path, "w") as f:
        f.write("\n".join(out) + "\n")


def read(path):
    cases, cur, arr = {}, None, None
    with open(path) as f:
        lines = [ln.rstrip("\n") for ln in f]
    k = 0
    while k < len(lines):
        ln = lines[k]
        k += 1
        if not ln or ln.startswith("#"):
            continue
        if ln.startswith("@case "):
            cur = cases.setdefault(ln.split()[1], {})
        elif ln == "@end":
            cur = None
        elif ln.startswith("@array "):
            parts = ln.split()
            name, d0 = parts[1], int(parts[2])
            d1 = int(parts[3]) if len(parts) > 3 else None
            rows = [lines[k + i].split() for i in range(d0)]
            k += d0
            integer = all("e" not in v and "." not in v for r in rows for v in r)
            arr = np.array([[int(v) if integer else float(v) for v in r] for r in rows],
                           dtype=np.int64 if integer else np.float64)
            cur[name] = arr.reshape(d0) if d1 is None else arr.reshape(d0, d1)
        else:
            raise ValueError(f"{path}:{k}: unexpected line {ln[:40]!r}")
    return cases


def _cases():
    """(fixture file, its header, [(case, model, params, frame, compressed)])."""
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.dirname(HERE))
    from paper_2304_09409_gb300 import inputs as I
    from _cases import (tiny_frame, tiny_model, tiny_model_e3, tiny_model_hybrid, tiny_model_hybrid_e3,
                        tiny_model_r)

    water = I.water_model()
    tiny = [("tiny_se_e2_a", tiny_model()), ("tiny_se_e2_a_one_side", tiny_model(type_one_side=1)),
            ("tiny_se_e2_r", tiny_model_r()), ("tiny_hybrid_se_e2_a_se_e2_r", tiny_model_hybrid()),
            ("tiny_se_e3", tiny_model_e3()), ("tiny_hybrid_se_e2_a_se_e3", tiny_model_hybrid_e3())]
    return [
        ("water192.txt",
         ["192-atom water-like frame (seed 0: O on a jittered 4^3 lattice, two H at 0.96 A, box 12.42 A),",
          "se_e2_a r_c 6, r_s 0.5, sel [46, 92], embedding 25/50/100, M_< 16, fitting 240^3, Xavier-normal",
          "weights from seed 0.  Energy (eV), virial (eV), per-atom energies, forces (eV/A).",
          "water192_network: the embedding net of Eq. (G2) evaluated directly (Sec. II.A.1, II.A.2).",
          "water192_compressed: the same weights through the Eq. (compress) quintic tables (stride 0.01 to",
          "90 % of s_max, 0.1 after)."],
         [("water192_network", water, I.make_params(water, 0), I.water_frame(0), False),
          ("water192_compressed", water, I.make_params(water, 0), I.water_frame(0), True)]),
        ("fcc108.txt",
         ["108-atom Cu-like FCC crystal (3^3 conventional cells, a 3.634 A, jitter 0.05 A, seed 1),",
          "se_e2_a r_c 8, r_s 0.5, sel [512], embedding 32/64/128, M_< 16, fitting 240^3, Xavier-normal",
          "weights from seed 0; the box is narrower than 2 r_c, so each atom sees several images of its",
          "neighbours.  Network embedding (Sec. II.A.1)."],
         [("fcc108_network", I.metal_model(), I.make_params(I.metal_model(), 0), I.fcc_frame((3, 3, 3), seed=1),
           False)]),
        ("tiny14.txt",
         ["14-atom two-species frame (seed 3) in a triclinic cell narrower than 2 r_c, so that images of",
          "one atom and of the centre itself are neighbours; r_c 3.5, sel [12, 20], fitting 12/12,",
          "seed-0 weights, one case per descriptor of Sec. II.A.1 (se_e2_a two-sided and one-sided,",
          "se_e2_r, se_e3 and the two hybrids).  tiny_se_e2_a also stores the brute-force neighbour",
          "list: per centre the sel_t slots of each type, nearest first, -1 padding (nl_j), and each",
          "slot's periodic image (nl_shift, 3 integers per slot, flattened per centre)."],
         [(name, cfg, I.make_params(cfg, 0), tiny_frame(3), False) for name, cfg in tiny]),
    ]


def main():
    sys.path.insert(0, ROOT)
    import oracle

    cmd = "python tests/golden/make_golden.py"
    for fname, header, cases in _cases():
        out = []
        for name, cfg, p, fr, compressed in cases:
            tab = oracle.table_build(cfg, p) if compressed else None
            res = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box, table=tab)
            arrays = {"energy": np.array([res.energy]), "virial": res.virial, "atom_energy": res.atom_energy,
                      "force": res.force}
            if name == "tiny_se_e2_a":
                nl_j, nl_s, _, _ = oracle.nlist(cfg, fr.coord, fr.atype, fr.box)
                arrays["nl_j"] = nl_j
                arrays["nl_shift"] = nl_s.reshape(nl_s.shape[0], -1)
            out.append((name, arrays))
        head = header + ["", "Values: the FP64 oracle's, written by `" + cmd + "` (no GPU involved)."]
        write(os.path.join(HERE, fname), head, out)
        print("wrote", fname)


if __name__ == "__main__":
    main()
