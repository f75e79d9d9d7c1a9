"""The FP64 GPU path, through the C-ABI, against the stored expected values under tests/golden/
(written from the FP64 oracle alone; no oracle code runs here).

Tolerances are those of the FP64 path: |dE|/atom <= 1e-10 eV, |dF| <= 1e-9 eV/A, per-atom energies
within 1e-10 eV, virial within 1e-10 of its largest entry (1e-9 through the compressed tables, whose
interval coefficients the GPU builds itself); the stored neighbour list bit-exact.
"""
import os
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_golden  # noqa: E402

CASES = [(fname, name, cfg, p, fr, comp)
         for fname, _, cases in make_golden._cases() for name, cfg, p, fr, comp in cases]


@pytest.mark.parametrize("fname,name,cfg,p,fr,comp", CASES, ids=[c[1] for c in CASES])
def test_fp64_gpu_matches_stored_oracle_values(fname, name, cfg, p, fr, comp):
    from paper_2304_09409_gb300 import dpgb
    g = make_golden.read(os.path.join(HERE, "golden", fname))[name]
    m = dpgb.Model(cfg, p, precision="fp64", compressed=comp)
    e, f, v, ae = m.compute(fr.coord, fr.atype, fr.box, atom_energy=True)
    assert abs(float(e[0]) - g["energy"][0]) / fr.natoms <= 1e-10
    assert np.abs(ae - g["atom_energy"]).max() <= 1e-10
    assert np.abs(f - g["force"]).max() <= 1e-9
    assert np.abs(v - g["virial"]).max() / np.abs(g["virial"]).max() <= (1e-9 if comp else 1e-10)
    if "nl_j" in g:
        gj, gs = m.build_nlist(fr.coord, fr.atype, fr.box).export()
        np.testing.assert_array_equal(gj, g["nl_j"])
        np.testing.assert_array_equal(np.asarray(gs).reshape(fr.natoms, -1), g["nl_shift"])
    m.free()
