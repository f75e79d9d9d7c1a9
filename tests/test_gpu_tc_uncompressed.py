"""Uncompressed path with the embedding and fitting GEMMs on the tensor cores (csrc/emb_tc.cu).

TF32 (10-bit mantissa) and BF16 (7-bit) operands with FP32 accumulation, against the FP64
oracle (the network itself, no table): on the tiny two-species model (type-pair nets and one-side
nets, tiles cut short at every net's end), the water model (widths 25/50/100 padded to 32/64/112)
and the metal model (32/64/128), at the realistic force scale (~1 eV/A RMS).  The errors are
those of one rounding of every operand (2^-11 for TF32, 2^-9 for BF16) carried through the
network and the force chain; a wrong layer, skip or gate would give errors of the size of the
forces themselves.
"""
import numpy as np
import pytest

import oracle
from paper_2304_09409_gb300 import inputs as I
from _cases import tiny_frame, tiny_model

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# relative bars (of the largest force / atomic energy) for each operand type
BARS = {"tf32": (1e-2, 1e-3), "bf16": (6e-2, 6e-3)}


def _run(cfg, p, frames, prec):
    from paper_2304_09409_gb300 import dpgb
    m = dpgb.Model(cfg, p, precision=prec)
    out = []
    for fr in frames:
        out.append(m.compute(fr.coord, fr.atype, fr.box, atom_energy=True))
    m.free()
    return out


def _check(cfg, p, frames, prec, tag):
    fbar, ebar = BARS[prec]
    for fr, (e, f, v, ae) in zip(frames, _run(cfg, p, frames, prec)):
        ref = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box)
        fmax = np.abs(ref.force).max()
        ferr = np.abs(f - ref.force).max()
        aerr = np.abs(ae - ref.atom_energy).max()
        escale = np.abs(ref.atom_energy).max()
        verr = np.abs(v - ref.virial).max() / np.abs(ref.virial).max()
        print(f"{tag} {prec}: |dF|max/|F|max {ferr / fmax:.2e} |dEi|max/|Ei|max {aerr / escale:.2e} "
              f"virial rel {verr:.2e} (|F|max {fmax:.3e})")
        assert ferr <= fbar * fmax, (tag, prec, ferr, fmax)
        assert aerr <= ebar * escale, (tag, prec, aerr, escale)
        assert verr <= 10 * fbar


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
@pytest.mark.parametrize("one_side", [0, 1])
def test_tiny_model(prec, one_side):
    cfg = tiny_model(one_side)
    p = I.make_params(cfg, 2)
    _check(cfg, p, [tiny_frame(seed=3), tiny_frame(seed=9, n=75)], prec, f"tiny one_side={one_side}")


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_water192_scaled(prec):
    cfg = I.water_model()
    _check(cfg, I.water_params_scaled(0), [I.water_frame(0)], prec, "water192")


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_fcc256_scaled(prec):
    cfg = I.metal_model()
    _check(cfg, I.metal_params_scaled(0), [I.fcc_frame((4, 4, 4), seed=3)], prec, "fcc256")


def test_fcc32000_sampled_vs_oracle():
    """The 32,000-atom FCC frame of the precision sweep: forces of sampled atoms against the oracle."""
    from paper_2304_09409_gb300 import dpgb
    cfg = I.metal_model()
    p = I.metal_params_scaled(0)
    fr = I.fcc_frame((20, 20, 20), seed=0)
    idx = np.array([0, 777, 12345, 31999])
    f_orc, e_orc = oracle.force_subset(cfg, p, fr.coord, fr.atype, fr.box, idx)
    coord = torch.tensor(fr.coord, device="cuda")
    atype = torch.tensor(fr.atype, device="cuda")
    for prec in ("tf32", "bf16"):
        m = dpgb.Model(cfg, p, precision=prec)
        _, f, _, ae = m.compute(coord, atype, fr.box, atom_energy=True)
        f = f.cpu().numpy()[idx]
        err = np.abs(f - f_orc).max()
        print(f"fcc32000 {prec} uncompressed: |dF|max (sampled, vs oracle) {err:.3e} eV/A")
        assert err <= BARS[prec][0] * 3 * np.abs(f_orc).max()
        m.free()
