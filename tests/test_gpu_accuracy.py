"""Accuracy of every precision path at a realistic force scale (about 1 eV/A RMS).

The seed-0 random-weight models have tiny forces (5e-4 eV/A RMS for water, 8e-6 for the FCC
metal), so an absolute bar of 1e-3 eV/A says nothing there.  These tests use the force-scaled
variants (the output layer multiplied so that the force RMS is about 1 eV/A; energies, forces
and virials scale exactly) and hold each path to the oracle:

  FP64 path                       |dF| <= 1e-9 eV/A
  FP32 compressed (split tensor-core fitting, three-pass moment contraction)
                                  |dF| <= 1e-3 eV/A   (the mixed-precision bar)
  BF16 compressed                 reported, held only to 10 % of the force RMS: it does not
                                  meet 1e-3 eV/A at this scale (one BF16 rounding is 2^-9)

on the 192-atom water frame (full oracle), the 12,288-atom tiled water frame (every replica
has the environment of the 192-atom cell) and the 32,000-atom FCC frame (oracle forces of
sampled atoms).
"""
import numpy as np
import pytest

import oracle
from paper_2304_09409_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

BAR = 1e-3  # eV/A, mixed-precision force bar


def _dp():
    from paper_2304_09409_gb300 import dpgb
    return dpgb


@pytest.fixture(scope="module")
def water_ref():
    cfg = I.water_model()
    p = I.water_params_scaled(0)
    fr = I.water_frame(0)
    ref = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box)
    return cfg, p, fr, ref


def _errs(f, e, fref, eref, n):
    return float(np.abs(f - fref).max()), abs(float(e) - eref) / n


@pytest.mark.parametrize("prec,compressed", [("fp64", False), ("fp32", False), ("fp32", True), ("bf16", True)])
def test_water192_scaled(water_ref, prec, compressed):
    cfg, p, fr, ref = water_ref
    frms = float(np.sqrt((ref.force ** 2).mean()))
    assert 0.7 < frms < 1.5
    m = _dp().Model(cfg, p, precision=prec, compressed=compressed)
    e, f, v, _ = m.compute(fr.coord, fr.atype, fr.box)
    ferr, eerr = _errs(f, e[0], ref.force, ref.energy, fr.natoms)
    verr = float(np.abs(v - ref.virial).max())
    print(f"water192 x{I.WATER_FORCE_SCALE:g} {prec}{' compressed' if compressed else ''}: F rms {frms:.3f} "
          f"|dF|max {ferr:.3e} ({ferr / frms:.2e} of rms) |dE|/atom {eerr:.3e} |dXi|max {verr:.3e}")
    if prec == "fp64":
        assert ferr <= 1e-9
        assert eerr <= 1e-10 * I.WATER_FORCE_SCALE  # energies scale with the output layer
    elif prec == "fp32":
        assert ferr <= BAR
    else:
        assert ferr <= 0.1 * frms
    m.free()


def test_water12288_scaled_fp32_compressed(water_ref):
    """The benchmark's water workload at the realistic force scale: the FP32 compressed path
    (split tensor-core fitting net) within the bar everywhere against the oracle."""
    cfg, p, fr, ref = water_ref
    big = I.replicate(fr, (4, 4, 4))
    m = _dp().Model(cfg, p, precision="fp32", compressed=True)
    e, f, v, ae = m.compute(big.coord, big.atype, big.box, atom_energy=True)
    ferr = float(np.abs(f - np.tile(ref.force, (64, 1))).max())
    print(f"water12288 fp32 compressed: |dF|max {ferr:.3e} eV/A")
    assert ferr <= BAR
    np.testing.assert_allclose(v, 64 * ref.virial, rtol=0, atol=64 * 1e-3 * np.abs(ref.virial).max())
    m.free()


def test_fcc32000_scaled_sampled_vs_oracle():
    """The 32,000-atom FCC metal frame at about 1 eV/A RMS: forces of sampled atoms against the
    oracle (their neighbourhoods by brute force), and every force against the FP64 GPU path."""
    dp = _dp()
    cfg = I.metal_model()
    p = I.metal_params_scaled(0)
    fr = I.fcc_frame((20, 20, 20), seed=0)
    idx = np.array([0, 777, 12345, 20000, 31999])
    f_orc, e_orc = oracle.force_subset(cfg, p, fr.coord, fr.atype, fr.box, idx, nthreads=0)
    coord = torch.tensor(fr.coord, device="cuda")
    atype = torch.tensor(fr.atype, device="cuda")
    m64 = dp.Model(cfg, p, precision="fp64")
    _, f64, _, ae64 = m64.compute(coord, atype, fr.box, atom_energy=True)
    f64 = f64.cpu().numpy()
    m64.free()
    assert np.abs(f64[idx] - f_orc).max() <= 1e-9
    np.testing.assert_allclose(ae64.cpu().numpy()[idx], e_orc, rtol=1e-12)
    frms = float(np.sqrt((f64 ** 2).mean()))
    assert 0.7 < frms < 1.5
    for prec in ("fp32", "bf16"):
        m = dp.Model(cfg, p, precision=prec, compressed=True)
        _, f, _, _ = m.compute(coord, atype, fr.box)
        f = f.cpu().numpy()
        e_all = float(np.abs(f - f64).max())
        e_smp = float(np.abs(f[idx] - f_orc).max())
        print(f"fcc32000 {prec} compressed: F rms {frms:.3f} |dF|max vs FP64 GPU {e_all:.3e}, "
              f"vs oracle (sampled) {e_smp:.3e}")
        if prec == "fp32":
            assert e_all <= BAR and e_smp <= BAR
        else:
            assert e_all <= 0.1 * frms * 3  # BF16: reported; the FCC forces amplify its rounding more
        m.free()
