"""Compressed embedding on the tensor cores (interval moments, csrc/mom.cu).

The FP32 mode runs the contraction with BF16 high/low operands in three passes; the mixed
mode with FP16 operands in one pass.  Both are compared with the FP64 compressed path (CUDA
cores, same tables; itself pinned to the oracle's compressed result) on frames that cover
every branch: two-sided and one-sided type nets, M = 16 / 100 / 128 (padded widths 16, 112,
128), tiles cut short at the end of a type, atoms without neighbours, several frames in one
batch, and a full 12,288-atom frame against the oracle's value on sampled atoms.
"""
import numpy as np
import pytest

import oracle
from paper_2304_09409_gb300 import inputs as I
from _cases import tiny_frame, tiny_model

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dp():
    from paper_2304_09409_gb300 import dpgb
    return dpgb


def _pair(cfg, p, frames, prec):
    """(test path, FP64 compressed) results of a batch of frames."""
    dp = _dp()
    nat = np.array([f.natoms for f in frames], dtype=np.int32)
    coord = np.concatenate([f.coord for f in frames])
    atype = np.concatenate([f.atype for f in frames]).astype(np.int32)
    boxes = np.stack([f.box for f in frames])
    m = dp.Model(cfg, p, precision=prec, compressed=True)
    ref = dp.Model(cfg, p, precision="fp64", compressed=True)
    out = dp.compute_batch(m, nat, coord, atype, boxes, atom_energy=True)
    exp = dp.compute_batch(ref, nat, coord, atype, boxes, atom_energy=True)
    return nat, out, exp


def _check(nat, out, exp, f_rel, e_rel, tag):
    e, f, v, ae = out
    e0, f0, v0, ae0 = exp
    fmax = np.abs(f0).max()
    ferr = np.abs(f - f0).max()
    eerr = np.abs(e - e0).max() / nat.min()
    aerr = np.abs(ae - ae0).max()
    escale = max(np.abs(ae0).max(), 1e-12)
    verr = np.abs(v - v0).max() / max(np.abs(v0).max(), 1e-12)
    print(f"{tag}: |dF|max/|F|max={ferr / fmax:.2e} |dE|/atom={eerr:.2e} |dEi|={aerr:.2e} (|Ei| {escale:.2e}) "
          f"virial rel={verr:.2e}")
    assert ferr <= f_rel * fmax, (tag, ferr, fmax)
    assert aerr <= e_rel * escale, (tag, aerr, escale)
    assert verr <= 10 * f_rel, (tag, verr)


@pytest.mark.parametrize("prec,f_rel,e_rel", [("fp32", 1e-4, 1e-5), ("bf16", 3e-2, 3e-3)])
def test_water192(prec, f_rel, e_rel):
    cfg = I.water_model()
    p = I.make_params(cfg, 0)
    nat, out, exp = _pair(cfg, p, [I.water_frame(0)], prec)
    _check(nat, out, exp, f_rel, e_rel, f"water192 {prec}")


@pytest.mark.parametrize("one_side", [0, 1])
def test_tiny_nets_and_ragged_tiles(one_side):
    """M = 16, M_< = 4; 14 + 40 + 75 atoms: type counts that are not multiples of 32.  (FP32
    mode only: the mixed mode's tensor-core fitting net needs widths that are multiples of 16.)"""
    prec, f_rel, e_rel = "fp32", 1e-4, 1e-5
    cfg = tiny_model(one_side)
    p = I.make_params(cfg, 2)
    frames = [tiny_frame(seed=3), tiny_frame(seed=8, n=40), tiny_frame(seed=9, n=75)]
    nat, out, exp = _pair(cfg, p, frames, prec)
    _check(nat, out, exp, f_rel, e_rel, f"tiny one_side={one_side} {prec}")


@pytest.mark.parametrize("prec,f_rel,e_rel", [("fp32", 1e-4, 1e-5), ("bf16", 3e-2, 3e-3)])
def test_metal_m128(prec, f_rel, e_rel):
    cfg = I.metal_model()
    p = I.make_params(cfg, 0)
    nat, out, exp = _pair(cfg, p, [I.fcc_frame((4, 4, 4), seed=3)], prec)
    _check(nat, out, exp, f_rel, e_rel, f"fcc256 {prec}")


def test_isolated_atoms_and_mixed_batch():
    """A frame whose atoms have no neighbours next to dense frames: zero forces there, and the
    dense frames unchanged by the company."""
    cfg = I.water_model()
    p = I.make_params(cfg, 0)
    lone = I.Frame(coord=np.array([[1.0, 1.0, 1.0], [15.0, 15.0, 15.0]]), atype=np.array([0, 1], dtype=np.int32),
                   box=np.eye(3) * 30.0)
    frames = [I.water_frame_n(27, seed=5), lone, I.water_frame(0)]
    nat, out, exp = _pair(cfg, p, frames, "fp32")
    _check(nat, out, exp, 1e-4, 1e-5, "mixed batch fp32")
    f = out[1]
    assert np.abs(f[nat[0]:nat[0] + 2]).max() == 0.0
    dp = _dp()
    m = dp.Model(cfg, p, precision="fp32", compressed=True)
    fr = I.water_frame(0)
    e1, f1, v1, _ = m.compute(fr.coord, fr.atype, fr.box)
    np.testing.assert_allclose(out[1][-fr.natoms:], f1, rtol=0, atol=1e-6 * np.abs(f1).max())


def test_water12288_sampled_vs_oracle():
    """Full-size frame (the bench workload): per-atom energies of sampled atoms against the
    oracle's compressed evaluation of the 192-atom cell (every replica has its environment)."""
    cfg = I.water_model()
    p = I.make_params(cfg, 0)
    small = I.water_frame(0)
    big = I.replicate(small, (4, 4, 4))
    tab = oracle.table_build(cfg, p)
    ref = oracle.compute(cfg, p, small.coord, small.atype, small.box, table=tab)
    for prec, tol in (("fp32", 1e-5), ("bf16", 3e-3)):
        m = _dp().Model(cfg, p, precision=prec, compressed=True)
        e, f, v, ae = m.compute(big.coord, big.atype, big.box, atom_energy=True)
        idx = np.array([0, 5, 191, 192, 4000, 12287])
        scale = np.abs(ref.atom_energy).max()
        assert np.abs(ae[idx] - ref.atom_energy[idx % 192]).max() <= tol * scale, prec
        fs = np.abs(ref.force).max()
        assert np.abs(f[idx] - ref.force[idx % 192]).max() <= (1e-4 if prec == "fp32" else 3e-2) * fs, prec
        assert np.abs(f.sum(0)).max() <= 1e-6 * fs * big.natoms
