"""se_e2_r, se_e3 and hybrid descriptors (Sec. II.A.1) on the GPU's CUDA-core path vs the FP64 oracle.

The hybrids here give their parts different cutoffs and sel (both parts read one list built with
the larger), as the paper's hybrid models do.

Tolerances: FP64 as the se_e2_a path (|dE|/atom <= 1e-10 eV, |dF| <= 1e-9 eV/A, virial relative
<= 1e-10); FP32 on models scaled to forces of about 1 eV/A RMS: |dF| <= 1e-3 eV/A, the total
energy per atom within 1e-6 of its value, single atomic energies within 1e-5 of the largest (FP32
networks and contractions, FP64 accumulation of energy, force, virial).
"""
import numpy as np
import pytest

import oracle
from paper_2304_09409_gb300 import inputs as I

from _cases import tiny_frame, tiny_model_e3, tiny_model_hybrid, tiny_model_hybrid_e3, tiny_model_r

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dp():
    from paper_2304_09409_gb300 import dpgb
    return dpgb


KINDS = ["r", "hybrid", "e3", "hybrid_e3"]


def _tiny(kind, tos=0):
    import dataclasses
    cfg = {"r": tiny_model_r, "hybrid": tiny_model_hybrid, "e3": tiny_model_e3, "hybrid_e3": tiny_model_hybrid_e3}[kind]()
    return dataclasses.replace(cfg, type_one_side=tos)


def _water(kind):
    return {"r": (I.water_model_r(), I.water_r_params_scaled(0)),
            "hybrid": (I.water_model_hybrid(), I.water_hybrid_params_scaled(0)),
            "e3": (I.water_model_e3(), I.water_e3_params_scaled(0)),
            "hybrid_e3": (I.water_model_hybrid_e3(), I.water_hybrid_e3_params_scaled(0))}[kind]


def _assert_fp64(res, ref, natoms):
    e, f, v, ae = res
    assert abs(float(e[0]) - ref.energy) / natoms <= 1e-10
    assert np.abs(f - ref.force).max() <= 1e-9
    assert np.abs(v - ref.virial).max() / max(np.abs(ref.virial).max(), 1e-30) <= 1e-10
    if ae is not None:
        assert np.abs(ae - ref.atom_energy).max() <= 1e-10


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("tos", [0, 1])
@pytest.mark.parametrize("seed", [3, 5])
def test_fp64_tiny_triclinic(kind, tos, seed):
    cfg = _tiny(kind, tos)
    fr = tiny_frame(seed=seed)
    p = I.make_params(cfg, 1)
    ref = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box)
    m = _dp().Model(cfg, p, precision="fp64")
    _assert_fp64(m.compute(fr.coord, fr.atype, fr.box, atom_energy=True), ref, fr.natoms)
    m.free()


@pytest.mark.parametrize("kind", KINDS)
def test_fp64_open_boundary(kind):
    cfg = _tiny(kind)
    fr = tiny_frame(seed=8)
    p = I.make_params(cfg, 2)
    ref = oracle.compute(cfg, p, fr.coord, fr.atype, None)
    m = _dp().Model(cfg, p, precision="fp64")
    _assert_fp64(m.compute(fr.coord, fr.atype, None, atom_energy=True), ref, fr.natoms)
    m.free()


@pytest.mark.parametrize("kind", KINDS)
def test_fp64_water192(kind):
    cfg, p = _water(kind)
    fr = I.water_frame(0)
    ref = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box)
    m = _dp().Model(cfg, p, precision="fp64")
    e, f, v, ae = m.compute(fr.coord, fr.atype, fr.box, atom_energy=True)
    # scaled model: bars relative to its force / energy scale
    assert abs(float(e[0]) - ref.energy) <= 1e-12 * abs(ref.energy)
    assert np.abs(f - ref.force).max() <= 1e-10
    assert np.abs(v - ref.virial).max() <= 1e-12 * np.abs(ref.virial).max()
    m.free()


@pytest.mark.parametrize("kind", KINDS)
def test_fp32_water192_scaled(kind):
    cfg, p = _water(kind)
    fr = I.water_frame(0)
    ref = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box)
    m = _dp().Model(cfg, p, precision="fp32")
    e, f, v, _ = m.compute(fr.coord, fr.atype, fr.box)
    err = np.abs(f - ref.force).max()
    assert err <= 1e-3, err
    assert abs(float(e[0]) - ref.energy) / fr.natoms <= 1e-6 * abs(ref.energy) / fr.natoms
    assert np.abs(v - ref.virial).max() <= 1e-5 * np.abs(ref.virial).max()
    m.free()


@pytest.mark.parametrize("kind", KINDS)
def test_fp32_water12288_sampled(kind):
    """The 12,288-atom water box (the size the throughput figures use): forces of 12 sampled
    atoms and energies of 6 against the oracle's per-atom restriction."""
    cfg, p = _water(kind)
    fr = I.water_frame_n(4096, seed=0)
    m = _dp().Model(cfg, p, precision="fp32")
    e, f, v, ae = m.compute(fr.coord, fr.atype, fr.box, atom_energy=True)
    idx = np.array([0, 1, 2, 777, 2048, 4095, 6000, 8191, 9001, 10000, 12000, 12287], np.int32)
    fs, es = oracle.force_subset(cfg, p, fr.coord, fr.atype, fr.box, idx)
    assert np.abs(f[idx] - fs).max() <= 1e-3
    # FP32 networks on a model with |E_i| of a few hundred eV: 1e-5 relative, as the FP32 se_e2_a path
    assert np.abs(ae[idx[:6]] - es[:6]).max() <= 1e-5 * np.abs(es).max()
    assert np.abs(f.sum(0)).max() <= 1e-6 * fr.natoms
    m.free()


def test_batch_of_frames_equals_alone():
    dpgb = _dp()
    cfg, p = _water("hybrid")
    frames = [I.water_frame_n(n, seed=20 + n) for n in (8, 27, 64)]
    m = dpgb.Model(cfg, p, precision="fp64")
    nat = np.array([fr.natoms for fr in frames], np.int32)
    coord = np.concatenate([fr.coord for fr in frames])
    atype = np.concatenate([fr.atype for fr in frames])
    boxes = np.stack([fr.box for fr in frames])
    e, f, v, _ = dpgb.compute_batch(m, nat, coord, atype, boxes)
    off = 0
    for k, fr in enumerate(frames):
        e1, f1, v1, _ = m.compute(fr.coord, fr.atype, fr.box)
        assert abs(e[k] - e1[0]) <= 1e-12 * abs(e1[0])
        assert np.abs(f[off:off + fr.natoms] - f1).max() <= 1e-11
        assert np.abs(v[k] - v1).max() <= 1e-12 * np.abs(v1).max()
        off += fr.natoms
    m.free()


def test_weight_file_roundtrip(tmp_path):
    dpgb = _dp()
    cfg = _tiny("hybrid")
    p = I.make_params(cfg, 4)
    path = str(tmp_path / "hyb.bin")
    dpgb.write_weight_file(path, cfg, p)
    fr = tiny_frame(seed=3)
    a = dpgb.Model(cfg, p, precision="fp64")
    b = dpgb.Model.from_file(path, cfg, precision="fp64")
    ea, fa, va, _ = a.compute(fr.coord, fr.atype, fr.box)
    eb, fb, vb, _ = b.compute(fr.coord, fr.atype, fr.box)
    # same model, same frame: only the order of the FP64 force atomics may differ
    assert float(ea[0]) == float(eb[0])
    np.testing.assert_allclose(fb, fa, rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose(vb, va, rtol=1e-13, atol=1e-16)
    a.free()
    b.free()


@pytest.mark.parametrize("kind,prec,compressed", [("hybrid", "fp64", True), ("hybrid_e3", "fp32", True),
                                                  ("r", "bf16", False), ("e3", "tf32", False), ("e3", "bf16", True)])
def test_other_paths_refuse(kind, prec, compressed):
    dpgb = _dp()
    cfg = _tiny(kind)
    with pytest.raises(dpgb.DPError) as ei:
        dpgb.Model(cfg, I.make_params(cfg, 0), precision=prec, compressed=compressed)
    assert ei.value.code == dpgb.DP_E_UNSUPPORTED


# ---- compressed se_e2_r and se_e3 (Eq. (compress); se_e3 pieces in theta) -------------------------

@pytest.mark.parametrize("kind", ["r", "e3"])
def test_compressed_tables_equal_oracle(kind):
    dpgb = _dp()
    cfg = _water(kind)[0]
    p = I.make_params(cfg, 0)
    m = dpgb.Model(cfg, p, precision="fp64", compressed=True)
    got = m.export_table()
    x0, h1, n1, h2, n2 = oracle.table_layout(cfg)
    want = oracle.table_build(cfg, p, x0, h1, n1, h2, n2)
    assert got.shape == want.shape
    # the t^5..t^3 coefficients divide node data by dx^5..dx^3 (ulp-level node differences show
    # there magnified): compare the low coefficients, and the pieces where they are used
    np.testing.assert_allclose(got[..., 3:], want[..., 3:], rtol=1e-11, atol=1e-12)
    nodes = np.concatenate([x0 + np.arange(n1 + 1) * h1, x0 + n1 * h1 + np.arange(1, n2 + 1) * h2])
    dx = np.diff(nodes)[None, :, None]
    scale = max(1.0, np.abs(want[..., 5]).max())
    for frac in (0.0, 0.3, 0.7, 1.0):
        t = frac * dx
        g = lambda c: ((((c[..., 0] * t + c[..., 1]) * t + c[..., 2]) * t + c[..., 3]) * t + c[..., 4]) * t + c[..., 5]  # noqa: E731
        assert np.abs(g(got) - g(want)).max() <= 1e-12 * scale
    m.free()


@pytest.mark.parametrize("kind", ["r", "e3"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_compressed_water192_vs_oracle(kind, prec):
    """Against the oracle's compressed result on the same pieces: FP64 to the FP64 bars, FP32 to the
    FP32 ones (forces of ~1 eV/A RMS)."""
    dpgb = _dp()
    cfg, p = _water(kind)
    fr = I.water_frame(0)
    lay = oracle.table_layout(cfg)
    ref = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box, table=oracle.table_build(cfg, p, *lay), table_layout=lay)
    assert ref.status == 0
    m = dpgb.Model(cfg, p, precision=prec, compressed=True)
    e, f, v, ae = m.compute(fr.coord, fr.atype, fr.box, atom_energy=True)
    if prec == "fp64":
        assert abs(float(e[0]) - ref.energy) <= 1e-12 * abs(ref.energy)
        assert np.abs(f - ref.force).max() <= 1e-10
        assert np.abs(v - ref.virial).max() <= 1e-12 * np.abs(ref.virial).max()
    else:
        assert np.abs(f - ref.force).max() <= 1e-3
        assert abs(float(e[0]) - ref.energy) / fr.natoms <= 1e-6 * abs(ref.energy) / fr.natoms
        assert np.abs(v - ref.virial).max() <= 1e-5 * np.abs(ref.virial).max()
    m.free()


@pytest.mark.parametrize("kind", ["r", "e3"])
def test_compressed_tiny_triclinic_fp64(kind):
    dpgb = _dp()
    cfg = _tiny(kind)
    fr = tiny_frame(seed=5)
    p = I.make_params(cfg, 1)
    lay = oracle.table_layout(cfg)
    ref = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box, table=oracle.table_build(cfg, p, *lay), table_layout=lay)
    m = dpgb.Model(cfg, p, precision="fp64", compressed=True)
    _assert_fp64(m.compute(fr.coord, fr.atype, fr.box, atom_energy=True), ref, fr.natoms)
    m.free()


def test_param_grad_refuses():
    dpgb = _dp()
    cfg = _tiny("hybrid")
    fr = tiny_frame(seed=3)
    m = dpgb.Model(cfg, I.make_params(cfg, 0), precision="fp64")
    with pytest.raises(dpgb.DPError) as ei:
        dpgb.param_grad(m, [fr.natoms], fr.coord, fr.atype, fr.box[None], np.ones(1), np.zeros((fr.natoms, 3)))
    assert ei.value.code == dpgb.DP_E_UNSUPPORTED
    m.free()


# ---- one neighbour type: every pair of the se_e3 part has one net both ways ---------------------

def _single_type(descriptor, embed):
    return I.ModelConfig(ntypes=1, rcut=5.0, rcut_smth=0.5, sel=(64,), embed=embed, axis=0, fit=(16, 16),
                         descriptor=descriptor)


@pytest.mark.parametrize("descriptor,embed", [(3, (2, 4, 8)), (3, (3, 6, 12)), (1, (10, 20, 40)), (1, (5, 10, 20))])
def test_single_type_fcc_vs_oracle(descriptor, embed):
    """A 108-atom FCC box with ~44 neighbours per atom in one type block: the se_e3 kernels take
    every pair once with weight 2 (rows of 32 partners and more, and shorter ones), and the se_e2_r
    kernel its nets on the same neighbours; fixed-shape and general evaluators, FP64 against the
    oracle and FP32 within 1e-4 of the force scale."""
    cfg = _single_type(descriptor, embed)
    fr = I.fcc_frame((3, 3, 3), seed=11)
    p = I.make_params(cfg, 3)
    ref = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box)
    m = _dp().Model(cfg, p, precision="fp64")
    _assert_fp64(m.compute(fr.coord, fr.atype, fr.box, atom_energy=True), ref, fr.natoms)
    m.free()
    m = _dp().Model(cfg, p, precision="fp32")
    e, f, v, _ = m.compute(fr.coord, fr.atype, fr.box)
    fs = np.abs(ref.force).max()
    assert np.abs(f - ref.force).max() <= 1e-4 * fs
    assert abs(float(e[0]) - ref.energy) <= 1e-5 * max(abs(ref.energy), 1.0)
    m.free()
