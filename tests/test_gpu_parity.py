"""GPU path vs the FP64 CPU oracle, through the C-ABI (libdpgb.so).

Tolerances (from the contract of this path):
  FP64 network path   |dE|/atom <= 1e-10 eV, |dF| <= 1e-9 eV/A, virial relative <= 1e-10
  FP32 network path   |dF| <= 1e-3 eV/A absolute; we also hold it to 1e-4 relative to the
                      force RMS, because the random-weight models here have small forces
  neighbour lists     bit-exact (same j and same image for every slot)
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


@pytest.fixture(scope="module")
def water():
    cfg = I.water_model()
    p = I.make_params(cfg, 0)
    fr = I.water_frame(0)
    ref = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box)
    return cfg, p, fr, ref


def _assert_fp64(res, ref, natoms):
    e, f, v, ae = res
    assert abs(float(e[0]) - ref.energy) / natoms <= 1e-10
    assert np.abs(f - ref.force).max() <= 1e-9
    scale = max(np.abs(ref.virial).max(), 1e-30)
    assert np.abs(v - ref.virial).max() / scale <= 1e-10
    if ae is not None:
        assert np.abs(ae - ref.atom_energy).max() <= 1e-10


def _assert_fp32(res, ref, natoms, rel=1e-4):
    e, f, v, ae = res
    frms = np.sqrt((ref.force ** 2).mean())
    err = np.abs(f - ref.force).max()
    assert err <= 1e-3
    assert err <= rel * max(frms, 1e-12) * 10, (err, frms)
    assert abs(float(e[0]) - ref.energy) / natoms <= 1e-5
    assert np.abs(v - ref.virial).max() <= rel * max(np.abs(ref.virial).max(), 1e-12) * 10


# ---------------------------------------------------------------------------------------------
# neighbour lists: bit-exact
# ---------------------------------------------------------------------------------------------

def _nl_cases():
    out = []
    for seed, tri in ((3, True), (4, False), (5, True)):
        fr = tiny_frame(seed=seed, triclinic=tri)
        c = fr.coord.copy()
        c[0] += 2 * fr.box[0] - 3 * fr.box[2]
        c[5] -= fr.box[1]
        out.append((f"tiny{seed}", tiny_model(), I.Frame(c, fr.atype, fr.box)))
    out.append(("water192", I.water_model(), I.water_frame(0)))
    out.append(("fcc256", I.metal_model(), I.fcc_frame((4, 4, 4), seed=1)))
    out.append(("water24", I.water_model(), I.water_frame_n(8, seed=2)))
    return out


@pytest.mark.parametrize("name,cfg,fr", _nl_cases(), ids=[c[0] for c in _nl_cases()])
def test_nlist_bit_exact(name, cfg, fr):
    dpgb = _dp()
    m = dpgb.Model(cfg, I.make_params(cfg, 0), precision="fp64")
    nl = m.build_nlist(fr.coord, fr.atype, fr.box)
    gj, gs = nl.export()
    rj, rs, counts, ov = oracle.nlist(cfg, fr.coord, fr.atype, fr.box)
    assert nl.n_overflow == ov
    np.testing.assert_array_equal(gj, rj)
    np.testing.assert_array_equal(gs, rs)


# Frames built to reach the rarely taken branches of the list builder: exact and near-exact
# distance ties (ordered by j, then image, under the exact FP64 r^2), pairs at r_c and within
# 1e-15 .. 1e-4 of it (the FP64 membership test), coincident atoms (r = 0), coordinates a
# thousand boxes away from the origin, and cells so large that the FP32 screening window is
# widest.
def _shell_frame():
    rng = np.random.default_rng(11)
    L, rc = 20.0, 6.0
    c0 = np.array([5.0, 5.0, 5.0])
    pts = [c0, c0 + [6, 0, 0], c0 + [0, 6, 0], c0 + [0, 0, -6], c0 + [3, 4, 0], c0 + [4, 3, 0], c0 + [0, 5, 0],
           c0 + [0, 0, 5], c0 + [-5, 0, 0], c0 + 6 / np.sqrt(3) * np.ones(3)]
    for rel in (1e-15, 1e-12, 1e-9, 1e-7, 1e-6, 1e-5, 1e-4):
        for sgn in (-1.0, 1.0):
            u = rng.normal(size=3)
            u /= np.linalg.norm(u)
            pts.append(c0 + u * rc * (1 + sgn * rel))
    # the same distances across the periodic boundary
    c1 = np.array([L - 1.0, 10.0, 10.0])
    pts += [c1, c1 + [6, 0, 0], c1 + [6 * (1 + 1e-12), 0, 0], c1 + [6 * (1 - 1e-12), 0, 0.0]]
    coord = np.array(pts, dtype=np.float64)
    atype = (np.arange(len(pts)) % 2).astype(np.int32)
    cfg = I.ModelConfig(ntypes=2, rcut=rc, rcut_smth=0.5, sel=(24, 24), embed=(4, 8, 16), axis=4, fit=(12, 12))
    return cfg, I.Frame(coord, atype, np.eye(3) * L)


def _hard_nl_cases():
    out = []
    out.append(("fcc_perfect_images", I.metal_model(), I.fcc_frame((3, 3, 3), sigma=0.0, seed=0)))
    out.append(("fcc_perfect", I.metal_model(), I.fcc_frame((5, 5, 5), sigma=0.0, seed=0)))
    cfg, fr = _shell_frame()
    out.append(("cutoff_shell", cfg, fr))
    w = I.water_frame(0)
    dup = np.concatenate([w.coord, w.coord[:10]])
    out.append(("water_coincident", I.water_model(),
                I.Frame(dup, np.concatenate([w.atype, w.atype[:10]]).astype(np.int32), w.box)))
    out.append(("water_far_images", I.water_model(),
                I.Frame(w.coord + 1000 * w.box[0] - 700 * w.box[1] + 3 * w.box[2], w.atype, w.box)))
    rng = np.random.default_rng(5)
    centres = rng.uniform(0, 3000.0, size=(20, 3))
    pts = (centres[:, None, :] + rng.uniform(-4, 4, size=(20, 12, 3))).reshape(-1, 3)
    out.append(("sparse_3000A", I.water_model(),
                I.Frame(pts, (np.arange(len(pts)) % 2).astype(np.int32), np.eye(3) * 3000.0)))
    return out


@pytest.mark.parametrize("name,cfg,fr", _hard_nl_cases(), ids=[c[0] for c in _hard_nl_cases()])
def test_nlist_ties_cutoff_and_extremes_bit_exact(name, cfg, fr):
    dpgb = _dp()
    m = dpgb.Model(cfg, I.make_params(cfg, 0), precision="fp64")
    nl = m.build_nlist(fr.coord, fr.atype, fr.box)
    gj, gs = nl.export()
    rj, rs, counts, ov = oracle.nlist(cfg, fr.coord, fr.atype, fr.box)
    assert nl.n_overflow == ov
    np.testing.assert_array_equal(gj, rj)
    np.testing.assert_array_equal(gs, rs)


def test_nlist_open_boundary_bit_exact():
    dpgb = _dp()
    cfg = tiny_model()
    fr = tiny_frame(seed=7)
    m = dpgb.Model(cfg, I.make_params(cfg, 0), precision="fp64")
    nl = m.build_nlist(fr.coord, fr.atype, None)
    gj, gs = nl.export()
    rj, rs, _, _ = oracle.nlist(cfg, fr.coord, fr.atype, None)
    np.testing.assert_array_equal(gj, rj)
    np.testing.assert_array_equal(gs, rs)


def test_nlist_overflow_reported_and_truncated():
    dpgb = _dp()
    cfg = I.ModelConfig(ntypes=2, rcut=3.5, rcut_smth=0.5, sel=(3, 4), embed=(4, 8, 16), axis=4, fit=(12, 12))
    fr = tiny_frame(seed=6)
    m = dpgb.Model(cfg, I.make_params(cfg, 0), precision="fp64")
    nl = m.build_nlist(fr.coord, fr.atype, fr.box)
    rj, rs, counts, ov = oracle.nlist(cfg, fr.coord, fr.atype, fr.box)
    assert ov > 0 and nl.n_overflow == ov
    gj, gs = nl.export()
    np.testing.assert_array_equal(gj, rj)
    np.testing.assert_array_equal(gs, rs)


def _dense_clump():
    """1331 atoms on a jittered 1.75 A lattice (about twice water's density) in one corner of an
    otherwise empty 60 A box: the cells around the clump hold far more candidates than the mean
    density of the box predicts, so the cell-centred search reports that its staging buffer is
    too small and the call is retried on the per-atom kernel."""
    rng = np.random.default_rng(11)
    g = np.arange(11) * 1.75
    lat = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    pts = lat + rng.uniform(-0.3, 0.3, lat.shape) + 20.0
    cfg = I.ModelConfig(ntypes=2, rcut=6.0, rcut_smth=0.5, sel=(200, 200), embed=(8, 16, 32), axis=4,
                        fit=(32, 32))
    return cfg, I.Frame(pts, (np.arange(len(pts)) % 2).astype(np.int32), np.eye(3) * 60.0)


def test_nlist_dense_clump_bit_exact():
    dpgb = _dp()
    cfg, fr = _dense_clump()
    m = dpgb.Model(cfg, I.make_params(cfg, 0), precision="fp64")
    nl = m.build_nlist(fr.coord, fr.atype, fr.box)
    gj, gs = nl.export()
    rj, rs, counts, ov = oracle.nlist(cfg, fr.coord, fr.atype, fr.box)
    assert ov == 0 and nl.n_overflow == 0
    np.testing.assert_array_equal(gj, rj)
    np.testing.assert_array_equal(gs, rs)


def test_fp64_dense_clump():
    """The kernels after the list run on the first (reported, retried) attempt too: the rows the
    cell-centred search could not fill must be left empty, not uninitialised."""
    cfg, fr = _dense_clump()
    p = I.make_params(cfg, 0)
    ref = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box)
    m = _dp().Model(cfg, p, precision="fp64")
    _assert_fp64(m.compute(fr.coord, fr.atype, fr.box, atom_energy=True), ref, fr.natoms)


# ---------------------------------------------------------------------------------------------
# FP64 path: energy, forces, virial
# ---------------------------------------------------------------------------------------------

def test_fp64_water192(water):
    cfg, p, fr, ref = water
    m = _dp().Model(cfg, p, precision="fp64")
    _assert_fp64(m.compute(fr.coord, fr.atype, fr.box, atom_energy=True), ref, fr.natoms)


@pytest.mark.parametrize("tos", [0, 1])
@pytest.mark.parametrize("seed", [3, 5])
def test_fp64_tiny_triclinic(tos, seed):
    cfg = tiny_model(type_one_side=tos)
    fr = tiny_frame(seed=seed)
    p = I.make_params(cfg, 1)
    ref = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box)
    m = _dp().Model(cfg, p, precision="fp64")
    _assert_fp64(m.compute(fr.coord, fr.atype, fr.box, atom_energy=True), ref, fr.natoms)


def test_fp64_open_boundary():
    cfg = tiny_model()
    fr = tiny_frame(seed=8)
    p = I.make_params(cfg, 2)
    ref = oracle.compute(cfg, p, fr.coord, fr.atype, None)
    m = _dp().Model(cfg, p, precision="fp64")
    _assert_fp64(m.compute(fr.coord, fr.atype, None, atom_energy=True), ref, fr.natoms)


def test_fp64_fcc_metal_small():
    cfg = I.metal_model()
    fr = I.fcc_frame((4, 4, 4), seed=1)
    p = I.make_params(cfg, 0)
    ref = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box)
    m = _dp().Model(cfg, p, precision="fp64")
    _assert_fp64(m.compute(fr.coord, fr.atype, fr.box), ref, fr.natoms)


def test_device_and_host_pointers_agree(water):
    cfg, p, fr, ref = water
    m = _dp().Model(cfg, p, precision="fp64")
    eh, fh, vh, _ = m.compute(fr.coord, fr.atype, fr.box)
    c = torch.tensor(fr.coord, device="cuda")
    t = torch.tensor(fr.atype, device="cuda")
    ed, fd, vd, _ = m.compute(c, t, fr.box)
    torch.cuda.synchronize()
    assert abs(float(ed.cpu()[0]) - float(eh[0])) <= 1e-12 * fr.natoms
    assert np.abs(fd.cpu().numpy() - fh).max() <= 1e-12
    assert np.abs(vd.cpu().numpy() - vh).max() <= 1e-12


def test_external_nlist_equals_internal(water):
    cfg, p, fr, ref = water
    m = _dp().Model(cfg, p, precision="fp64")
    nl = m.build_nlist(fr.coord, fr.atype, fr.box)
    _assert_fp64(m.compute(fr.coord, fr.atype, fr.box, nlist=nl), ref, fr.natoms)


def test_single_atom_and_isolated_atoms():
    """Degenerate cases: one atom in a periodic cell (only its own images are neighbours),
    and an open-boundary frame with an atom that has no neighbour at all."""
    cfg = tiny_model()
    p = I.make_params(cfg, 3)
    coord = np.array([[0.3, 0.2, 0.1]])
    atype = np.array([1], np.int32)
    box = np.eye(3) * 3.0
    ref = oracle.compute(cfg, p, coord, atype, box)
    m = _dp().Model(cfg, p, precision="fp64")
    _assert_fp64(m.compute(coord, atype, box), ref, 1)
    coord = np.array([[0.0, 0.0, 0.0], [1.1, 0.2, 0.0], [50.0, 50.0, 50.0]])
    atype = np.array([0, 1, 0], np.int32)
    ref = oracle.compute(cfg, p, coord, atype, None)
    _assert_fp64(m.compute(coord, atype, None, atom_energy=True), ref, 3)


def test_bad_type_is_an_error():
    dpgb = _dp()
    cfg = tiny_model()
    fr = tiny_frame(seed=3)
    m = dpgb.Model(cfg, I.make_params(cfg, 0), precision="fp64")
    bad = fr.atype.copy()
    bad[2] = 5
    with pytest.raises(dpgb.DPError) as ei:
        m.compute(fr.coord, bad, fr.box)
    assert ei.value.code == dpgb.DP_E_ARG
    badd = torch.tensor(bad, device="cuda")
    with pytest.raises(dpgb.DPError) as ei:
        m.compute(torch.tensor(fr.coord, device="cuda"), badd, fr.box)
    assert ei.value.code == dpgb.DP_E_ARG


# ---------------------------------------------------------------------------------------------
# FP32 path
# ---------------------------------------------------------------------------------------------

def test_fp32_water192(water):
    cfg, p, fr, ref = water
    m = _dp().Model(cfg, p, precision="fp32")
    _assert_fp32(m.compute(fr.coord, fr.atype, fr.box), ref, fr.natoms)


def test_fp32_tiny():
    cfg = tiny_model()
    fr = tiny_frame(seed=3)
    p = I.make_params(cfg, 1)
    ref = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box)
    m = _dp().Model(cfg, p, precision="fp32")
    _assert_fp32(m.compute(fr.coord, fr.atype, fr.box), ref, fr.natoms)


# ---------------------------------------------------------------------------------------------
# Compressed path (Eq. (compress))
# ---------------------------------------------------------------------------------------------

def test_table_matches_oracle_table():
    cfg = I.water_model()
    p = I.make_params(cfg, 0)
    m = _dp().Model(cfg, p, precision="fp64", compressed=True)
    gt = m.export_table()
    ot = oracle.table_build(cfg, p)
    assert gt.shape == ot.shape
    # The t^5..t^3 coefficients divide node data by dx^5..dx^3, so ulp-level differences in
    # the node values appear there magnified; compare the pieces where they are used instead.
    nodes = np.concatenate([np.arange(181) * 0.01, 1.8 + np.arange(1, 3) * 0.1])
    dx = np.diff(nodes)[None, :, None]
    np.testing.assert_allclose(gt[..., 3:], ot[..., 3:], rtol=1e-11, atol=1e-12)
    for frac in (0.0, 0.3, 0.7, 1.0):
        t = frac * dx
        g = lambda c: ((((c[..., 0] * t + c[..., 1]) * t + c[..., 2]) * t + c[..., 3]) * t + c[..., 4]) * t + c[..., 5]
        gp = lambda c: (((5 * c[..., 0] * t + 4 * c[..., 1]) * t + 3 * c[..., 2]) * t + 2 * c[..., 3]) * t + c[..., 4]
        assert np.abs(g(gt) - g(ot)).max() <= 1e-12
        assert np.abs(gp(gt) - gp(ot)).max() <= 1e-9


def test_compressed_fp64_vs_oracle_compressed(water):
    cfg, p, fr, _ = water
    tab = oracle.table_build(cfg, p)
    ref = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box, table=tab)
    m = _dp().Model(cfg, p, precision="fp64", compressed=True)
    res = m.compute(fr.coord, fr.atype, fr.box, atom_energy=True)
    e, f, v, ae = res
    assert abs(float(e[0]) - ref.energy) / fr.natoms <= 1e-10
    assert np.abs(f - ref.force).max() <= 1e-9
    assert np.abs(v - ref.virial).max() / np.abs(ref.virial).max() <= 1e-9


def test_compressed_fp32_vs_oracle(water):
    cfg, p, fr, ref = water
    m = _dp().Model(cfg, p, precision="fp32", compressed=True)
    _assert_fp32(m.compute(fr.coord, fr.atype, fr.box), ref, fr.natoms)


def test_compressed_tiny_type_one_side():
    cfg = tiny_model(type_one_side=1)
    fr = tiny_frame(seed=5)
    p = I.make_params(cfg, 4)
    tab = oracle.table_build(cfg, p)
    ref = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box, table=tab)
    m = _dp().Model(cfg, p, precision="fp64", compressed=True)
    e, f, v, _ = m.compute(fr.coord, fr.atype, fr.box)
    assert abs(float(e[0]) - ref.energy) / fr.natoms <= 1e-10
    assert np.abs(f - ref.force).max() <= 1e-9


# ---------------------------------------------------------------------------------------------
# Full-size frames: properties that hold at any size, plus sampled oracle values
# ---------------------------------------------------------------------------------------------

def test_water12288_is_64_replicas(water):
    """The 12,288-atom box is the 192-atom frame tiled 4x4x4 (the 12.42 A cell is wider than
    2 r_c), so every replica has the same energy and forces as the small frame."""
    cfg, p, fr, ref = water
    big = I.replicate(fr, (4, 4, 4))
    for prec, ftol, etol in (("fp64", 1e-9, 1e-10), ("fp32", 1e-3, 1e-5)):
        m = _dp().Model(cfg, p, precision=prec)
        e, f, v, ae = m.compute(big.coord, big.atype, big.box, atom_energy=True)
        assert abs(float(e[0]) - 64 * ref.energy) / big.natoms <= etol
        assert np.abs(f - np.tile(ref.force, (64, 1))).max() <= ftol
        assert np.abs(ae - np.tile(ref.atom_energy, 64)).max() <= etol * 10
        np.testing.assert_allclose(v, 64 * ref.virial, rtol=1e-4 if prec == "fp32" else 1e-9, atol=1e-12)


def test_water12288_nlist_rows_sampled(water):
    cfg, p, fr, _ = water
    big = I.replicate(fr, (4, 4, 4))
    m = _dp().Model(cfg, p, precision="fp64")
    nl = m.build_nlist(big.coord, big.atype, big.box)
    gj, gs = nl.export()
    idx = np.array([0, 1, 777, 5000, 12287])
    rj, rs, _ = oracle.atom_subset(cfg, p, big.coord, big.atype, big.box, idx)
    np.testing.assert_array_equal(gj[idx], rj)
    np.testing.assert_array_equal(gs[idx], rs)


def test_fcc32000_sampled_and_properties():
    cfg = I.metal_model()
    fr = I.fcc_frame((20, 20, 20), seed=0)
    p = I.make_params(cfg, 0)
    idx = np.array([0, 4321, 31999])
    rj, rs, re = oracle.atom_subset(cfg, p, fr.coord, fr.atype, fr.box, idx)
    m = _dp().Model(cfg, p, precision="fp64")
    nl = m.build_nlist(fr.coord, fr.atype, fr.box)
    gj, gs = nl.export()
    np.testing.assert_array_equal(gj[idx], rj)
    np.testing.assert_array_equal(gs[idx], rs)
    e, f, v, ae = m.compute(fr.coord, fr.atype, fr.box, nlist=nl, atom_energy=True)
    assert np.abs(ae[idx] - re).max() <= 1e-10
    assert np.abs(f.sum(0)).max() <= 1e-8
    np.testing.assert_allclose(v, v.T, atol=1e-8)
