"""The synthetic inputs the tests and the benchmark share: geometry and composition of the water
and FCC frames, replication, and seeded parameters."""
import math

import numpy as np
import pytest

from paper_2304_09409_gb300 import inputs as I


def _min_image(d, L):
    return d - L * np.round(d / L)


def test_water_frame_geometry():
    fr = I.water_frame(0)
    assert fr.natoms == 192 and fr.coord.shape == (192, 3)
    np.testing.assert_array_equal(fr.atype, np.tile([0, 1, 1], 64))
    L = 4 * 3.105
    np.testing.assert_allclose(fr.box, np.eye(3) * L)
    o, h1, h2 = fr.coord[0::3], fr.coord[1::3], fr.coord[2::3]
    # every H at the O-H bond length from its O, at the HOH angle
    v1, v2 = h1 - o, h2 - o
    np.testing.assert_allclose(np.linalg.norm(v1, axis=1), I.OH_BOND, rtol=1e-12)
    np.testing.assert_allclose(np.linalg.norm(v2, axis=1), I.OH_BOND, rtol=1e-12)
    cosang = (v1 * v2).sum(1) / (I.OH_BOND ** 2)
    np.testing.assert_allclose(np.degrees(np.arccos(cosang)), I.HOH_ANGLE_DEG, atol=1e-9)
    # O on the jittered lattice: minimum image O-O distance at least 2.5 A
    d = _min_image(o[:, None, :] - o[None, :, :], L)
    r = np.sqrt((d * d).sum(-1)) + np.eye(64) * 1e9
    assert r.min() >= 2.5
    # about 1 g/cm^3
    assert L ** 3 / 64 == pytest.approx(I.WATER_ML_PER_MOL_A3, rel=0.01)


def test_water_frame_n_random_addition_density_and_spacing():
    fr = I.water_frame_n(50, seed=3)  # not a cube: random sequential addition
    assert fr.natoms == 150
    L = fr.box[0, 0]
    assert L ** 3 / 50 == pytest.approx(I.WATER_ML_PER_MOL_A3, rel=1e-12)
    o = fr.coord[0::3]
    d = _min_image(o[:, None, :] - o[None, :, :], L)
    r = np.sqrt((d * d).sum(-1)) + np.eye(50) * 1e9
    assert r.min() >= 2.5


def test_fcc_frame_lattice():
    a = 3.634
    fr = I.fcc_frame((3, 4, 5), seed=1)
    assert fr.natoms == 4 * 3 * 4 * 5
    np.testing.assert_allclose(np.diag(fr.box), [3 * a, 4 * a, 5 * a])
    assert np.all(fr.atype == 0)
    # nearest neighbours at a / sqrt(2), up to the 0.05 A jitter
    d = _min_image(fr.coord[:, None, :] - fr.coord[None, :, :], np.diag(fr.box))
    r = np.sqrt((d * d).sum(-1)) + np.eye(fr.natoms) * 1e9
    nn = r.min(1)
    assert np.all(np.abs(nn - a / math.sqrt(2)) < 0.4)


def test_replicate_tiles_the_frame():
    base = I.water_frame(0)
    big = I.replicate(base, (4, 4, 4))
    assert big.natoms == 64 * base.natoms == 12288
    np.testing.assert_allclose(big.box, base.box * 4)
    np.testing.assert_array_equal(big.coord[:192], base.coord)
    np.testing.assert_allclose(big.coord[192:384], base.coord + base.box[2])  # image (0, 0, 1)
    np.testing.assert_array_equal(big.atype, np.tile(base.atype, 64))


def test_parameters_are_seeded_and_laid_out():
    cfg = I.water_model()
    p0, p0b, p1 = I.make_params(cfg, 0), I.make_params(cfg, 0), I.make_params(cfg, 1)
    assert p0.dtype == np.float64 and p0.size == cfg.n_params()
    np.testing.assert_array_equal(p0, p0b)
    assert not np.array_equal(p0, p1)
    # first embedding layer 1 -> 25: W ~ N(0, 2/26), 25 weights, then 25 biases ~ N(0, 1)
    w = p0[:25]
    assert np.abs(w).max() < 6 * math.sqrt(2 / 26)


def test_force_scaled_models_reach_about_one_ev_per_angstrom():
    """The force-scaled variants scale only the output layer: the oracle's energies, forces and
    virial scale by exactly the factor, and the force RMS lands near 1 eV/A on the water frame
    and on an FCC frame of the metal model (the scale at which the 1e-3 eV/A bar means
    something)."""
    import oracle
    cfg = I.water_model()
    p = I.make_params(cfg, 0)
    ps = I.water_params_scaled(0)
    changed = np.nonzero(ps != p)[0]
    assert changed.size == 2 * (cfg.fit[-1] + 1)  # W and b of the last layer of both types
    fr = I.water_frame(0)
    a = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box)
    b = oracle.compute(cfg, ps, fr.coord, fr.atype, fr.box)
    s = I.WATER_FORCE_SCALE
    np.testing.assert_allclose(b.force, s * a.force, rtol=1e-10, atol=1e-12 * s)
    np.testing.assert_allclose(b.virial, s * a.virial, rtol=1e-10, atol=1e-12 * s)
    assert b.energy == pytest.approx(s * a.energy, rel=1e-12)
    assert 0.7 < np.sqrt((b.force ** 2).mean()) < 1.5
    cfg = I.metal_model()
    fr = I.fcc_frame((4, 4, 4), seed=0)
    r = oracle.compute(cfg, I.metal_params_scaled(0), fr.coord, fr.atype, fr.box)
    assert 0.7 < np.sqrt((r.force ** 2).mean()) < 1.5
