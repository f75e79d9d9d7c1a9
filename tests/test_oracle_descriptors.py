"""Pins of the oracle's se_e2_r and hybrid descriptors (Sec. II.A.1).

se_e2_r keeps only the radial column of R: D^i = G^T s / N_c, M values per atom.  The hybrid
descriptor concatenates the se_e2_a block (M x M_<) and the se_e2_r block.  Closed forms on
dimers and trimers fix the formula (the s weight, the 1/N_c, no angular information); the
decomposition of a hybrid model with a linear fitting net into its two parts fixes the
concatenation order and the parameter layout; dual numbers, finite differences and the
symmetries fix the reverse pass.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2304_09409_gb300 import inputs as I

from _cases import tiny_frame, tiny_model_hybrid, tiny_model_r


def _pair_model_r(M=1, sel=(4,), rc=4.0):
    return I.ModelConfig(ntypes=1, rcut=rc, rcut_smth=0.5, sel=sel, embed=(M,), axis=0, fit=(), descriptor=1)


def test_se_e2_r_dimer_closed_form_energy_and_force():
    """Isolated pair, M = 1, linear fitting: E = 2 (wf G(s) s / Nc + bf) with
    G(s) = tanh(w s + b) + s, and F_1 = -dE/dr u, dE/dr = 2 wf/Nc (G'(s) s + G(s)) s'(r)."""
    cfg = _pair_model_r()
    w, b, wf, bf = 0.7, -0.3, 1.9, 0.25
    p = np.array([w, b, wf, bf])
    for r in (0.4, 1.3, 2.7, 3.9):
        u = np.array([0.3, -0.8, math.sqrt(1 - 0.73)])
        coord = np.array([[0.0, 0.0, 0.0], r * u])
        res = oracle.compute(cfg, p, coord, np.zeros(2, np.int32), None)
        s, ds = oracle.switch(r, 0.5, 4.0)
        t = math.tanh(w * s + b)
        G, dG = t + s, w * (1 - t * t) + 1.0
        assert res.energy == pytest.approx(2 * (wf * G * s / 4 + bf), rel=1e-13)
        dEdr = 2 * wf / 4 * (dG * s + G) * ds
        np.testing.assert_allclose(res.force[1], -dEdr * u, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(res.force[0], dEdr * u, rtol=1e-12, atol=1e-15)
        # Xi_ab = -sum (dE/dr_ij)_a (r_ij)_b over both ordered pairs
        np.testing.assert_allclose(res.virial, -dEdr * r * np.outer(u, u), rtol=1e-12, atol=1e-15)


def test_se_e2_r_trimer_carries_no_angle():
    """Atom i with neighbours at r_j, r_k: D_i = (g(r_j) + g(r_k)) / Nc, g(r) = G(s(r)) s(r),
    whatever the angle between them."""
    cfg = _pair_model_r(sel=(5,), rc=3.0)
    w, b = 0.4, 0.1
    p = np.array([w, b, 1.0, 0.0])
    rj, rk = 1.1, 1.7

    def g(r):
        s = oracle.switch(r, 0.5, 3.0)[0]
        return (math.tanh(w * s + b) + s) * s

    for th in (0.7, 1.2, 2.9):
        coord = np.array([[0.0, 0.0, 0.0], [rj, 0.0, 0.0], [rk * math.cos(th), rk * math.sin(th), 0.0]])
        res = oracle.compute(cfg, p, coord, np.zeros(3, np.int32), None)
        assert res.atom_energy[0] == pytest.approx((g(rj) + g(rk)) / 5.0, rel=1e-13)


def test_se_e2_r_padding_scales_descriptor_by_inverse_nc():
    """Growing sel with no new neighbours scales the se_e2_r D by Nc/Nc' (one power, where
    se_e2_a's D, a product of two contractions, takes two)."""
    cfg1 = _pair_model_r(M=3, sel=(24,), rc=3.0)
    cfg2 = _pair_model_r(M=3, sel=(60,), rc=3.0)
    rng = I.Rng(5)
    p = np.concatenate([rng.normal(6), rng.normal(3), [0.0]])
    fr = tiny_frame(seed=8)
    e1 = oracle.compute(cfg1, p, fr.coord, np.zeros(fr.natoms, np.int32), fr.box)
    e2 = oracle.compute(cfg2, p, fr.coord, np.zeros(fr.natoms, np.int32), fr.box)
    assert e1.status == 0 and e2.status == 0
    assert e2.energy == pytest.approx(e1.energy * 24 / 60, rel=1e-12)
    np.testing.assert_allclose(e2.force, e1.force * 24 / 60, rtol=1e-11, atol=1e-14)


def _linear_parts(seed=3):
    """A hybrid model with a linear fitting net, and its se_e2_a and se_e2_r halves."""
    hyb = I.ModelConfig(ntypes=2, rcut=3.5, rcut_smth=0.5, sel=(12, 20), embed=(4, 8), axis=3, fit=(),
                        descriptor=2, embed_r=(2, 4, 5))
    ang = I.ModelConfig(ntypes=2, rcut=3.5, rcut_smth=0.5, sel=(12, 20), embed=(4, 8), axis=3, fit=())
    rad = I.ModelConfig(ntypes=2, rcut=3.5, rcut_smth=0.5, sel=(12, 20), embed=(2, 4, 5), axis=0, fit=(),
                        descriptor=1)
    p = I.make_params(hyb, seed)
    na = ang.n_embed_nets * sum(a * b + b for a, b in ang.embed_layer_shapes())
    nr = rad.n_embed_nets * sum(a * b + b for a, b in rad.embed_layer_shapes())
    da, dr = 8 * 3, 5
    pa, pr, pf = p[:na], p[na:na + nr], p[na + nr:]
    fa, fr_ = [], []
    for t in range(2):  # per type: W [da + dr] then b
        blk = pf[t * (da + dr + 1):(t + 1) * (da + dr + 1)]
        fa.append(np.concatenate([blk[:da], blk[-1:]]))
        fr_.append(np.concatenate([blk[da:da + dr], [0.0]]))
    return (hyb, p), (ang, np.concatenate([pa] + fa)), (rad, np.concatenate([pr] + fr_))


def test_hybrid_with_linear_fitting_is_sum_of_its_parts():
    """E_i = W . [D_a, D_r] + b splits into an se_e2_a model with (W_a, b) and an se_e2_r model
    with (W_r, 0): energies, per-atom energies, forces and virials add."""
    (hyb, ph), (ang, pa), (rad, pr) = _linear_parts()
    # the two halves each carry one bias per type; the hybrid carries one
    assert hyb.n_params() == oracle.n_params(hyb) == pa.size + pr.size - hyb.ntypes
    fr = tiny_frame(seed=6)
    h = oracle.compute(hyb, ph, fr.coord, fr.atype, fr.box)
    a = oracle.compute(ang, pa, fr.coord, fr.atype, fr.box)
    r = oracle.compute(rad, pr, fr.coord, fr.atype, fr.box)
    assert abs(r.energy) > 1e-3 and abs(a.energy) > 1e-3
    assert h.energy == pytest.approx(a.energy + r.energy, rel=1e-13)
    np.testing.assert_allclose(h.atom_energy, a.atom_energy + r.atom_energy, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(h.force, a.force + r.force, rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(h.virial, a.virial + r.virial, rtol=1e-11, atol=1e-13)


def _case(kind, seed=3):
    cfg = tiny_model_r() if kind == "r" else tiny_model_hybrid()
    fr = tiny_frame(seed=seed)
    p = I.make_params(cfg, 1)
    nl = oracle.nlist(cfg, fr.coord, fr.atype, fr.box)[:2]
    return cfg, fr, p, nl


@pytest.mark.parametrize("kind", ["r", "hybrid"])
def test_forces_and_virial_vs_dual_numbers(kind):
    cfg, fr, p, nl = _case(kind)
    r = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box, nl=nl)
    assert r.energy == pytest.approx(oracle.energy_plain(cfg, p, fr.coord, fr.atype, fr.box, nl), rel=1e-13)
    rng = I.Rng(2)
    for _ in range(3):
        u = rng.normal(fr.coord.size).reshape(fr.coord.shape)
        _, dE = oracle.energy_dual(cfg, p, fr.coord, fr.atype, fr.box, nl, dcoord=u)
        assert -(r.force * u).sum() == pytest.approx(dE, rel=1e-11, abs=1e-14)
    for b_ in range(3):
        for a in range(3):
            eps = np.zeros((3, 3))
            eps[b_, a] = 1.0
            _, dE = oracle.energy_dual(cfg, p, fr.coord, fr.atype, fr.box, nl, dcoord=fr.coord @ eps,
                                       dbox=fr.box @ eps)
            assert r.virial[a, b_] == pytest.approx(-dE, rel=1e-10, abs=1e-13)


@pytest.mark.parametrize("kind", ["r", "hybrid"])
def test_forces_vs_central_differences(kind):
    cfg, fr, p, nl = _case(kind)
    r = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box, nl=nl)
    hh = 1e-5
    for i in (0, 4, 9, 13):
        for a in range(3):
            cp = fr.coord.copy()
            cm = fr.coord.copy()
            cp[i, a] += hh
            cm[i, a] -= hh
            ep = oracle.compute(cfg, p, cp, fr.atype, fr.box, nl=nl).energy
            em = oracle.compute(cfg, p, cm, fr.atype, fr.box, nl=nl).energy
            assert r.force[i, a] == pytest.approx(-(ep - em) / (2 * hh), abs=2e-7)


def _rotation(seed):
    q, _ = np.linalg.qr(I.Rng(seed).normal(9).reshape(3, 3))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    return q


@pytest.mark.parametrize("kind", ["r", "hybrid"])
def test_symmetries(kind):
    cfg, fr, p, _ = _case(kind, seed=9)
    base = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box)
    t = oracle.compute(cfg, p, fr.coord + np.array([3.3, -7.1, 12.9]), fr.atype, fr.box)
    assert t.energy == pytest.approx(base.energy, rel=1e-12)
    np.testing.assert_allclose(t.force, base.force, atol=1e-11)
    Q = _rotation(4)
    rr = oracle.compute(cfg, p, fr.coord @ Q, fr.atype, fr.box @ Q)
    assert rr.energy == pytest.approx(base.energy, rel=1e-12)
    np.testing.assert_allclose(rr.force, base.force @ Q, atol=1e-11)
    np.testing.assert_allclose(rr.virial, Q.T @ base.virial @ Q, atol=1e-11)
    np.testing.assert_allclose(base.virial, base.virial.T, atol=1e-11)
    assert np.abs(base.force.sum(0)).max() < 1e-12
    perm = np.arange(fr.natoms)
    same = [i for i in range(fr.natoms) if fr.atype[i] == fr.atype[0]]
    perm[same] = same[::-1]
    pr = oracle.compute(cfg, p, fr.coord[perm], fr.atype[perm], fr.box)
    assert pr.energy == pytest.approx(base.energy, rel=1e-12)
    np.testing.assert_allclose(pr.force, base.force[perm], atol=1e-11)


@pytest.mark.parametrize("kind", ["r", "hybrid"])
def test_energy_continuous_across_cutoff(kind):
    """Move one atom radially across r_c of another: E(r_c - d) - E(r_c + d) = O(d^3)."""
    cfg = tiny_model_r() if kind == "r" else tiny_model_hybrid()
    p = I.make_params(cfg, 2)
    rc = cfg.rcut
    base = np.array([[0.0, 0.0, 0.0], [1.2, 0.3, -0.4], [-0.5, 1.1, 0.2], [0.0, 0.0, 0.0]])
    atype = np.array([0, 1, 0, 1], np.int32)
    direction = np.array([0.36, -0.48, 0.8])

    def e(r):
        c = base.copy()
        c[3] = r * direction
        return oracle.compute(cfg, p, c, atype, None).energy

    jumps = [abs(e(rc - d) - e(rc + d)) for d in (4e-2, 2e-2, 1e-2)]
    assert jumps[0] > 0
    assert jumps[0] / jumps[1] > 7.0 and jumps[1] / jumps[2] > 7.0
