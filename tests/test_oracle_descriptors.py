"""Pins of the oracle's se_e2_r, se_e3 and hybrid descriptors (Sec. II.A.1).

se_e2_r keeps only the radial column of R: D^i = G^T s / N_c, M values per atom.  se_e3
contracts R R^T with the three-body embedding: D^i = (R R^T) : G / N_c^2 with
G_jk = N^{a_j,a_k}(R_j . R_k).  A hybrid descriptor concatenates its parts, each with its own
cutoff, sel and nets.  Closed forms on dimers and trimers fix the formulas (the s weight, the
1/N_c and 1/N_c^2, the angle, the type-pair nets); the decomposition of a hybrid model with a
linear fitting net into stand-alone parts fixes the concatenation order, the parameter layout
and the per-part neighbour lists; dual numbers, finite differences and the symmetries fix the
reverse pass.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2304_09409_gb300 import inputs as I

from _cases import tiny_frame, tiny_model_e3, tiny_model_hybrid, tiny_model_hybrid_e3, tiny_model_r


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


def _linear_parts(second="r", rc=(3.0, 3.5), sel=((8, 14), (12, 20)), seed=3):
    """A hybrid model with a linear fitting net, and its two parts as stand-alone models with their
    own cutoffs and sel (each builds its own list by brute force)."""
    kind2, emb2 = (1, (2, 4, 5)) if second == "r" else (3, (2, 4))
    hyb = I.ModelConfig(ntypes=2, rcut=rc[0], rcut_smth=0.5, sel=sel[0], embed=(4, 8), axis=3, fit=(),
                        descriptor=2 if second == "r" else 4, rcut_2=rc[1], rcut_smth_2=0.4, sel_2=sel[1],
                        embed_2=emb2)
    ang = I.ModelConfig(ntypes=2, rcut=rc[0], rcut_smth=0.5, sel=sel[0], embed=(4, 8), axis=3, fit=())
    two = I.ModelConfig(ntypes=2, rcut=rc[1], rcut_smth=0.4, sel=sel[1], embed=emb2, axis=0, fit=(),
                        descriptor=kind2)
    p = I.make_params(hyb, seed)
    na = ang.embed_params()
    n2 = two.embed_params()
    da, d2 = ang.descriptor_dim, two.descriptor_dim
    pa, p2, pf = p[:na], p[na:na + n2], p[na + n2:]
    fa, f2 = [], []
    for t in range(2):  # per type: W [da + d2] then b
        blk = pf[t * (da + d2 + 1):(t + 1) * (da + d2 + 1)]
        fa.append(np.concatenate([blk[:da], blk[-1:]]))
        f2.append(np.concatenate([blk[da:da + d2], [0.0]]))
    return (hyb, p), (ang, np.concatenate([pa] + fa)), (two, np.concatenate([p2] + f2))


@pytest.mark.parametrize("second", ["r", "e3"])
@pytest.mark.parametrize("rc,sel", [((3.0, 3.5), ((8, 14), (12, 20))), ((3.5, 2.8), ((12, 20), (6, 9))),
                                    ((3.5, 3.5), ((12, 20), (12, 20)))], ids=["wider2", "wider1", "same"])
def test_hybrid_with_linear_fitting_is_sum_of_its_parts(second, rc, sel):
    """E_i = W . [D_1, D_2] + b splits into the first part with (W_1, b) and the second part with
    (W_2, 0), each a stand-alone model with its own cutoff, sel and brute-force list: energies,
    per-atom energies, forces and virials add.  This fixes the concatenation order, the parameter
    layout, and that a part reads the nearest sel_2 neighbours within its own r_c from the one list
    built at the wider cutoff."""
    (hyb, ph), (ang, pa), (two, p2) = _linear_parts(second, rc, sel)
    # the two halves each carry one bias per type; the hybrid carries one
    assert hyb.n_params() == oracle.n_params(hyb) == pa.size + p2.size - hyb.ntypes
    fr = tiny_frame(seed=6)
    h = oracle.compute(hyb, ph, fr.coord, fr.atype, fr.box)
    a = oracle.compute(ang, pa, fr.coord, fr.atype, fr.box)
    r = oracle.compute(two, p2, fr.coord, fr.atype, fr.box)
    assert abs(r.energy) > 1e-4 and abs(a.energy) > 1e-4
    assert h.energy == pytest.approx(a.energy + r.energy, rel=1e-13)
    np.testing.assert_allclose(h.atom_energy, a.atom_energy + r.atom_energy, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(h.force, a.force + r.force, rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(h.virial, a.virial + r.virial, rtol=1e-11, atol=1e-13)


# ----------------------------------------------------------------------------------------
# se_e3: closed forms
# ----------------------------------------------------------------------------------------


def _e3_model(ntypes=1, sel=(4,), rc=4.0, M=1):
    return I.ModelConfig(ntypes=ntypes, rcut=rc, rcut_smth=0.5, sel=sel, embed=(M,), axis=0, fit=(), descriptor=3)


def test_se_e3_dimer_closed_form_energy_and_force():
    """Isolated pair, M = 1, linear fitting: atom i's only pair is (j, j) with theta = R_j . R_j
    = 2 s^2, so E = 2 (wf theta G(theta) / Nc^2 + bf), G(x) = tanh(w x + b) + x; and
    dE/dr = 2 wf / Nc^2 (G + theta G') 4 s s'(r)."""
    cfg = _e3_model()
    w, b, wf, bf = 0.35, -0.2, 1.3, 0.1
    p = np.array([w, b, wf, bf])
    for r in (0.4, 1.3, 2.7, 3.9):
        u = np.array([0.3, -0.8, np.sqrt(1 - 0.73)])
        coord = np.array([[0.0, 0.0, 0.0], r * u])
        res = oracle.compute(cfg, p, coord, np.zeros(2, np.int32), None)
        s, ds = oracle.switch(r, 0.5, 4.0)
        th = 2 * s * s
        t = np.tanh(w * th + b)
        G, dG = t + th, w * (1 - t * t) + 1.0
        assert res.energy == pytest.approx(2 * (wf * th * G / 16 + bf), rel=1e-13)
        dEdr = 2 * wf / 16 * (G + th * dG) * 4 * s * ds
        np.testing.assert_allclose(res.force[1], -dEdr * u, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(res.virial, -dEdr * r * np.outer(u, u), rtol=1e-12, atol=1e-15)


def test_se_e3_trimer_type_pair_nets_and_angle():
    """Centre of type 0 with neighbours j (type 0) and k (type 1) at angle gamma, M = 1:
    D = [th_jj G00(th_jj) + th_kk G11(th_kk) + th_jk (G01(th_jk) + G10(th_jk))] / Nc^2 with
    th_jj = 2 s_j^2, th_kk = 2 s_k^2, th_jk = s_j s_k (1 + cos gamma); nets N^{a_j, a_k} stored
    in the order (0,0), (0,1), (1,0), (1,1)."""
    cfg = _e3_model(ntypes=2, sel=(2, 3), rc=3.0)
    nets = [(0.4, 0.1), (-0.3, 0.2), (0.7, -0.5), (0.25, 0.05)]
    p = np.concatenate([np.array(nets).ravel(), [1.0, 0.0], [0.0, 0.0]])
    rj, rk = 1.1, 1.7
    G = lambda n, x: np.tanh(nets[n][0] * x + nets[n][1]) + x  # noqa: E731
    sw = lambda r: oracle.switch(r, 0.5, 3.0)[0]  # noqa: E731
    for gam in (0.7, 1.9, 2.8):
        coord = np.array([[0.0, 0.0, 0.0], [rj, 0.0, 0.0], [rk * np.cos(gam), rk * np.sin(gam), 0.0]])
        res = oracle.compute(cfg, p, coord, np.array([0, 0, 1], np.int32), None)
        sj, sk = sw(rj), sw(rk)
        tjj, tkk, tjk = 2 * sj * sj, 2 * sk * sk, sj * sk * (1 + np.cos(gam))
        D = (tjj * G(0, tjj) + tkk * G(3, tkk) + tjk * (G(1, tjk) + G(2, tjk))) / 25.0
        assert res.atom_energy[0] == pytest.approx(D, rel=1e-13)


def test_se_e3_padding_scales_descriptor_by_inverse_nc_squared():
    cfg1 = _e3_model(sel=(24,), rc=3.0, M=3)
    cfg2 = _e3_model(sel=(60,), rc=3.0, M=3)
    rng = I.Rng(5)
    p = np.concatenate([rng.normal(6), rng.normal(3), [0.0]])
    fr = tiny_frame(seed=8)
    e1 = oracle.compute(cfg1, p, fr.coord, np.zeros(fr.natoms, np.int32), fr.box)
    e2 = oracle.compute(cfg2, p, fr.coord, np.zeros(fr.natoms, np.int32), fr.box)
    assert e1.status == 0 and e2.status == 0
    assert e2.energy == pytest.approx(e1.energy * (24 / 60) ** 2, rel=1e-12)


KINDS = ["r", "hybrid", "e3", "hybrid_e3"]


def _model(kind):
    return {"r": tiny_model_r, "hybrid": tiny_model_hybrid, "e3": tiny_model_e3,
            "hybrid_e3": tiny_model_hybrid_e3}[kind]()


def _case(kind, seed=3):
    cfg = _model(kind)
    fr = tiny_frame(seed=seed)
    p = I.make_params(cfg, 1)
    nl = oracle.nlist(cfg, fr.coord, fr.atype, fr.box)[:2]
    return cfg, fr, p, nl


@pytest.mark.parametrize("kind", KINDS)
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


@pytest.mark.parametrize("kind", KINDS)
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


@pytest.mark.parametrize("kind", KINDS)
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


@pytest.mark.parametrize("kind", KINDS)
def test_energy_continuous_across_cutoff(kind):
    """Move one atom radially across r_c of another: E(r_c - d) - E(r_c + d) = O(d^3)."""
    cfg = _model(kind)
    p = I.make_params(cfg, 2)
    rc = cfg.list_rcut  # the outer cutoff: every part's terms in the moved atom vanish there
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


# ----------------------------------------------------------------------------------------
# Compressed se_e2_r and se_e3 (Eq. (compress); for se_e3 the pieces are in theta)
# ----------------------------------------------------------------------------------------


@pytest.mark.parametrize("kind", ["r", "e3"])
def test_table_layout_and_nodes(kind):
    """The e3 grid covers theta in [0, 2 / r_s^2] (R_j . R_k <= |R_j| |R_k| = 2 s_j s_k); at every
    node each piece reproduces the net's value, slope and curvature, and its right end the next value."""
    cfg = I.water_model_r() if kind == "r" else I.water_model_e3()
    p = I.make_params(cfg, 0)
    lay = oracle.table_layout(cfg)
    x0, h1, n1, h2, n2 = lay
    top = x0 + n1 * h1 + n2 * h2
    assert top == pytest.approx(1 / cfg.rcut_smth if kind == "r" else 2 / cfg.rcut_smth ** 2, rel=1e-12)
    tab = oracle.table_build(cfg, p, *lay)
    nodes = np.concatenate([x0 + np.arange(n1 + 1) * h1, x0 + n1 * h1 + np.arange(1, n2 + 1) * h2])
    for net in range(cfg.n_embed_nets):
        y, y1, y2 = oracle.embed_jets(cfg, p, net, nodes)
        c = tab[net]
        np.testing.assert_allclose(c[:, :, 5], y[:-1], rtol=0, atol=1e-13)
        np.testing.assert_allclose(c[:, :, 4], y1[:-1], rtol=0, atol=1e-12)
        np.testing.assert_allclose(2 * c[:, :, 3], y2[:-1], rtol=0, atol=1e-11)
        dx = np.diff(nodes)[:, None]
        right = ((((c[..., 0] * dx + c[..., 1]) * dx + c[..., 2]) * dx + c[..., 3]) * dx + c[..., 4]) * dx + c[..., 5]
        np.testing.assert_allclose(right, y[1:], rtol=0, atol=1e-9)


@pytest.mark.parametrize("kind", ["r", "e3"])
def test_compressed_close_to_network(kind):
    cfg = I.water_model_r() if kind == "r" else I.water_model_e3()
    p = I.make_params(cfg, 0)
    fr = I.water_frame(0)
    lay = oracle.table_layout(cfg)
    tab = oracle.table_build(cfg, p, *lay)
    a = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box)
    b = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box, table=tab, table_layout=lay)
    assert b.status == 0
    assert abs(a.energy - b.energy) / fr.natoms < 1e-8
    assert np.abs(a.force - b.force).max() < 1e-7
    np.testing.assert_allclose(b.virial, a.virial, atol=1e-7)


@pytest.mark.parametrize("kind", ["r", "e3"])
def test_compressed_forces_vs_differences_of_compressed_energy(kind):
    """The compressed reverse pass uses each piece's analytic slope (in s, or in theta for se_e3)."""
    cfg = tiny_model_r() if kind == "r" else tiny_model_e3()
    fr = tiny_frame(seed=3)
    p = I.make_params(cfg, 1)
    nl = oracle.nlist(cfg, fr.coord, fr.atype, fr.box)[:2]
    lay = oracle.table_layout(cfg)
    tab = oracle.table_build(cfg, p, *lay)
    r = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box, nl=nl, table=tab, table_layout=lay)
    assert r.status == 0
    h = 1e-5
    for i, a in ((0, 0), (3, 1), (7, 2), (11, 0)):
        cp = fr.coord.copy()
        cm = fr.coord.copy()
        cp[i, a] += h
        cm[i, a] -= h
        ep = oracle.compute(cfg, p, cp, fr.atype, fr.box, nl=nl, table=tab, table_layout=lay).energy
        em = oracle.compute(cfg, p, cm, fr.atype, fr.box, nl=nl, table=tab, table_layout=lay).energy
        assert r.force[i, a] == pytest.approx(-(ep - em) / (2 * h), abs=2e-7)
