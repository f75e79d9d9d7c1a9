"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

None of these checks re-types an oracle formula: each one compares the oracle with an
independent fact -- a closed form, a derivative by another mechanism (central finite
differences, forward-mode dual numbers), a symmetry of the energy, or brute force.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2304_09409_gb300 import inputs as I

from _cases import tiny_frame, tiny_model

# ----------------------------------------------------------------------------------------
# Eq. (switch)
# ----------------------------------------------------------------------------------------


def test_switch_closed_form_and_smoothness():
    rs, rc = 0.5, 6.0
    # r < r_s: plain 1/r
    for r in (0.1, 0.3, 0.49999):
        s, ds = oracle.switch(r, rs, rc)
        assert s == pytest.approx(1.0 / r, rel=1e-15)
        assert ds == pytest.approx(-1.0 / r ** 2, rel=1e-14)
    # x = 1/2 gives the polynomial value 1/2: s = 1/(2 r)
    rm = 0.5 * (rs + rc)
    assert oracle.switch(rm, rs, rc)[0] == pytest.approx(0.5 / rm, rel=1e-14)
    # beyond the cutoff
    assert oracle.switch(rc, rs, rc) == (0.0, 0.0)
    assert oracle.switch(rc + 1.0, rs, rc) == (0.0, 0.0)

    # s, s', s'' continuous at r_s and r_c (the switch is C^2): one-sided difference quotients
    def d2(r, h=1e-4):
        return (oracle.switch(r + h, rs, rc)[1] - oracle.switch(r - h, rs, rc)[1]) / (2 * h)

    for knot in (rs, rc):
        e = 1e-7
        sl, dl = oracle.switch(knot - e, rs, rc)
        sr, dr = oracle.switch(knot + e, rs, rc)
        assert abs(sl - sr) < 1e-5 and abs(dl - dr) < 1e-5
        assert abs(d2(knot - 1e-3) - d2(knot + 1e-3)) < 5e-2 * max(1.0, abs(d2(knot - 1e-3)))
    # s' against central differences of s everywhere on the smooth part
    for r in np.linspace(0.2, 5.9, 23):
        h = 1e-6
        fd = (oracle.switch(r + h, rs, rc)[0] - oracle.switch(r - h, rs, rc)[0]) / (2 * h)
        assert oracle.switch(r, rs, rc)[1] == pytest.approx(fd, rel=1e-6, abs=1e-8)


# ----------------------------------------------------------------------------------------
# Eq. (compress): the quintic of one interval
# ----------------------------------------------------------------------------------------


def _poly(c, t):
    return ((((c[0] * t + c[1]) * t + c[2]) * t + c[3]) * t + c[4]) * t + c[5]


def test_quintic_hermite_conditions():
    rng = I.Rng(7)
    for _ in range(20):
        y0, y1, d0, d1, dd0, dd1 = rng.normal(6)
        dx = 0.01 + rng.uniform(1)[0]
        c = oracle.quintic(y0, y1, d0, d1, dd0, dd1, dx)
        p1 = np.polyder(c)
        p2 = np.polyder(p1)
        for t, y, d, dd in ((0.0, y0, d0, dd0), (dx, y1, d1, dd1)):
            assert np.polyval(c, t) == pytest.approx(y, abs=1e-10)
            assert np.polyval(p1, t) == pytest.approx(d, abs=1e-9)
            assert np.polyval(p2, t) == pytest.approx(dd, abs=1e-7)


def test_quintic_reproduces_degree5_polynomial():
    rng = I.Rng(11)
    q = rng.normal(6)  # q[0] t^5 + ... + q[5]
    dx = 0.37
    q1, q2 = np.polyder(q), np.polyder(q, 2)
    c = oracle.quintic(np.polyval(q, 0), np.polyval(q, dx), np.polyval(q1, 0), np.polyval(q1, dx),
                       np.polyval(q2, 0), np.polyval(q2, dx), dx)
    np.testing.assert_allclose(c, q, rtol=1e-9, atol=1e-9)


# ----------------------------------------------------------------------------------------
# Embedding network and its node derivatives (Eq. NN; library special case)
# ----------------------------------------------------------------------------------------


def _numpy_net(cfg, params, net, s):
    """Eq. (NN) with numpy matmul/tanh (ResNet on, w_hat = 1)."""
    off = 0
    per_net = sum(a * b + b for a, b in cfg.embed_layer_shapes())
    off = net * per_net
    x = np.atleast_2d(np.asarray(s, dtype=np.float64)).T
    for fi, fo in cfg.embed_layer_shapes():
        W = params[off:off + fi * fo].reshape(fi, fo)
        b = params[off + fi * fo: off + fi * fo + fo]
        off += fi * fo + fo
        y = np.tanh(x @ W + b)
        if fo == fi:
            y = y + x
        elif fo == 2 * fi:
            y = y + np.concatenate([x, x], axis=1)
        x = y
    return x


@pytest.mark.parametrize("cfg_fn", [tiny_model, I.water_model])
def test_embedding_jets_vs_library_and_differences(cfg_fn):
    cfg = cfg_fn()
    p = I.make_params(cfg, 0)
    xs = np.linspace(0.0, 2.0, 9)
    for net in range(cfg.n_embed_nets):
        y, y1, y2 = oracle.embed_jets(cfg, p, net, xs)
        np.testing.assert_allclose(y, _numpy_net(cfg, p, net, xs), rtol=1e-13, atol=1e-13)
        h = 1e-4
        yp = _numpy_net(cfg, p, net, xs + h)
        ym = _numpy_net(cfg, p, net, xs - h)
        np.testing.assert_allclose(y1, (yp - ym) / (2 * h), rtol=1e-6, atol=1e-7)
        np.testing.assert_allclose(y2, (yp - 2 * y + ym) / h ** 2, rtol=1e-4, atol=1e-4)


# ----------------------------------------------------------------------------------------
# Neighbour list: brute force vs an independent enumeration
# ----------------------------------------------------------------------------------------


def _numpy_neighbours(coord, atype, box, rc, K=3):
    """All (j, shift) with |r_j + n h - r_i| < r_c for n in [-K, K]^3 (coordinates far
    outside the cell are folded first so K = 3 suffices for these small cases)."""
    inv = np.linalg.inv(box)
    f = coord @ inv
    wrap = np.floor(f)
    base = (f - wrap) @ box
    out = []
    rng = np.arange(-K, K + 1)
    shifts = np.stack(np.meshgrid(rng, rng, rng, indexing="ij"), -1).reshape(-1, 3)
    for i in range(coord.shape[0]):
        neigh = []
        for j in range(coord.shape[0]):
            d = base[j] + shifts @ box - base[i]
            r = np.sqrt((d * d).sum(1))
            for s_idx in np.nonzero(r < rc)[0]:
                n = tuple(int(v) for v in shifts[s_idx] - wrap[j] + wrap[i])
                if j == i and n == (0, 0, 0):
                    continue
                neigh.append((int(atype[j]), float(r[s_idx]), j, n))
        out.append(neigh)
    return out


@pytest.mark.parametrize("seed,triclinic", [(3, True), (4, False), (5, True)])
def test_nlist_matches_independent_enumeration(seed, triclinic):
    cfg = tiny_model()
    fr = tiny_frame(seed=seed, triclinic=triclinic)
    # move a few atoms far outside the cell: the list is defined on raw coordinates
    coord = fr.coord.copy()
    coord[0] += 2 * fr.box[0] - 3 * fr.box[2]
    coord[5] -= fr.box[1]
    nl_j, nl_s, counts, ov = oracle.nlist(cfg, coord, fr.atype, fr.box)
    ref = _numpy_neighbours(coord, fr.atype, fr.box, cfg.rcut)
    for i, neigh in enumerate(ref):
        for t in range(cfg.ntypes):
            mine = sorted([e for e in neigh if e[0] == t], key=lambda e: (e[1], e[2], e[3]))
            assert counts[i, t] == len(mine)
            off = sum(cfg.sel[:t])
            keep = mine[:cfg.sel[t]]
            got = [(int(nl_j[i, off + q]), tuple(int(v) for v in nl_s[i, off + q])) for q in range(len(keep))]
            assert got == [(e[2], e[3]) for e in keep]
            assert np.all(nl_j[i, off + len(keep): off + cfg.sel[t]] == -1)
    assert ov == int((counts > np.array(cfg.sel)).sum())


def test_nlist_overflow_truncates_to_nearest():
    cfg = I.ModelConfig(ntypes=2, rcut=3.5, rcut_smth=0.5, sel=(3, 4), embed=(4, 8, 16), axis=4, fit=(12, 12))
    fr = tiny_frame(seed=6)
    nl_j, nl_s, counts, ov = oracle.nlist(cfg, fr.coord, fr.atype, fr.box)
    assert ov > 0
    ref = _numpy_neighbours(fr.coord, fr.atype, fr.box, cfg.rcut)
    for i, neigh in enumerate(ref):
        for t in range(2):
            mine = sorted([e for e in neigh if e[0] == t], key=lambda e: (e[1], e[2], e[3]))[:cfg.sel[t]]
            off = sum(cfg.sel[:t])
            assert [int(v) for v in nl_j[i, off:off + len(mine)]] == [e[2] for e in mine]


def test_water_neighbour_counts_within_sel():
    cfg = I.water_model()
    fr = I.water_frame(0)
    _, _, counts, ov = oracle.nlist(cfg, fr.coord, fr.atype, fr.box)
    assert ov == 0
    assert counts[:, 0].max() <= 46 and counts[:, 1].max() <= 92
    # density 1 g/cm^3 -> about 0.0334 molecules / A^3 -> ~30 O and ~60 H inside 6 A
    assert 20 < counts[:, 0].mean() < 40 and 45 < counts[:, 1].mean() < 75


# ----------------------------------------------------------------------------------------
# Energy: generic forward vs reverse-pass forward; descriptor closed forms
# ----------------------------------------------------------------------------------------


def _tiny_case(seed=3, scale=1.0):
    cfg = tiny_model()
    fr = tiny_frame(seed=seed)
    p = I.make_params(cfg, 1) * scale
    nl = oracle.nlist(cfg, fr.coord, fr.atype, fr.box)[:2]
    return cfg, fr, p, nl


def test_generic_forward_equals_reverse_pass_forward():
    cfg, fr, p, nl = _tiny_case()
    r = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box, nl=nl)
    e2 = oracle.energy_plain(cfg, p, fr.coord, fr.atype, fr.box, nl)
    assert r.energy == pytest.approx(e2, rel=1e-13)
    assert r.atom_energy.sum() == pytest.approx(r.energy, rel=1e-14)


def _pair_model(M=1, axis=1, sel=(4,), rc=4.0):
    return I.ModelConfig(ntypes=1, rcut=rc, rcut_smth=0.5, sel=sel, embed=(M,), axis=axis, fit=())


def _linear_fit_params(cfg, w_emb, b_emb, w_fit, b_fit):
    # embedding 1 -> M (tanh, with +x skip when M == 1); fitting D (M*axis) -> 1 linear
    return np.concatenate([np.atleast_1d(w_emb), np.atleast_1d(b_emb), np.atleast_1d(w_fit), [b_fit]]).astype(float)


def test_descriptor_dimer_closed_form():
    """Isolated pair, M = M_< = 1: R_j = (s, s u) with |u| = 1, so D = 2 (G(s) s)^2 / Nc^2,
    with G(s) = tanh(w s + b) + s (the 1 -> 1 layer carries the +x skip)."""
    cfg = _pair_model()
    w, b, wf, bf = 0.7, -0.3, 1.9, 0.25
    p = _linear_fit_params(cfg, w, b, wf, bf)
    for r in (0.4, 1.3, 2.7, 3.9):
        coord = np.array([[0.0, 0.0, 0.0], [0.3 * r, -0.8 * r, math.sqrt(1 - 0.73) * r]])
        res = oracle.compute(cfg, p, coord, np.zeros(2, np.int32), None)
        s = oracle.switch(r, 0.5, 4.0)[0]
        G = math.tanh(w * s + b) + s
        D = 2.0 * (G * s) ** 2 / 4 ** 2
        assert res.energy == pytest.approx(2 * (wf * D + bf), rel=1e-13)


def test_descriptor_trimer_law_of_cosines():
    """Atom i with two neighbours j, k at angle theta, M = M_< = 1:
    D_i = [(a+b)^2 + a^2 + b^2 + 2ab cos(theta)] / Nc^2 with a = G(s_j) s_j, b = G(s_k) s_k."""
    cfg = _pair_model(sel=(5,), rc=3.0)
    w, b = 0.4, 0.1
    p = _linear_fit_params(cfg, w, b, 1.0, 0.0)
    rj, rk, th = 1.1, 1.7, 1.2
    coord = np.array([[0.0, 0.0, 0.0], [rj, 0.0, 0.0], [rk * math.cos(th), rk * math.sin(th), 0.0]])
    res = oracle.compute(cfg, p, coord, np.zeros(3, np.int32), None)
    g = lambda r: (math.tanh(w * oracle.switch(r, 0.5, 3.0)[0] + b) + oracle.switch(r, 0.5, 3.0)[0]) * \
        oracle.switch(r, 0.5, 3.0)[0]
    a_, b_ = g(rj), g(rk)
    Di = ((a_ + b_) ** 2 + a_ ** 2 + b_ ** 2 + 2 * a_ * b_ * math.cos(th)) / 25.0
    assert res.atom_energy[0] == pytest.approx(Di, rel=1e-13)


def test_padding_scales_descriptor_by_inverse_nc_squared():
    """Nc is the padded constant: growing sel with no new neighbours scales D by (Nc/Nc')^2;
    with a linear fitting net without bias E scales the same way."""
    cfg1 = _pair_model(M=3, axis=2, sel=(24,), rc=3.0)
    cfg2 = _pair_model(M=3, axis=2, sel=(60,), rc=3.0)
    rng = I.Rng(5)
    pe = rng.normal(6)
    pf = rng.normal(6)
    p = np.concatenate([pe, pf, [0.0]])
    fr = tiny_frame(seed=8)
    e1 = oracle.compute(cfg1, p, fr.coord, np.zeros(fr.natoms, np.int32), fr.box)
    e2 = oracle.compute(cfg2, p, fr.coord, np.zeros(fr.natoms, np.int32), fr.box)
    assert e1.status == 0 and e2.status == 0
    assert e2.energy == pytest.approx(e1.energy * (24 / 60) ** 2, rel=1e-12)


# ----------------------------------------------------------------------------------------
# Forces and virial: finite differences, dual numbers, invariants
# ----------------------------------------------------------------------------------------


def test_forces_vs_dual_numbers_exact():
    cfg, fr, p, nl = _tiny_case()
    r = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box, nl=nl)
    rng = I.Rng(2)
    for _ in range(4):
        u = rng.normal(fr.coord.size).reshape(fr.coord.shape)
        _, dE = oracle.energy_dual(cfg, p, fr.coord, fr.atype, fr.box, nl, dcoord=u)
        assert -(r.force * u).sum() == pytest.approx(dE, rel=1e-11, abs=1e-14)
    # per-component on a few atoms
    for i in (0, 5, 13):
        for a in range(3):
            u = np.zeros_like(fr.coord)
            u[i, a] = 1.0
            _, dE = oracle.energy_dual(cfg, p, fr.coord, fr.atype, fr.box, nl, dcoord=u)
            assert -r.force[i, a] == pytest.approx(dE, rel=1e-10, abs=1e-14)


def test_virial_vs_dual_numbers_strain():
    """Xi_ab = -dE/d eps_ba under r -> r (I + eps), h -> h (I + eps) (fractional coordinates fixed)."""
    cfg, fr, p, nl = _tiny_case()
    r = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box, nl=nl)
    for b_ in range(3):
        for a in range(3):
            eps = np.zeros((3, 3))
            eps[b_, a] = 1.0
            _, dE = oracle.energy_dual(cfg, p, fr.coord, fr.atype, fr.box, nl, dcoord=fr.coord @ eps,
                                       dbox=fr.box @ eps)
            assert r.virial[a, b_] == pytest.approx(-dE, rel=1e-10, abs=1e-13)


def test_forces_vs_central_differences():
    cfg, fr, p, nl = _tiny_case()
    r = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box, nl=nl)
    h = 1e-5
    for i in range(fr.natoms):
        for a in range(3):
            cp = fr.coord.copy()
            cm = fr.coord.copy()
            cp[i, a] += h
            cm[i, a] -= h
            ep = oracle.compute(cfg, p, cp, fr.atype, fr.box, nl=nl).energy
            em = oracle.compute(cfg, p, cm, fr.atype, fr.box, nl=nl).energy
            assert r.force[i, a] == pytest.approx(-(ep - em) / (2 * h), abs=2e-7)


def test_virial_vs_central_difference_strain():
    cfg, fr, p, _ = _tiny_case()
    r = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box)
    h = 1e-6
    for b_ in range(3):
        for a in range(3):
            eps = np.zeros((3, 3))
            eps[b_, a] = h
            ep = oracle.compute(cfg, p, fr.coord @ (np.eye(3) + eps), fr.atype, fr.box @ (np.eye(3) + eps)).energy
            em = oracle.compute(cfg, p, fr.coord @ (np.eye(3) - eps), fr.atype, fr.box @ (np.eye(3) - eps)).energy
            assert r.virial[a, b_] == pytest.approx(-(ep - em) / (2 * h), abs=1e-7)
    # rotational invariance makes the virial symmetric
    np.testing.assert_allclose(r.virial, r.virial.T, atol=1e-11)


def test_water_forces_sum_to_zero_and_virial_symmetric():
    cfg = I.water_model()
    fr = I.water_frame(0)
    p = I.make_params(cfg, 0)
    r = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box)
    assert np.abs(r.force.sum(0)).max() < 1e-12 * fr.natoms
    np.testing.assert_allclose(r.virial, r.virial.T, atol=1e-12)


def test_water_forces_spot_central_differences():
    cfg = I.water_model()
    fr = I.water_frame(0)
    p = I.make_params(cfg, 0)
    r = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box, nthreads=0)
    h = 1e-5
    for i, a in ((0, 0), (1, 2), (100, 1)):
        cp = fr.coord.copy()
        cm = fr.coord.copy()
        cp[i, a] += h
        cm[i, a] -= h
        ep = oracle.compute(cfg, p, cp, fr.atype, fr.box).energy
        em = oracle.compute(cfg, p, cm, fr.atype, fr.box).energy
        assert r.force[i, a] == pytest.approx(-(ep - em) / (2 * h), abs=5e-8)


def _rotation(seed):
    q, _ = np.linalg.qr(I.Rng(seed).normal(9).reshape(3, 3))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    return q


def test_translation_rotation_permutation_invariance():
    cfg, fr, p, _ = _tiny_case(seed=9)
    base = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box)
    # translation (neighbour list rebuilt from the moved coordinates)
    t = oracle.compute(cfg, p, fr.coord + np.array([3.3, -7.1, 12.9]), fr.atype, fr.box)
    assert t.energy == pytest.approx(base.energy, rel=1e-12)
    np.testing.assert_allclose(t.force, base.force, atol=1e-11)
    # rotation of coordinates and cell
    Q = _rotation(4)
    rr = oracle.compute(cfg, p, fr.coord @ Q, fr.atype, fr.box @ Q)
    assert rr.energy == pytest.approx(base.energy, rel=1e-12)
    np.testing.assert_allclose(rr.force, base.force @ Q, atol=1e-11)
    np.testing.assert_allclose(rr.virial, Q.T @ base.virial @ Q, atol=1e-11)
    # permutation of same-type atoms
    perm = np.arange(fr.natoms)
    same = [i for i in range(fr.natoms) if fr.atype[i] == fr.atype[0]]
    perm[same] = same[::-1]
    pr = oracle.compute(cfg, p, fr.coord[perm], fr.atype[perm], fr.box)
    assert pr.energy == pytest.approx(base.energy, rel=1e-12)
    np.testing.assert_allclose(pr.force, base.force[perm], atol=1e-11)


def test_energy_continuous_across_cutoff():
    """Move one atom radially across r_c of another: E(r_c - d) - E(r_c + d) = O(d^3)."""
    cfg = tiny_model()
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


# ----------------------------------------------------------------------------------------
# Compressed embedding (Eq. compress) against the network
# ----------------------------------------------------------------------------------------


def test_table_reproduces_nodes_and_bounds_error():
    cfg = I.water_model()
    p = I.make_params(cfg, 0)
    tab = oracle.table_build(cfg, p)
    nodes = np.concatenate([np.arange(181) * 0.01, 1.8 + np.arange(1, 3) * 0.1])
    for net in (0, 3):
        y, y1, y2 = oracle.embed_jets(cfg, p, net, nodes)
        c = tab[net]
        # value, slope, curvature of each piece at its left node and of the previous at its right node
        np.testing.assert_allclose(c[:, :, 5], y[:-1], rtol=0, atol=1e-14)
        np.testing.assert_allclose(c[:, :, 4], y1[:-1], rtol=0, atol=1e-14)
        np.testing.assert_allclose(2 * c[:, :, 3], y2[:-1], rtol=0, atol=1e-13)
        dx = np.diff(nodes)[:, None]
        right = ((((c[..., 0] * dx + c[..., 1]) * dx + c[..., 2]) * dx + c[..., 3]) * dx + c[..., 4]) * dx + c[..., 5]
        np.testing.assert_allclose(right, y[1:], rtol=0, atol=1e-11)
        # error on a fine grid inside the tabulated range
        xs = np.linspace(0.0, 2.0, 4001)[:-1]
        ref = oracle.embed_jets(cfg, p, net, xs)[0]
        li = np.where(xs < 1.8, np.floor(xs / 0.01), 180 + np.floor((xs - 1.8) / 0.1)).astype(int)
        li = np.minimum(li, 181)
        t = xs - nodes[li]
        cc = c[li]
        g = ((((cc[..., 0] * t[:, None] + cc[..., 1]) * t[:, None] + cc[..., 2]) * t[:, None] + cc[..., 3])
             * t[:, None] + cc[..., 4]) * t[:, None] + cc[..., 5]
        err = np.abs(g - ref)
        assert err[xs < 1.8].max() < 1e-9    # stride 0.01
        assert err.max() < 1e-4              # last 10 % at stride 0.1


def test_compressed_energy_and_forces_close_to_network():
    cfg = I.water_model()
    fr = I.water_frame(0)
    p = I.make_params(cfg, 0)
    tab = oracle.table_build(cfg, p)
    a = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box)
    b = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box, table=tab)
    assert b.status == 0
    assert abs(a.energy - b.energy) / fr.natoms < 1e-9
    assert np.abs(a.force - b.force).max() < 1e-9
    np.testing.assert_allclose(a.virial, b.virial, atol=1e-9)


def test_compressed_forces_vs_dual_of_compressed_energy():
    """The compressed reverse pass uses the analytic derivative of each quintic piece;
    check it against central differences of the compressed energy."""
    cfg, fr, p, nl = _tiny_case()
    tab = oracle.table_build(cfg, p)
    r = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box, nl=nl, table=tab)
    h = 1e-5
    for i, a in ((0, 0), (3, 1), (7, 2), (11, 0)):
        cp = fr.coord.copy()
        cm = fr.coord.copy()
        cp[i, a] += h
        cm[i, a] -= h
        ep = oracle.compute(cfg, p, cp, fr.atype, fr.box, nl=nl, table=tab).energy
        em = oracle.compute(cfg, p, cm, fr.atype, fr.box, nl=nl, table=tab).energy
        assert r.force[i, a] == pytest.approx(-(ep - em) / (2 * h), abs=2e-7)


def _loss_from_compute(cfg, p, frames, e_ref, f_ref, pE, pF, pV=0.0, v_ref=None):
    """The Sec. II.B loss (Eq. (loss)) evaluated from the oracle's plain energy/force/virial results."""
    L = 0.0
    for k, (fr, er, fref) in enumerate(zip(frames, e_ref, f_ref)):
        r = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box)
        n = fr.natoms
        L += pE * (r.energy - er) ** 2 / n + pF * float(((r.force - fref) ** 2).sum()) / (3 * n)
        if v_ref is not None:
            L += pV * float(((r.virial - v_ref[k]) ** 2).sum()) / (9 * n)
    return L / len(frames)


def test_loss_direction_derivative_vs_central_differences():
    """The hyper-dual loss derivative (energy and force terms, the latter a mixed second
    derivative of E) against central differences of the loss computed from plain results,
    for random parameter directions and for directions confined to one net."""
    cfg = tiny_model()
    p = I.make_params(cfg, 5)
    frames = [tiny_frame(seed=s) for s in (3, 4)]
    q = I.make_params(cfg, 6)
    e_ref, f_ref = [], []
    for fr in frames:
        r = oracle.compute(cfg, q, fr.coord, fr.atype, fr.box)
        e_ref.append(r.energy)
        f_ref.append(r.force)
    e_ref = np.array(e_ref)
    rng = I.Rng(17)
    n = p.size
    n_emb = sum(a * b + b for a, b in cfg.embed_layer_shapes()) * cfg.n_embed_nets
    dirs = [rng.normal(n), np.r_[rng.normal(n_emb), np.zeros(n - n_emb)], np.r_[np.zeros(n_emb), rng.normal(n - n_emb)]]
    for pE, pF in ((1.0, 0.0), (0.0, 1.0), (0.3, 2.0)):
        L0 = _loss_from_compute(cfg, p, frames, e_ref, f_ref, pE, pF)
        for v in dirs:
            L, dL = oracle.loss_dir(cfg, p, v, frames, e_ref, f_ref, pE, pF)
            assert abs(L - L0) <= 1e-12 * max(1.0, abs(L0))
            h = 1e-5
            fd = (_loss_from_compute(cfg, p + h * v, frames, e_ref, f_ref, pE, pF)
                  - _loss_from_compute(cfg, p - h * v, frames, e_ref, f_ref, pE, pF)) / (2 * h)
            assert abs(dL - fd) <= 1e-6 * max(abs(fd), 1e-3 * abs(L0)), (pE, pF, dL, fd)


# ----------------------------------------------------------------------------------------
# Whole forward (descriptor assembly and the fitting net's hidden layers) against numpy
# ----------------------------------------------------------------------------------------


def _numpy_fit(cfg, params, ai, D):
    """Eq. (NN) for the fitting net of type ai on descriptor rows D [n, M M_<]: tanh hidden
    layers with the identity skip where the width is kept (the {x,x} skip where it doubles),
    then the linear width-1 output layer (Eq. (fitting_energy)); numpy matmul and tanh."""
    off = cfg.n_embed_nets * sum(a * b + b for a, b in cfg.embed_layer_shapes())
    off += ai * sum(a * b + b for a, b in cfg.fit_layer_shapes())
    shapes = cfg.fit_layer_shapes()
    x = D
    for k, (fi, fo) in enumerate(shapes):
        W = params[off:off + fi * fo].reshape(fi, fo)
        b = params[off + fi * fo: off + fi * fo + fo]
        off += fi * fo + fo
        z = x @ W + b
        if k == len(shapes) - 1:
            x = z
            continue
        y = np.tanh(z)
        if fo == fi:
            y = y + x
        elif fo == 2 * fi:
            y = y + np.concatenate([x, x], axis=1)
        x = y
    return x[:, 0]


def _numpy_atom_energies(cfg, params, fr, nl_j, nl_shift):
    """E_i from a given neighbour list with numpy only: r_ij = r_j + n.h - r_i, R rows
    (s, s x/r, s y/r, s z/r) (s from the pinned switch), G by `_numpy_net`, T = G^T R / Nc,
    D = T T_<^T flattened row-major, then `_numpy_fit`."""
    N, nc, M, A = fr.natoms, cfg.nc, cfg.m, cfg.axis
    valid = nl_j >= 0
    j = np.where(valid, nl_j, 0)
    d = fr.coord[j] + nl_shift.astype(np.float64) @ fr.box - fr.coord[:, None, :]
    r = np.sqrt((d * d).sum(-1))
    s = np.zeros_like(r)
    for idx in zip(*np.nonzero(valid)):
        s[idx] = oracle.switch(float(r[idx]), cfg.rcut_smth, cfg.rcut)[0]
    R = np.zeros((N, nc, 4))
    R[..., 0] = s
    R[..., 1:] = s[..., None] * d / np.where(valid, r, 1.0)[..., None]
    G = np.zeros((N, nc, M))
    off = np.cumsum([0] + list(cfg.sel))
    for ai in range(cfg.ntypes):
        rows = np.nonzero(fr.atype == ai)[0]
        for t in range(cfg.ntypes):
            net = t if cfg.type_one_side else ai * cfg.ntypes + t
            blk = s[np.ix_(rows, np.arange(off[t], off[t + 1]))]
            G[np.ix_(rows, np.arange(off[t], off[t + 1]))] = _numpy_net(cfg, params, net, blk.ravel()).reshape(
                blk.shape + (M,))
    T = np.einsum("ikm,ikc->imc", G, R) / nc
    D = np.einsum("imc,ilc->iml", T, T[:, :A, :]).reshape(N, M * A)
    e = np.zeros(N)
    for ai in range(cfg.ntypes):
        rows = fr.atype == ai
        e[rows] = _numpy_fit(cfg, params, ai, D[rows])
    return e


@pytest.mark.parametrize("case", ["water", "tiny", "tiny_one_side"])
def test_atom_energies_vs_numpy_forward(case):
    """The oracle's atomic energies against an independent numpy evaluation of the whole forward
    (R, embedding, descriptor, and the fitting net with its tanh hidden layers, identity skips
    and linear output layer) on the oracle's own neighbour list (pinned separately against an
    independent enumeration).  A wrong skip, activation, layer order or flatten order of D in
    the oracle's fitting net changes every E_i."""
    if case == "water":
        cfg, fr = I.water_model(), I.water_frame(0)
    else:
        cfg, fr = tiny_model(type_one_side=int(case == "tiny_one_side")), tiny_frame(seed=4)
    p = I.make_params(cfg, 2)
    nl_j, nl_s, _, _ = oracle.nlist(cfg, fr.coord, fr.atype, fr.box)
    res = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box, nl=(nl_j, nl_s))
    ref = _numpy_atom_energies(cfg, p, fr, nl_j, nl_s)
    np.testing.assert_allclose(res.atom_energy, ref, rtol=1e-12, atol=1e-12)


# ----------------------------------------------------------------------------------------
# Sampled-atom oracle (reference of the full-size GPU checks) against the full oracle
# ----------------------------------------------------------------------------------------


@pytest.mark.parametrize("case", ["tiny_triclinic", "water_far_images", "fcc"])
def test_atom_subset_equals_full_oracle(case):
    """orc_atom_subset builds each sampled atom's rows by its own brute force; they must equal
    the full oracle's rows bit for bit and its atomic energies, also with coordinates several
    boxes outside the cell and in a cell narrower than 2 r_c."""
    if case == "tiny_triclinic":
        cfg, fr = tiny_model(), tiny_frame(seed=6)
    elif case == "water_far_images":
        cfg, fr = I.water_model(), I.water_frame(1)
        k = np.arange(fr.natoms) % 5 - 2  # shift atoms by -2 .. +2 box vectors
        fr = I.Frame(fr.coord + k[:, None] * fr.box[0] - (k[:, None] // 2) * fr.box[2], fr.atype, fr.box)
    else:
        cfg = I.ModelConfig(ntypes=1, rcut=5.0, rcut_smth=0.5, sel=(80,), embed=(8, 16), axis=4, fit=(16, 16))
        fr = I.fcc_frame((3, 3, 3), seed=2)
    p = I.make_params(cfg, 3)
    nl_j, nl_s, _, _ = oracle.nlist(cfg, fr.coord, fr.atype, fr.box)  # sel overflow included
    full = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box, nl=(nl_j, nl_s))
    idx = np.arange(0, fr.natoms, 3)
    sj, ss, se = oracle.atom_subset(cfg, p, fr.coord, fr.atype, fr.box, idx)
    np.testing.assert_array_equal(sj, nl_j[idx])
    np.testing.assert_array_equal(ss, nl_s[idx])
    np.testing.assert_allclose(se, full.atom_energy[idx], rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("case", ["tiny_triclinic", "water", "fcc"])
def test_force_subset_equals_full_oracle(case):
    """orc_force_subset forms only the sampled atoms' neighbourhoods; their forces and energies
    must equal the full oracle's (up to summation order), including periodic images of the atom
    itself in a cell narrower than 2 r_c and sel truncation."""
    if case == "tiny_triclinic":
        cfg, fr = tiny_model(), tiny_frame(seed=6)
    elif case == "water":
        cfg, fr = I.water_model(), I.water_frame(2)
    else:
        cfg = I.ModelConfig(ntypes=1, rcut=5.0, rcut_smth=0.5, sel=(80,), embed=(8, 16), axis=4, fit=(16, 16))
        fr = I.fcc_frame((3, 3, 3), seed=2)
    p = I.make_params(cfg, 4)
    full = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box)
    idx = np.array([0, 1, fr.natoms // 2, fr.natoms - 1])
    f, e = oracle.force_subset(cfg, p, fr.coord, fr.atype, fr.box, idx)
    fs = np.abs(full.force).max()
    np.testing.assert_allclose(f, full.force[idx], rtol=0, atol=1e-12 * fs)
    np.testing.assert_allclose(e, full.atom_energy[idx], rtol=1e-13, atol=1e-13)


def test_loss_direction_derivative_with_virial_term():
    """The virial term of Eq. (loss): its hyper-dual derivative (a homogeneous deformation in the
    e1 direction) against central differences of the loss computed from plain oracle energies,
    forces and virials, alone and together with the energy and force terms."""
    cfg = tiny_model()
    p = I.make_params(cfg, 5)
    frames = [tiny_frame(seed=s) for s in (3, 4)]
    q = I.make_params(cfg, 6)
    e_ref, f_ref, v_ref = [], [], []
    for fr in frames:
        r = oracle.compute(cfg, q, fr.coord, fr.atype, fr.box)
        e_ref.append(r.energy)
        f_ref.append(r.force)
        v_ref.append(r.virial)
    e_ref, v_ref = np.array(e_ref), np.array(v_ref)
    rng = I.Rng(23)
    n = p.size
    n_emb = sum(a * b + b for a, b in cfg.embed_layer_shapes()) * cfg.n_embed_nets
    dirs = [rng.normal(n), np.r_[rng.normal(n_emb), np.zeros(n - n_emb)], np.r_[np.zeros(n_emb), rng.normal(n - n_emb)]]
    for pE, pF, pV in ((0.0, 0.0, 1.0), (0.3, 2.0, 0.7)):
        L0 = _loss_from_compute(cfg, p, frames, e_ref, f_ref, pE, pF, pV, v_ref)
        for v in dirs:
            L, dL = oracle.loss_dir(cfg, p, v, frames, e_ref, f_ref, pE, pF, pV, v_ref)
            assert abs(L - L0) <= 1e-12 * max(1.0, abs(L0))
            h = 1e-5
            fd = (_loss_from_compute(cfg, p + h * v, frames, e_ref, f_ref, pE, pF, pV, v_ref)
                  - _loss_from_compute(cfg, p - h * v, frames, e_ref, f_ref, pE, pF, pV, v_ref)) / (2 * h)
            assert abs(dL - fd) <= 1e-6 * max(abs(fd), 1e-3 * abs(L0)), (pE, pF, pV, dL, fd)


# ----------------------------------------------------------------------------------------
# Model deviation (Sec. II.C)
# ----------------------------------------------------------------------------------------


def test_model_deviation_special_cases():
    """Identical models deviate by zero; for two models the deviation of atom i is exactly half
    the distance between their forces, |F_i^1 - F_i^2| / 2 (and the virial one |Xi^1 - Xi^2| /(2N)),
    and the statistics are the largest, mean and smallest of those; the relative form divides by
    |<F_i>| + nu."""
    cfg, fr = tiny_model(), tiny_frame(seed=5)
    p1, p2 = I.make_params(cfg, 1), I.make_params(cfg, 2)
    ef, ev, st, fm = oracle.model_deviation([(cfg, p1), (cfg, p1), (cfg, p1)], fr.coord, fr.atype, fr.box)
    a = oracle.compute(cfg, p1, fr.coord, fr.atype, fr.box)
    scale = np.abs(a.force).max()  # zero up to the rounding of a mean of equal values
    assert np.abs(ef).max() <= 1e-15 * scale and np.abs(st).max() <= 1e-15 * scale
    assert np.abs(ev).max() <= 1e-15 * np.abs(a.virial).max() / fr.natoms
    b = oracle.compute(cfg, p2, fr.coord, fr.atype, fr.box)
    ef, ev, st, fm = oracle.model_deviation([(cfg, p1), (cfg, p2)], fr.coord, fr.atype, fr.box)
    half = np.linalg.norm(a.force - b.force, axis=1) / 2
    np.testing.assert_allclose(ef, half, rtol=1e-12)
    np.testing.assert_allclose(ev, np.abs(a.virial - b.virial) / (2 * fr.natoms), rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose(fm, (a.force + b.force) / 2, rtol=1e-12)
    assert st[0] == half.max() and st[2] == half.min() and st[1] == pytest.approx(half.mean(), rel=1e-12)
    nu = 0.1
    er, _, _, _ = oracle.model_deviation([(cfg, p1), (cfg, p2)], fr.coord, fr.atype, fr.box, nu=nu)
    np.testing.assert_allclose(er, half / (np.linalg.norm((a.force + b.force) / 2, axis=1) + nu), rtol=1e-12)
