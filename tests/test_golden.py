"""The stored expected values under tests/golden/ (written from the FP64 oracle alone by
tests/golden/make_golden.py) against the oracle as it stands, and against the laws the stored values
must obey whatever produced them.

A mismatch with the oracle means that the oracle's arithmetic or the seeded input generators changed
since the fixtures were written: such a change names, in its commit, the passage of the paper (or the
reading of it) that justifies it, and the fixtures are rewritten by the same command.
"""
import os
import sys

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_golden  # noqa: E402

CASES = [(fname, name, cfg, p, fr, comp)
         for fname, _, cases in make_golden._cases() for name, cfg, p, fr, comp in cases]
IDS = [c[1] for c in CASES]


def _stored(fname, name):
    return make_golden.read(os.path.join(HERE, "golden", fname))[name]


def test_every_fixture_case_is_listed():
    for fname, _, cases in make_golden._cases():
        stored = make_golden.read(os.path.join(HERE, "golden", fname))
        assert sorted(stored) == sorted(c[0] for c in cases)


@pytest.mark.parametrize("fname,name,cfg,p,fr,comp", CASES, ids=IDS)
def test_oracle_reproduces_fixture(fname, name, cfg, p, fr, comp):
    g = _stored(fname, name)
    tab = oracle.table_build(cfg, p) if comp else None
    res = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box, table=tab)
    # the oracle is deterministic up to the order of its threaded sums: 1e-12 relative is far above
    # that rounding and far below any change of a term
    escale = max(1.0, np.abs(g["atom_energy"]).max())
    assert abs(res.energy - g["energy"][0]) <= 1e-12 * escale * fr.natoms
    assert np.abs(res.atom_energy - g["atom_energy"]).max() <= 1e-12 * escale
    assert np.abs(res.force - g["force"]).max() <= 1e-12 * np.abs(g["force"]).max()
    assert np.abs(res.virial - g["virial"]).max() <= 1e-12 * np.abs(g["virial"]).max()
    if "nl_j" in g:
        nl_j, nl_s, _, _ = oracle.nlist(cfg, fr.coord, fr.atype, fr.box)
        np.testing.assert_array_equal(nl_j, g["nl_j"])
        np.testing.assert_array_equal(nl_s.reshape(nl_s.shape[0], -1), g["nl_shift"])


@pytest.mark.parametrize("fname,name,cfg,p,fr,comp", CASES, ids=IDS)
def test_fixture_obeys_invariants(fname, name, cfg, p, fr, comp):
    """E = sum of the atomic energies (Sec. II.A.2); sum of F = 0 (translation invariance);
    the virial is symmetric (rotation invariance)."""
    g = _stored(fname, name)
    n = fr.natoms
    assert abs(g["atom_energy"].sum() - g["energy"][0]) <= 1e-13 * np.abs(g["atom_energy"]).sum()
    fmax = np.abs(g["force"]).max()
    assert np.abs(g["force"].sum(axis=0)).max() <= 1e-13 * n * fmax
    v = g["virial"]
    assert np.abs(v - v.T).max() <= 1e-13 * np.abs(v).max()
    assert fmax > 0 and np.all(np.isfinite(g["force"]))


def test_compressed_fixture_within_table_error_of_network():
    """The Eq. (compress) tables interpolate each embedding output by a quintic on steps of 0.01 and
    0.1; the stored compressed result lies within that interpolation error of the network one."""
    net = _stored("water192.txt", "water192_network")
    tab = _stored("water192.txt", "water192_compressed")
    assert np.abs(tab["atom_energy"] - net["atom_energy"]).max() <= 1e-9
    assert np.abs(tab["force"] - net["force"]).max() <= 1e-9 * max(1.0, np.abs(net["force"]).max())


def test_stored_list_is_nearest_first_with_padding_last():
    """Sec. II.A.1 list layout: per centre, sel_t slots for each type t, filled nearest first and
    padded with -1; each listed j of type t at r < r_c."""
    fname, name, cfg, p, fr, _ = next(c for c in CASES if c[1] == "tiny_se_e2_a")
    g = _stored(fname, name)
    nl_j, sh = g["nl_j"], g["nl_shift"].reshape(fr.natoms, -1, 3)
    off = 0
    for t, sel in enumerate(cfg.sel):
        for i in range(fr.natoms):
            js = nl_j[i, off:off + sel]
            real = js >= 0
            assert np.all(real[:real.sum()]), "padding before a real slot"
            r2 = []
            for q in np.nonzero(real)[0]:
                j = js[q]
                assert fr.atype[j] == t
                d = fr.coord[j] + sh[i, off + q] @ fr.box - fr.coord[i]
                r2.append(float(d @ d))
            assert all(0.0 < x < cfg.rcut ** 2 for x in r2)
            assert all(a <= b for a, b in zip(r2, r2[1:]))
        off += sel
