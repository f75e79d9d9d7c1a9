"""Plain FP64 CPU oracle for the Deep Potential energy / force / virial path (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py.  The product path never imports it.

The C++ source (dp_oracle.cpp) restates the DeePMD-kit v2 paper (arXiv 2304.09409)
directly; see its header for the equation-by-equation map.  This wrapper only marshals
numpy arrays.  Model configurations are duck-typed: any object with attributes
ntypes, sel, rcut, rcut_smth, embed, axis, fit, type_one_side, and optionally descriptor
(0 se_e2_a, 1 se_e2_r, 2 hybrid se_e2_a + se_e2_r, 3 se_e3, 4 hybrid se_e2_a + se_e3) with the
hybrid's second part in rcut_2, rcut_smth_2, sel_2, embed_2.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dp_oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libdporacle.so")

# Quintic table layout used by the paper's workloads: s in [0, 2]; stride 0.01 on the
# first 90 % of the range (180 intervals) and 0.1 on the last 10 % (2 intervals).
TABLE_S0 = 0.0
TABLE_STRIDE1 = 0.01
TABLE_N1 = 180
TABLE_STRIDE2 = 0.1
TABLE_N2 = 2


def compile_source(src: str, out: str) -> str:
    """Compile one oracle source file into the shared library `out` with g++ (no fused
    multiply-add contraction, OpenMP over atoms)."""
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           src, "-o", out]
    subprocess.run(cmd, check=True)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle (dp_oracle.cpp) into oracle/_build, unless the library is newer than it."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    compile_source(_SRC, tmp)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Cfg(ctypes.Structure):
    _fields_ = [
        ("ntypes", ctypes.c_int),
        ("sel", ctypes.c_int * 8),
        ("rcut", ctypes.c_double),
        ("rcut_smth", ctypes.c_double),
        ("n_embed", ctypes.c_int),
        ("embed", ctypes.c_int * 8),
        ("axis", ctypes.c_int),
        ("n_fit", ctypes.c_int),
        ("fit", ctypes.c_int * 8),
        ("type_one_side", ctypes.c_int),
        ("descriptor", ctypes.c_int),
        ("rcut_2", ctypes.c_double),
        ("rcut_smth_2", ctypes.c_double),
        ("sel_2", ctypes.c_int * 8),
        ("n_embed_2", ctypes.c_int),
        ("embed_2", ctypes.c_int * 8),
    ]


_lib = None


def _L():
    global _lib
    if _lib is None:
        # DP_ORACLE_LIB names a library compiled from a modified copy of dp_oracle.cpp: the
        # pin-strength test plants one mistake per copy and runs the pins against each
        _lib = ctypes.CDLL(os.environ.get("DP_ORACLE_LIB") or build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        cp = ctypes.POINTER(_Cfg)
        _lib.orc_n_params.argtypes = [cp]
        _lib.orc_n_params.restype = ctypes.c_long
        _lib.orc_switch.argtypes = [ctypes.c_double] * 3 + [dp, dp]
        _lib.orc_quintic.argtypes = [ctypes.c_double] * 7 + [dp]
        _lib.orc_nlist.argtypes = [cp, ctypes.c_int, dp, ip, dp, ip, ip, ip]
        _lib.orc_nlist.restype = ctypes.c_int
        _lib.orc_embed_jets.argtypes = [cp, dp, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
        _lib.orc_table_build.argtypes = [cp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_int, dp]
        _lib.orc_compute.argtypes = [cp, dp, ctypes.c_int, dp, ip, dp, ip, ip, dp, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int, ctypes.c_double, ctypes.c_int, dp, dp, dp, dp, ctypes.c_int]
        _lib.orc_compute.restype = ctypes.c_int
        _lib.orc_energy_dual.argtypes = [cp, dp, ctypes.c_int, dp, dp, ip, dp, dp, ip, ip, dp, dp]
        _lib.orc_energy_dual.restype = ctypes.c_double
        _lib.orc_energy_plain.argtypes = [cp, dp, ctypes.c_int, dp, ip, dp, ip, ip]
        _lib.orc_energy_plain.restype = ctypes.c_double
        _lib.orc_atom_subset.argtypes = [cp, dp, ctypes.c_int, dp, ip, dp, ctypes.c_int, ip, ip, ip, dp]
        _lib.orc_atom_subset.restype = ctypes.c_int
        _lib.orc_force_subset.argtypes = [cp, dp, ctypes.c_int, dp, ip, dp, ctypes.c_int, ip, dp, dp, ctypes.c_int]
        _lib.orc_force_subset.restype = ctypes.c_int
    return _lib


def _cfg(cfg) -> _Cfg:
    c = _Cfg()
    c.ntypes = int(cfg.ntypes)
    for t, v in enumerate(cfg.sel):
        c.sel[t] = int(v)
    c.rcut = float(cfg.rcut)
    c.rcut_smth = float(cfg.rcut_smth)
    c.n_embed = len(cfg.embed)
    for k, v in enumerate(cfg.embed):
        c.embed[k] = int(v)
    c.axis = int(cfg.axis)
    c.n_fit = len(cfg.fit)
    for k, v in enumerate(cfg.fit):
        c.fit[k] = int(v)
    c.type_one_side = int(getattr(cfg, "type_one_side", 0))
    c.descriptor = int(getattr(cfg, "descriptor", 0))
    if c.descriptor in (2, 4):  # hybrid: the second part's cutoffs, sel and nets
        c.rcut_2 = float(getattr(cfg, "rcut_2", 0.0) or cfg.rcut)
        c.rcut_smth_2 = float(getattr(cfg, "rcut_smth_2", 0.0) or cfg.rcut_smth)
        sel_2 = tuple(getattr(cfg, "sel_2", ()) or cfg.sel)
        for t, v in enumerate(sel_2):
            c.sel_2[t] = int(v)
        embed_2 = tuple(cfg.embed_2)
        c.n_embed_2 = len(embed_2)
        for k, v in enumerate(embed_2):
            c.embed_2[k] = int(v)
    return c


def _d(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.int32)


def n_params(cfg) -> int:
    c = _cfg(cfg)
    return int(_L().orc_n_params(ctypes.byref(c)))


def switch(r: float, rs: float, rc: float):
    """Eq. (switch): returns (s(r), ds/dr)."""
    s = ctypes.c_double()
    ds = ctypes.c_double()
    _L().orc_switch(r, rs, rc, ctypes.byref(s), ctypes.byref(ds))
    return s.value, ds.value


def quintic(y0, y1, d0, d1, dd0, dd1, dx) -> np.ndarray:
    """Eq. (compress): coefficients (a, b, c, d, e, f) of one interval."""
    out = np.zeros(6)
    _L().orc_quintic(y0, y1, d0, d1, dd0, dd1, dx, _d(out))
    return out


def nlist(cfg, coord, atype, box):
    """Brute-force neighbour list.  Returns (nl_j [N, Nc] int32, nl_shift [N, Nc, 3] int32,
    counts [N, ntypes] int32, n_overflow)."""
    coord = _f64(coord)
    atype = _i32(atype)
    box = _f64(box)
    N = coord.shape[0]
    nc = int(cfg.nc)
    nl_j = np.zeros((N, nc), dtype=np.int32)
    nl_s = np.zeros((N, nc, 3), dtype=np.int32)
    counts = np.zeros((N, cfg.ntypes), dtype=np.int32)
    c = _cfg(cfg)
    ov = _L().orc_nlist(ctypes.byref(c), N, _d(coord), _i(atype), _d(box), _i(nl_j), _i(nl_s), _i(counts))
    return nl_j, nl_s, counts, ov


def embed_jets(cfg, params, net: int, xs):
    """Embedding-net outputs y and derivatives y', y'' (w.r.t. the scalar input) at xs."""
    xs = _f64(np.atleast_1d(xs))
    M = int(cfg.embed[-1])
    y = np.zeros((xs.size, M))
    y1 = np.zeros_like(y)
    y2 = np.zeros_like(y)
    c = _cfg(cfg)
    _L().orc_embed_jets(ctypes.byref(c), _d(_f64(params)), net, xs.size, _d(xs), _d(y), _d(y1), _d(y2))
    return y, y1, y2


def table_layout(cfg):
    """Node grid (x0, stride1, n1, stride2, n2) of the first part's tables: s in [0, 1/r_s] with stride
    0.01 on the first 90 % and 0.1 on the rest; for se_e3 the pieces are in theta = R_j . R_k, which
    lies in [0, 2 s_max^2] (|R_j|^2 = 2 s_j^2 and 1 + cos >= 0), the same grid scaled by 2 / r_s."""
    smax = 1.0 / cfg.rcut_smth
    n1 = int(np.floor(0.9 * smax / 0.01 + 0.5))
    rest = smax - n1 * 0.01
    n2 = max(1, int(np.ceil(rest / 0.1 - 1e-9))) if rest > 0 else 1
    scale = 2.0 / cfg.rcut_smth if getattr(cfg, "descriptor", 0) == 3 else 1.0
    return (0.0, 0.01 * scale, n1, 0.1 * scale, n2)


def table_build(cfg, params, s0=TABLE_S0, stride1=TABLE_STRIDE1, n1=TABLE_N1, stride2=TABLE_STRIDE2, n2=TABLE_N2):
    """Eq. (compress) tables for every embedding net: [nets, n1+n2, M, 6] (a..f)."""
    nets = int(cfg.n_embed_nets) if hasattr(cfg, "n_embed_nets") else (
        cfg.ntypes if getattr(cfg, "type_one_side", 0) else cfg.ntypes ** 2)
    M = int(cfg.embed[-1])
    tab = np.zeros((nets, n1 + n2, M, 6))
    c = _cfg(cfg)
    _L().orc_table_build(ctypes.byref(c), _d(_f64(params)), s0, stride1, n1, stride2, n2, _d(tab))
    return tab


class Result:
    def __init__(self, energy, force, virial, atom_energy, status):
        self.energy = energy
        self.force = force
        self.virial = virial
        self.atom_energy = atom_energy
        self.status = status


def compute(cfg, params, coord, atype, box, nl=None, table=None, table_layout=None, nthreads: int = 0) -> Result:
    """E, F [N,3], virial [3,3], per-atom E.  nl = (nl_j, nl_shift) or None (brute force).
    table = quintic table from `table_build` (compressed embedding) or None (network)."""
    coord = _f64(coord)
    atype = _i32(atype)
    box = _f64(box)
    params = _f64(params)
    N = coord.shape[0]
    force = np.zeros((N, 3))
    virial = np.zeros((3, 3))
    ae = np.zeros(N)
    e = ctypes.c_double()
    nl_j = nl_s = None
    if nl is not None:
        nl_j = _i32(nl[0])
        nl_s = _i32(nl[1])
    tab = _f64(table)
    lay = table_layout or (TABLE_S0, TABLE_STRIDE1, TABLE_N1, TABLE_STRIDE2, TABLE_N2)
    c = _cfg(cfg)
    st = _L().orc_compute(ctypes.byref(c), _d(params), N, _d(coord), _i(atype), _d(box), _i(nl_j), _i(nl_s), _d(tab),
                          lay[0], lay[1], lay[2], lay[3], lay[4], ctypes.byref(e), _d(force), _d(virial), _d(ae),
                          int(nthreads))
    return Result(e.value, force, virial, ae, st)


def energy_dual(cfg, params, coord, atype, box, nl, dcoord=None, dbox=None):
    """Forward-mode dual-number derivative of E along (dcoord, dbox), nlist held fixed.
    Returns (E, dE)."""
    coord = _f64(coord)
    N = coord.shape[0]
    dE = ctypes.c_double()
    c = _cfg(cfg)
    E = _L().orc_energy_dual(ctypes.byref(c), _d(_f64(params)), N, _d(coord), _d(_f64(dcoord)), _i(_i32(atype)),
                             _d(_f64(box)), _d(_f64(dbox)), _i(_i32(nl[0])), _i(_i32(nl[1])), ctypes.byref(dE), None)
    return E, dE.value


def energy_plain(cfg, params, coord, atype, box, nl) -> float:
    """E through the generic (templated) forward in plain doubles."""
    coord = _f64(coord)
    c = _cfg(cfg)
    return _L().orc_energy_plain(ctypes.byref(c), _d(_f64(params)), coord.shape[0], _d(coord), _i(_i32(atype)),
                                 _d(_f64(box)), _i(_i32(nl[0])), _i(_i32(nl[1])))


def atom_subset(cfg, params, coord, atype, box, idx):
    """Neighbour rows (nl_j [S, Nc], nl_shift [S, Nc, 3]) and atomic energies [S] of the atoms
    `idx` only, for sampled checks of frames too large for the full oracle."""
    coord = _f64(coord)
    idx = _i32(np.atleast_1d(idx))
    S = idx.size
    nc = int(cfg.nc)
    nl_j = np.zeros((S, nc), dtype=np.int32)
    nl_s = np.zeros((S, nc, 3), dtype=np.int32)
    e = np.zeros(S)
    c = _cfg(cfg)
    _L().orc_atom_subset(ctypes.byref(c), _d(_f64(params)), coord.shape[0], _d(coord), _i(_i32(atype)), _d(_f64(box)),
                         S, _i(idx), _i(nl_j), _i(nl_s), _d(e))
    return nl_j, nl_s, e


def force_subset(cfg, params, coord, atype, box, idx, nthreads: int = 0):
    """Forces [S, 3] and atomic energies [S] of the atoms `idx` only (their neighbourhoods
    within r_c evaluated by brute force), for sampled checks of frames too large for the full
    oracle.  Network embedding."""
    coord = _f64(coord)
    idx = _i32(np.atleast_1d(idx))
    S = idx.size
    f = np.zeros((S, 3))
    e = np.zeros(S)
    c = _cfg(cfg)
    _L().orc_force_subset(ctypes.byref(c), _d(_f64(params)), coord.shape[0], _d(coord), _i(_i32(atype)),
                          _d(_f64(box)), S, _i(idx), _d(f), _d(e), int(nthreads))
    return f, e


def _pack_frames(cfg, frames):
    nat = np.array([f.natoms for f in frames], dtype=np.int32)
    coord = np.ascontiguousarray(np.concatenate([f.coord for f in frames]), dtype=np.float64)
    atype = np.ascontiguousarray(np.concatenate([f.atype for f in frames]), dtype=np.int32)
    boxes = np.ascontiguousarray(np.stack([f.box for f in frames]).reshape(-1, 9), dtype=np.float64)
    njs, nss, off = [], [], 0
    for f in frames:
        nj, ns, _, _ = nlist(cfg, f.coord, f.atype, f.box)
        njs.append(np.where(nj >= 0, nj + off, -1))
        nss.append(ns)
        off += f.natoms
    return nat, coord, atype, boxes, np.ascontiguousarray(np.concatenate(njs), dtype=np.int32), \
        np.ascontiguousarray(np.concatenate(nss), dtype=np.int32)


def loss_dir(cfg, params, vdir, frames, e_ref, f_ref, pE=1.0, pF=1.0, pV=0.0, v_ref=None):
    """Energy + force (+ virial) loss of a batch of frames (Sec. II.B, Eq. (loss)) and its
    derivative along the parameter direction vdir (hyper-dual numbers).  v_ref: [B, 3, 3]
    reference virials, or None for no virial term.  Returns (L, dL . vdir)."""
    L_ = _L()
    if not hasattr(L_, "_loss_set"):
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        L_.orc_loss_dir.argtypes = [ctypes.POINTER(_Cfg), dp, dp, ctypes.c_int, ip, dp, ip, dp, ip, ip, dp, dp,
                                    ctypes.c_double, ctypes.c_double, dp, dp, ctypes.c_double]
        L_.orc_loss_dir.restype = ctypes.c_double
        L_._loss_set = True
    nat, coord, atype, boxes, nj, ns = _pack_frames(cfg, frames)
    dL = ctypes.c_double()
    c = _cfg(cfg)
    vr = None if v_ref is None else np.ascontiguousarray(np.asarray(v_ref, dtype=np.float64).reshape(-1, 9))
    val = L_.orc_loss_dir(ctypes.byref(c), _d(_f64(params)), _d(_f64(vdir)), len(frames), _i(nat), _d(coord),
                          _i(atype), _d(boxes), _i(nj), _i(ns), _d(_f64(e_ref)), _d(_f64(np.concatenate(f_ref))),
                          float(pE), float(pF), ctypes.byref(dL), _d(vr), float(pV))
    return val, dL.value


def model_deviation(cfg_params, coord, atype, box, nu: float = 0.0):
    """Model deviation of an ensemble on one frame (Sec. II.C), from the oracle's forces and
    virials of every model: eps_F,i = sqrt(<|F_i - <F_i>|^2>) and
    eps_Xi,ab = (1/N) sqrt(<(Xi_ab - <Xi_ab>)^2>), <.> the ensemble mean; with nu > 0 the
    relative forms eps_F,i / (|<F_i>| + nu) and eps_Xi,ab / (|<Xi>| + nu) (Frobenius norm).
    cfg_params: [(cfg, params), ...].  Returns (devi_f [N], devi_v [3, 3], stats [6] =
    (max, mean, min of eps_F,i, max, mean, min of eps_Xi,ab), force_mean [N, 3])."""
    res = [compute(c, p, coord, atype, box) for c, p in cfg_params]
    Fk = np.stack([r.force for r in res])      # [n_m, N, 3]
    Vk = np.stack([r.virial for r in res])     # [n_m, 3, 3]
    N = Fk.shape[1]
    fm = Fk.mean(axis=0)
    ef = np.sqrt(((Fk - fm[None]) ** 2).sum(axis=2).mean(axis=0))
    vm = Vk.mean(axis=0)
    ev = np.sqrt(((Vk - vm[None]) ** 2).mean(axis=0)) / N
    if nu > 0.0:
        ef = ef / (np.linalg.norm(fm, axis=1) + nu)
        ev = ev / (np.linalg.norm(vm) + nu)
    stats = np.array([ef.max(), ef.mean(), ef.min(), ev.max(), ev.mean(), ev.min()])
    return ef, ev, stats, fm
