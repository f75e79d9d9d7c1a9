"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module holds no arithmetic of the Deep Potential method itself: it only draws
random numbers and lays out atoms, model configurations and network parameters.
Both the oracle and the CUDA path receive the arrays produced here.

Random numbers: a counter-based SplitMix64 stream (Steele, Lea, Flood 2014) turned
into uniforms on [0, 1) with the top 53 bits, and into normals with the Box-Muller
transform.  The paper's datasets (water, Cu) are not available; the generators below
stand in for them with the system sizes and densities of the workloads described in
the paper's benchmark section (Sec. IV): liquid-water-like boxes at 1 g/cm^3 and a
Cu-like FCC crystal with a = 3.634 A.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _splitmix64(counter: np.ndarray) -> np.ndarray:
    """SplitMix64 output for each 64-bit counter value (state = counter * golden)."""
    with np.errstate(over="ignore"):
        z = counter * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


class Rng:
    """Counter-based SplitMix64 stream: value k of stream `seed` is mix((seed<<32) + k + 1)."""

    def __init__(self, seed: int):
        self.base = np.uint64((int(seed) & 0xFFFFFFFF) << 32)
        self.k = 0

    def bits(self, n: int) -> np.ndarray:
        ctr = self.base + np.arange(self.k + 1, self.k + 1 + n, dtype=np.uint64)
        self.k += n
        return _splitmix64(ctr)

    def uniform(self, n: int) -> np.ndarray:
        return (self.bits(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def normal(self, n: int) -> np.ndarray:
        m = (n + 1) // 2
        u1 = 1.0 - self.uniform(m)  # (0, 1]
        u2 = self.uniform(m)
        rad = np.sqrt(-2.0 * np.log(u1))
        z = np.concatenate([rad * np.cos(2.0 * math.pi * u2), rad * np.sin(2.0 * math.pi * u2)])
        return z[:n]


# ----------------------------------------------------------------------------------------------
# Model configuration (se_e2_a, Sec. II.A.1 and II.A.2) and parameter layout
# ----------------------------------------------------------------------------------------------

MAX_TYPES = 8
MAX_LAYERS = 8


@dataclasses.dataclass
class ModelConfig:
    ntypes: int
    rcut: float
    rcut_smth: float
    sel: Tuple[int, ...]
    embed: Tuple[int, ...]        # embedding net widths, input width 1 implied
    axis: int                     # M_<
    fit: Tuple[int, ...]          # fitting net hidden widths; a final width-1 linear layer is implied
    type_one_side: int = 0        # 0: nets N^{a_i,a_j}; 1: nets N^{a_j}
    # 0: se_e2_a; 1: se_e2_r; 2: hybrid se_e2_a + se_e2_r; 3: se_e3; 4: hybrid se_e2_a + se_e3
    descriptor: int = 0
    # hybrids: the second part's cutoffs (0: those of the first), sel (empty: that of the first)
    # and embedding widths
    rcut_2: float = 0.0
    rcut_smth_2: float = 0.0
    sel_2: Tuple[int, ...] = ()
    embed_2: Tuple[int, ...] = ()

    @property
    def hybrid(self) -> bool:
        return self.descriptor in (2, 4)

    @property
    def list_sel(self) -> Tuple[int, ...]:
        """Per-type width of the neighbour list all parts read: the larger sel of the parts."""
        if not self.hybrid:
            return tuple(self.sel)
        sel_2 = tuple(self.sel_2) or tuple(self.sel)
        return tuple(max(a, b) for a, b in zip(self.sel, sel_2))

    @property
    def list_rcut(self) -> float:
        return max(self.rcut, self.rcut_2 or self.rcut) if self.hybrid else self.rcut

    @property
    def nc(self) -> int:
        """Width of the neighbour list (sum of list_sel)."""
        return int(sum(self.list_sel))

    @property
    def m(self) -> int:
        return int(self.embed[-1])

    @property
    def n_embed_nets(self) -> int:
        """Nets of the first part: N^{a_i,a_j} or N^{a_j}; se_e3 nets N^{a_j,a_k}."""
        if self.descriptor == 3:
            return self.ntypes * self.ntypes
        return self.ntypes if self.type_one_side else self.ntypes * self.ntypes

    @property
    def n_embed_nets_2(self) -> int:
        if not self.hybrid:
            return 0
        if self.descriptor == 4:
            return self.ntypes * self.ntypes
        return self.ntypes if self.type_one_side else self.ntypes * self.ntypes

    @property
    def descriptor_dim(self) -> int:
        """Width of D: M * M_< (se_e2_a), M (se_e2_r, se_e3), or the sum of the parts (hybrid)."""
        if self.descriptor in (1, 3):
            return self.m
        if self.hybrid:
            return self.m * self.axis + int(self.embed_2[-1])
        return self.m * self.axis

    def embed_layer_shapes(self) -> List[Tuple[int, int]]:
        dims = [1] + list(self.embed)
        return [(dims[k], dims[k + 1]) for k in range(len(self.embed))]

    def embed_2_layer_shapes(self) -> List[Tuple[int, int]]:
        """Layer shapes of the hybrid's second-part nets (empty for the other descriptors)."""
        if not self.hybrid:
            return []
        dims = [1] + list(self.embed_2)
        return [(dims[k], dims[k + 1]) for k in range(len(self.embed_2))]

    def embed_params(self) -> int:
        """Parameters of all embedding nets (those of `embed`, then the hybrid's second part)."""
        p1 = sum(a * b + b for a, b in self.embed_layer_shapes())
        p2 = sum(a * b + b for a, b in self.embed_2_layer_shapes())
        return self.n_embed_nets * p1 + self.n_embed_nets_2 * p2

    def fit_layer_shapes(self) -> List[Tuple[int, int]]:
        dims = [self.descriptor_dim] + list(self.fit) + [1]
        return [(dims[k], dims[k + 1]) for k in range(len(dims) - 1)]

    def n_params(self) -> int:
        nf = sum(a * b + b for a, b in self.fit_layer_shapes())
        return self.embed_params() + self.ntypes * nf


def water_model() -> ModelConfig:
    """Water-like se_e2_a model: r_c 6, r_s 0.5, sel [46, 92], embedding 25/50/100, M_< 16, fitting 240^3."""
    return ModelConfig(ntypes=2, rcut=6.0, rcut_smth=0.5, sel=(46, 92), embed=(25, 50, 100), axis=16,
                       fit=(240, 240, 240))


def metal_model() -> ModelConfig:
    """Metal-like single-type model: r_c 8, r_s 0.5, sel [512], embedding 32/64/128, M_< 16, fitting 240^3."""
    return ModelConfig(ntypes=1, rcut=8.0, rcut_smth=0.5, sel=(512,), embed=(32, 64, 128), axis=16,
                       fit=(240, 240, 240))


def water_model_r() -> ModelConfig:
    """Water-like se_e2_r model: the water model's list (r_c 6, r_s 0.5, sel [46, 92]) with
    embedding 10/20/40 and the same fitting net (D has 40 values)."""
    return ModelConfig(ntypes=2, rcut=6.0, rcut_smth=0.5, sel=(46, 92), embed=(10, 20, 40), axis=0,
                       fit=(240, 240, 240), descriptor=1)


def water_model_hybrid() -> ModelConfig:
    """Water-like hybrid se_e2_a + se_e2_r: an se_e2_a part with r_c 4 (sel [20, 40], embedding
    25/50/100, M_< 16) and an se_e2_r part with r_c 6 (sel [46, 92], embedding 10/20/40); D has
    1640 values."""
    return ModelConfig(ntypes=2, rcut=4.0, rcut_smth=0.5, sel=(20, 40), embed=(25, 50, 100), axis=16,
                       fit=(240, 240, 240), descriptor=2, rcut_2=6.0, rcut_smth_2=0.5, sel_2=(46, 92),
                       embed_2=(10, 20, 40))


def water_model_e3() -> ModelConfig:
    """Water-like se_e3 model: r_c 6, r_s 0.5, sel [46, 92], embedding 2/4/8 (D has 8 values)."""
    return ModelConfig(ntypes=2, rcut=6.0, rcut_smth=0.5, sel=(46, 92), embed=(2, 4, 8), axis=0,
                       fit=(240, 240, 240), descriptor=3)


def water_model_hybrid_e3() -> ModelConfig:
    """Water-like hybrid se_e2_a + se_e3: the se_e2_a part with r_c 4 as in water_model_hybrid and
    an se_e3 part with r_c 6 (sel [46, 92], embedding 2/4/8); D has 1608 values."""
    return ModelConfig(ntypes=2, rcut=4.0, rcut_smth=0.5, sel=(20, 40), embed=(25, 50, 100), axis=16,
                       fit=(240, 240, 240), descriptor=4, rcut_2=6.0, rcut_smth_2=0.5, sel_2=(46, 92),
                       embed_2=(2, 4, 8))


def make_params(cfg: ModelConfig, seed: int = 0) -> np.ndarray:
    """Xavier-normal weights W ~ N(0, 2/(fan_in+fan_out)) and biases b ~ N(0, 1), FP64, flat.

    Layout (shared by every consumer): embedding nets in order of net index
    (a_i * ntypes + a_j, or a_j when type_one_side; a_j * ntypes + a_k for se_e3), then
    (hybrids only) the second part's embedding nets in the same order, then fitting nets by
    type; inside a net, layer by layer, W row-major [in][out] followed by b [out].
    """
    rng = Rng(seed)
    out = []
    nets = [(cfg.embed_layer_shapes(), cfg.n_embed_nets), (cfg.embed_2_layer_shapes(), cfg.n_embed_nets_2),
            (cfg.fit_layer_shapes(), cfg.ntypes)]
    for shapes, count in nets:
        for _ in range(count):
            for fi, fo in shapes:
                std = math.sqrt(2.0 / (fi + fo))
                out.append(rng.normal(fi * fo) * std)
                out.append(rng.normal(fo))
    p = np.concatenate(out).astype(np.float64)
    assert p.size == cfg.n_params()
    return p


# Output-layer scales that bring the seed-0 random-weight models to forces of about 1 eV/A RMS,
# the magnitude of forces in condensed-phase data: the seed-0 water model gives 5.0e-4 eV/A RMS
# on the water frames, the seed-0 metal model 8.2e-6 eV/A on the FCC frames.  Accuracy bars in
# eV/A (1e-3 eV/A for the mixed-precision path) are only meaningful at that force scale.
WATER_FORCE_SCALE = 2000.0
METAL_FORCE_SCALE = 1.2e5
# the same for the water-like se_e2_r (seed 0: 4.4e-3 eV/A RMS), hybrid se_e2_a + se_e2_r (1.1e-3),
# se_e3 (5.2e-4) and hybrid se_e2_a + se_e3 (3.9e-3) models
WATER_R_FORCE_SCALE = 230.0
WATER_HYBRID_FORCE_SCALE = 900.0
WATER_E3_FORCE_SCALE = 1950.0
WATER_HYBRID_E3_FORCE_SCALE = 255.0


def force_scaled(cfg: ModelConfig, params: np.ndarray, scale: float) -> np.ndarray:
    """Copy of `params` with the final (linear, width-1) fitting layer of every type -- its
    weights and its bias -- multiplied by `scale`: atomic energies, forces and virials all
    scale by exactly that factor, while every other layer is unchanged."""
    out = np.array(params, dtype=np.float64, copy=True)
    off = cfg.embed_params()
    shapes = cfg.fit_layer_shapes()
    per_type = sum(a * b + b for a, b in shapes)
    last_in = shapes[-1][0]
    for t in range(cfg.ntypes):
        o = off + t * per_type + sum(a * b + b for a, b in shapes[:-1])
        out[o:o + last_in + 1] *= scale  # W [last_in][1] then b [1]
    return out


def water_params_scaled(seed: int = 0) -> np.ndarray:
    """The water model's parameters with forces of about 1 eV/A RMS."""
    cfg = water_model()
    return force_scaled(cfg, make_params(cfg, seed), WATER_FORCE_SCALE)


def water_r_params_scaled(seed: int = 0) -> np.ndarray:
    """The water-like se_e2_r model's parameters with forces of about 1 eV/A RMS."""
    cfg = water_model_r()
    return force_scaled(cfg, make_params(cfg, seed), WATER_R_FORCE_SCALE)


def water_hybrid_params_scaled(seed: int = 0) -> np.ndarray:
    """The water-like hybrid model's parameters with forces of about 1 eV/A RMS."""
    cfg = water_model_hybrid()
    return force_scaled(cfg, make_params(cfg, seed), WATER_HYBRID_FORCE_SCALE)


def water_e3_params_scaled(seed: int = 0) -> np.ndarray:
    """The water-like se_e3 model's parameters with forces of about 1 eV/A RMS."""
    cfg = water_model_e3()
    return force_scaled(cfg, make_params(cfg, seed), WATER_E3_FORCE_SCALE)


def water_hybrid_e3_params_scaled(seed: int = 0) -> np.ndarray:
    """The water-like hybrid se_e2_a + se_e3 model's parameters with forces of about 1 eV/A RMS."""
    cfg = water_model_hybrid_e3()
    return force_scaled(cfg, make_params(cfg, seed), WATER_HYBRID_E3_FORCE_SCALE)


def metal_params_scaled(seed: int = 0) -> np.ndarray:
    """The metal model's parameters with forces of about 1 eV/A RMS."""
    cfg = metal_model()
    return force_scaled(cfg, make_params(cfg, seed), METAL_FORCE_SCALE)


# ----------------------------------------------------------------------------------------------
# Configurations (atoms)
# ----------------------------------------------------------------------------------------------

@dataclasses.dataclass
class Frame:
    coord: np.ndarray  # [N, 3] float64
    atype: np.ndarray  # [N] int32
    box: np.ndarray    # [3, 3] float64, rows are the cell vectors h_0, h_1, h_2

    @property
    def natoms(self) -> int:
        return int(self.coord.shape[0])


WATER_ML_PER_MOL_A3 = 18.01528 / 0.602214076  # A^3 per molecule at 1 g/cm^3 (29.915)
OH_BOND = 0.96
HOH_ANGLE_DEG = 104.52


def _unit_vectors(rng: Rng, n: int) -> np.ndarray:
    z = 2.0 * rng.uniform(n) - 1.0
    phi = 2.0 * math.pi * rng.uniform(n)
    rxy = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([rxy * np.cos(phi), rxy * np.sin(phi), z], axis=1)


def _place_hydrogens(rng: Rng, o: np.ndarray) -> np.ndarray:
    """Two H per O at 0.96 A: the first direction uniform on the sphere, the second at the
    HOH angle from it with a uniformly random azimuth."""
    n = o.shape[0]
    u = _unit_vectors(rng, n)
    # a vector not parallel to u, then an orthonormal pair (e1, e2) perpendicular to u
    helper = np.where(np.abs(u[:, :1]) < 0.9, np.array([[1.0, 0.0, 0.0]]), np.array([[0.0, 1.0, 0.0]]))
    e1 = np.cross(u, helper)
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(u, e1)
    psi = 2.0 * math.pi * rng.uniform(n)
    th = math.radians(HOH_ANGLE_DEG)
    v = math.cos(th) * u + math.sin(th) * (np.cos(psi)[:, None] * e1 + np.sin(psi)[:, None] * e2)
    h1 = o + OH_BOND * u
    h2 = o + OH_BOND * v
    return h1, h2


def _min_image_dist(o: np.ndarray, L: float) -> float:
    d = o[:, None, :] - o[None, :, :]
    d -= L * np.round(d / L)
    r = np.sqrt((d * d).sum(-1))
    np.fill_diagonal(r, np.inf)
    return float(r.min()) if o.shape[0] > 1 else np.inf


def water_frame(seed: int = 0, n_side: int = 4, spacing: float = 3.105, jitter: float = 0.2,
                min_oo: float = 2.5) -> Frame:
    """Water-like frame: O on an n_side^3 cubic lattice (spacing 3.105 A, box 12.42 A for
    n_side = 4, i.e. 1 g/cm^3) with uniform jitter of +-0.2 A, resampled until the minimum
    image O-O distance is >= 2.5 A; two H per O (see `_place_hydrogens`).  Atom order is
    O, H, H per molecule (types 0, 1, 1)."""
    rng = Rng(seed)
    L = n_side * spacing
    g = np.arange(n_side) * spacing
    lat = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    for _ in range(1000):
        o = lat + (2.0 * rng.uniform(lat.size).reshape(lat.shape) - 1.0) * jitter
        if _min_image_dist(o, L) >= min_oo:
            break
    h1, h2 = _place_hydrogens(rng, o)
    coord = np.stack([o, h1, h2], axis=1).reshape(-1, 3)
    atype = np.tile(np.array([0, 1, 1], dtype=np.int32), o.shape[0])
    return Frame(coord.astype(np.float64), atype, np.eye(3) * L)


def water_frame_n(n_mol: int, seed: int, min_oo: float = 2.5) -> Frame:
    """Water-like frame with n_mol molecules at 1 g/cm^3: when n_mol is a cube the lattice
    generator above is used; otherwise O atoms are placed by random sequential addition
    with a 2.5 A minimum image O-O distance."""
    L = (n_mol * WATER_ML_PER_MOL_A3) ** (1.0 / 3.0)
    k = round(n_mol ** (1.0 / 3.0))
    if k ** 3 == n_mol:
        return water_frame(seed=seed, n_side=k, spacing=L / k)
    rng = Rng(seed)
    o = np.zeros((0, 3))
    tries = 0
    while o.shape[0] < n_mol:
        c = rng.uniform(3) * L
        if o.shape[0]:
            d = o - c
            d -= L * np.round(d / L)
            if (d * d).sum(-1).min() < min_oo * min_oo:
                tries += 1
                if tries > 200000:
                    raise RuntimeError("random sequential addition failed")
                continue
        o = np.vstack([o, c[None]])
    h1, h2 = _place_hydrogens(rng, o)
    coord = np.stack([o, h1, h2], axis=1).reshape(-1, 3)
    atype = np.tile(np.array([0, 1, 1], dtype=np.int32), n_mol)
    return Frame(coord.astype(np.float64), atype, np.eye(3) * L)


def replicate(fr: Frame, reps: Sequence[int]) -> Frame:
    """Tile a periodic frame reps[0] x reps[1] x reps[2] times (atom order: image-major)."""
    out = []
    for a in range(reps[0]):
        for b in range(reps[1]):
            for c in range(reps[2]):
                out.append(fr.coord + a * fr.box[0] + b * fr.box[1] + c * fr.box[2])
    box = fr.box * np.array(reps, dtype=np.float64)[:, None]
    n = int(np.prod(reps))
    return Frame(np.concatenate(out), np.tile(fr.atype, n), box)


def fcc_frame(n_cells: Sequence[int] = (20, 20, 20), a: float = 3.634, sigma: float = 0.05,
              seed: int = 0) -> Frame:
    """Cu-like FCC crystal: conventional 4-atom cell of edge a, n_cells copies, Gaussian
    jitter N(0, sigma^2) per Cartesian component; single type 0."""
    rng = Rng(seed)
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]], dtype=np.float64)
    nx, ny, nz = n_cells
    g = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"), -1).reshape(-1, 3)
    pos = ((g[:, None, :] + basis[None]) * a).reshape(-1, 3)
    pos = pos + rng.normal(pos.size).reshape(pos.shape) * sigma
    box = np.diag([nx * a, ny * a, nz * a]).astype(np.float64)
    return Frame(pos, np.zeros(pos.shape[0], dtype=np.int32), box)


def perturbed(fr: Frame, seed: int, sigma: float) -> Frame:
    """Copy of a frame with N(0, sigma^2) noise added to every coordinate."""
    rng = Rng(seed)
    return Frame(fr.coord + rng.normal(fr.coord.size).reshape(fr.coord.shape) * sigma, fr.atype.copy(),
                 fr.box.copy())


def triclinic_box(L: float, tilt: Tuple[float, float, float]) -> np.ndarray:
    """Lower-triangular cell (rows h_0, h_1, h_2) with off-diagonal tilts (xy, xz, yz)."""
    xy, xz, yz = tilt
    return np.array([[L, 0.0, 0.0], [xy, L, 0.0], [xz, yz, L]], dtype=np.float64)


def random_frame(n: int, ntypes: int, box: np.ndarray, seed: int, min_dist: float = 0.8) -> Frame:
    """Random atoms in a (possibly triclinic) periodic cell with a minimum image distance,
    types drawn uniformly; used for small edge-case tests."""
    rng = Rng(seed)
    inv = np.linalg.inv(box)
    pts = []
    tries = 0
    while len(pts) < n:
        f = rng.uniform(3)
        c = f @ box
        ok = True
        for p in pts:
            d = (c - p) @ inv
            d -= np.round(d)
            if np.linalg.norm(d @ box) < min_dist:
                ok = False
                break
        tries += 1
        if tries > 100000:
            raise RuntimeError("could not place atoms")
        if ok:
            pts.append(c)
    atype = (rng.bits(n) % np.uint64(ntypes)).astype(np.int32)
    return Frame(np.array(pts), atype, box.astype(np.float64))
