"""Small seeded cases shared by the oracle pins and the GPU parity tests."""
import numpy as np

from paper_2304_09409_gb300 import inputs as I


def tiny_model(type_one_side: int = 0) -> I.ModelConfig:
    """Two species, short cutoff, narrow nets: every code path of the full model
    (type-pair nets, {x,x} and +x skips, linear output layer) at a size the oracle's
    dual-number and finite-difference checks finish quickly."""
    return I.ModelConfig(ntypes=2, rcut=3.5, rcut_smth=0.5, sel=(12, 20), embed=(4, 8, 16), axis=4,
                         fit=(12, 12), type_one_side=type_one_side)


def tiny_frame(seed: int = 3, n: int = 14, triclinic: bool = True) -> I.Frame:
    """14 atoms in a small triclinic cell narrower than 2 r_c, so periodic images of the
    same atom (and of atom i itself) appear in the neighbour list."""
    box = I.triclinic_box(5.2, (0.9, -0.6, 0.4)) if triclinic else np.eye(3) * 5.2
    return I.random_frame(n, 2, box, seed=seed, min_dist=1.0)


def scaled_params(cfg, seed=0, scale=1.0):
    return I.make_params(cfg, seed) * scale


def tiny_model_r(type_one_side: int = 0) -> I.ModelConfig:
    """The tiny model's list and fitting net with the se_e2_r descriptor (embedding 4/8/16)."""
    return I.ModelConfig(ntypes=2, rcut=3.5, rcut_smth=0.5, sel=(12, 20), embed=(4, 8, 16), axis=0,
                         fit=(12, 12), type_one_side=type_one_side, descriptor=1)


def tiny_model_hybrid(type_one_side: int = 0) -> I.ModelConfig:
    """The tiny model with an se_e2_r part (same list, embedding 3/6/12) beside its se_e2_a part."""
    return I.ModelConfig(ntypes=2, rcut=3.5, rcut_smth=0.5, sel=(12, 20), embed=(4, 8, 16), axis=4,
                         fit=(12, 12), type_one_side=type_one_side, descriptor=2, embed_2=(3, 6, 12))


def tiny_model_e3() -> I.ModelConfig:
    """The tiny model's list and fitting net with the se_e3 descriptor (embedding 2/4/8)."""
    return I.ModelConfig(ntypes=2, rcut=3.5, rcut_smth=0.5, sel=(12, 20), embed=(2, 4, 8), axis=0,
                         fit=(12, 12), descriptor=3)


def tiny_model_hybrid_e3() -> I.ModelConfig:
    """Hybrid se_e2_a (r_c 3.0, sel [8, 14], embedding 4/8/16, M_< 4) + se_e3 (r_c 3.5, sel
    [12, 20], embedding 2/4/8): parts with different cutoffs and sel on one list."""
    return I.ModelConfig(ntypes=2, rcut=3.0, rcut_smth=0.5, sel=(8, 14), embed=(4, 8, 16), axis=4,
                         fit=(12, 12), descriptor=4, rcut_2=3.5, rcut_smth_2=0.4, sel_2=(12, 20),
                         embed_2=(2, 4, 8))
