"""Batched evaluation of frames with uneven atom counts (dp_compute_batch).

Each frame's energy, forces, virial and atomic energies from a mixed batch must match the
FP64 oracle (FP64 path: contract tolerances) and must match the same frame evaluated alone
with the same model (any precision: only the order of floating-point accumulation differs).
"""
import numpy as np
import pytest

import oracle
from paper_2304_09409_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _water_mix():
    frames = [I.water_frame_n(8, seed=11), I.water_frame_n(27, seed=12), I.water_frame_n(40, seed=13),
              I.water_frame(0), I.water_frame_n(125, seed=14)]
    return I.water_model(), frames


def _pack(frames):
    nat = np.array([f.natoms for f in frames], dtype=np.int32)
    coord = np.concatenate([f.coord for f in frames])
    atype = np.concatenate([f.atype for f in frames]).astype(np.int32)
    boxes = np.stack([f.box for f in frames])
    return nat, coord, atype, boxes


def _split(x, nat):
    return np.split(np.asarray(x), np.cumsum(nat)[:-1])


def test_batch_fp64_matches_oracle_per_frame():
    from paper_2304_09409_gb300 import dpgb
    cfg, frames = _water_mix()
    p = I.make_params(cfg, 0)
    m = dpgb.Model(cfg, p, precision="fp64")
    nat, coord, atype, boxes = _pack(frames)
    e, f, v, ae = dpgb.compute_batch(m, nat, coord, atype, boxes, atom_energy=True)
    for k, (fr, fk, aek) in enumerate(zip(frames, _split(f, nat), _split(ae, nat))):
        ref = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box)
        assert abs(e[k] - ref.energy) / fr.natoms <= 1e-10, k
        assert np.abs(fk - ref.force).max() <= 1e-9, k
        assert np.abs(v[k] - ref.virial).max() <= 1e-10 * max(1.0, np.abs(ref.virial).max()), k
        assert np.abs(aek - ref.atom_energy).max() <= 1e-10, k


@pytest.mark.parametrize("prec,comp", [("fp64", False), ("fp32", True), ("bf16", True)])
def test_batch_equals_alone(prec, comp):
    from paper_2304_09409_gb300 import dpgb
    cfg, frames = _water_mix()
    p = I.make_params(cfg, 0)
    m = dpgb.Model(cfg, p, precision=prec, compressed=comp)
    nat, coord, atype, boxes = _pack(frames)
    e, f, v, ae = dpgb.compute_batch(m, nat, torch.tensor(coord, device="cuda"), torch.tensor(atype, device="cuda"),
                                     boxes, atom_energy=True)
    e, f, v, ae = (x.cpu().numpy() for x in (e, f, v, ae))
    for k, (fr, fk, aek) in enumerate(zip(frames, _split(f, nat), _split(ae, nat))):
        e1, f1, v1, ae1 = m.compute(fr.coord, fr.atype, fr.box, atom_energy=True)
        assert abs(e[k] - e1[0]) <= 1e-10 * fr.natoms, (prec, k)
        assert np.abs(fk - f1).max() <= 1e-9, (prec, k)
        assert np.abs(v[k] - v1).max() <= 1e-9 * max(1.0, np.abs(v1).max()), (prec, k)
        assert np.abs(aek - ae1).max() <= 1e-10, (prec, k)


def test_batch_metal_frames_and_host_pointers():
    from paper_2304_09409_gb300 import dpgb
    cfg = I.metal_model()
    p = I.make_params(cfg, 0)
    frames = [I.fcc_frame((3, 3, 3), seed=1), I.fcc_frame((4, 4, 4), seed=2), I.fcc_frame((3, 4, 5), seed=3)]
    m = dpgb.Model(cfg, p, precision="fp64")
    nat, coord, atype, boxes = _pack(frames)
    e, f, v, _ = dpgb.compute_batch(m, nat, coord, atype, boxes)
    for k, (fr, fk) in enumerate(zip(frames, _split(f, nat))):
        ref = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box)
        assert abs(e[k] - ref.energy) / fr.natoms <= 1e-10
        assert np.abs(fk - ref.force).max() <= 1e-9


def test_batch_single_frame_equals_compute():
    from paper_2304_09409_gb300 import dpgb
    cfg = I.water_model()
    p = I.make_params(cfg, 0)
    fr = I.water_frame(0)
    m = dpgb.Model(cfg, p, precision="bf16", compressed=True)
    e, f, v, _ = dpgb.compute_batch(m, [fr.natoms], fr.coord, fr.atype, fr.box[None])
    e1, f1, v1, _ = m.compute(fr.coord, fr.atype, fr.box)
    assert abs(e[0] - e1[0]) <= 1e-12 * fr.natoms
    assert np.abs(f - f1).max() <= 1e-12
