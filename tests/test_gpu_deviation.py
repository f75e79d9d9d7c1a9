"""Model deviation of an ensemble (Sec. II.C) on the GPU (dp_model_deviation), and frames of
several models in one batched call (dp_compute_batch with frame_model).

The deviation of four independently initialised water models on the 192-atom frame against the
oracle's (FP64 path: 1e-9 relative; FP32 compressed path: within the force bar of each model's
forces), absolute and relative forms, host and device arrays; the multi-model batch against
each model alone.
"""
import numpy as np
import pytest

import oracle
from paper_2304_09409_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _ensemble(n=4):
    cfg = I.water_model()
    return cfg, [I.force_scaled(cfg, I.make_params(cfg, s), I.WATER_FORCE_SCALE) for s in range(n)]


@pytest.mark.parametrize("nu", [0.0, 0.5])
def test_deviation_fp64_vs_oracle(nu):
    from paper_2304_09409_gb300 import dpgb
    cfg, ps = _ensemble()
    fr = I.water_frame(3)
    ref_f, ref_v, ref_s, ref_m = oracle.model_deviation([(cfg, p) for p in ps], fr.coord, fr.atype, fr.box, nu=nu)
    models = [dpgb.Model(cfg, p, precision="fp64") for p in ps]
    for dev in (False, True):
        c = torch.tensor(fr.coord, device="cuda") if dev else fr.coord
        t = torch.tensor(fr.atype, device="cuda") if dev else fr.atype
        df, dv, st, fm = dpgb.model_deviation(models, c, t, fr.box, nu=nu)
        if dev:
            df, dv, st, fm = (x.cpu().numpy() for x in (df, dv, st, fm))
        np.testing.assert_allclose(df, ref_f, rtol=1e-9, atol=1e-12 * np.abs(ref_f).max())
        np.testing.assert_allclose(dv, ref_v, rtol=1e-9, atol=1e-12 * np.abs(ref_v).max())
        np.testing.assert_allclose(st, ref_s, rtol=1e-9, atol=1e-12 * np.abs(ref_s).max())
        np.testing.assert_allclose(fm, ref_m, rtol=0, atol=1e-9)
    for m in models:
        m.free()


def test_deviation_fp32_compressed_close_to_oracle():
    """The mixed path's ensemble: each model's forces are within 1e-3 eV/A, so the deviation is too."""
    from paper_2304_09409_gb300 import dpgb
    cfg, ps = _ensemble()
    fr = I.water_frame(3)
    ref_f, _, ref_s, _ = oracle.model_deviation([(cfg, p) for p in ps], fr.coord, fr.atype, fr.box)
    models = [dpgb.Model(cfg, p, precision="fp32", compressed=True) for p in ps]
    df, dv, st, fm = dpgb.model_deviation(models, fr.coord, fr.atype, fr.box)
    print(f"eps_F max {st[0]:.4f} (oracle {ref_s[0]:.4f}), |d eps_F|max {np.abs(df - ref_f).max():.2e}")
    assert np.abs(df - ref_f).max() <= 1e-3
    assert abs(st[0] - ref_s[0]) <= 1e-3
    for m in models:
        m.free()


def test_multi_model_batch_equals_each_model_alone():
    """Water and metal frames of two resident models in one dp_compute_batch call (frames of each
    model in runs, in an interleaved order) equal each model's own single-model batch."""
    from paper_2304_09409_gb300 import dpgb
    wc, mc = I.water_model(), I.metal_model()
    mw = dpgb.Model(wc, I.water_params_scaled(0), precision="fp32", compressed=True)
    mm = dpgb.Model(mc, I.metal_params_scaled(0), precision="fp32", compressed=True)
    frames = [I.water_frame_n(27, seed=1), I.water_frame(2), I.fcc_frame((3, 3, 4), seed=1),
              I.water_frame_n(40, seed=3), I.fcc_frame((4, 4, 4), seed=2)]
    fmodel = np.array([0, 0, 1, 0, 1], dtype=np.int32)
    nat = np.array([f.natoms for f in frames], dtype=np.int32)
    coord = torch.tensor(np.concatenate([f.coord for f in frames]), device="cuda")
    atype = torch.tensor(np.concatenate([f.atype for f in frames]).astype(np.int32), device="cuda")
    boxes = np.stack([f.box for f in frames])
    e, f, v, ae = dpgb.compute_batch([mw, mm], nat, coord, atype, boxes, atom_energy=True, frame_model=fmodel)
    off = np.concatenate([[0], np.cumsum(nat)])
    for k, fr in enumerate(frames):
        m = mw if fmodel[k] == 0 else mm
        e1, f1, v1, _ = dpgb.compute_batch(m, nat[k:k + 1], fr.coord, fr.atype, fr.box[None])
        fk = f[off[k]:off[k + 1]].cpu().numpy()
        scale = max(np.abs(f1).max(), 1.0)
        assert np.abs(fk - f1).max() <= 1e-6 * scale, k
        assert abs(float(e[k]) - float(e1[0])) <= 1e-9 * max(1.0, abs(float(e1[0]))), k
        np.testing.assert_allclose(v[k].cpu().numpy(), v1[0], rtol=1e-6, atol=1e-6 * np.abs(v1).max())
    with pytest.raises(dpgb.DPError):
        dpgb.compute_batch([mw, mm], nat, coord, atype, boxes, frame_model=np.array([0, 0, 2, 0, 1], np.int32))
    mw.free()
    mm.free()
