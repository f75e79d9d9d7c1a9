"""dp_build_nlist_noalloc: the neighbour-list entry point that allocates nothing.

It exists for callers that cannot allocate device memory when they need a list (an MD
engine that owns all device memory, or a loop being captured into a CUDA graph).  Its
result must equal the allocating entry point's (dp_build_nlist, exported with
dp_nlist_export) bit for bit, like every neighbour list here, and a call must not be
affected by the previous call's leftovers in the shared static scratch: two calls in a row
on different frames (the larger one first) are both checked.

This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_2304_09409_gb300 import inputs as I

from _cases import tiny_frame, tiny_model

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _reference(cfg, fr):
    from paper_2304_09409_gb300 import dpgb
    m = dpgb.Model(cfg, I.make_params(cfg, 0), precision="fp64")
    nl = m.build_nlist(fr.coord, fr.atype, fr.box)
    j, s = nl.export()
    ov = nl.n_overflow
    nl.free()
    m.free()
    return j, s, ov


def test_noalloc_nlist_equals_allocating_entry_point_on_two_calls():
    from paper_2304_09409_gb300 import dpgb
    cases = [(I.water_model(), I.replicate(I.water_frame(0), (2, 2, 2))),   # 1,536 atoms
             (tiny_model(), tiny_frame(seed=3))]                            # 14 atoms, triclinic
    for cfg, fr in cases:
        rj, rs, rov = _reference(cfg, fr)
        c = torch.tensor(fr.coord, device="cuda")
        t = torch.tensor(fr.atype, device="cuda")
        gj, gs, gov = dpgb.build_nlist_noalloc(cfg, c, t, fr.box)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(gj.cpu().numpy(), rj)
        np.testing.assert_array_equal(gs.cpu().numpy(), rs)
        assert gov == rov


def test_noalloc_on_dense_fcc_and_hybrid_lists():
    """The per-atom kernel this entry point always runs against the cell-centred kernel the
    allocating entry point prefers, on a dense FCC frame (sel [512], lattice shells whose FP32
    keys fall inside the tie window) and on a hybrid model's list (the larger cutoff and sel of
    its two parts)."""
    from paper_2304_09409_gb300 import dpgb
    cases = [(I.metal_model(), I.fcc_frame((6, 6, 6), seed=3)),                   # 864 atoms
             (I.water_model_hybrid(), I.replicate(I.water_frame(0), (2, 2, 2)))]  # r_c 4 + 6
    for cfg, fr in cases:
        rj, rs, rov = _reference(cfg, fr)
        assert rj.shape[1] == cfg.nc
        c = torch.tensor(fr.coord, device="cuda")
        t = torch.tensor(fr.atype, device="cuda")
        gj, gs, gov = dpgb.build_nlist_noalloc(cfg, c, t, fr.box)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(gj.cpu().numpy(), rj)
        np.testing.assert_array_equal(gs.cpu().numpy(), rs)
        assert gov == rov


def test_noalloc_rejects_frames_beyond_its_limit():
    from paper_2304_09409_gb300 import dpgb
    cfg = I.water_model()
    n = 16000  # 16,000 x 138 slots > 2,097,152
    c = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    t = torch.zeros(n, dtype=torch.int32, device="cuda")
    with pytest.raises(dpgb.DPError) as ei:
        dpgb.build_nlist_noalloc(cfg, c, t, np.eye(3) * 60.0)
    assert ei.value.code == dpgb.DP_E_ARG
    assert "at most" in str(ei.value)
