"""The C-ABI library loads on a machine without a GPU and exports every declared symbol."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(dp_\w+)\s*\(", src, flags=re.M))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2304_09409_gb300 import build, dpgb
    if not os.path.exists(dpgb.LIB_PATH):
        build.build()
    lib = ctypes.CDLL(dpgb.LIB_PATH)
    declared = _declared()
    assert "dp_compute" in declared and "dp_build_nlist" in declared and "dp_init_model" in declared
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert set(dpgb.EXPORTED) <= declared


def test_n_params_matches_inputs_layout():
    from paper_2304_09409_gb300 import dpgb
    from paper_2304_09409_gb300 import inputs as I
    for cfg in (I.water_model(), I.metal_model(), I.water_model_r(), I.water_model_hybrid()):
        assert dpgb.n_params(cfg) == cfg.n_params()


def test_weight_file_roundtrip_header(tmp_path):
    import numpy as np
    from paper_2304_09409_gb300 import dpgb
    from paper_2304_09409_gb300 import inputs as I
    cfg = I.water_model()
    p = I.make_params(cfg, 0)
    path = tmp_path / "w.bin"
    dpgb.write_weight_file(str(path), cfg, p)
    raw = path.read_bytes()
    assert raw[:8] == b"DPGBW002"
    n = ctypes.sizeof(dpgb.Config)
    assert np.frombuffer(raw[8 + n: 16 + n], dtype=np.int64)[0] == p.size
    np.testing.assert_array_equal(np.frombuffer(raw[16 + n:], dtype=np.float64), p)


def test_config_checks_descriptor_fields():
    """dp_model_n_params is host-only: it refuses unknown descriptors, a hybrid without
    second-part nets or with a bad second cutoff, and accepts se_e2_r without M_<; se_e3 nets
    are N_t^2 whatever type_one_side says."""
    import dataclasses
    from paper_2304_09409_gb300 import dpgb
    from paper_2304_09409_gb300 import inputs as I
    hyb = I.water_model_hybrid()
    assert dpgb.n_params(hyb) == hyb.n_params()
    assert dpgb.n_params(dataclasses.replace(hyb, embed_2=())) == -1
    assert dpgb.n_params(dataclasses.replace(hyb, descriptor=5)) == -1
    assert dpgb.n_params(dataclasses.replace(hyb, rcut_2=0.4)) == -1  # r_s of the second part above its r_c
    for cfg in (I.water_model_e3(), I.water_model_hybrid_e3(), dataclasses.replace(I.water_model_e3(), type_one_side=1)):
        assert dpgb.n_params(cfg) == cfg.n_params()
    assert dpgb.n_params(dataclasses.replace(I.water_model_r(), axis=0)) == I.water_model_r().n_params()
    assert dpgb.n_params(dataclasses.replace(I.water_model(), axis=0)) == -1
