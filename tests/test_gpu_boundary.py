"""The C ABI's own contract on the GPU: the weight-file entry point, error reporting, rejection of
non-finite coordinates, and the bounded device waits (failure detection without a GPU fault).
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2304_09409_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_init_model_from_weight_file_matches_oracle(tmp_path):
    """dp_init_model: a weight file written by the binding, loaded by the library, evaluated on
    the FP64 path and compared with the oracle on the same parameters."""
    from paper_2304_09409_gb300 import dpgb
    cfg = I.water_model()
    p = I.make_params(cfg, 4)
    path = str(tmp_path / "water.dpgbw")
    dpgb.write_weight_file(path, cfg, p)
    fr = I.water_frame(5)
    ref = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box)
    m = dpgb.Model.from_file(path, cfg, precision="fp64")
    e, f, v, ae = m.compute(fr.coord, fr.atype, fr.box, atom_energy=True)
    assert abs(float(e[0]) - ref.energy) / fr.natoms <= 1e-10
    assert np.abs(f - ref.force).max() <= 1e-9
    np.testing.assert_allclose(v, ref.virial, rtol=1e-10, atol=1e-12)
    m.free()
    # and the compressed FP32 path from the same file
    m = dpgb.Model.from_file(path, cfg, precision="fp32", compressed=True)
    _, f, _, _ = m.compute(fr.coord, fr.atype, fr.box)
    assert np.abs(f - ref.force).max() <= 1e-4 * max(np.abs(ref.force).max(), 1e-3)
    m.free()


def test_init_model_rejects_missing_and_malformed_files(tmp_path):
    from paper_2304_09409_gb300 import dpgb
    with pytest.raises(dpgb.DPError) as ei:
        dpgb.load_model_file(str(tmp_path / "absent.dpgbw"))
    assert ei.value.code == dpgb.DP_E_ARG and "cannot open" in str(ei.value)
    bad = tmp_path / "bad.dpgbw"
    bad.write_bytes(b"NOTAWEIGHTFILE" * 4)
    with pytest.raises(dpgb.DPError) as ei:
        dpgb.load_model_file(str(bad))
    assert ei.value.code == dpgb.DP_E_ARG and "malformed" in str(ei.value)


def test_last_error_copies_and_truncates():
    """dp_last_error(buf, len): returns the full length, copies at most len - 1 characters."""
    from paper_2304_09409_gb300 import dpgb
    with pytest.raises(dpgb.DPError):
        dpgb.load_model_file("/nonexistent/dir/file.dpgbw")
    L = dpgb.lib()
    n = L.dp_last_error(None, 0)
    full = dpgb.last_error()
    assert n == len(full.encode()) and n > 10
    buf = ctypes.create_string_buffer(8)
    assert L.dp_last_error(buf, 8) == n
    assert buf.value == full.encode()[:7]


def test_non_finite_coordinates_rejected():
    """NaN / Inf coordinates from host arrays are rejected before any work is queued, with
    DP_E_ARG and a message naming the atom; the model keeps working afterwards."""
    from paper_2304_09409_gb300 import dpgb
    cfg = I.water_model()
    m = dpgb.Model(cfg, I.make_params(cfg, 0), precision="fp32", compressed=True)
    fr = I.water_frame(0)
    e0, f0, _, _ = m.compute(fr.coord, fr.atype, fr.box)
    for bad in (np.nan, np.inf, -np.inf):
        c = fr.coord.copy()
        c[17, 1] = bad
        with pytest.raises(dpgb.DPError) as ei:
            m.compute(c, fr.atype, fr.box)
        assert ei.value.code == dpgb.DP_E_ARG and "non-finite" in str(ei.value) and "atom 17" in str(ei.value)
        with pytest.raises(dpgb.DPError) as ei:
            dpgb.compute_batch(m, np.array([fr.natoms, fr.natoms], np.int32), np.concatenate([fr.coord, c]),
                               np.concatenate([fr.atype, fr.atype]), np.stack([fr.box, fr.box]))
        assert ei.value.code == dpgb.DP_E_ARG
    e1, f1, _, _ = m.compute(fr.coord, fr.atype, fr.box)
    assert float(e1[0]) == float(e0[0]) and np.abs(f1 - f0).max() <= 1e-12
    m.free()


def test_bounded_wait_gives_up_and_context_stays_usable():
    """dp_wait_selftest: an mbarrier nothing arrives at, waited on by the kernels' bounded-wait
    routine, gives up and reports DP_E_TIMEOUT (with a short poll limit and with the kernels' own
    limit); the context then runs a full evaluation correctly."""
    import time
    from paper_2304_09409_gb300 import dpgb
    times = {}
    for limit in (1000, 100000):
        t0 = time.perf_counter()
        rc = dpgb.wait_selftest(limit)
        times[limit] = time.perf_counter() - t0
        assert rc == dpgb.DP_E_TIMEOUT, (rc, dpgb.last_error())
        assert "gave up" in dpgb.last_error()
    per_poll = (times[100000] - times[1000]) / 99000
    print(f"bounded wait: {per_poll * 1e9:.1f} ns per poll; the kernels' limit of 2^24 polls gives up after "
          f"about {per_poll * 2 ** 24:.2f} s")
    assert times[100000] < 30.0
    cfg = I.water_model()
    p = I.make_params(cfg, 0)
    fr = I.water_frame(0)
    ref = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box)
    m = dpgb.Model(cfg, p, precision="fp64")
    _, f, _, _ = m.compute(fr.coord, fr.atype, fr.box)
    assert np.abs(f - ref.force).max() <= 1e-9
    m.free()
