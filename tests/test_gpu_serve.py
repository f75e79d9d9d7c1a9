"""Continuous-batching server: every result in the mix equals the frame evaluated alone.

A Poisson stream of water and FCC requests of uneven size is served with several batches in
flight, batches holding frames of both resident models; each request's energy, forces and
virial must equal a stand-alone dp_compute of the same frame with the same model (only the
accumulation order differs), and the server must report latency percentiles for every request.
With no free-memory share left, admission by device memory must split the stream into
single-frame batches, with the same results.
"""
import numpy as np
import pytest

from paper_2304_09409_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _models():
    return {"water": (I.water_model(), I.water_params_scaled(0)),
            "metal": (I.metal_model(), I.metal_params_scaled(0))}


def _pools():
    water = [I.water_frame_n(n, seed=30 + n) for n in (8, 27, 50, 64, 90)]
    fcc = [I.fcc_frame(abc, seed=40 + k) for k, abc in enumerate([(3, 3, 3), (3, 4, 5), (4, 4, 4), (5, 5, 3)])]
    return water, fcc


def _check_alone(srv, models):
    from paper_2304_09409_gb300 import dpgb
    alone = {k: dpgb.Model(cfg, p, precision="fp32", compressed=True) for k, (cfg, p) in models.items()}
    for r in srv.completed:
        e1, f1, v1, _ = alone[r.model].compute(r.frame.coord, r.frame.atype, r.frame.box)
        scale = max(1.0, float(np.abs(f1).max()))
        assert abs(r.energy - e1[0]) <= 1e-9 * max(1.0, abs(float(e1[0])))
        assert np.abs(r.force - f1).max() <= 1e-9 * scale
        assert np.abs(r.virial - v1).max() <= 1e-9 * max(1.0, np.abs(v1).max())
    for m in alone.values():
        m.free()


def test_served_results_equal_alone():
    from paper_2304_09409_gb300 import serve
    models = _models()
    water, fcc = _pools()
    reqs = serve.poisson_stream(water, fcc, n=64, rate=20000.0, seed=5)
    srv = serve.Server(models, precision="fp32", compressed=True, slots=2, max_batch_atoms=6000)
    st = srv.run(reqs, realtime=True)
    assert st["frames"] == len(reqs) and not st["errors"], st["errors"][:3]
    assert st["p50_ms"] is not None and st["p99_ms"] >= st["p50_ms"]
    assert st["mean_batch_frames"] > 1.0 and st["mixed_model_batches"] > 0, st
    _check_alone(srv, models)
    srv.close()


def test_memory_admission_splits_batches():
    from paper_2304_09409_gb300 import serve
    models = _models()
    water, _ = _pools()
    same = [water[2]] * 12  # equal frames, all waiting at once
    reqs = [serve.Request(k, "water", fr, 0.0) for k, fr in enumerate(same)]
    srv = serve.Server(models, precision="fp32", compressed=True, slots=1, max_batch_atoms=10 ** 6,
                       hbm_fraction=0.0)  # no share of the free memory: only what the slot already holds
    st = srv.run(reqs, realtime=False)
    assert st["frames"] == len(reqs) and not st["errors"], st["errors"][:3]
    assert max(b[0] for b in srv.batches) == 1, srv.batches
    _check_alone(srv, models)
    srv.close()
