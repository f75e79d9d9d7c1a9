"""Continuous-batching server: every result in the mix equals the frame evaluated alone.

A short Poisson stream of water and FCC requests of uneven size is served with several
batches in flight; each request's energy, forces and virial must equal a stand-alone
dp_compute of the same frame with the same model (only accumulation order differs), and
the server must report latency percentiles for every request.
"""
import numpy as np
import pytest

from paper_2304_09409_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_served_results_equal_alone():
    from paper_2304_09409_gb300 import dpgb, serve
    models = {"water": (I.water_model(), I.make_params(I.water_model(), 0)),
              "metal": (I.metal_model(), I.make_params(I.metal_model(), 0))}
    water = [I.water_frame_n(n, seed=30 + n) for n in (8, 27, 50, 64, 90)]
    fcc = [I.fcc_frame(abc, seed=40 + k) for k, abc in enumerate([(3, 3, 3), (3, 4, 5), (4, 4, 4), (5, 5, 3)])]
    reqs = serve.poisson_stream(water, fcc, n=48, rate=4000.0, seed=5)
    srv = serve.Server(models, precision="bf16", compressed=True, slots=3, max_batch_atoms=4000)
    st = srv.run(reqs, realtime=True)
    assert st["frames"] == len(reqs) and not st["errors"], st["errors"][:3]
    assert st["p50_ms"] is not None and st["p99_ms"] >= st["p50_ms"]
    alone = {k: dpgb.Model(cfg, p, precision="bf16", compressed=True) for k, (cfg, p) in models.items()}
    for r in srv.completed:
        e1, f1, v1, _ = alone[r.model].compute(r.frame.coord, r.frame.atype, r.frame.box)
        assert abs(r.energy - e1[0]) <= 1e-10 * r.frame.natoms
        assert np.abs(r.force - f1).max() <= 1e-9
        assert np.abs(r.virial - v1).max() <= 1e-9 * max(1.0, np.abs(v1).max())
    srv.close()
