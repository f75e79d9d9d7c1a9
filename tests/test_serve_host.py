"""Host side of the continuous-batching server (no GPU): which requests a free execution slot
takes, in what order, and how large a batch may grow."""
import collections
import threading

import numpy as np
import pytest

from paper_2304_09409_gb300 import inputs as I
from paper_2304_09409_gb300 import serve


def _server(max_batch_atoms=1000, hbm_budget=10 ** 15):
    """A server with its queues and admission state only (no models, no streams)."""
    srv = serve.Server.__new__(serve.Server)
    srv.cfgs = {"water": I.water_model(), "metal": I.metal_model()}
    srv.queues = {k: collections.deque() for k in srv.cfgs}
    srv.cv = threading.Condition()
    srv.closed = False
    srv.max_batch_atoms = max_batch_atoms
    srv.hbm_budget = hbm_budget
    srv.precision = "bf16"
    return srv


def _req(rid, model, natoms, arrival):
    fr = I.Frame(np.zeros((natoms, 3)), np.zeros(natoms, dtype=np.int32), np.eye(3) * 10.0)
    return serve.Request(rid, model, fr, arrival)


def test_oldest_model_first_then_fifo_up_to_the_budget():
    srv = _server(max_batch_atoms=1000)
    for r in (_req(0, "water", 300, 0.10), _req(1, "metal", 500, 0.05), _req(2, "water", 400, 0.20),
              _req(3, "metal", 600, 0.30)):
        srv.submit(r)
    # the oldest waiting request is metal #1; metal #3 would take the batch past 1000 atoms
    assert [r.rid for r in srv._take()] == [1]
    # then water (#0 at 0.10 is now the oldest head): both water frames fit together
    assert [r.rid for r in srv._take()] == [0, 2]
    assert [r.rid for r in srv._take()] == [3]
    srv.closed = True
    assert srv._take() is None  # closed and nothing waiting: the worker leaves


def test_a_frame_above_the_budget_is_admitted_alone():
    srv = _server(max_batch_atoms=1000)
    srv.submit(_req(0, "metal", 5000, 0.0))
    srv.submit(_req(1, "metal", 10, 0.1))
    assert [r.rid for r in srv._take()] == [0]
    assert [r.rid for r in srv._take()] == [1]


def test_atom_budget_is_the_smaller_of_the_cap_and_free_memory():
    per = serve.scratch_bytes_per_atom(I.water_model(), "bf16")
    assert per > 0
    srv = _server(max_batch_atoms=1000, hbm_budget=per * 250)
    assert srv.atom_budget("water") == 250  # free memory decides
    srv = _server(max_batch_atoms=100, hbm_budget=per * 250)
    assert srv.atom_budget("water") == 100  # the cap decides
    srv = _server(max_batch_atoms=100, hbm_budget=0)
    assert srv.atom_budget("water") == 1  # never zero: one frame is always admitted


def test_scratch_estimate_grows_with_the_list_and_precision():
    w, m = I.water_model(), I.metal_model()
    assert serve.scratch_bytes_per_atom(m, "bf16") > serve.scratch_bytes_per_atom(w, "bf16")  # 512 vs 138 slots
    assert serve.scratch_bytes_per_atom(w, "fp64") == pytest.approx(2 * serve.scratch_bytes_per_atom(w, "bf16"), rel=1e-6)


def test_poisson_stream_is_seeded_and_has_the_requested_rate():
    water = [I.water_frame_n(8, seed=1)]
    fcc = [I.fcc_frame((3, 3, 3), seed=2)]
    a = serve.poisson_stream(water, fcc, n=4000, rate=2000.0, seed=7)
    b = serve.poisson_stream(water, fcc, n=4000, rate=2000.0, seed=7)
    assert [(r.model, r.arrival) for r in a] == [(r.model, r.arrival) for r in b]
    t = np.array([r.arrival for r in a])
    assert np.all(np.diff(t) > 0)
    assert (t[-1] / len(t)) == pytest.approx(1 / 2000.0, rel=0.05)  # mean gap 1/rate
    frac_water = np.mean([r.model == "water" for r in a])
    assert frac_water == pytest.approx(0.5, abs=0.03)
