"""Host side of the continuous-batching server (no GPU): which requests a free execution slot
takes, in what order, and how large a batch may grow."""
import collections
import threading

import numpy as np
import pytest

from paper_2304_09409_gb300 import inputs as I
from paper_2304_09409_gb300 import serve


def _server(max_batch_atoms=1000, free=10 ** 15, fraction=1.0, slots=1):
    """A server with its queue and admission state only (no models, no streams, no device)."""
    srv = serve.Server.__new__(serve.Server)
    srv.names = ["water", "metal"]
    srv.cfgs = {"water": I.water_model(), "metal": I.metal_model()}
    srv.queue = collections.deque()
    srv.cv = threading.Condition()
    srv.closed = False
    srv.max_batch_atoms = max_batch_atoms
    srv.hbm_fraction = fraction
    srv.slots = slots
    srv.slot_bytes = [0] * slots
    srv.precision = "fp32"
    srv.upload = None
    srv.torch = None
    srv.free_bytes = lambda: free
    return srv


def _req(rid, model, natoms, arrival):
    fr = I.Frame(np.zeros((natoms, 3)), np.zeros(natoms, dtype=np.int32), np.eye(3) * 10.0)
    return serve.Request(rid, model, fr, arrival)


def _submit_in_arrival_order(srv, reqs):
    for r in sorted(reqs, key=lambda r: r.arrival):
        srv.submit(r)


def test_oldest_first_then_arrival_order_across_models_up_to_the_budget():
    srv = _server(max_batch_atoms=1000)
    _submit_in_arrival_order(srv, [_req(0, "water", 300, 0.10), _req(1, "metal", 500, 0.05),
                                   _req(2, "water", 400, 0.20), _req(3, "metal", 600, 0.30)])
    # metal #1 (oldest), then water #0; water #2 would take the batch past 1000 atoms
    assert [r.rid for r in srv._take()] == [1, 0]
    assert [r.rid for r in srv._take()] == [2, 3]  # 400 + 600: one batch of both models
    srv.closed = True
    assert srv._take() is None  # closed and nothing waiting: the worker leaves


def test_a_frame_above_the_budget_is_admitted_alone():
    srv = _server(max_batch_atoms=1000)
    srv.submit(_req(0, "metal", 5000, 0.0))
    srv.submit(_req(1, "metal", 10, 0.1))
    assert [r.rid for r in srv._take()] == [0]
    assert [r.rid for r in srv._take()] == [1]


def test_free_memory_measured_at_admission_limits_the_batch():
    per = serve.scratch_bytes_per_atom(I.water_model(), "fp32")
    srv = _server(max_batch_atoms=10 ** 6, free=per * 250, slots=1)
    _submit_in_arrival_order(srv, [_req(k, "water", 100, 0.01 * k) for k in range(5)])
    assert [r.rid for r in srv._take()] == [0, 1]  # 200 atoms fit the 250-atom share, 300 do not
    # the slot now holds the scratch of 200 atoms; free memory dropped to nothing: it may reuse it
    srv.free_bytes = lambda: 0
    assert [r.rid for r in srv._take()] == [2, 3]
    # more free memory at the next admission: a larger batch
    srv.free_bytes = lambda: per * 10 ** 4
    srv.submit(_req(9, "water", 100, 1.0))
    assert [r.rid for r in srv._take()] == [4, 9]
    # the share is divided among the slots
    srv = _server(max_batch_atoms=10 ** 6, free=per * 250, slots=2)
    _submit_in_arrival_order(srv, [_req(k, "water", 100, 0.01 * k) for k in range(3)])
    assert [r.rid for r in srv._take(0)] == [0]  # 125-atom share per slot


def test_atom_budget_is_the_smaller_of_the_cap_and_free_memory():
    per = serve.scratch_bytes_per_atom(I.water_model(), "fp32")
    assert per > 0
    assert _server(max_batch_atoms=1000, free=per * 250).atom_budget("water") == 250  # free memory decides
    assert _server(max_batch_atoms=100, free=per * 250).atom_budget("water") == 100  # the cap decides
    assert _server(max_batch_atoms=100, free=0).atom_budget("water") == 1  # never zero


def test_scratch_estimate_grows_with_the_list_and_precision():
    w, m = I.water_model(), I.metal_model()
    assert serve.scratch_bytes_per_atom(m, "fp32") > serve.scratch_bytes_per_atom(w, "fp32")  # 512 vs 138 slots
    assert serve.scratch_bytes_per_atom(w, "fp64") == pytest.approx(2 * serve.scratch_bytes_per_atom(w, "fp32"), rel=1e-6)


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


def test_prefill_queues_every_request_at_time_zero_in_arrival_order():
    """The capacity operating point: every request is queued (arrival 0) before a slot starts, in
    arrival order, and the first batch takes the oldest ones up to the budget."""
    srv = _server(max_batch_atoms=1000)
    srv._worker = lambda slot: None  # no device work: only the queue is examined
    reqs = [_req(0, "water", 300, 0.30), _req(1, "metal", 500, 0.05), _req(2, "water", 400, 0.20)]
    srv.stats = lambda wall: {}
    srv.run(reqs, prefill=True)
    assert [r.rid for r in srv.queue] == [1, 2, 0]
    assert all(r.arrival == 0.0 for r in reqs)
    srv.closed = False
    assert [r.rid for r in srv._take()] == [1, 2]
