"""Continuous-batching evaluation service for energy/force/virial requests.

Requests are frames (coordinates, types, cell) for one of several resident models.  They
arrive over time; a frame that arrives while others are on the GPU waits in its model's
queue only until an execution slot frees up.  Each slot is a worker thread that owns its
own model instance (and so its own device scratch) and its own CUDA stream: up to `slots`
batches are in flight at once and overlap on the device.  When a slot frees up it takes
the oldest waiting request's model and admits that model's queued frames in arrival order
until the batch reaches its atom budget; the budget is the smaller of `max_batch_atoms` and
what the free device memory allows (admission by free HBM).  Every batch is one
dp_compute_batch call.  Latency of a request = completion time - arrival time.
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time
from typing import Dict, List, Optional

import numpy as np

from . import dpgb
from . import inputs as I


@dataclasses.dataclass
class Request:
    rid: int
    model: str
    frame: I.Frame
    arrival: float = 0.0      # scheduled arrival (seconds from the start of the run)
    admitted: float = 0.0
    done: float = 0.0
    energy: float = 0.0
    force: Optional[np.ndarray] = None
    virial: Optional[np.ndarray] = None


def scratch_bytes_per_atom(cfg, precision: str) -> int:
    """Upper estimate of the device scratch one atom of a batch needs: per neighbour slot the
    list (8 B), its FP32 displacement (16 B), the environment records and run index (36 B) and
    the per-run moment / P records of the compressed path (136 B); per atom the descriptor and
    its gradient, the fitting activations and the sort and cell arrays."""
    nc, M, A = cfg.nc, cfg.m, cfg.axis
    w = max(cfg.fit) if cfg.fit else 1
    b = nc * (8 + 16 + 36 + 136) + M * 4 * 4 * 2 + M * A * (2 + 4 + 4) + 6 * w * 6 + 512
    return int(b * (2 if precision == "fp64" else 1) * 1.25)


class Server:
    def __init__(self, models: Dict[str, tuple], precision: str = "bf16", compressed: bool = True, slots: int = 3,
                 max_batch_atoms: int = 65536, hbm_fraction: float = 0.5, device: int = 0):
        import torch
        self.torch = torch
        self.cfgs = {k: v[0] for k, v in models.items()}
        self.slots = slots
        self.max_batch_atoms = max_batch_atoms
        self.device = device
        free, _ = torch.cuda.mem_get_info(device)
        self.hbm_budget = int(free * hbm_fraction / max(slots, 1))
        self.precision = precision
        # one model instance per (slot, model): each slot has private scratch
        self.inst = [{k: dpgb.Model(cfg, p, device=device, precision=precision, compressed=compressed)
                      for k, (cfg, p) in models.items()} for _ in range(slots)]
        self.streams = [torch.cuda.Stream(device=device) for _ in range(slots)]
        self.queues: Dict[str, collections.deque] = {k: collections.deque() for k in models}
        self.cv = threading.Condition()
        self.closed = False
        self.completed: List[Request] = []
        self.batches: List[tuple] = []  # (model, frames, atoms, seconds)
        self.t0 = 0.0
        self.errors: List[str] = []

    # ---- admission -------------------------------------------------------------------------
    def atom_budget(self, model: str) -> int:
        per = scratch_bytes_per_atom(self.cfgs[model], self.precision)
        return max(1, min(self.max_batch_atoms, self.hbm_budget // per))

    def submit(self, req: Request):
        with self.cv:
            self.queues[req.model].append(req)
            self.cv.notify()

    def _take(self) -> Optional[List[Request]]:
        """Oldest waiting model's queue head, then FIFO until the atom budget is reached."""
        with self.cv:
            while True:
                heads = [(q[0].arrival, k) for k, q in self.queues.items() if q]
                if heads:
                    break
                if self.closed:
                    return None
                self.cv.wait(timeout=0.05)
            _, model = min(heads)
            q = self.queues[model]
            budget = self.atom_budget(model)
            batch, atoms = [], 0
            while q and (not batch or atoms + q[0].frame.natoms <= budget):
                r = q.popleft()
                atoms += r.frame.natoms
                batch.append(r)
            return batch

    # ---- execution -------------------------------------------------------------------------
    def _worker(self, slot: int):
        torch = self.torch
        torch.cuda.set_device(self.device)
        stream = self.streams[slot]
        while True:
            batch = self._take()
            if batch is None:
                return
            model = batch[0].model
            now = time.perf_counter() - self.t0
            for r in batch:
                r.admitted = now
            nat = np.array([r.frame.natoms for r in batch], dtype=np.int32)
            coord = np.concatenate([r.frame.coord for r in batch])
            atype = np.concatenate([r.frame.atype for r in batch]).astype(np.int32)
            boxes = np.stack([r.frame.box for r in batch])
            try:
                t_start = time.perf_counter()
                e, f, v, _ = dpgb.compute_batch(self.inst[slot][model], nat, coord, atype, boxes, stream=stream)
                t_end = time.perf_counter()
            except Exception as exc:  # keep serving; report at the end
                self.errors.append(repr(exc))
                continue
            done = t_end - self.t0
            off = np.concatenate([[0], np.cumsum(nat)])
            for k, r in enumerate(batch):
                r.done = done
                r.energy = float(e[k])
                r.force = f[off[k]:off[k + 1]]
                r.virial = v[k]
            with self.cv:
                self.completed.extend(batch)
                self.batches.append((model, len(batch), int(nat.sum()), t_end - t_start))

    def run(self, requests: List[Request], realtime: bool = True) -> dict:
        """Replay `requests` (arrival times in seconds) and serve them; returns statistics."""
        threads = [threading.Thread(target=self._worker, args=(s,), daemon=True) for s in range(self.slots)]
        self.t0 = time.perf_counter()
        for t in threads:
            t.start()
        for r in sorted(requests, key=lambda r: r.arrival):
            if realtime:
                delay = r.arrival - (time.perf_counter() - self.t0)
                if delay > 0:
                    time.sleep(delay)
            self.submit(r)
        with self.cv:
            self.closed = True
            self.cv.notify_all()
        for t in threads:
            t.join()
        wall = time.perf_counter() - self.t0
        return self.stats(wall)

    def stats(self, wall: float) -> dict:
        lat = np.array([r.done - r.arrival for r in self.completed]) * 1e3
        atoms = sum(r.frame.natoms for r in self.completed)
        first = min((r.arrival for r in self.completed), default=0.0)
        last = max((r.done for r in self.completed), default=wall)
        span = max(last - first, 1e-9)
        return {
            "frames": len(self.completed),
            "atoms": int(atoms),
            "atom_evals_per_s": atoms / span,
            "frames_per_s": len(self.completed) / span,
            "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
            "mean_batch_frames": float(np.mean([b[1] for b in self.batches])) if self.batches else 0.0,
            "mean_batch_atoms": float(np.mean([b[2] for b in self.batches])) if self.batches else 0.0,
            "batches": len(self.batches),
            "errors": self.errors[:3],
        }

    def close(self):
        for d in self.inst:
            for m in d.values():
                m.free()


# ---- synthetic request streams --------------------------------------------------------------

def frame_pool(seed: int = 0, n_water: int = 12, n_fcc: int = 12):
    """Frames for the serving workload: water-like boxes of 8-1000 molecules (24-3000 atoms)
    at 1 g/cm^3 and FCC crystals of 4abc atoms, 3 <= a, b, c <= 17 (108-19,652 atoms)."""
    rng = I.Rng(seed)
    water, fcc = [], []
    nm = 8 + (rng.bits(n_water) % np.uint64(993)).astype(int)
    for k, n in enumerate(nm):
        water.append(I.water_frame_n(int(n), seed=1000 + k))
    abc = 3 + (rng.bits(3 * n_fcc) % np.uint64(15)).astype(int).reshape(n_fcc, 3)
    for k, (a, b, c) in enumerate(abc):
        fcc.append(I.fcc_frame((int(a), int(b), int(c)), seed=2000 + k))
    return water, fcc


def poisson_stream(water, fcc, n: int, rate: float, seed: int = 0) -> List[Request]:
    """n requests with exponential inter-arrival times (mean 1/rate), each uniformly a water
    or an FCC frame drawn from the pools."""
    rng = I.Rng(seed)
    gaps = -np.log(1.0 - rng.uniform(n)) / rate
    arrivals = np.cumsum(gaps)
    pick = rng.uniform(n)
    idx = rng.bits(n)
    reqs = []
    for k in range(n):
        if pick[k] < 0.5:
            fr = water[int(idx[k] % np.uint64(len(water)))]
            reqs.append(Request(k, "water", fr, float(arrivals[k])))
        else:
            fr = fcc[int(idx[k] % np.uint64(len(fcc)))]
            reqs.append(Request(k, "metal", fr, float(arrivals[k])))
    return reqs
