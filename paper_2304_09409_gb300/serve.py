"""Continuous-batching evaluation service for energy/force/virial requests.

Requests are frames (coordinates, types, cell) for one of several resident models.  A request's
coordinates and types are copied to the device once, when it arrives (pinned host memory, a copy
stream of its own), and stay there until its result is read back.  A frame that arrives while
others are on the GPU waits only until an execution slot frees up.  Each slot is a worker thread
with its own instance of every model (and so its own device scratch), its own CUDA stream and its
own device batch buffers: up to `slots` batches are in flight at once and overlap on the device.
When a slot frees up it takes the oldest waiting request and then the next oldest requests of any
model, in arrival order, until the batch reaches its budget: `max_batch_atoms` and the device
memory the batch's scratch may take, from the free HBM measured at that moment (admission by
free memory; the batching of frames of Sec. III.B).  The batch's frames are gathered device to
device into the slot's buffers, grouped by model, and evaluated by one dp_compute_batch call
over all resident models.  Latency of a request = completion time - arrival time.
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
    seq: int = 0              # submission order
    dcoord: object = None     # device copies made at arrival
    dtype: object = None
    ready: object = None      # CUDA event: the copies have landed


def scratch_bytes_per_atom(cfg, precision: str) -> int:
    """Upper estimate of the device scratch one atom of a batch needs: per neighbour slot the
    list (8 B), its FP32 displacement (16 B), the environment records and run index (36 B) and
    the per-run moment / P records of the compressed path (136 B); per atom the descriptor and
    its gradient (split operands in the FP32 mode), the fitting activations and the sort and cell
    arrays."""
    nc, M, A = cfg.nc, cfg.m, cfg.axis
    w = max(cfg.fit) if cfg.fit else 1
    b = nc * (8 + 16 + 36 + 136) + M * 4 * 4 * 2 + M * A * (2 + 4 + 4 + 4) + 12 * w * 6 + 512
    return int(b * (2 if precision == "fp64" else 1) * 1.25)


class Server:
    def __init__(self, models: Dict[str, tuple], precision: str = "fp32", compressed: bool = True, slots: int = 3,
                 max_batch_atoms: int = 65536, hbm_fraction: float = 0.5, device: int = 0):
        import torch
        self.torch = torch
        self.names = list(models)
        self.cfgs = {k: v[0] for k, v in models.items()}
        self.slots = slots
        self.max_batch_atoms = max_batch_atoms
        self.hbm_fraction = hbm_fraction
        self.device = device
        self.precision = precision
        # one model instance per (slot, model): each slot has private scratch
        self.inst = [{k: dpgb.Model(cfg, p, device=device, precision=precision, compressed=compressed)
                      for k, (cfg, p) in models.items()} for _ in range(slots)]
        self.streams = [torch.cuda.Stream(device=device) for _ in range(slots)]
        self.upload = torch.cuda.Stream(device=device)
        self.pinned: Dict[int, tuple] = {}  # host frame -> its pinned copies (made once per frame)
        self.last_ready = None              # event of the latest upload (the upload stream is in order)
        # per-slot device batch buffers (grown on demand) and per-slot largest admitted scratch
        self.buf = [None] * slots
        self.slot_bytes = [0] * slots
        self.queue: collections.deque = collections.deque()  # all models, arrival order
        self.cv = threading.Condition()
        self.closed = False
        self.completed: List[Request] = []
        self.batches: List[tuple] = []  # (frames, atoms, seconds, models in the batch)
        self.t0 = 0.0
        self.errors: List[str] = []

    # ---- admission -------------------------------------------------------------------------
    def free_bytes(self) -> int:
        return int(self.torch.cuda.mem_get_info(self.device)[0])

    def byte_budget(self, slot: int) -> int:
        """Device bytes a batch of this slot may take: its share of the free HBM now, plus what
        the slot already holds from earlier batches (its scratch is reused)."""
        return int(self.free_bytes() * self.hbm_fraction / max(self.slots, 1)) + self.slot_bytes[slot]

    def atom_budget(self, model: str) -> int:
        per = scratch_bytes_per_atom(self.cfgs[model], self.precision)
        return max(1, min(self.max_batch_atoms, int(self.free_bytes() * self.hbm_fraction / max(self.slots, 1)) // per))

    def submit(self, req: Request):
        """Arrival: the frame's coordinates and types go to the device once, then it queues."""
        torch = self.torch
        if self.upload is None:  # scheduler-only use (no device)
            with self.cv:
                self.queue.append(req)
                self.cv.notify()
            return
        self._seq = getattr(self, "_seq", 0) + 1
        req.seq = self._seq
        key = id(req.frame)
        if key not in self.pinned:  # the client's host arrays, pinned once (the cache holds the frame)
            if len(self.pinned) >= 4096:
                self.pinned.clear()
            self.pinned[key] = (torch.from_numpy(np.ascontiguousarray(req.frame.coord)).pin_memory(),
                                torch.from_numpy(np.ascontiguousarray(req.frame.atype, dtype=np.int32)).pin_memory(),
                                req.frame)
        hc, ht, _ = self.pinned[key]
        dev = f"cuda:{self.device}"
        with torch.cuda.stream(self.upload):
            req.dcoord = torch.empty(hc.shape, dtype=hc.dtype, device=dev)
            req.dcoord.copy_(hc, non_blocking=True)
            req.dtype = torch.empty(ht.shape, dtype=ht.dtype, device=dev)
            req.dtype.copy_(ht, non_blocking=True)
            req.ready = torch.cuda.Event()
            req.ready.record(self.upload)
        with self.cv:
            self.queue.append(req)
            self.cv.notify()

    def _take(self, slot: int = 0) -> Optional[List[Request]]:
        """The oldest waiting request, then the next oldest of any model while the batch stays
        within max_batch_atoms and the slot's device-memory budget."""
        with self.cv:
            while not self.queue:
                if self.closed:
                    return None
                self.cv.wait(timeout=0.05)
            budget = self.byte_budget(slot)
            batch, atoms, nbytes = [], 0, 0
            while self.queue:
                r = self.queue[0]
                n = r.frame.natoms
                b = n * scratch_bytes_per_atom(self.cfgs[r.model], self.precision)
                if batch and (atoms + n > self.max_batch_atoms or nbytes + b > budget):
                    break
                self.queue.popleft()
                atoms += n
                nbytes += b
                batch.append(r)
            self.slot_bytes[slot] = max(self.slot_bytes[slot], nbytes)
            return batch

    # ---- execution -------------------------------------------------------------------------
    def _buffers(self, slot: int, atoms: int):
        torch = self.torch
        b = self.buf[slot]
        if b is None or b["cap"] < atoms:
            cap = max(atoms, 1024)
            dev = f"cuda:{self.device}"
            b = {"cap": cap, "coord": torch.empty((cap, 3), dtype=torch.float64, device=dev),
                 "type": torch.empty(cap, dtype=torch.int32, device=dev),
                 "force": torch.empty((cap, 3), dtype=torch.float64, device=dev),
                 # results: energies [F], virials [F][9], forces [N][3] in one pinned host block
                 "host": torch.empty(cap * 4 + 10 * 4096, dtype=torch.float64).pin_memory()}
            self.buf[slot] = b
        return b

    def _newest(self, batch):
        """The upload event of the most recently submitted request of the batch."""
        return max(batch, key=lambda r: r.seq).ready

    def _worker(self, slot: int):
        torch = self.torch
        torch.cuda.set_device(self.device)
        stream = self.streams[slot]
        models = [self.inst[slot][k] for k in self.names]
        while True:
            batch = self._take(slot)
            if batch is None:
                return
            now = time.perf_counter() - self.t0
            for r in batch:
                r.admitted = now
            # group by model (stable within a model): one pass of each model's kernels
            order = sorted(range(len(batch)), key=lambda k: self.names.index(batch[k].model))
            batch = [batch[k] for k in order]
            nat = np.array([r.frame.natoms for r in batch], dtype=np.int32)
            fmodel = np.array([self.names.index(r.model) for r in batch], dtype=np.int32)
            boxes = np.stack([r.frame.box for r in batch])
            N = int(nat.sum())
            try:
                t_start = time.perf_counter()
                b = self._buffers(slot, N)
                F = len(batch)
                with torch.cuda.stream(stream):
                    # the uploads are in order: the newest request's event covers the others
                    stream.wait_event(self._newest(batch))
                    # device-to-device gather of the resident inputs into the slot's buffers
                    torch.cat([r.dcoord for r in batch], out=b["coord"][:N])
                    torch.cat([r.dtype for r in batch], out=b["type"][:N])
                    e = torch.empty(F, dtype=torch.float64, device=b["coord"].device)
                    v = torch.empty((F, 3, 3), dtype=torch.float64, device=b["coord"].device)
                    f = b["force"][:N]
                    dpgb.compute_batch(models, nat, b["coord"][:N], b["type"][:N], boxes, stream=stream,
                                       out=(e, f, v, None), frame_model=fmodel)
                    h = b["host"]  # the results go back to the requesters: one copy each, one wait
                    h[:F].copy_(e, non_blocking=True)
                    h[F:10 * F].copy_(v.reshape(-1), non_blocking=True)
                    h[10 * F:10 * F + 3 * N].copy_(f.reshape(-1), non_blocking=True)
                stream.synchronize()
                e_h = h[:F].numpy().copy()
                v_h = h[F:10 * F].numpy().reshape(F, 3, 3).copy()
                f_h = h[10 * F:10 * F + 3 * N].numpy().reshape(N, 3).copy()
                t_end = time.perf_counter()
            except Exception as exc:  # keep serving; report at the end
                self.errors.append(repr(exc))
                continue
            done = t_end - self.t0
            off = np.concatenate([[0], np.cumsum(nat)])
            for k, r in enumerate(batch):
                r.done = done
                r.energy = float(e_h[k])
                r.force = f_h[off[k]:off[k + 1]]
                r.virial = v_h[k]
                r.dcoord = r.dtype = r.ready = None
            with self.cv:
                self.completed.extend(batch)
                self.batches.append((len(batch), N, t_end - t_start, len(set(fmodel.tolist()))))

    def run(self, requests: List[Request], realtime: bool = True, prefill: bool = False) -> dict:
        """Replay `requests` (arrival times in seconds) and serve them; returns statistics.

        prefill: every request arrives (and is uploaded) before the slots start, all at time 0 --
        the operating point of a queue that never runs dry, whose throughput is the capacity of
        the GPU path rather than of the submitting thread."""
        threads = [threading.Thread(target=self._worker, args=(s,), daemon=True) for s in range(self.slots)]
        if prefill:
            for r in sorted(requests, key=lambda r: r.arrival):
                r.arrival = 0.0
                self.submit(r)
            if self.upload is not None:
                self.upload.synchronize()
        self.t0 = time.perf_counter()
        for t in threads:
            t.start()
        for r in ([] if prefill else sorted(requests, key=lambda r: r.arrival)):
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
        sizes = np.array([b[0] for b in self.batches]) if self.batches else np.zeros(1)
        hist = {str(k): int(c) for k, c in zip(*np.unique(np.minimum(sizes, 16), return_counts=True))}
        return {
            "frames": len(self.completed),
            "atoms": int(atoms),
            "atom_evals_per_s": atoms / span,
            "frames_per_s": len(self.completed) / span,
            "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
            "mean_batch_frames": float(np.mean(sizes)) if self.batches else 0.0,
            "mean_batch_atoms": float(np.mean([b[1] for b in self.batches])) if self.batches else 0.0,
            "batch_frames_histogram": hist,  # batch size (16 = 16 or more) -> batches
            "mixed_model_batches": int(sum(1 for b in self.batches if b[3] > 1)),
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
