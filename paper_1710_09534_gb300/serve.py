"""Continuous-batching request loop for many independent lattice simulations.

Requests (a workload: size, geometry, parameters, initial fields, a step
count and a storage precision) arrive over time.  The server keeps every
admitted lattice resident on the device inside one batch per precision
(`Batch`: all members advance together in one persistent kernel per step),
admits waiting requests first-come first-served whenever their device
footprint (tlb_workspace_bytes) fits the HBM budget and the batch has a free
slot, advances the batches in chunks no longer than the smallest remaining
step count, and returns each finished lattice's fields (read back to host
memory) as soon as it completes, freeing its memory for the next requests.
Requests that arrive while others run join the running batch at the next
chunk boundary, so their work shares the device with the others'.

Time to result = completion time - arrival time (host clock).  The loop is
single-threaded host Python: it only launches work and moves data; every
lattice update runs in the library's CUDA kernels.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import Batch, Lattice, load_library, PRECISIONS


@dataclass
class Request:
    rid: int
    workload: object          # workloads.Workload
    steps: int
    precision: str = "fp32"
    arrival: float = 0.0      # seconds after the server starts
    # filled in by the server
    admitted: float | None = None
    done: float | None = None
    fields: dict | None = None

    @property
    def latency(self):
        return None if self.done is None else self.done - self.arrival


@dataclass
class _Active:
    req: Request
    lattice: Lattice
    remaining: int
    nbytes: int


@dataclass
class ServeStats:
    requests: int = 0
    node_updates: int = 0
    makespan: float = 0.0
    latencies: list = field(default_factory=list)
    peak_bytes: int = 0
    peak_members: int = 0

    def summary(self):
        lat = np.array(self.latencies) if self.latencies else np.zeros(1)
        return {"requests": self.requests, "node_updates": self.node_updates,
                "makespan_s": round(self.makespan, 3),
                "aggregate_mlups": round(self.node_updates / max(self.makespan, 1e-9) / 1e6, 1),
                "p50_s": round(float(np.percentile(lat, 50)), 3),
                "p99_s": round(float(np.percentile(lat, 99)), 3),
                "peak_resident_bytes": self.peak_bytes, "peak_resident_lattices": self.peak_members}


class Server:
    """One batch per storage precision, an HBM budget and a chunk length."""

    def __init__(self, hbm_budget_bytes: int, max_lattices: int = 256, chunk: int = 200,
                 max_tiles: int = 1 << 20, max_wall_nodes: int = 1 << 23):
        self.lib = load_library()
        self.budget = int(hbm_budget_bytes)
        self.max_lattices = int(max_lattices)
        self.chunk = int(chunk)
        self.caps = (int(max_tiles), int(max_wall_nodes))
        self.batches = {}
        self.active: list[_Active] = []
        self.used = 0
        self.tiles_used = {}
        self.wall_used = {}

    def footprint(self, req: Request) -> int:
        w = req.workload
        return int(self.lib.tlb_workspace_bytes(w.nx, w.ny, PRECISIONS[req.precision]))

    def _batch(self, precision):
        if precision not in self.batches:
            b = Batch(precision, self.max_lattices, *self.caps)
            # the shape the batch tuner picked on the 256-lattice workload
            b.config(threads=64, rows_small=8, rows_large=32, small_ny=128)
            self.batches[precision] = b
            self.tiles_used[precision] = 0
            self.wall_used[precision] = 0
        return self.batches[precision]

    def _fits(self, req: Request) -> bool:
        if self.used + self.footprint(req) > self.budget:
            return False
        b = self.batches.get(req.precision)
        if b is not None and len(b.members) >= self.max_lattices:
            return False
        w = req.workload
        tiles = Batch.tiles_needed(w.nx, w.ny)
        return self.tiles_used.get(req.precision, 0) + tiles <= self.caps[0]

    def _admit(self, req: Request, now: float):
        w = req.workload
        L = Lattice(w.nx, w.ny, req.precision, w.edges)
        L.set_geometry(w.mask)
        L.set_params(w.params)
        L.set_fields(w.c1, w.c2, w.ux, w.uy, w.p)
        b = self._batch(req.precision)
        if self.wall_used[req.precision] + L.wall_nodes() > self.caps[1]:
            raise RuntimeError("batch wall-node capacity exceeded")
        b.add(L)
        nb = self.footprint(req)
        self.used += nb
        self.tiles_used[req.precision] += Batch.tiles_needed(w.nx, w.ny)
        self.wall_used[req.precision] += L.wall_nodes()
        req.admitted = now
        self.active.append(_Active(req, L, req.steps, nb))

    def _retire(self, a: _Active, now: float):
        b = self.batches[a.req.precision]
        b.remove(a.lattice)
        a.req.fields = a.lattice.fields()
        a.req.done = now
        self.used -= a.nbytes
        w = a.req.workload
        self.tiles_used[a.req.precision] -= Batch.tiles_needed(w.nx, w.ny)
        self.wall_used[a.req.precision] -= a.lattice.wall_nodes()
        a.lattice.close()
        self.active.remove(a)

    def run(self, requests: list[Request]) -> ServeStats:
        """Serve `requests` (sorted by arrival) to completion; returns stats."""
        stats = ServeStats(requests=len(requests))
        waiting = []
        incoming = sorted(requests, key=lambda r: r.arrival)
        i = 0
        t0 = time.perf_counter()
        clock = lambda: time.perf_counter() - t0
        for r in requests:
            if self.footprint(r) > self.budget:
                raise ValueError(f"request {r.rid} alone exceeds the HBM budget")
        while i < len(incoming) or waiting or self.active:
            now = clock()
            while i < len(incoming) and incoming[i].arrival <= now:
                waiting.append(incoming[i])
                i += 1
            while waiting and self._fits(waiting[0]):
                self._admit(waiting.pop(0), clock())
            stats.peak_bytes = max(stats.peak_bytes, self.used)
            stats.peak_members = max(stats.peak_members, len(self.active))
            if not self.active:
                if i < len(incoming):
                    time.sleep(max(0.0, min(incoming[i].arrival - clock(), 0.05)))
                continue
            k = min(self.chunk, min(a.remaining for a in self.active))
            if k > 0:
                for p, b in self.batches.items():
                    if b.members:
                        b.step(k)
                for b in self.batches.values():
                    b.synchronize()
                for a in self.active:
                    a.remaining -= k
                    stats.node_updates += a.req.workload.nodes * k
            now = clock()
            for a in [a for a in self.active if a.remaining <= 0]:
                self._retire(a, now)
                stats.latencies.append(a.req.latency)
        stats.makespan = clock()
        return stats

    def close(self):
        for a in list(self.active):
            a.lattice.close()
        self.active = []
        for b in self.batches.values():
            b.close()
        self.batches = {}


def poisson_arrivals(n: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Arrival times of n requests of a Poisson process with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, n))
