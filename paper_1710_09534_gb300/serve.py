"""Continuous-batching request loop for many independent lattice simulations.

Requests (a workload: size, geometry, parameters, initial fields, a step
count and a storage precision) arrive over time.  The server keeps every
admitted lattice resident on the device inside one batch per precision
(`Batch`: all members advance together in one persistent kernel per step),
admits waiting requests first-come first-served whenever their device
footprint (tlb_workspace_bytes, plus the batch's own workspace when the
request opens a batch) fits the HBM budget and the batch has a free slot and
room for the request's tiles and near-wall nodes, advances the batches in
chunks no longer than the smallest remaining step count, and returns each
finished lattice's fields (read back to host memory) as soon as it completes,
freeing its memory for the next requests.  Requests that arrive while others
run join the running batch at the next chunk boundary, so their work shares
the device with the others'.

The host work overlaps the device work: a chunk is launched first, and while
it runs the server reads back the lattices that finished in the previous
chunk and sets up the lattices of newly admitted requests (on a stream of its
own); at the chunk boundary it only removes finished members, adds the new
ones and launches the next chunk.  Whenever a batch's size mix changes
materially (the number of tiles by a factor of two, or the share of small
members by a quarter), the batch tuner picks the tile shape again on the live
members, which it leaves unchanged; shapes already tuned for a mix are reused.

Time to result = completion time (fields on the host) - arrival time (host
clock).  The loop is single-threaded host Python: it only launches work and
moves data; every lattice update runs in the library's CUDA kernels.
"""
from __future__ import annotations

import math
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
    tiles: int
    wall: int


@dataclass
class ServeStats:
    requests: int = 0
    node_updates: int = 0
    makespan: float = 0.0
    latencies: list = field(default_factory=list)
    peak_bytes: int = 0
    peak_members: int = 0
    gpu_busy: float = 0.0
    chunks: int = 0
    tune_s: float = 0.0   # wall time spent in the tuner (its trial steps leave the state unchanged)
    tuned: list = field(default_factory=list)

    def summary(self):
        lat = np.array(self.latencies) if self.latencies else np.zeros(1)
        return {"requests": self.requests, "node_updates": self.node_updates,
                "makespan_s": round(self.makespan, 3),
                "aggregate_mlups": round(self.node_updates / max(self.makespan, 1e-9) / 1e6, 1),
                "p50_s": round(float(np.percentile(lat, 50)), 3),
                "p99_s": round(float(np.percentile(lat, 99)), 3),
                "peak_resident_bytes": self.peak_bytes, "peak_resident_lattices": self.peak_members,
                "chunks": self.chunks,
                "gpu_busy_s": round(self.gpu_busy, 3),
                "gpu_idle_frac": round(max(0.0, 1.0 - self.gpu_busy / max(self.makespan, 1e-9)), 3),
                "tune_s": round(self.tune_s, 3),
                "tuned": self.tuned}


class Server:
    """One batch per storage precision, an HBM budget and a chunk length."""

    def __init__(self, hbm_budget_bytes: int, max_lattices: int = 256, chunk: int = 200,
                 max_tiles: int = 1 << 20, max_wall_nodes: int = 1 << 23, tune: bool = True,
                 tune_steps: int = 2):
        import torch
        self.torch = torch
        self.lib = load_library()
        self.budget = int(hbm_budget_bytes)
        self.max_lattices = int(max_lattices)
        self.chunk = int(chunk)
        self.caps = (int(max_tiles), int(max_wall_nodes))
        self.batch_bytes = int(self.lib.tlb_batch_workspace_bytes(self.max_lattices, *self.caps))
        self.tune, self.tune_steps = bool(tune), int(tune_steps)
        self.batches = {}
        self.active: list[_Active] = []
        self.used = 0
        self.tiles_used = {}
        self.wall_used = {}
        self.mix_key = {}       # precision -> size mix the batch's shape was picked for
        self.tune_cache = {}    # (precision, mix) -> shape
        self.setup_stream = torch.cuda.Stream()

    def footprint(self, req: Request) -> int:
        w = req.workload
        return int(self.lib.tlb_workspace_bytes(w.nx, w.ny, PRECISIONS[req.precision]))

    def _batch(self, precision):
        if precision not in self.batches:
            b = Batch(precision, self.max_lattices, *self.caps)
            # until the tuner has seen a mix: the shape it picked on the
            # 256-lattice workload
            b.config(threads=64, rows_small=8, rows_large=32, small_ny=128)
            self.batches[precision] = b
            self.used += self.batch_bytes
            self.tiles_used[precision] = 0
            self.wall_used[precision] = 0
        return self.batches[precision]

    def _fits(self, req: Request) -> bool:
        extra = 0 if req.precision in self.batches else self.batch_bytes
        if self.used + self.footprint(req) + extra > self.budget:
            return False
        members = sum(1 for a in self.active if a.req.precision == req.precision)
        if members >= self.max_lattices:
            return False
        w = req.workload
        return self.tiles_used.get(req.precision, 0) + Batch.tiles_needed(w.nx, w.ny) <= self.caps[0]

    def _admit(self, req: Request, now: float) -> bool:
        """Build the request's lattice on the set-up stream and reserve its
        memory; False (request stays queued) if its near-wall nodes do not fit
        the batch's capacity."""
        w = req.workload
        with self.torch.cuda.stream(self.setup_stream):
            L = Lattice(w.nx, w.ny, req.precision, w.edges, stream=self.setup_stream)
            L.set_geometry(w.mask)
        wall = L.wall_nodes()
        if self.wall_used.get(req.precision, 0) + wall > self.caps[1]:
            L.close()
            return False
        L.set_params(w.params)
        L.set_fields(w.c1, w.c2, w.ux, w.uy, w.p)
        self._batch(req.precision)
        nb = self.footprint(req)
        tiles = Batch.tiles_needed(w.nx, w.ny)
        self.used += nb
        self.tiles_used[req.precision] += tiles
        self.wall_used[req.precision] += wall
        req.admitted = now
        self.active.append(_Active(req, L, req.steps, nb, tiles, wall))
        return True

    def _release(self, a: _Active):
        self.used -= a.nbytes
        self.tiles_used[a.req.precision] -= a.tiles
        self.wall_used[a.req.precision] -= a.wall
        a.lattice.close()

    def _mix(self, b: Batch):
        """Size mix of a batch: the order of magnitude (base 2) of its tile
        count and the share of members at or below the small-row threshold,
        in quarters."""
        tiles = sum(Batch.tiles_needed(L.nx, L.ny) for L in b.members)
        small = sum(1 for L in b.members if L.ny <= 128) / max(len(b.members), 1)
        return (int(round(math.log2(max(tiles, 1)))), int(round(4 * small)))

    def _retune(self, precision, b: Batch, stats: ServeStats):
        key = self._mix(b)
        if not self.tune or self.mix_key.get(precision) == key:
            return
        cached = self.tune_cache.get((precision, key))
        if cached is not None:
            b.config(cached["threads"], cached["rows_small"], cached["rows_large"], cached["small_ny"])
        else:
            # the tuner's scratch holds the members' c_i u planes while it runs
            scratch = int(self.lib.tlb_batch_tune_scratch_bytes(b._h))
            if self.used + scratch > self.budget:
                return
            t0 = time.perf_counter()
            cfg = b.tune(trial_steps=self.tune_steps)
            stats.tune_s += time.perf_counter() - t0
            self.tune_cache[(precision, key)] = cfg
            stats.tuned.append({"precision": precision, "members": len(b.members),
                                "tiles_log2": key[0], "small_quarters": key[1],
                                "threads": cfg["threads"], "rows_small": cfg["rows_small"],
                                "rows_large": cfg["rows_large"], "ms_per_step": round(cfg["ms_per_step"], 4)})
        self.mix_key[precision] = key

    def run(self, requests: list[Request]) -> ServeStats:
        """Serve `requests` to completion (in order of arrival); returns stats."""
        torch = self.torch
        stats = ServeStats(requests=len(requests))
        for r in requests:
            if self.footprint(r) + self.batch_bytes > self.budget:
                raise ValueError(f"request {r.rid} alone exceeds the HBM budget")
        waiting: list[Request] = []
        incoming = sorted(requests, key=lambda r: r.arrival)
        nxt = 0
        retired: list[_Active] = []   # finished, fields not yet read back
        t0 = time.perf_counter()
        clock = lambda: time.perf_counter() - t0

        def arrivals_and_admissions():
            nonlocal nxt
            now = clock()
            while nxt < len(incoming) and incoming[nxt].arrival <= now:
                waiting.append(incoming[nxt])
                nxt += 1
            while waiting and self._fits(waiting[0]):
                if not self._admit(waiting[0], clock()):
                    break
                waiting.pop(0)

        def read_back():
            for a in retired:
                a.req.fields = a.lattice.fields()
                a.req.done = clock()
                stats.latencies.append(a.req.latency)
                self._release(a)
            retired.clear()

        while nxt < len(incoming) or waiting or self.active or retired:
            # with lattices on the GPU, admissions happen while a chunk runs
            # (below), so that their set-up overlaps the device work
            if not self.active:
                arrivals_and_admissions()
            stats.peak_bytes = max(stats.peak_bytes, self.used)
            stats.peak_members = max(stats.peak_members, len(self.active))
            if not self.active:
                read_back()
                if nxt < len(incoming) and not waiting:
                    time.sleep(max(0.0, min(incoming[nxt].arrival - clock(), 0.05)))
                continue
            # chunk boundary: new members join, shapes follow the mix
            for a in self.active:
                b = self.batches[a.req.precision]
                if a.lattice not in b.members:
                    b.add(a.lattice)
            for p, b in self.batches.items():
                if b.members:
                    self._retune(p, b, stats)
            k = min(self.chunk, min(a.remaining for a in self.active))
            ev = []
            for b in self.batches.values():
                if b.members:
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(b.stream)
                    b.step(k)
                    e1.record(b.stream)
                    ev.append((e0, e1))
            # while the chunk runs: results of the previous chunk, new arrivals
            read_back()
            arrivals_and_admissions()
            stats.peak_bytes = max(stats.peak_bytes, self.used)
            for b in self.batches.values():
                b.synchronize()
            stats.gpu_busy += max(e0.elapsed_time(e1) for e0, e1 in ev) / 1e3
            stats.chunks += 1
            running = [a for a in self.active if a.lattice in self.batches[a.req.precision].members]
            for a in running:
                a.remaining -= k
                stats.node_updates += a.req.workload.nodes * k
            for a in [a for a in running if a.remaining <= 0]:
                self.batches[a.req.precision].remove(a.lattice)
                self.active.remove(a)
                retired.append(a)
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
