"""Serving loop: continuous batching of limited-LBM solves on one GPU.

Requests (a lattice, its initial state and a number of steps) arrive over
time.  The server keeps every admitted lattice resident in a Batch
(include/lbm_batch.h) and advances all of them together, one quantum of steps
at a time.  Between quanta it admits waiting requests, first come first
served, as long as their device footprint (lbm_footprint_bytes) fits in the
memory budget, and retires the ones that reached their step count, reading
their density and velocity fields back.  Work of different requests therefore
overlaps on the device: every batched launch covers all resident lattices.
A lattice's result does not depend on the mix it ran in (the batched kernels
evaluate each site exactly as a lone run does).

Host-side scheduling only; every step runs in the CUDA library.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import inputs as _inputs
from . import lbm


@dataclass
class Request:
    rid: int
    arrival: float              # seconds after the start of the run
    workload: _inputs.Workload
    rho: np.ndarray = None
    ux: np.ndarray = None
    uy: np.ndarray = None


@dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    steps: int
    sites: int
    rho: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    stats: dict = field(default_factory=dict)
    status: str = "ok"          # "ok", or "nonfinite" for a solve that blew up (no fields)

    @property
    def latency(self) -> float:
        return self.finished - self.arrival

    @property
    def queued(self) -> float:
        return self.admitted - self.arrival


def lattice_config(w: _inputs.Workload) -> dict:
    """The lbm_config fields of one workload (FP32 storage)."""
    if w.lattice == lbm.D1Q3:
        return dict(lattice=lbm.D1Q3, nx=w.nx, ny=1, boundary=lbm.BC_WALLS, precision=lbm.FP32,
                    beta=w.beta, limiters=w.limiters, delta_median=w.delta_median,
                    delta_ehrenfest=w.delta_ehrenfest, k_max=w.k_max, rho_ref=1.0)
    return dict(lattice=lbm.D2Q9, nx=w.nx, ny=w.ny, boundary=lbm.BC_WALLS, precision=lbm.FP32,
                beta=w.beta, u_lid=w.u_lid, rho_wall=w.rho0, limiters=w.limiters,
                delta_median=w.delta_median, delta_ehrenfest=w.delta_ehrenfest, k_max=w.k_max)


def initial_state(w: _inputs.Workload):
    """Rest state of a cavity, or the two-density shock tube."""
    if w.lattice == lbm.D1Q3:
        rho, ux = _inputs.shock_tube(w.nx, 1.0, w.rho_right)
        return rho, ux, None
    return _inputs.cavity_rest(w.nx, w.ny, w.rho0)


def requests_from_trace(trace) -> list:
    return [Request(i, t, w) for i, (t, w) in enumerate(trace)]


class Server:
    """Continuous-batching server over one Batch.

    memory_bytes: device budget for resident lattices (admission by footprint).
    quantum: steps per batched round between admission / retirement decisions.
    graph_steps: CUDA-graph replay length inside a round (0: plain launches).
    batch: the batch to serve from (default: a new lbm.Batch on `stream`); any
    object with lbm.Batch's add / init / step / synchronize / lattice_status /
    moments / stats / remove methods.
    """

    def __init__(self, memory_bytes: int, quantum: int = 500, graph_steps: int = 0,
                 stream: int | None = None, clock=time.perf_counter, batch=None):
        self.batch = lbm.Batch(stream) if batch is None else batch
        if graph_steps:
            self.batch.set_graph(graph_steps)
        self.memory_bytes = int(memory_bytes)
        self.quantum = int(quantum)
        self.clock = clock
        self.rounds = 0
        self.steps_run = 0
        self.site_updates = 0

    def close(self):
        self.batch.close()

    def run(self, requests, realtime: bool = True, on_round=None) -> list:
        """Serves `requests` (sorted by arrival).  With realtime, a request is
        visible only once the wall clock passes its arrival time; otherwise all
        arrivals are visible at once (a closed queue).  Returns the results in
        completion order."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting = collections.deque()
        active = {}  # slot -> [request, remaining, admitted, footprint]
        used = 0
        results = []
        t0 = self.clock()
        while pending or waiting or active:
            now = self.clock() - t0
            while pending and (not realtime or pending[0].arrival <= now):
                waiting.append(pending.popleft())
            # admission: first come first served while the footprint fits
            while waiting:
                req = waiting[0]
                cfg = lattice_config(req.workload)
                need = lbm.footprint_bytes(**cfg)
                if need > self.memory_bytes:
                    raise ValueError(f"request {req.rid} needs {need} bytes, above the memory budget")
                if used + need > self.memory_bytes:
                    break
                waiting.popleft()
                slot = self.batch.add(**cfg)
                if req.rho is None:
                    req.rho, req.ux, req.uy = initial_state(req.workload)
                self.batch.init(slot, req.rho, req.ux, req.uy)
                active[slot] = [req, req.workload.steps, self.clock() - t0, need]
                used += need
            if not active:
                if pending:  # idle until the next arrival
                    delay = pending[0].arrival - (self.clock() - t0)
                    if delay > 0:
                        time.sleep(min(delay, 0.05))
                continue
            q = min(self.quantum, min(a[1] for a in active.values()))
            self.batch.step(q)
            failed = set()
            try:
                self.batch.synchronize()
            except lbm.LBMError as e:
                # a solve that met a nonfinite site is retired as failed; the
                # other lattices of the batch are independent and carry on
                if e.status != lbm.ERR_NONFINITE:
                    raise
                failed = {s for s in active if self.batch.lattice_status(s) != lbm.OK}
            self.rounds += 1
            self.steps_run += q
            self.site_updates += q * sum(a[0].workload.sites for a in active.values())
            done = [s for s, a in active.items() if a[1] - q <= 0 or s in failed]
            for s, a in active.items():
                a[1] -= q
            for s in done:
                req, left, admitted, need = active.pop(s)
                if s in failed:
                    rho = ux = uy = None
                    st, status = {}, "nonfinite"
                else:
                    rho, ux, uy = self.batch.moments(s)
                    st, status = self.batch.stats(s), "ok"
                self.batch.remove(s)
                used -= need
                results.append(Result(req.rid, req.arrival, admitted, self.clock() - t0,
                                      req.workload.steps - max(left, 0), req.workload.sites, rho, ux, uy, st,
                                      status))
            if on_round is not None:
                on_round(self, active)
        return results


def summarize(results, wall_s: float, site_updates: int) -> dict:
    """Latency percentiles over the completed solves; failed ones are counted."""
    ok = [r for r in results if r.status == "ok"]
    lat = np.array([r.latency for r in ok]) if ok else np.zeros(1)
    que = np.array([r.queued for r in ok]) if ok else np.zeros(1)
    return {"requests": len(results), "failed": len(results) - len(ok),
            "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)), "mean_latency_s": float(lat.mean()),
            "p50_queue_s": float(np.percentile(que, 50)), "p99_queue_s": float(np.percentile(que, 99)),
            "wall_s": wall_s, "aggregate_mlups": site_updates / wall_s / 1e6}
