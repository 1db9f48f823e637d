"""Continuous-batching server of Shack-Hartmann frame requests.

Many concurrent Monte-Carlo runs (the parameter sweeps used to tune a system) each ask for
their next wavefront-sensor frame: a request is (run, step), the frame time is step * dt.
The server

* admits runs in arrival order while their device footprint (screens + the handle's
  tables and scratch) fits the HBM budget, and retires a run once its last request is
  served, which frees budget for the next;
* keeps up to ``slots`` batches in flight, each on its own CUDA stream; whenever a slot is
  free and requests are pending, it launches one batch made of the oldest pending request
  of every admitted run that has no request on the GPU (``wfs_batch_measure_subset``), so
  requests that arrive while others run join the next batch and their work overlaps on the
  device;
* records each request's latency (completion seen by the host minus arrival).

Every request's slopes are those of ``wfs_measure`` on its run's handle: batching changes
neither the arithmetic nor the noise stream (counter-based on seed, t, WFS, pixel).
This module is scheduling only; all arithmetic runs in the library's kernels.
"""
from __future__ import annotations

import dataclasses
import heapq
import math
import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np

from . import inputs, native


def footprint_bytes(cfg: inputs.Config) -> int:
    """Device bytes one run holds: its screens and the handle's tables and scratch."""
    L = cfg.layers
    total = L.n_layers * L.screen_size ** 2 * 4
    for s in cfg.stars:
        g = cfg.geometries[s.geometry_index]
        n_sub = g.n_sub
        nv = n_sub * n_sub  # upper bound on valid subapertures
        n = g.n_pix_sub
        per = n * n * 4 + 8 + 4 * ((n * n + 31) // 32) + 8
        if s.is_lgs:
            per += (2 * n - 1) * n * 8
        total += nv * per
    return int(total)


@dataclass
class Run:
    run_id: int
    cfg: inputs.Config
    seed: int
    screens_host: np.ndarray
    footprint: int = 0
    # device state while admitted
    wfs: Optional[native.Wfs] = None
    screens: object = None
    slopes: object = None
    in_flight: bool = False
    pending: List = field(default_factory=list)   # (arrival_time, step)
    remaining: int = 0                            # requests not yet completed
    index: int = -1                               # position in the current batch


@dataclass
class Stats:
    latencies_ms: List[float] = field(default_factory=list)
    completed: int = 0
    spots: int = 0
    batches: int = 0
    batch_sizes: List[int] = field(default_factory=list)
    admitted_max: int = 0
    duration_s: float = 0.0

    def summary(self) -> Dict:
        lat = np.asarray(self.latencies_ms) if self.latencies_ms else np.zeros(1)
        return {"requests": self.completed, "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
                "frames_per_s": self.completed / max(self.duration_s, 1e-9),
                "spots_per_s": self.spots / max(self.duration_s, 1e-9),
                "batches": self.batches,
                "mean_batch": float(np.mean(self.batch_sizes)) if self.batch_sizes else 0.0,
                "max_admitted": self.admitted_max, "duration_s": self.duration_s}


class Server:
    def __init__(self, runs: List[Run], hbm_budget_bytes: int, slots: int = 3, keep_results: bool = False,
                 noise: bool = True):
        import torch
        self.torch = torch
        self.dev = torch.device("cuda", torch.cuda.current_device())
        self.runs = runs
        self.budget = hbm_budget_bytes
        self.slots = max(1, min(slots, 8))
        self.keep = keep_results
        self.noise = noise
        self.results: Dict = {}
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(self.slots)]
        self.events = [None] * self.slots          # completion event per slot
        self.slot_reqs = [[] for _ in range(self.slots)]  # (run, arrival, step) per slot
        self.admitted: List[Run] = []
        self.used = 0
        self.batch = None
        self.old_batches = []                       # (batch, set of slots still using it)
        self.batch_dirty = True
        for r in runs:
            r.footprint = footprint_bytes(r.cfg)

    # ---------------------------------------------------------------- admission
    def _admit(self, r: Run):
        r.wfs = native.Wfs(r.cfg, seed=r.seed, noise=self.noise)
        r.screens = self.torch.as_tensor(r.screens_host).to(self.dev)
        r.slopes = self.torch.zeros((max(r.wfs.total, 1), 2), device=self.dev)
        self.admitted.append(r)
        self.used += r.footprint
        self.batch_dirty = True

    def _retire(self, r: Run):
        self.admitted.remove(r)
        self.used -= r.footprint
        self.batch_dirty = True
        self._retired.append(r)

    def _rebuild_batch(self):
        if self.batch is not None:
            busy = {k for k in range(self.slots) if self.events[k] is not None}
            self.old_batches.append((self.batch, busy))
        self.batch = native.wfs_batch_create([r.wfs.h for r in self.admitted]) if self.admitted else None
        for i, r in enumerate(self.admitted):
            r.index = i
        self.batch_dirty = False

    def _collect_old(self):
        keep = []
        for b, busy in self.old_batches:
            busy = {k for k in busy if self.events[k] is not None}
            if busy:
                keep.append((b, busy))
            else:
                native.wfs_batch_destroy(b)
        self.old_batches = keep

    def _free_retired(self):
        # a retired run's device memory is released once no slot can still be using it
        if any(e is not None for e in self.events):
            return
        for r in self._retired:
            if r.wfs is not None:
                r.wfs.close()
                r.wfs = None
            r.screens = None
            r.slopes = None
        self._retired = []

    def preadmit(self):
        """Admit, before the clock starts, every run that fits the budget (runs whose state
        is already device-resident when their traffic begins)."""
        for r in self.runs:
            if r.wfs is None and self.used + r.footprint <= self.budget:
                self._admit(r)
        if self.batch_dirty:
            self._rebuild_batch()
        self.torch.cuda.synchronize()

    # ---------------------------------------------------------------- main loop
    def serve(self, arrivals: List, max_seconds: float = 120.0) -> Stats:
        """arrivals: list of (arrival_offset_s, run_id, step), any order; offsets are from the
        start of this call."""
        st = Stats()
        self._retired = []
        by_run = {r.run_id: r for r in self.runs}
        for r in self.runs:
            r.remaining = 0
            r.pending = []
            r.in_flight = False
        queue = []
        for a, rid, step in arrivals:
            heapq.heappush(queue, (a, rid, step))
            by_run[rid].remaining += 1
        first = {}
        for a, rid, _ in arrivals:
            first[rid] = min(a, first.get(rid, math.inf))
        waiting = [by_run[rid] for rid in sorted(first, key=lambda rid: first[rid])
                   if by_run[rid].wfs is None]
        t0 = time.perf_counter()
        deadline = t0 + max_seconds
        while True:
            now = time.perf_counter() - t0
            while queue and queue[0][0] <= now:
                a, rid, step = heapq.heappop(queue)
                by_run[rid].pending.append((a, step))
            # completions
            for k in range(self.slots):
                ev = self.events[k]
                if ev is not None and ev.query():
                    tdone = time.perf_counter() - t0
                    for r, a, step in self.slot_reqs[k]:
                        st.latencies_ms.append(1e3 * (tdone - a))
                        st.completed += 1
                        st.spots += r.wfs.total
                        r.in_flight = False
                        r.remaining -= 1
                        if self.keep:
                            self.results[(r.run_id, step)] = r.slopes[: r.wfs.total].cpu().numpy().copy()
                        if r.remaining == 0:
                            self._retire(r)
                    self.slot_reqs[k] = []
                    self.events[k] = None
            self._collect_old()
            self._free_retired()
            # admission (arrival order of the runs' first request)
            while waiting and self.used + waiting[0].footprint <= self.budget:
                self._admit(waiting.pop(0))
            st.admitted_max = max(st.admitted_max, len(self.admitted))
            if self.batch_dirty:
                self._rebuild_batch()
            # launch into a free slot
            ready = [r for r in self.admitted if r.pending and not r.in_flight]
            free = [k for k in range(self.slots) if self.events[k] is None]
            if ready and free and self.batch is not None:
                k = free[0]
                reqs = []
                for r in ready:
                    a, step = r.pending.pop(0)
                    reqs.append((r, a, step))
                    r.in_flight = True
                s = self.streams[k]
                native.wfs_batch_measure_subset(
                    self.batch, k, [r.index for r, _, _ in reqs], [r.screens.data_ptr() for r, _, _ in reqs],
                    [step * r.cfg.dt_s for r, _, step in reqs], [r.slopes.data_ptr() for r, _, _ in reqs],
                    s.cuda_stream)
                ev = self.torch.cuda.Event()
                ev.record(s)
                self.events[k] = ev
                self.slot_reqs[k] = reqs
                st.batches += 1
                st.batch_sizes.append(len(reqs))
                continue
            if not queue and all(e is None for e in self.events) and not any(r.pending for r in self.admitted) \
                    and not waiting:
                break
            if time.perf_counter() > deadline:
                break
            time.sleep(2e-5)
        st.duration_s = time.perf_counter() - t0
        self.torch.cuda.synchronize()
        self._free_retired()
        for r in list(self.admitted):
            self._retire(r)
        self._free_retired()
        if self.batch is not None:
            native.wfs_batch_destroy(self.batch)
            self.batch = None
        for b, _ in self.old_batches:
            native.wfs_batch_destroy(b)
        self.old_batches = []
        return st


# ---------------------------------------------------------------- the serving workload

def make_runs(n_runs: int = 32, seed: int = 5000, dt_s: float = 1e-3,
              mix=(inputs.config1, inputs.config2, inputs.config3)) -> List[Run]:
    """n_runs Monte-Carlo runs drawn from the configurations (seeded).  Runs of one
    configuration share one screen set (generated once) but sample it at their own
    layer offsets, so each run sees its own turbulence."""
    rng = np.random.default_rng(seed)
    cache = {}
    runs = []
    for i in range(n_runs):
        k = int(rng.integers(len(mix)))
        cfg = mix[k](inputs.PREC_FP32)
        cfg.layers = dataclasses.replace(cfg.layers)
        span = cfg.layers.screen_size * cfg.layers.screen_dx_m
        cfg.layers.x0_m = rng.uniform(0, span, cfg.layers.n_layers)
        cfg.layers.y0_m = rng.uniform(0, span, cfg.layers.n_layers)
        cfg.dt_s = dt_s
        if k not in cache:
            cache[k] = inputs.make_screens(cfg.layers, cfg.seed)
        runs.append(Run(run_id=i, cfg=cfg, seed=seed + 1 + i, screens_host=cache[k]))
    return runs


def poisson_arrivals(runs: List[Run], rate_per_run: float, duration_s: float, seed: int = 1,
                     stagger_s: float = 0.0, max_per_run: Optional[int] = None) -> List:
    """Per-run Poisson arrivals of next-step requests; run i starts at i * stagger_s."""
    rng = np.random.default_rng(seed)
    out = []
    for i, r in enumerate(runs):
        t = i * stagger_s
        step = 0
        while True:
            t += rng.exponential(1.0 / rate_per_run)
            if t > duration_s + i * stagger_s:
                break
            out.append((t, r.run_id, step))
            step += 1
            if max_per_run and step >= max_per_run:
                break
    return out


def capacity(runs: List[Run], hbm_budget_bytes: int, slots: int = 3, frames: int = 400) -> float:
    """Saturated throughput (frames/s) with the runs pre-admitted: every run has
    `frames // len(runs)` requests at t = 0."""
    per = max(1, frames // len(runs))
    arrivals = [(0.0, r.run_id, s) for r in runs for s in range(per)]
    srv = Server(runs, hbm_budget_bytes, slots)
    srv.preadmit()
    st = srv.serve(arrivals)
    return st.completed / st.duration_s
