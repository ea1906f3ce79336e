"""Serving many independent MHD runs with continuous batching, admitted by free device memory.

Requests (grid size N, initial condition, nu, eta, Mach, step budget) arrive as a Poisson stream.
Runs of one grid size are batched in "slabs": fixed-capacity `mhd_pool`s (C ABI) whose slots hold
device-resident runs stepped together in one launch per kernel.  Slabs are not planned ahead:

  * admission: a waiting request goes to an idle slab of its size with a free slot; if there is
    none, a new slab is created when the device's free memory at that moment (the driver's free
    memory plus what PyTorch's caching allocator holds unused, less a reserve) covers its
    footprint (mhd_footprint_bytes), with as many slots as fit, up to a per-size cap;
  * retirement: a run that has reached its step budget is copied out (D2H) and its slot freed; a
    slab with no live run left is destroyed at once, so the memory a retired 32^3 run frees can
    admit a waiting 256^3 run;
  * each slab advances k steps at a time on its own CUDA stream and is polled through its own
    events, so slabs of different sizes overlap on the device and a run's per-step latency is the
    device time of its own slab's steps (event to event, divided by k), not a global round's.

Runs never interact, so a run's result is bitwise the same alone and in the mix.

Reported: per-step latency (one sample per live run and slab batch), per-run latency
(retirement time - arrival time), queueing time, p50 and p99 of each overall and per grid size,
and aggregate throughput in grid-point-steps/s.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import inputs, mhd

SIZES = (32, 64, 128, 256)
WEIGHTS = (0.4, 0.3, 0.2, 0.1)
IC_SEEDS = 4  # initial states per (N, kind); requests pick one, the host caches them
# most slots one slab of a size gets (larger N: fewer instances already fill the device)
SLAB_CAP = {16: 64, 32: 64, 64: 32, 128: 8, 256: 4, 512: 1, 1024: 1}


@dataclass
class Request:
    rid: int
    arrival: float
    n: int
    ic: str
    seed: int
    nu: float
    eta: float
    mach: float
    nsteps: int

    @property
    def work(self) -> float:
        return float(self.n) ** 3 * self.nsteps


def make_requests(count: int, rate: float, seed: int = 5, sizes=SIZES, weights=WEIGHTS,
                  steps=(100, 1000)) -> list:
    """Poisson stream of `count` requests at `rate` per second, all parameters from
    default_rng(seed): N by `weights`, ABC or Orszag-Tang 50/50, nu, eta ~ U[1e-3, 1e-2],
    Mach ~ U[0.05, 0.5], steps ~ U{steps[0]..steps[1]}."""
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, count))
    ns = rng.choice(np.array(sizes), p=np.array(weights), size=count)
    ics = rng.choice(np.array(["abc", "ot"]), size=count)
    nu = rng.uniform(1e-3, 1e-2, count)
    eta = rng.uniform(1e-3, 1e-2, count)
    mach = rng.uniform(0.05, 0.5, count)
    nsteps = rng.integers(steps[0], steps[1] + 1, count)
    seeds = rng.integers(0, IC_SEEDS, count)
    return [Request(i, float(arrivals[i]), int(ns[i]), str(ics[i]), int(seeds[i]), float(nu[i]), float(eta[i]),
                    float(mach[i]), int(nsteps[i])) for i in range(count)]


class ICCache:
    """Host-side initial states keyed by (N, kind, seed); parameters are set per request."""

    def __init__(self):
        self._c = {}

    def get(self, req: Request):
        key = (req.n, req.ic, req.seed)
        if key not in self._c:
            if req.ic == "abc":
                ic = inputs.abc_dynamo(req.n, seed=req.seed, b_energy=1e-5)
            else:
                ic = inputs.orszag_tang(req.n, seed=req.seed)
            self._c[key] = (np.ascontiguousarray(ic.rho), np.ascontiguousarray(ic.u), np.ascontiguousarray(ic.b))
        return self._c[key]


def slab_capacity(n: int, precision: int, available_bytes: float, cap: int | None = None) -> int:
    """Slots of a new slab of size n: the most, up to `cap` (SLAB_CAP[n] by default), whose
    footprint fits in `available_bytes`; 0 if not even one slot fits."""
    cap = SLAB_CAP.get(n, 1) if cap is None else cap
    c = cap
    while c > 0 and mhd.mhd_footprint_bytes(n, precision, c) > available_bytes:
        c -= 1
    return c


def pct(a, q):
    return float(np.percentile(a, q)) if len(a) else None


@dataclass
class ServeStats:
    completed: int = 0
    work: float = 0.0
    wall: float = 0.0
    step_latency_ms: list = field(default_factory=list)
    run_latency_s: list = field(default_factory=list)
    queue_s: list = field(default_factory=list)
    outputs: dict = field(default_factory=dict)
    by_size: dict = field(default_factory=dict)  # n -> {"step_ms": [...], "run_s": [...]}
    admitted_at: dict = field(default_factory=dict)  # request id -> seconds from the start
    retired_at: dict = field(default_factory=dict)
    slabs_created: int = 0
    peak_bytes: float = 0.0

    def summary(self) -> dict:
        out = {"completed": self.completed, "wall_s": self.wall,
               "throughput": self.work / self.wall if self.wall > 0 else 0.0,
               "step_latency_ms_p50": pct(self.step_latency_ms, 50), "step_latency_ms_p99": pct(self.step_latency_ms, 99),
               "run_latency_s_p50": pct(self.run_latency_s, 50), "run_latency_s_p99": pct(self.run_latency_s, 99),
               "queue_s_p50": pct(self.queue_s, 50), "queue_s_p99": pct(self.queue_s, 99)}
        if self.by_size:
            out["per_size"] = {str(n): {"runs": len(v["run_s"]), "step_latency_ms_p50": pct(v["step_ms"], 50),
                                        "step_latency_ms_p99": pct(v["step_ms"], 99),
                                        "run_latency_s_p50": pct(v["run_s"], 50), "run_latency_s_p99": pct(v["run_s"], 99)}
                               for n, v in sorted(self.by_size.items())}
            out["slabs_created"] = self.slabs_created
            out["peak_slab_bytes"] = self.peak_bytes
        return out


class Slab:
    """One pool of a grid size on a stream of its own."""

    def __init__(self, torch, n: int, capacity: int, precision: int):
        self.n, self.capacity = n, capacity
        self.stream = torch.cuda.Stream()
        with torch.cuda.stream(self.stream):
            self.pool = mhd.mhd_pool_create(n, capacity, precision=precision)
        self.footprint = mhd.mhd_footprint_bytes(n, precision, capacity)
        self.live = {}  # slot -> request
        self.busy = False
        self.ev0 = torch.cuda.Event(enable_timing=True)
        self.ev1 = torch.cuda.Event(enable_timing=True)

    def close(self):
        mhd.mhd_pool_destroy(self.pool)


class Server:
    """Continuous-batching scheduler over slabs (see the module docstring).

    `memory_limit` (bytes, optional) caps the slabs' total footprint below what the device has
    free, so that admission by memory can be exercised at any device size; `reserve` bytes of
    device memory are always left free."""

    def __init__(self, precision: int = mhd.MHD_FP32_MIXED, k: int = 10, cache: ICCache | None = None,
                 memory_limit: float | None = None, reserve: float = 2e9, slab_cap: dict | None = None):
        import torch
        self.torch = torch
        self.k = k
        self.precision = precision
        self.cache = cache or ICCache()
        self.memory_limit = memory_limit
        self.reserve = reserve
        self.slab_cap = dict(SLAB_CAP)
        self.slab_cap.update(slab_cap or {})
        self.slabs = []

    def close(self):
        for s in self.slabs:
            s.close()
        self.slabs.clear()

    def used_bytes(self) -> float:
        return float(sum(s.footprint for s in self.slabs))

    def available_bytes(self) -> float:
        t = self.torch
        free, _ = t.cuda.mem_get_info()
        cached = t.cuda.memory_reserved() - t.cuda.memory_allocated()
        avail = free + cached - self.reserve
        if self.memory_limit is not None:
            avail = min(avail, self.memory_limit - self.used_bytes())
        return avail

    def _admit_into(self, slab: Slab, req: Request) -> bool:
        rho, u, b = self.cache.get(req)
        with self.torch.cuda.stream(slab.stream):
            slot = mhd.mhd_pool_admit(slab.pool, (req.nu, req.eta, 1.0 / req.mach), rho, u, b, req.nsteps)
        if slot is None:
            return False
        slab.live[slot] = req
        return True

    def _place(self, req: Request, stats: ServeStats) -> str:
        """Admit `req` into an idle slab of its size with a free slot ("admitted"); if a slab of
        its size has a free slot but is stepping, wait for it, at most one batch of k steps
        ("wait"); else open a new slab if the free memory allows, or report "memory"."""
        room = [s for s in self.slabs if s.n == req.n and len(s.live) < s.capacity]
        for s in room:
            if not s.busy:
                return "admitted" if self._admit_into(s, req) else "wait"
        if room:
            return "wait"
        cap = slab_capacity(req.n, self.precision, self.available_bytes(), self.slab_cap.get(req.n, 1))
        if cap < 1:
            return "memory"
        slab = Slab(self.torch, req.n, cap, self.precision)
        self.slabs.append(slab)
        stats.slabs_created += 1
        stats.peak_bytes = max(stats.peak_bytes, self.used_bytes())
        return "admitted" if self._admit_into(slab, req) else "wait"

    def _issue(self, slab: Slab):
        with self.torch.cuda.stream(slab.stream):
            slab.ev0.record(slab.stream)
            mhd.mhd_pool_step(slab.pool, self.k)
            slab.ev1.record(slab.stream)
        slab.busy = True

    def _finish(self, slab: Slab, stats: ServeStats, t0: float, keep: set, stop: bool) -> float:
        """Collect a completed batch of steps; returns the grid-point-steps it advanced."""
        step_ms = slab.ev0.elapsed_time(slab.ev1) / self.k
        bucket = stats.by_size.setdefault(slab.n, {"step_ms": [], "run_s": []})
        stats.step_latency_ms += [step_ms] * len(slab.live)
        bucket["step_ms"] += [step_ms] * len(slab.live)
        steps, _, fin = mhd.mhd_pool_progress(slab.pool)
        advanced = 0.0
        for s in list(slab.live):
            req = slab.live[s]
            done_before = getattr(req, "_counted", 0)
            advanced += float(req.n) ** 3 * (int(steps[s]) - done_before)
            req._counted = int(steps[s])
            if fin[s] or stop:
                out = mhd.mhd_pool_retire(slab.pool, s, copy_out=(req.rid in keep) and fin[s])
                slab.live.pop(s)
                if out is not None:
                    stats.outputs[req.rid] = out
                if fin[s]:
                    t = time.perf_counter() - t0
                    stats.completed += 1
                    stats.work += req.work
                    stats.run_latency_s.append(t - req.arrival)
                    bucket["run_s"].append(t - req.arrival)
                    stats.retired_at[req.rid] = t
        slab.busy = False
        return advanced

    def run(self, requests: list, keep_outputs=(), stop_after_s: float | None = None) -> ServeStats:
        """Serve `requests` in real time (arrival times relative to the start).  Outputs of the
        request ids in `keep_outputs` are returned in stats.outputs.  With `stop_after_s`, no
        request is admitted after that many seconds and the runs in flight are dropped once their
        current steps complete; stats.work then counts the steps actually taken (a closed-loop
        capacity measurement)."""
        keep = set(keep_outputs)
        stats = ServeStats()
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting = collections.deque()
        for r in requests:
            r._counted = 0
        t0 = time.perf_counter()
        steps_work = 0.0
        while True:
            now = time.perf_counter() - t0
            stop = stop_after_s is not None and now >= stop_after_s
            # completed batches: progress, retirements, empty slabs destroyed
            for slab in list(self.slabs):
                if slab.busy and slab.ev1.query():
                    steps_work += self._finish(slab, stats, t0, keep, stop)
                    if not slab.live:
                        slab.close()
                        self.slabs.remove(slab)
            if stop:
                pending.clear()
                waiting.clear()
                if not any(s.busy for s in self.slabs):
                    for slab in list(self.slabs):
                        for s in list(slab.live):
                            mhd.mhd_pool_retire(slab.pool, s, copy_out=False)
                            slab.live.pop(s)
                        slab.close()
                        self.slabs.remove(slab)
                    break
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            # admission in arrival order.  A request whose slab is stepping waits for it while
            # later ones go ahead; a request that no free memory can take stops admission for
            # the round, so that the slabs of smaller runs drain and free the memory it needs
            # (a large run is not starved by a stream of small ones)
            still = collections.deque()
            while waiting:
                req = waiting.popleft()
                outcome = self._place(req, stats)
                if outcome == "admitted":
                    stats.admitted_at[req.rid] = time.perf_counter() - t0
                    stats.queue_s.append(stats.admitted_at[req.rid] - req.arrival)
                    continue
                still.append(req)
                if outcome == "memory":
                    still.extend(waiting)
                    waiting.clear()
            waiting = still
            for slab in self.slabs:
                if not slab.busy and slab.live and not stop:
                    self._issue(slab)
            if not pending and not waiting and not self.slabs:
                break
            if not any(s.busy for s in self.slabs):
                if pending:
                    time.sleep(max(0.0, min(0.002, pending[0].arrival - (time.perf_counter() - t0))))
                elif waiting:
                    raise RuntimeError("a waiting request fits no slab even with the device idle")
            else:
                time.sleep(0.0002)
        stats.wall = time.perf_counter() - t0
        if stop_after_s is not None:
            stats.work = steps_work
        return stats


def run_alone(req: Request, precision: int = mhd.MHD_FP32_MIXED, cache: ICCache | None = None):
    """The same run in a pool of its own (reference for the alone-versus-mix check)."""
    cache = cache or ICCache()
    rho, u, b = cache.get(req)
    pool = mhd.mhd_pool_create(req.n, 1, precision=precision)
    slot = mhd.mhd_pool_admit(pool, (req.nu, req.eta, 1.0 / req.mach), rho, u, b, req.nsteps)
    while True:
        mhd.mhd_pool_step(pool, 50)
        _, _, fin = mhd.mhd_pool_progress(pool)
        if fin[slot]:
            break
    out = mhd.mhd_pool_retire(pool, slot)
    mhd.mhd_pool_destroy(pool)
    return out


def measure_capacity(server: Server, requests: list, duration_s: float = 10.0) -> float:
    """Closed-loop throughput (grid-point-steps/s): every request available at once, admission
    as fast as memory and slabs allow, for `duration_s`; the work counted is the steps the runs
    actually took."""
    closed = [Request(r.rid, 0.0, r.n, r.ic, r.seed, r.nu, r.eta, r.mach, r.nsteps) for r in requests]
    stats = server.run(closed, stop_after_s=duration_s)
    return stats.work / stats.wall
