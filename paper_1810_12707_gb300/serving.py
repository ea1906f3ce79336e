"""Serving many independent MHD runs with continuous batching.

Requests (grid size N, initial condition, nu, eta, Mach, step budget) arrive as a Poisson stream.
Each grid size has one `mhd_pool` (C ABI) whose slots hold device-resident runs; the number of
slots per size is set once from the free device memory and the request mix (admission by free
HBM).  A scheduler round admits every arrived request that has a free slot (H2D of its initial
state), advances every pool by k steps -- pools of different sizes on their own CUDA streams, so
their work overlaps on the device -- and retires the runs that reached their budget (D2H of the
final state).  Runs never interact, so a run's result is bitwise the same alone and in the mix.

Reported: per-step latency (round wall time / k, one sample per live run and round), per-run
latency (retirement time - arrival time), p50 and p99 of both, and aggregate throughput in
grid-point-steps/s.
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


def plan_slots(free_bytes: float, precision: int = mhd.MHD_FP32_MIXED, sizes=SIZES, weights=WEIGHTS,
               fraction: float = 0.8, max_slots: int = 64) -> dict:
    """Slots per grid size, at least one each, total footprint (mhd_footprint_bytes of every pool)
    within `fraction` of the free device memory.  Every live run advances the same k steps per
    scheduler round, so by Little's law the runs of size N in flight are proportional to that
    size's arrival share: slots are given in proportion to the request weights."""
    share = np.array(weights, dtype=np.float64)
    share /= share.sum()
    budget = free_bytes * fraction
    slots = {n: 1 for n in sizes}
    used = sum(mhd.mhd_footprint_bytes(n, precision, 1) for n in sizes)
    # grow the size whose slots are furthest below its work share, while memory lasts
    while True:
        total = sum(slots.values())
        best = None
        for i, n in enumerate(sizes):
            if slots[n] >= max_slots:
                continue
            extra = mhd.mhd_footprint_bytes(n, precision, slots[n] + 1) - mhd.mhd_footprint_bytes(n, precision, slots[n])
            if used + extra > budget:
                continue
            key = (share[i] * (total + 1) - slots[n], n, extra)
            if best is None or key > best:
                best = key
        if best is None:
            return slots
        slots[best[1]] += 1
        used += best[2]


@dataclass
class ServeStats:
    completed: int = 0
    work: float = 0.0
    wall: float = 0.0
    step_latency_ms: list = field(default_factory=list)
    run_latency_s: list = field(default_factory=list)
    queue_s: list = field(default_factory=list)
    outputs: dict = field(default_factory=dict)

    def summary(self) -> dict:
        pct = lambda a, q: float(np.percentile(a, q)) if len(a) else None
        return {"completed": self.completed, "wall_s": self.wall,
                "throughput": self.work / self.wall if self.wall > 0 else 0.0,
                "step_latency_ms_p50": pct(self.step_latency_ms, 50), "step_latency_ms_p99": pct(self.step_latency_ms, 99),
                "run_latency_s_p50": pct(self.run_latency_s, 50), "run_latency_s_p99": pct(self.run_latency_s, 99),
                "queue_s_p50": pct(self.queue_s, 50), "queue_s_p99": pct(self.queue_s, 99)}


class Server:
    def __init__(self, slots: dict, precision: int = mhd.MHD_FP32_MIXED, k: int = 10, cache: ICCache | None = None):
        import torch
        self.torch = torch
        self.k = k
        self.precision = precision
        self.cache = cache or ICCache()
        self.pools, self.streams = {}, {}
        for n, s in slots.items():
            st = torch.cuda.Stream()
            with torch.cuda.stream(st):
                self.pools[n] = mhd.mhd_pool_create(n, s, precision=precision)
            self.streams[n] = st
        self.slots = dict(slots)

    def close(self):
        for p in self.pools.values():
            mhd.mhd_pool_destroy(p)
        self.pools.clear()

    def _admit(self, req: Request) -> int | None:
        rho, u, b = self.cache.get(req)
        pool = self.pools[req.n]
        with self.torch.cuda.stream(self.streams[req.n]):
            return mhd.mhd_pool_admit(pool, (req.nu, req.eta, 1.0 / req.mach), rho, u, b, req.nsteps)

    def run(self, requests: list, keep_outputs=()) -> ServeStats:
        """Serve `requests` in real time (arrival times relative to the start).  Outputs of the
        request ids in `keep_outputs` are returned in stats.outputs."""
        keep = set(keep_outputs)
        stats = ServeStats()
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting = collections.deque()
        live = {n: {} for n in self.pools}  # slot -> request
        admitted_at = {}
        t0 = time.perf_counter()
        while pending or waiting or any(live[n] for n in live):
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            still = collections.deque()
            while waiting:
                req = waiting.popleft()
                slot = self._admit(req) if len(live[req.n]) < self.slots[req.n] else None
                if slot is None:
                    still.append(req)
                else:
                    live[req.n][slot] = req
                    admitted_at[req.rid] = time.perf_counter() - t0
            waiting = still
            if not any(live[n] for n in live):
                if pending:
                    time.sleep(max(0.0, min(0.002, pending[0].arrival - (time.perf_counter() - t0))))
                continue
            tr = time.perf_counter()
            for n, pool in self.pools.items():
                if live[n]:
                    with self.torch.cuda.stream(self.streams[n]):
                        mhd.mhd_pool_step(pool, self.k)
            done = []
            for n, pool in self.pools.items():
                if live[n]:
                    steps, status, fin = mhd.mhd_pool_progress(pool)
                    done += [(n, s) for s in list(live[n]) if fin[s]]
            round_ms = (time.perf_counter() - tr) * 1e3
            nlive = sum(len(live[n]) for n in live)
            stats.step_latency_ms += [round_ms / self.k] * nlive
            for n, s in done:
                req = live[n].pop(s)
                out = mhd.mhd_pool_retire(self.pools[n], s, copy_out=req.rid in keep)
                if out is not None:
                    stats.outputs[req.rid] = out
                t = time.perf_counter() - t0
                stats.completed += 1
                stats.work += req.work
                stats.run_latency_s.append(t - req.arrival)
                stats.queue_s.append(admitted_at[req.rid] - req.arrival)
        stats.wall = time.perf_counter() - t0
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
    """Closed-loop throughput (grid-point-steps/s) with every slot kept busy by requests admitted
    back to back; the work counted is the steps the runs actually took."""
    queue = {n: collections.deque(r for r in requests if r.n == n) for n in server.pools}
    live = {n: {} for n in server.pools}   # slot -> steps already counted
    work, t0 = 0.0, time.perf_counter()
    while time.perf_counter() - t0 < duration_s:
        for n in server.pools:
            while len(live[n]) < server.slots[n] and queue[n]:
                r = queue[n].popleft()
                live[n][server._admit(r)] = 0
                queue[n].append(r)
        for n, pool in server.pools.items():
            if live[n]:
                with server.torch.cuda.stream(server.streams[n]):
                    mhd.mhd_pool_step(pool, server.k)
        for n, pool in server.pools.items():
            if not live[n]:
                continue
            steps, _, fin = mhd.mhd_pool_progress(pool)
            for s in list(live[n]):
                work += float(n) ** 3 * (steps[s] - live[n][s])
                live[n][s] = steps[s]
                if fin[s]:
                    live[n].pop(s)
                    mhd.mhd_pool_retire(pool, s, copy_out=False)
    wall = time.perf_counter() - t0
    for n, pool in server.pools.items():
        for s in list(live[n]):
            mhd.mhd_pool_retire(pool, s, copy_out=False)
    return work / wall
