#!/usr/bin/env python
"""Throughput benchmark of the MHD time step on GB300.

Default workload (`--config tg512`): N = 512^3 Taylor-Green flow u = (sin x cos y cos z,
-cos x sin y cos z, 0) with a seeded random |k| <= 4 magnetic field at <|B|^2>/2 = 1e-3 (seed 2),
Mach 0.3, nu = eta = 1e-3, rho0 = 1, CFL-limited dt, in the FP64-tolerance double-float mode
(MHD_FP64_DF: every value a pair of FP32 numbers, 48-bit significand; parity with the FP64 oracle
to <= 1e-10 after 100 steps).  The same line carries, as extra keys, the same workload in IEEE
FP64 and in the FP32 mixed mode with each mode's relative L2 error per field against IEEE FP64
after 100 steps, the plain cuFFT build at 512^3 FP64, and a short served segment of the serving
configuration (Poisson requests N in {32, 64, 128, 256}) with p50/p99 latencies.  Other
configurations: `abc256` (256^3 ABC dynamo, FP64), `ot32` (Orszag-Tang type, 32^3 FP64, fixed dt
1e-3), `ens64` (64 independent 64^3 Orszag-Tang instances, mixed precision, one batched launch
per kernel, CUDA-graph replay); `--precision` overrides a configuration's mode.

One bench step is one Adams-Bashforth step of every instance through the whole hot path (inverse
transforms, fluxes, forward transforms, spectral assembly, CFL dt, update).  The per-step
working set of the default configuration (about 40 GB moved per step) is far larger than the
129 MB L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config NAME] [--impl ours|reference|cufft]

Prints one JSON line (rank 0).  Under torchrun every rank runs an independent replica (the
instances share nothing), the timed region is bracketed by barriers and the slowest rank's time
is used.  `--impl reference` times the FP64 CPU oracle on the host cores instead (at 512^3 on a
256^3 sample of the same flow: the oracle would hold about 130 GB of host memory at 512^3).
`--serve` runs the full serving configuration (1000 requests at 0.8x and 1.2x capacity).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MHD grid-point-steps/s & HBM GB/s vs peak; served p50/p99 at rel err ≤1e-5"
UNIT = "grid-point-steps/s"
# Paper, Table III: 256^3 on a Tesla V100 at 0.22 s per step (FP64, OpenACC + cuFFT, unified
# memory) -> 256^3 / 0.22 grid-point-steps/s.  Another machine: context for the ratio only.
PAPER_256_V100 = 256 ** 3 / 0.22
# Table III at 512^3: the paper's fastest GPU figure, a P100 at 80.97 s per step (FP64, out-of-core
# unified memory).  Another machine: context only.
PAPER_512_P100 = 512 ** 3 / 80.97


def paper_baseline(n: int):
    return {256: PAPER_256_V100, 512: PAPER_512_P100}.get(n)
FP64_PEAK_TFLOPS = 1.26   # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (nominal 1.25 TFLOP/s)
FP32_PEAK_TFLOPS = 80.5   # 152 SMs x 128 FP32 FMA/clk x 2 flop x 2.07 GHz
FP32_PEAK_TOPS = 40.27    # FP32 lane operations per second: 152 SMs x 128 lanes x 2.07 GHz (x 1e12)
ORACLE_MAX_N = 256        # largest grid the oracle is timed on (about 16 GB of host memory)

CONFIGS = {
    "tg512": dict(n=512, batch=1, precision="fp64df", ic="tg", dt=0.0),
    "abc256": dict(n=256, batch=1, precision="fp64", ic="abc", dt=0.0),
    "ot32": dict(n=32, batch=1, precision="fp64", ic="ot", dt=1e-3),
    "ens64": dict(n=64, batch=64, precision="fp32", ic="ens", dt=0.0),
}
DEFAULT_CONFIG = "tg512"
DTYPES = {"fp64": "f64", "fp64df": "f32x2 double-float (48-bit significand, FP64 tolerance)",
          "fp32": "f32 (double-float state)"}
IC_DESC = {
    "abc": ("abc_dynamo", "ABC A=B=C=1 + seed-1 random B (|k|<=4, E_B=1e-5), Mach 0.1, nu=eta=2e-3"),
    "tg": ("taylor_green", "Taylor-Green + seed-2 random B (|k|<=4, E_B=1e-3), Mach 0.3, nu=eta=1e-3"),
    "ot": ("orszag_tang", "Orszag-Tang type + seed-0 1e-3 perturbation, Mach 0.1, nu=eta=1e-2"),
    "ens": ("ensemble_orszag_tang", "Orszag-Tang type, seeds 1000.., nu,eta log-U[1e-3,1e-2], Mach U[0.05,0.5] (rng 4)"),
}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def workload(n: int, ic: str, batch: int = 1):
    """List of `batch` initial conditions."""
    from paper_1810_12707_gb300 import inputs
    if ic == "tg":
        return [inputs.taylor_green(n, seed=2, b_energy=1e-3, mach=0.3, nu=1e-3, eta=1e-3)] * batch
    if ic == "ot":
        return [inputs.orszag_tang(n, seed=0, mach=0.1, nu=1e-2, eta=1e-2)] * batch
    if ic == "ens":
        nu, eta, mach = inputs.ensemble_params(batch, seed=4)
        return [inputs.orszag_tang(n, seed=1000 + i, mach=float(mach[i]), nu=float(nu[i]), eta=float(eta[i]))
                for i in range(batch)]
    return [inputs.abc_dynamo(n, seed=1, b_energy=1e-5, mach=0.1, nu=2e-3, eta=2e-3)] * batch


# ---------------------------------------------------------------------------------------------
# Algorithmic work per launch of each kernel.  Bytes are the compulsory HBM reads + writes of the
# pass; flops count 5 N log2 N per complex FFT of length N plus the pointwise arithmetic.
# ---------------------------------------------------------------------------------------------
def kernel_model(n: int, batch: int = 1, precision: str = "fp64"):
    k = (n - 1) // 3
    nx, nk = k + 1, 2 * k + 1
    spec = nk * nk * nx
    # complex value of the passes: 16 B in FP64, 8 B in the mixed mode, whose state is a pair of
    # FP32 arrays (hi, lo) and whose history is FP32
    # (the double-float mode moves FP64-sized values: hi + lo FP32 pairs)
    wide = precision in ("fp64", "fp64df")
    c = 16.0 if wide else 8.0
    state_read = 16.0 if wide else 8.0   # the mixed mode's inverse z pass reads hi only
    # assembly per mode: 12 products + state + history read, state + history written
    asm = (12 * 16 + 4 * 7 * 16) if wide else (12 + 7 * 2 + 7 + 7 * 3) * 8
    fft = 5.0 * n * math.log2(n)
    m = {
        "inverse_z": (7 * (spec * state_read + n * nk * nx * c), 7 * nk * nx * fft),
        "inverse_y": (7 * (n * nk * nx + n * n * nx) * c, 7 * n * nx * fft),
        "flux_x": ((7 + 12) * n * n * nx * c, (7 + 12) * (n * n / 2) * fft + 49.0 * n ** 3),
        "step_dt": (8.0 * n * n / 2, 0.0),
        "forward_y": (12 * (n * n * nx + n * nk * nx) * c, 12 * n * nx * fft),
        "forward_z": (12 * (n * nk * nx + spec) * c, 12 * nk * nx * fft),
        "assemble_ab2": (asm * spec, 110.0 * spec),
        # the fused assembly: the assembly's traffic plus the z pass's output (its state read is
        # the assembly's own)
        "assemble_iz": (asm * spec + 7 * n * nk * nx * c, 110.0 * spec + 7 * nk * nx * fft),
    }
    if precision == "fp64df":
        # the double-float kernels are bound by their FP32 arithmetic: "flops" become the FP32
        # lane operations the double-float method performs (dfloat_ops)
        ops = dfloat_ops(n)
        m = {key: (b, ops[key]) for key, (b, f) in m.items()}
    return {key: (b * batch, f * batch) for key, (b, f) in m.items()}


def dfloat_fft_ops(n: int) -> float:
    """FP32 lane operations of one length-n complex transform in double-float: radix-8 stages
    (the first untwiddled) and one radix-4 or radix-2 stage for the remaining factor.  Primitive
    costs: a double-float sum 8 (TwoSum 6, low parts 2), product 4 (TwoProd 2, cross terms 2),
    product with an FP32 number 3, renormalisation 3; a complex sum 16, a complex twiddle product
    32.  Radix-8 DFT: 24 complex sums and the two W8 products (2 sums and 2 products by
    sqrt(2)/2 each) = 432; twiddled radix-8 = 432 + 7 x 32; radix-4 = 8 x 16 + 3 x 32; radix-2 =
    2 x 16 + 32."""
    stages, rem = 0, n
    while rem >= 8:
        rem //= 8
        stages += 1
    ops = (n / 8) * 432.0 + (stages - 1) * (n / 8) * (432.0 + 7 * 32)
    if rem == 4:
        ops += (n / 4) * (8 * 16 + 3 * 32)
    elif rem == 2:
        ops += (n / 2) * (2 * 16 + 32)
    return ops


def dfloat_ops(n: int) -> dict:
    """FP32 lane operations per launch of each double-float kernel (one instance): transforms
    (dfloat_fft_ops) plus the renormalisation of every stored value (3 per real), the packing of
    the x pass (two complex sums per kept mode in, two per mode out), the grid products (about
    286 per grid value: 7 renormalisations, a reciprocal, 3 velocity products, 3 squares, the 12
    products and the CFL speed's squares) and the spectral assembly with the update (about 930 per
    mode)."""
    k = (n - 1) // 3
    nx, nk = k + 1, 2 * k + 1
    spec = nk * nk * nx
    f = dfloat_fft_ops(n)
    store = 6.0  # renormalisation of one complex value
    return {
        "inverse_z": 7 * nk * nx * (f + n * store),
        "inverse_y": 7 * n * nx * (f + n * store),
        "flux_x": (n * n / 2) * (19 * f + 7 * nx * 2 * 16 + 12 * nx * (2 * 16 + 2 * store) + 2 * n * 286.0),
        "step_dt": 0.0,
        "forward_y": 12 * n * nx * (f + nk * store),
        "forward_z": 12 * nk * nx * (f + nk * store),
        "assemble_ab2": 930.0 * spec,
        "assemble_iz": 930.0 * spec + 7 * nk * nx * (f + n * store),
    }


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch, from one ncu capture
# per entry (summarised under profiles/).  A figure stands only while the sources that build the
# kernel are the ones it was taken on: the entry keeps a hash of those files and is dropped
# (traffic reported as null) as soon as they change.
KERNEL_SOURCES = {
    "flux_x": ("kernels_x.cu", "fft_device.cuh"),
    "col": ("kernels_col.cu", "fft_device.cuh"),
}
TRAFFIC = {
    # (kernel, n, batch, precision): (bytes per launch, source hash, capture)
    ("flux_x", 256, 1, "fp64"): (634_281_728 + 1_029_447_000, "8098a458af43095a",
                                 "ncu --set full, profiles/ncu_flux_x_abc256_fp64.md"),
    ("flux_x", 256, 1, "fp32"): (315_693_312 + 489_866_752, "8098a458af43095a",
                                 "ncu --set full, profiles/ncu_abc256_fp32.md"),
    ("flux_x", 256, 1, "fp64df"): (631_424_000 + 1_028_800_512, "76c413daf911ef3f",
                                   "ncu --set full, profiles/ncu_df_kernels_abc256.md"),
    # the 512^3 launch, captured directly with these three metrics (one ncu pass, so nothing is
    # saved or restored around it), profiles/ncu_df_kernels_abc256.md
    ("flux_x", 512, 1, "fp64df"): (5_023_917_824 + 8_550_996_480, "76c413daf911ef3f",
                                   "ncu dram__bytes metrics on one 512^3 launch, profiles/ncu_df_kernels_abc256.md"),
}


def sources_hash(kernel: str) -> str:
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1810_12707_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel: str, n: int, batch: int, precision: str):
    entry = TRAFFIC.get((kernel, n, batch, precision))
    if entry is None:
        return None, "no capture for this kernel and workload"
    nbytes, digest, capture = entry
    if digest != sources_hash("col" if kernel.startswith(("inverse", "forward")) else kernel):
        return None, "kernel sources changed since the capture"
    return nbytes, capture


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        self.proc = None
        self.dev = device_index

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.dev), "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    smax.append(float(p[2]))
                except ValueError:
                    continue
                for name, v in zip(names, p[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The largest value of `x` over all ranks (the slowest rank's time); `x` itself alone."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def oracle_sample_n(n: int) -> int:
    """Grid the oracle is timed on for a workload of size n: n itself up to ORACLE_MAX_N, else a
    ORACLE_MAX_N^3 sample of the same flow (the oracle holds about fifty full n^3 complex arrays,
    some 130 GB of host memory at 512^3)."""
    return min(n, ORACLE_MAX_N)


def time_oracle(cfg, steps: int, budget_s: float = 30.0, warmup: int = 0, warmup_budget_s: float = 60.0):
    """Time the CPU oracle on the same workload (on its oracle_sample_n grid): after set_state and
    `warmup` untimed steps (fewer if they exceed `warmup_budget_s`), up to `steps` AB2 steps of the
    first instance, stopping once `budget_s` has passed.  Returns (grid-point-steps/s, steps timed,
    seconds, threads, warm-up steps done, grid)."""
    from oracle import oracle
    n = oracle_sample_n(cfg["n"])
    ic = workload(n, cfg["ic"], 1)[0]
    o = oracle.Oracle(n, ic.nu, ic.eta, ic.cs, dt=cfg["dt"])
    o.set_state(ic.rho, ic.u, ic.b)
    warm, t0 = 0, time.perf_counter()
    while warm < warmup and time.perf_counter() - t0 < warmup_budget_s:
        o.step(1)
        warm += 1
    done, t0 = 0, time.perf_counter()
    while done < steps:
        o.step(1)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    return n ** 3 * done / el, done, el, oracle.num_threads(), warm, n


def oracle_sample_text(cfg, done, warm, n, el=None):
    txt = f"{done} AB2 steps of one {n}^3 instance after set_state and {warm} untimed steps"
    if el is not None:
        txt += f" ({el:.1f} s)"
    if n != cfg["n"]:
        txt += (f"; a {n}^3 sample of the {cfg['n']}^3 workload (same flow and parameters): the oracle would "
                f"hold about 130 GB of host memory at {cfg['n']}^3")
    return txt


def config_block(name, cfg, world):
    ic_name, desc = IC_DESC[cfg["ic"]]
    n, b = cfg["n"], cfg["batch"]
    return {"workload": f"{name}: {b} x {ic_name} {n}^3 {cfg['precision']}", "n": n, "batch": b,
            "precision": cfg["precision"], "ic": desc, "dt": cfg["dt"] if cfg["dt"] > 0 else "cfl",
            "l2": "per-step working set > L2 (no flush)" if b * n ** 3 >= 128 ** 3 * 8 else "working set may fit L2",
            "parallelism": f"replicas x{world}",
            "baseline": {256: "paper Table III 256^3 V100 0.22 s/step (other hardware, context)",
                         512: "paper Table III 512^3 P100 80.97 s/step, out-of-core unified memory "
                              "(other hardware, context)"}.get(n, "none at this size")}


def run_reference(args, name, cfg):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    n = cfg["n"]
    # each bench step is one oracle step of (the first instance of) the same workload, after the
    # requested untimed warm-up steps; timed steps stop after two minutes of CPU work
    value, done, el, cores, warm, on = time_oracle(cfg, args.steps, budget_s=120.0, warmup=args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": done, "warmup": warm, "ms_per_step": 1e3 * el / done, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": value / PAPER_256_V100 if on == 256 else None, "dtype": "f64",
        "data": "synthetic", "config": config_block(name, cfg, 1),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": oracle_sample_text(cfg, done, warm, on)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, name, cfg):
    import torch

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1810_12707_gb300 import build_lib
    if rank == 0:
        build_lib.build()
    if dist:
        dist.barrier()
    from paper_1810_12707_gb300 import mhd

    n, batch, K, W = cfg["n"], cfg["batch"], args.steps, args.warmup
    prec = {"fp64": mhd.MHD_FP64, "fp64df": mhd.MHD_FP64_DF}.get(cfg["precision"], mhd.MHD_FP32_MIXED)
    ics = workload(n, cfg["ic"], batch)
    phys = [(ic.nu, ic.eta, ic.cs) for ic in ics]
    ctx = mhd.mhd_init(n, phys, dt=cfg["dt"], precision=prec)
    for i, ic in enumerate(ics):
        mhd.mhd_set_state(ctx, i, ic.rho, ic.u, ic.b)
    stream = torch.cuda.current_stream()
    # tile widths of the column FFT passes from the library's autotuner (before any timing)
    tuned = None if args.no_autotune else mhd.mhd_autotune(ctx, reps=3)
    if args.fused_update:
        mhd.mhd_set_option(ctx, mhd.MHD_OPT_FUSED_UPDATE, 1)
    tiles = tuned["tiles"] if tuned else None

    # per-kernel device times from a profiled run (direct launches, events on the library's
    # stream) of K steps, after the warm-up
    mhd.mhd_step(ctx, W)
    if mhd.mhd_synchronize(ctx) != mhd.MHD_OK:
        raise RuntimeError("non-finite state during warm-up")
    mhd.mhd_profile(ctx, True)
    mhd.mhd_step(ctx, K)
    prof = mhd.mhd_profile_read(ctx)
    mhd.mhd_profile(ctx, False)

    # the timed region: K steps as the library runs them (CUDA-graph replay)
    mhd.mhd_step(ctx, 2)
    sampler = ClockSampler(local)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    torch.cuda.nvtx.range_push("timed")  # lets a profiler select exactly the timed launches
    e0.record(stream)
    for _ in range(K):
        mhd.mhd_step(ctx, 1)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    st = mhd.mhd_synchronize(ctx)
    pts = batch * n ** 3
    value = world * pts * K / (ms / 1e3)
    diag = mhd.mhd_diagnostics(ctx, 0)
    mhd.mhd_destroy(ctx)  # the end-to-end context below must fit beside nothing else (1024^3: 150 GB)
    torch.cuda.empty_cache()

    # end to end through the C ABI with pinned host buffers: per step, H2D of every instance's
    # state (rho, u, B), one step, D2H of every instance's state (rho, m, B).  The D2H goes
    # through mhd_get_state_async, so a step's copies out overlap the next step's copies in; the
    # timed region ends with mhd_synchronize, after the last copy has landed.
    E = max(1, min(K, args.e2e_steps))
    pin = lambda shape: torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
    lib = mhd.load_library()
    hs = []
    for ic in ics[: min(batch, 64)]:
        h = (pin((n, n, n)), pin((3, n, n, n)), pin((3, n, n, n)))
        h[0][...] = ic.rho
        h[1][...] = ic.u
        h[2][...] = ic.b
        hs.append(h)
    outs = [(pin((n, n, n)), pin((3, n, n, n)), pin((3, n, n, n))) for _ in range(len(hs))]
    ectx = mhd.mhd_init(n, phys, dt=cfg["dt"], precision=prec)
    if tuned:
        for opt, t in zip((mhd.MHD_OPT_TILE_INV_Z, mhd.MHD_OPT_TILE_INV_Y, mhd.MHD_OPT_TILE_FWD_Y,
                           mhd.MHD_OPT_TILE_FWD_Z), tuned["tiles"]):
            mhd.mhd_set_option(ectx, opt, t)
        if prec == mhd.MHD_FP32_MIXED:
            for opt, r in zip((mhd.MHD_OPT_RADIX_INV_Z, mhd.MHD_OPT_RADIX_INV_Y, mhd.MHD_OPT_RADIX_FWD_Y,
                               mhd.MHD_OPT_RADIX_FWD_Z), tuned["radix"]):
                mhd.mhd_set_option(ectx, opt, r)

    phase = [0.0, 0.0, 0.0]  # host wall time in set_state, step (to completion), get_state_async
    lib_stream = torch.cuda.current_stream()  # the context's stream

    def e2e_step():
        t0 = time.perf_counter()
        for i in range(batch):
            h = hs[i % len(hs)]
            assert lib.mhd_set_state(ectx.handle, i, h[0].ctypes.data, h[1].ctypes.data, h[2].ctypes.data, 0) == 0
        t1 = time.perf_counter()
        assert lib.mhd_step(ectx.handle, 1) == 0
        lib_stream.synchronize()  # the step only (the previous copies out may still run)
        t2 = time.perf_counter()
        for i in range(batch):
            o = outs[i % len(outs)]
            assert lib.mhd_get_state_async(ectx.handle, i, o[0].ctypes.data, o[1].ctypes.data, o[2].ctypes.data) == 0
        t3 = time.perf_counter()
        phase[0] += t1 - t0
        phase[1] += t2 - t1
        phase[2] += t3 - t2

    # the first host transfers of fresh pinned buffers are several times slower (measured 140-780
    # ms for a 512^3 set_state against 41 ms after): three untimed steps
    for _ in range(3):
        e2e_step()
    assert lib.mhd_synchronize(ectx.handle) == 0
    phase[:] = [0.0, 0.0, 0.0]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(E):
        e2e_step()
    t_drain = time.perf_counter()
    assert lib.mhd_synchronize(ectx.handle) == 0  # the last step's copies out have landed
    t_end = time.perf_counter()
    te = max_over_ranks(t_end - t0, dist, "cuda")
    e2e = {"value": world * pts * E / te, "unit": UNIT, "h2d_bytes_per_step": 7 * pts * 8,
           "d2h_bytes_per_step": 7 * pts * 8, "steps": E,
           "phases_ms_per_step": {"set_state": phase[0] / E * 1e3, "step": phase[1] / E * 1e3,
                                  "get_state_async": phase[2] / E * 1e3},
           "final_drain_ms": (t_end - t_drain) * 1e3}
    mhd.mhd_destroy(ectx)

    # roofline of the dominant kernel (largest share of device time)
    hbm, hbm_src = peaks()
    model = kernel_model(n, batch, cfg["precision"])
    alu_peak = {"fp64": FP64_PEAK_TFLOPS, "fp64df": FP32_PEAK_TOPS}.get(cfg["precision"], FP32_PEAK_TFLOPS)
    total_ms = sum(v[0] for v in prof.values())
    per = {}
    for kname, (tot, cnt) in prof.items():
        if cnt:
            b, f = model[kname]
            avg = tot / cnt
            per[kname] = {"avg_ms": avg, "share": tot / max(total_ms, 1e-30),
                          "gbs": b / (avg * 1e-3) / 1e9, "tflops": f / (avg * 1e-3) / 1e12}
    top = max(per, key=lambda k: per[k]["share"])
    # algorithmic bytes of one step: each kernel's bytes times its launches per profiled step
    step_bytes = sum(model[kname][0] * cnt / K for kname, (tot, cnt) in prof.items() if cnt)
    tb, tf = model[top]
    traffic, traffic_src = measured_traffic(top, n, batch, cfg["precision"])
    t_mem = tb / (hbm * 1e9)
    t_alu = tf / (alu_peak * 1e12)
    if t_alu >= t_mem:
        if prec == mhd.MHD_FP64_DF:
            unit, src = ("T FP32-ops/s", "FP32 lanes x clock: 152 SMs x 128 x 2.07 GHz (one operation per lane "
                         "per clock; the algorithmic count is the double-float method's FP32 operations)")
        elif prec == mhd.MHD_FP64:
            unit, src = "TFLOP/s", "FP64 FMA units x clock (nominal 1.25 TFLOP/s; probe 1.19)"
        else:
            unit, src = "TFLOP/s", "FP32 FMA units x clock (probe 74.4 TFLOP/s)"
        roof = {"bound": "alu", "achieved": per[top]["tflops"], "peak": alu_peak, "unit": unit,
                "frac": per[top]["tflops"] / alu_peak, "traffic": traffic, "peak_source": src}
    else:
        roof = {"bound": "hbm", "achieved": per[top]["gbs"], "peak": hbm, "unit": "GB/s",
                "frac": per[top]["gbs"] / hbm, "traffic": traffic, "peak_source": f"{hbm_src} copy"}
    roof.update({"kernel": top, "traffic_source": traffic_src, "algorithmic_bytes": tb, "algorithmic_flops": tf,
                 "achieved_gbs": per[top]["gbs"], "frac_hbm_of_measured": per[top]["gbs"] / hbm,
                 "step_model_bytes": step_bytes,
                 "step_frac_hbm": step_bytes / (ms / K * 1e-3) / 1e9 / hbm})

    extras = {}
    if rank == 0 and world == 1 and not args.no_extras and name == DEFAULT_CONFIG:
        torch.cuda.empty_cache()
        extras = run_extras(args, cfg, ics, tuned)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, done, el, cores, warm, on = time_oracle(cfg, 5, budget_s=30.0, warmup=1)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": oracle_sample_text(cfg, done, warm, on, el)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": value / (world * paper_baseline(n)) if (paper_baseline(n) and batch == 1) else None,
            "dtype": DTYPES[cfg["precision"]], "data": "synthetic",
            "config": dict(config_block(name, cfg, world),
                           col_tiles=tiles if tiles else "library default (autotuner off)",
                           col_radix=tuned["radix"] if tuned else "library default",
                           fused_update=bool(args.fused_update)),
            "roofline": roof,
            "kernels": per,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": (6 if args.fused_update else 7) * K,
            "clocks": clocks,
            "status": mhd.STATUS_NAMES.get(st, st),
            "final": {"t": diag["t"], "dt": diag["dt"], "step": diag["step"], "ke": diag["ke"], "me": diag["me"]},
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def precision_study(cfg, ics, tuned, steps: int = 100, timed: int = 10):
    """The same workload in IEEE FP64, double-float and mixed precision: device time per step
    (`timed` graph-replayed steps after 3 warm-up steps, inside the first `steps`), and each mode's
    relative L2 error per field (rho; m and B as vectors) against IEEE FP64 after `steps` steps,
    computed on the device."""
    import torch
    from paper_1810_12707_gb300 import mhd
    n = cfg["n"]
    ic = ics[0]
    out, ref = {}, None
    for key, prec in (("fp64", mhd.MHD_FP64), ("fp64df", mhd.MHD_FP64_DF), ("fp32_mixed", mhd.MHD_FP32_MIXED)):
        ctx = mhd.mhd_init(n, [(ic.nu, ic.eta, ic.cs)], dt=cfg["dt"], precision=prec)
        mhd.mhd_set_state(ctx, 0, ic.rho, ic.u, ic.b)
        t = mhd.mhd_autotune(ctx, reps=2)
        stream = torch.cuda.current_stream()
        mhd.mhd_step(ctx, 3)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        mhd.mhd_step(ctx, timed)
        e1.record(stream)
        mhd.mhd_step(ctx, steps - 3 - timed)
        if mhd.mhd_synchronize(ctx) != mhd.MHD_OK:
            raise RuntimeError(f"{key}: non-finite state")
        ms = e0.elapsed_time(e1) / timed
        state = mhd.mhd_get_state(ctx, 0, device=True)
        d = mhd.mhd_diagnostics(ctx, 0)
        mhd.mhd_destroy(ctx)
        entry = {"ms_per_step": ms, "value": n ** 3 / (ms * 1e-3), "unit": UNIT, "dtype": DTYPES[
            {"fp64": "fp64", "fp64df": "fp64df", "fp32_mixed": "fp32"}[key]], "col_tiles": t["tiles"],
                 "t_after": d["t"], "steps": steps}
        if ref is None:
            ref = state
        else:
            errs = [float(torch.linalg.vector_norm(g - e) / torch.linalg.vector_norm(e)) for g, e in zip(state, ref)]
            entry[f"rel_l2_vs_fp64_after_{steps}_steps"] = {"rho": errs[0], "m": errs[1], "B": errs[2]}
        out[key] = entry
        del state
        torch.cuda.empty_cache()
    del ref
    torch.cuda.empty_cache()
    return out


def plain_cufft_time(cfg, ic, steps: int = 3, warmup: int = 2, dtype_name: str = "fp64"):
    import torch
    sys.path.insert(0, os.path.join(ROOT, "baseline"))
    from cufft_plain import PlainMHD
    dtype = torch.float64 if dtype_name == "fp64" else torch.float32
    p = PlainMHD(cfg["n"], ic.nu, ic.eta, ic.cs, dt=cfg["dt"], dtype=dtype)
    p.set_state(ic.rho, ic.u, ic.b)
    p.step(warmup)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    p.step(steps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    del p
    torch.cuda.empty_cache()
    return {"ms_per_step": ms, "value": cfg["n"] ** 3 / (ms * 1e-3), "unit": UNIT, "dtype": dtype_name,
            "steps": steps, "note": "full-spectrum cuFFT (torch.fft) per field, unfused elementwise products and update"}


def serve_segment(requests: int, load: float, k: int, capacity_s: float, precision=None, seed: int = 5,
                  alone_check: bool = True):
    """A served segment of the serving configuration: capacity measured closed-loop, then
    `requests` Poisson requests at `load` x capacity; summary with p50/p99 per step and per run,
    overall and per grid size, and the alone-versus-mix check on one request of each size."""
    import torch
    from paper_1810_12707_gb300 import mhd, serving
    precision = mhd.MHD_FP32_MIXED if precision is None else precision
    cache = serving.ICCache()
    probe = serving.make_requests(400, rate=1.0, seed=seed)
    for r in probe:  # every (N, kind, seed) initial state, generated before any timing
        cache.get(r)
    srv = serving.Server(precision=precision, k=k, cache=cache)
    capacity = serving.measure_capacity(srv, probe, duration_s=capacity_s)
    mean_work = float(np.mean([r.work for r in probe]))
    cap_rate = capacity / mean_work
    reqs = serving.make_requests(requests, rate=load * cap_rate, seed=seed + 1)
    keep = []
    for nn in serving.SIZES:
        rid = next((r.rid for r in reqs if r.n == nn), None)
        if rid is not None:
            keep.append(rid)
    stats = srv.run(reqs, keep_outputs=keep if alone_check else [])
    srv.close()
    checked = equal = 0
    if alone_check:
        for rid in keep:
            alone = serving.run_alone(reqs[rid], precision=precision, cache=cache)
            checked += 1
            equal += all(np.array_equal(g, e) for g, e in zip(stats.outputs[rid], alone))
    torch.cuda.empty_cache()
    return dict(stats.summary(), requests=requests, load=load, rate_req_s=load * cap_rate,
                capacity_pts_steps_s=capacity, capacity_req_s=cap_rate, k_steps_per_batch=k,
                alone_vs_mix=f"{equal}/{checked} bitwise equal",
                admission="slabs opened by the device's free memory at arrival, destroyed when empty")


def run_extras(args, cfg, ics, tuned):
    """Extra keys of the default line (outside the timed region): the precision study, the plain
    cuFFT build and a served segment.  A failing extra is reported, not raised."""
    out = {}
    for key, fn in (("precision_study", lambda: precision_study(cfg, ics, tuned)),
                    ("cufft_plain", lambda: plain_cufft_time(cfg, ics[0])),
                    ("serving", lambda: serve_segment(args.serve_segment, 0.8, args.serve_k, 8.0))):
        t0 = time.perf_counter()
        try:
            out[key] = fn()
        except Exception as e:  # reported in the line
            out[key] = {"error": f"{type(e).__name__}: {e}"}
        out[key]["wall_s"] = time.perf_counter() - t0
    ps, cu = out.get("precision_study", {}), out.get("cufft_plain", {})
    if "fp64" in ps and "ms_per_step" in cu:
        out["cufft_plain"]["speedup_of_fp64df"] = cu["ms_per_step"] / ps["fp64df"]["ms_per_step"]
        out["cufft_plain"]["speedup_of_fp64"] = cu["ms_per_step"] / ps["fp64"]["ms_per_step"]
    return out


def run_plain_cufft(args, name, cfg):
    """The same configuration on the plain cuFFT build (baseline/cufft_plain.py), device-timed."""
    import torch
    sys.path.insert(0, os.path.join(ROOT, "baseline"))
    from cufft_plain import PlainMHD
    torch.cuda.set_device(0)
    n, K, W = cfg["n"], args.steps, args.warmup
    ic = workload(n, cfg["ic"], 1)[0]
    dtype = torch.float64 if cfg["precision"] == "fp64" else torch.float32
    p = PlainMHD(n, ic.nu, ic.eta, ic.cs, dt=cfg["dt"], dtype=dtype)
    p.set_state(ic.rho, ic.u, ic.b)
    p.step(W)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    p.step(K)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    value = n ** 3 * K / (ms / 1e3)
    line = {"impl": "cufft_plain", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": K,
            "warmup": W, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": value / paper_baseline(n) if paper_baseline(n) else None,
            "dtype": "f64" if dtype == torch.float64 else "f32", "data": "synthetic",
            "config": config_block(name, cfg, 1),
            "note": "full-spectrum cuFFT (torch.fft) per field, unfused elementwise products and update"}
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    """Serving configuration: Poisson stream of run requests (N in {32,64,128,256} with weights
    .4/.3/.2/.1, ABC or Orszag-Tang, nu, eta ~ U[1e-3,1e-2], Mach ~ U[0.05,0.5], 100-1000 steps,
    mixed precision) served with continuous batching at 0.8x and 1.2x the measured capacity."""
    import torch

    from paper_1810_12707_gb300 import build_lib
    build_lib.build()
    torch.cuda.set_device(0)
    loads = {}
    for load in (0.8, 1.2):
        loads[f"{load}x"] = serve_segment(args.requests, load, args.serve_k, args.capacity_s,
                                          seed=5 if load < 1 else 7, alone_check=load < 1)
    hi = loads["1.2x"]
    line = {
        "metric": METRIC, "value": hi["throughput"], "unit": UNIT, "n_gpus": 1, "steps": args.requests,
        "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPES["fp32"], "data": "synthetic",
        "config": {"workload": f"serve: {args.requests} Poisson requests per load, N in {[32, 64, 128, 256]}",
                   "k_steps_per_batch": args.serve_k, "precision": "fp32",
                   "admission": "slabs opened by free device memory at arrival, destroyed when empty"},
        "serving": loads,
        "note": "value = aggregate grid-point-steps/s at 1.2x capacity; per-step latencies are in serving",
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--config", choices=sorted(CONFIGS), default=DEFAULT_CONFIG)
    ap.add_argument("--n", type=int)
    ap.add_argument("--batch", type=int)
    ap.add_argument("--precision", choices=("fp64", "fp64df", "fp32"))
    ap.add_argument("--ic", choices=("abc", "tg", "ot", "ens"))
    ap.add_argument("--impl", choices=("ours", "reference", "cufft"), default="ours")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the extra keys of the default line")
    ap.add_argument("--serve-segment", type=int, default=200, help="requests of the default line's served segment")
    ap.add_argument("--no-autotune", action="store_true", help="keep the library's default FFT tile widths")
    ap.add_argument("--fused-update", action="store_true",
                    help="AB2 steps with the assembly fused into the next inverse z pass (MHD_OPT_FUSED_UPDATE)")
    ap.add_argument("--serve", action="store_true", help="run the serving configuration instead")
    ap.add_argument("--requests", type=int, default=1000)
    ap.add_argument("--serve-k", type=int, default=20)
    ap.add_argument("--capacity-s", type=float, default=10.0)
    args = ap.parse_args()
    if args.serve:
        return run_serve(args)
    cfg = dict(CONFIGS[args.config])
    for key in ("n", "batch", "precision", "ic"):
        if getattr(args, key) is not None:
            cfg[key] = getattr(args, key)
    name = args.config
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args, name, cfg)
    if args.impl == "cufft":
        return run_plain_cufft(args, name, cfg)
    return run_ours(args, name, cfg)


if __name__ == "__main__":
    sys.exit(main())
