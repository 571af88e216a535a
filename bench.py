#!/usr/bin/env python3
"""Benchmark of the cuSten hot path on GB300 (one JSON line on stdout, rank 0).

Headline workload: the 2D stencil suite on 4096^2 and 8192^2 grids, FP64 and FP32 storage --
xy 9-point Laplacian, 13-point biharmonic, 4th-order d/dx and d/dy, each periodic and
non-periodic, plus the user function c^3 - c - Laplacian(c) -- on sums of 8 random-phase sines
(wavenumbers 1..32) plus 1e-3 uniform noise.  One step = one sweep of every stencil of the
suite (40 sweeps).  `value` = grid points updated per second over the suite (whole job,
all ranks).  The L2 (129 MB) is flushed before every sweep, outside the timed kernel intervals.

Other parts of the metric are measured after the timed steps and reported beside it:
Cahn-Hilliard ADI steps/s (N = 1024, 4096; FP64 and FP32 storage) and the ragged batched-1D
sweep (65536 lines, log-uniform 64..4096, FP32, persistent launch replayed from a CUDA graph),
the coarsening run of Sec. 5.1 (512^2 to t = 100, s(t) and k_1(t) on the device), and
host-resident grids streamed through 256 MiB of device band slots, and the periodic XY WENO
advection term (Sec. 4.2) at 8192^2, and the Cahn-Hilliard step with no-flux boundaries at 4096^2.

--impl reference runs the CPU oracle (the reference arm of this build: a plain FP64 C program)
on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "stencil Gpts/s and HBM GB/s vs ~8 TB/s; CH-ADI steps/s; served p50/p99 vs plain"
WORKLOAD = ("2D stencil suite: nx=ny in {4096, 8192}, FP64 and FP32 storage; xy 9-point "
            "Laplacian, 13-point biharmonic, 4th-order d/dx and d/dy, periodic and non-periodic, "
            "plus user function c^3-c-Lap(c) (periodic and non-periodic); A9 sine fields")
SIZES = (4096, 8192)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# FP64 pipe: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (nominal 1.25 TFLOP/s)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# FP64 instructions (DFMA, DADD, DMUL each one): 152 SMs x 2 per clock x 2.07 GHz
FP64_PEAK_GOPS = 152 * 2 * 2.07
# Instruction issue in lane operations: 152 SMs x 4 schedulers x 32 lanes x 2.07 GHz (also the
# FP32 FMA lane rate)
FP32_LANE_PEAK_TOPS = 152 * 128 * 2.07e9 / 1e12


def dd_ops_per_point(taps: int, name: str) -> int:
    """Integer / FP32 lane operations per output point of the FP64-storage formulation (exact
    integer digits; weights c * small integers): two integer multiply-adds per tap for the two
    digit sums, 13 to cut one input value into its two digits (exponent, significand, one
    shift, the sign as a two's complement, the two digits), 9 to round and assemble the 64-bit
    integer the one FP64 FMA scales.  The cubic user function adds 20: its u^3 - u in
    double-float on packed FP32x2 instructions (32 per pair of outputs), two exact int -> float
    conversions and two integer adds to join Q.  Loads, address arithmetic and control are not
    counted (the executed count is in the ncu summary)."""
    ops = 2 * taps + 13 + 9
    if name == "cubic_minus_lap":
        ops += 20
    return ops


def stencil_suite(h):
    lap9 = np.array([1, 4, 1, 4, -20, 4, 1, 4, 1.0]) / (6 * h * h)
    b = np.zeros((5, 5))
    b[2, 2] = 20
    b[1, 2] = b[3, 2] = b[2, 1] = b[2, 3] = -8
    b[1, 1] = b[1, 3] = b[3, 1] = b[3, 3] = 2
    b[0, 2] = b[4, 2] = b[2, 0] = b[2, 4] = 1
    d1 = np.array([1, -8, 0, 8, -1.0]) / (12 * h)
    return [
        # name, dir, L, R, T, B, weights, fn, coe, nonzero taps
        ("lap9", 2, 1, 1, 1, 1, lap9, 0, None, 9),
        ("biharm13", 2, 2, 2, 2, 2, b.ravel() / h ** 4, 0, None, 13),
        ("ddx4", 0, 2, 2, 0, 0, d1, 0, None, 4),
        ("ddy4", 1, 0, 0, 2, 2, d1, 0, None, 4),
        ("cubic_minus_lap", 2, 1, 1, 1, 1, None, 3, [1.0 / (h * h)], 5),
    ]


class Clocks:
    """nvidia-smi sampling during the timed region (clocks and throttle reasons)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
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
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
            os.unlink(self.path)
        except Exception:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_id(torch, local):
    """nvidia-smi identifier of the GPU this process uses (UUID when torch exposes it)."""
    try:
        u = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [v for v in vis.split(",") if v.strip()]
        return ids[local] if local < len(ids) else str(local)


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, value: float) -> float:
    """Largest value over all ranks (the slowest rank's time); NCCL on CUDA, gloo on CPU."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gpts(world: int, points_per_rank_step: int, ms_per_step: float) -> float:
    """Whole-job throughput: every rank updates its own grids (weak scaling), and the step
    lasts as long as the slowest rank."""
    return world * points_per_rank_step / (ms_per_step * 1e-3) / 1e9


# --------------------------------------------------------------------------------------------
def build_suite(cs, torch, rank, only=None):
    """Resident fields and one plan per (size, dtype, stencil, bc).  `only` = (name, n, dtype,
    bc) restricts the suite to one sweep (used to profile one kernel on its own)."""
    sweeps = []
    keep = []
    sizes = SIZES if only is None else (int(only[1]),)
    for n in sizes:
        h = 2 * np.pi / n
        base = W.sines_field(n, seed=1902 + n + 7 * rank)
        for dtype in (cs.CS_F64, cs.CS_F32):
            if only is not None and only[2] != ("f64" if dtype == cs.CS_F64 else "f32"):
                continue
            tdt = torch.float64 if dtype == cs.CS_F64 else torch.float32
            d_in = torch.from_numpy(base).to("cuda", tdt)
            d_out = torch.zeros_like(d_in)
            keep += [d_in, d_out]
            eb = 8 if dtype == cs.CS_F64 else 4
            for name, d, L, R, T, B, w, fn, coe, taps in stencil_suite(h):
                for bc in (cs.CS_BC_PERIODIC, cs.CS_BC_NONPERIODIC):
                    if only is not None and (only[0] != name or only[3] != ("p" if bc else "np")):
                        continue
                    desc = cs.StencilDesc(nx=n, ny=n, dir=d, bc=bc, dtype=dtype, left=L, right=R, top=T,
                                          bottom=B, weights=w, fn=fn, coe=coe)
                    plan = cs.cs_plan_create_2d(desc, d_in, d_out)
                    sweeps.append(dict(name=name, n=n, dtype="f64" if eb == 8 else "f32", bc="p" if bc else "np",
                                       plan=plan, points=n * n, bytes=2 * eb * n * n, taps=taps,
                                       d_in=d_in, d_out=d_out, eb=eb))
        del base
    # consecutive sweeps never share an input: round-robin over the (size, dtype) grids, so a
    # sweep's input was last touched several hundred MB of traffic ago (plus the flush)
    groups = {}
    for sw in sweeps:
        groups.setdefault((sw["n"], sw["dtype"]), []).append(sw)
    order = []
    lists = list(groups.values())
    for i in range(max(len(g) for g in lists)):
        for g in lists:
            if i < len(g):
                order.append(g[i])
    return order, keep


def flush_l2(buf):
    """Evicts the L2 (129 MB) by reading a 256 MB buffer: a read leaves only clean lines, so the
    next timed kernel does not pay for writing the flush back to HBM."""
    return buf.sum()


def timed_sweeps(cs, torch, sweeps, flush, stream, record):
    """One step: flush L2, then time each sweep with events on the launch stream."""
    evs = []
    for sw in sweeps:
        flush_l2(flush)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cs.cs_compute(sw["plan"], stream)
        e1.record(stream)
        evs.append((sw, e0, e1))
    if record is not None:
        record.append(evs)


def run_ours(args):
    import torch
    import paper_1902_09931_gb300 as cs
    world, rank, local = dist_setup(args)
    cs.load()
    hbm_peak, peak_kind = peaks()
    stream = torch.cuda.current_stream()
    only = tuple(args.only.split(",")) if args.only else None
    cached = bool(args.tune_file) and os.path.exists(args.tune_file)
    if cached:  # the tile choices of an earlier run (plans look the cache up when created)
        cs.cs_tune_load(args.tune_file)
    sweeps, keep = build_suite(cs, torch, rank, only)
    if args.tile_choice >= 0:
        for sw in sweeps:
            cs.cs_plan_set_tile_choice(sw["plan"], args.tile_choice)
    elif not args.no_autotune and not cached:
        for sw in sweeps:  # pick tile shapes with the project's autotuner
            cs.cs_autotune(sw["plan"], stream)
        if args.tune_file and rank == 0:
            cs.cs_tune_save(args.tune_file)
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2
    for _ in range(args.warmup):
        timed_sweeps(cs, torch, sweeps, flush, stream, None)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    clocks = Clocks(gpu_id(torch, local))
    clocks.start()
    launches0 = cs.cs_launch_count()
    record = []
    for _ in range(args.steps):
        timed_sweeps(cs, torch, sweeps, flush, stream, record)
    torch.cuda.synchronize()
    launches = cs.cs_launch_count() - launches0
    clk = clocks.stop()
    barrier(world)
    torch.cuda.synchronize()
    # per-sweep device times
    per = {}
    total_ms = 0.0
    for evs in record:
        for sw, e0, e1 in evs:
            ms = e0.elapsed_time(e1)
            key = f'{sw["name"]}|{sw["n"]}|{sw["dtype"]}|{sw["bc"]}'
            per.setdefault(key, []).append(ms)
            total_ms += ms
    ms_per_step = max_over_ranks(world, total_ms / args.steps)
    pts_per_step = sum(sw["points"] for sw in sweeps)
    bytes_per_step = sum(sw["bytes"] for sw in sweeps)
    value = whole_job_gpts(world, pts_per_step, ms_per_step)
    hbm_gbs = world * bytes_per_step / (ms_per_step * 1e-3) / 1e9

    # dominant kernel: largest share of the step.  Its roofline is the method's algorithmic work:
    # one read and one write of every grid point (2 s bytes, s the element size), against the
    # measured HBM copy rate; halo re-reads and the arithmetic formulation are not algorithmic.
    shares = {k: statistics.mean(v) for k, v in per.items()}
    dom_key = max(shares, key=shares.get)
    dom = [sw for sw in sweeps if f'{sw["name"]}|{sw["n"]}|{sw["dtype"]}|{sw["bc"]}' == dom_key][0]
    dom_ms = shares[dom_key]
    achieved = dom["bytes"] / (dom_ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
            "frac": round(achieved / hbm_peak, 4), "peak_kind": peak_kind, "kernel": dom_key,
            "bytes_per_launch": dom["bytes"], "launch_ms": round(dom_ms, 4),
            "traffic": traffic_for(dom_key)}
    if dom["eb"] == 8:
        # FP64 storage is evaluated on the integer / FP32 pipes (exact digits): the formulation's
        # own lane-operation count, against the instruction-issue peak in lane operations
        ops = dd_ops_per_point(dom["taps"], dom["name"]) * dom["points"]
        lane = ops / (dom_ms * 1e-3) / 1e12
        roof["formulation"] = {"ops_per_point": dd_ops_per_point(dom["taps"], dom["name"]),
                               "achieved_tops": round(lane, 3), "peak_tops": round(FP32_LANE_PEAK_TOPS, 3),
                               "frac": round(lane / FP32_LANE_PEAK_TOPS, 4),
                               "peak_kind": "derived: instruction issue, 152 SM x 4 schedulers x 32 lanes x 2.07 GHz"}

    # every sweep against the HBM roofline
    f32 = {}
    for k, v in shares.items():
        name, n, dt, bc = k.split("|")
        sw = [s for s in sweeps if s["name"] == name and s["n"] == int(n) and s["dtype"] == dt and s["bc"] == bc][0]
        gbs = sw["bytes"] / (v * 1e-3) / 1e9
        f32[k] = {"ms": round(v, 4), "gpts": round(sw["points"] / (v * 1e-3) / 1e9, 2),
                  "hbm_gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm_peak, 3),
                  "tile_choice": cs.cs_plan_get_tile_choice(sw["plan"])}

    by_dtype = {}
    for dt in ("f64", "f32"):
        sel = [(k, v) for k, v in shares.items() if k.split("|")[2] == dt]
        if not sel:
            continue
        ms_dt = sum(v for _, v in sel)
        pts_dt = sum(sw["points"] for sw in sweeps if sw["dtype"] == dt)
        bytes_dt = sum(sw["bytes"] for sw in sweeps if sw["dtype"] == dt)
        by_dtype[dt] = {"gpts": round(world * pts_dt / (ms_dt * 1e-3) / 1e9, 2), "ms_per_step": round(ms_dt, 4),
                        "hbm_gbs": round(world * bytes_dt / (ms_dt * 1e-3) / 1e9, 1),
                        "hbm_frac": round(bytes_dt / (ms_dt * 1e-3) / 1e9 / hbm_peak, 4)}
    e2e = e2e_host(cs, torch, sweeps, stream, max(1, min(args.steps, 3)), world)
    parts = {}
    if not args.skip_parts:
        parts["single_call"] = bench_single_call(cs, torch, stream)
        parts["group"] = bench_group(cs, torch, stream)
        parts["ch_adi"] = bench_ch(cs, torch, stream)
        parts["ch_runs"] = bench_ch_runs(cs, torch, stream)
        parts["batch1d"] = bench_batch1d(cs, torch, stream, hbm_peak)
        parts["serve"] = bench_serve(cs, torch)
        parts["coarsening"] = bench_coarsening(cs, torch, stream)
        parts["streamed"] = bench_streamed(cs, torch, stream)
        parts["weno"] = bench_weno(cs, torch, stream, hbm_peak)
        parts["ch_noflux"] = bench_ch(cs, torch, stream, [(4096, cs.CS_F64, 30, cs.CS_CH_NOFLUX),
                                                          (4096, cs.CS_F32, 30, cs.CS_CH_NOFLUX)])
    for sw in sweeps:
        cs.cs_destroy(sw["plan"])
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "Gpts/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sweeps_per_step": len(sweeps), "points_per_step": pts_per_step,
                   "l2": "evicted before every sweep by reading a 256 MB buffer (2x L2), outside the timed intervals",
                   "parallelism": f"replicas x{world} (independent grids per GPU)"},
        "hbm_gbs": round(hbm_gbs, 1), "hbm_frac_of_measured": round(hbm_gbs / hbm_peak, 4),
        "hbm_frac_of_8tbs": round(hbm_gbs / 8000.0, 4),
        "gpts_f64": by_dtype.get("f64", {}).get("gpts"), "gpts_f32": by_dtype.get("f32", {}).get("gpts"),
        "hbm_frac_f64": by_dtype.get("f64", {}).get("hbm_frac"), "hbm_frac_f32": by_dtype.get("f32", {}).get("hbm_frac"),
        "by_dtype": by_dtype,
        "roofline": roof, "clocks": clk, "gpu_launches": launches, "e2e": e2e,
        "per_sweep": f32, "parts": parts,
    }
    if rank == 0 and not args.skip_cpu:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
        if not args.skip_parts:
            line["cpu_baseline"]["rows"] = cpu_rows()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def traffic_for(key):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on this kernel."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        for line in open(path):
            if line.startswith("#") or not line.strip():
                continue
            k, b = line.split()[:2]
            if k == key:
                return int(float(b))
    except OSError:
        pass
    return None


def e2e_host(cs, torch, sweeps, stream, steps, world):
    """The suite through cs_compute_host: pinned host input copied in and output copied back
    every sweep, timed end to end."""
    host = {}
    for sw in sweeps:
        key = (sw["n"], sw["dtype"])
        if key not in host:
            host[key] = (sw["d_in"].cpu().pin_memory(), torch.empty(sw["d_out"].shape, dtype=sw["d_out"].dtype).pin_memory())
    for sw in sweeps:  # untimed: each plan creates its copy streams and events on first use
        h_in, h_out = host[(sw["n"], sw["dtype"])]
        cs.cs_compute_host(sw["plan"], h_in, h_out, stream)
    torch.cuda.synchronize()
    # each step timed on its own (wall clock; cs_compute_host synchronises), the median step
    # reported: a single host-side stall in one step of a few would otherwise set the figure
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        for sw in sweeps:
            h_in, h_out = host[(sw["n"], sw["dtype"])]
            cs.cs_compute_host(sw["plan"], h_in, h_out, stream)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    dt = max_over_ranks(world, statistics.median(times))
    pts = sum(sw["points"] for sw in sweeps)
    nbytes = sum(sw["points"] * sw["eb"] for sw in sweeps)
    return {"value": round(world * pts / dt / 1e9, 3), "unit": "Gpts/s",
            "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "steps": steps,
            "step_s": [round(t, 4) for t in times]}


def bench_ch(cs, torch, stream, cases=None, autotune=True):
    out = {}
    if cases is None:
        cases = [(1024, cs.CS_F64, 200), (4096, cs.CS_F64, 30), (1024, cs.CS_F32, 200), (4096, cs.CS_F32, 30)]
    for case in cases:
        n, storage, steps = case[:3]
        boundary = case[3] if len(case) > 3 else cs.CS_CH_PERIODIC
        h = 2 * np.pi / n
        tdt = torch.float64 if storage == cs.CS_F64 else torch.float32
        c0 = torch.from_numpy(W.ch_initial(n, seed=5)).to("cuda", tdt)
        f = [c0.clone(), c0.clone(), torch.zeros_like(c0)]
        plan = cs.cs_ch_create(cs.CHDesc(n=n, storage=storage, D=1.0, gamma=0.01, dt=0.1 * h,
                                         boundary=boundary), *f)
        if autotune:
            cs.cs_autotune(plan, stream)  # chunks per line of the partitioned line solves
        cs.cs_ch_step(plan, 5, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cs.cs_ch_step(plan, steps, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        chunks, m = cs.cs_ch_config(plan)
        cs.cs_destroy(plan)
        key = f"n{n}_{'f64' if storage == cs.CS_F64 else 'f32'}" + ("_noflux" if boundary == cs.CS_CH_NOFLUX else "")
        fp64_ops = ch_fp64_ops_per_point(chunks, m, storage == cs.CS_F32) * n * n
        out[key] = {"ms_per_step": round(ms, 4), "steps_per_s": round(1e3 / ms, 1),
                    "fp64_gops": round(fp64_ops / (ms * 1e-3) / 1e9, 1),
                    "fp64_frac": round(fp64_ops / (ms * 1e-3) / 1e9 / FP64_PEAK_GOPS, 3),
                    "chunks_per_line": chunks}
    return out


def bench_single_call(cs, torch, stream, n=256, calls=2000):
    """One compute call on a 256^2 periodic grid, FP64, 5-point Laplacian, h = 2 pi / 256, input
    U[-1, 1]: microseconds per call launched directly and replayed from a CUDA graph, each the
    mean of `calls` back-to-back calls between two CUDA events (the 1 MiB grid stays in L2, so
    this measures launch and latency, not HBM)."""
    h = 2 * np.pi / n
    x = torch.from_numpy(W.uniform_field(n, n, seed=256)).to("cuda", torch.float64)
    y = torch.zeros_like(x)
    w = np.array([0, 1, 0, 1, -4, 1, 0, 1, 0.0]) / h ** 2
    desc = cs.StencilDesc(nx=n, ny=n, dir=cs.CS_DIR_XY, bc=cs.CS_BC_PERIODIC, dtype=cs.CS_F64,
                          left=1, right=1, top=1, bottom=1, weights=w)
    plan = cs.cs_plan_create_2d(desc, x, y)
    cs.cs_autotune(plan, stream)
    out = {"n": n, "stencil": "5-point Laplacian, FP64, periodic", "calls": calls,
           "tile_choice": cs.cs_plan_get_tile_choice(plan)}
    for mode in ("plain", "graph"):
        cs.cs_plan_use_graph(plan, mode == "graph")
        for _ in range(20):
            cs.cs_compute(plan, stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(calls):
            cs.cs_compute(plan, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / calls
        out[mode] = {"us_per_call": round(us, 3), "gpts_per_s": round(n * n / (us * 1e-6) / 1e9, 2)}
    cs.cs_destroy(plan)
    return out


def bench_ch_runs(cs, torch, stream, steps=1000):
    """The 1000-step Cahn-Hilliard runs of the configuration (n = 1024, 4096; FP64 and FP32
    storage; deep quench C0 ~ U[-0.1, 0.1] with the mean removed, D = 1, gamma = 0.01,
    dt = 0.1 h) with the mass and free energy read back after every step: steps/s with the
    per-step invariants, the largest mass drift (of h^2 sum |C0|), and the energy's behaviour
    (steps where it rose, the first one, the largest rise), reported as they come."""
    out = {}
    for n in (1024, 4096):
        h = 2 * np.pi / n
        for storage in (cs.CS_F64, cs.CS_F32):
            tdt = torch.float64 if storage == cs.CS_F64 else torch.float32
            c0 = torch.from_numpy(W.ch_initial(n, seed=1902)).to("cuda", tdt)
            f = [c0.clone(), c0.clone(), torch.zeros_like(c0)]
            plan = cs.cs_ch_create(cs.CHDesc(n=n, storage=storage, D=1.0, gamma=0.01, dt=0.1 * h), *f)
            cs.cs_autotune(plan, stream)
            m0, e0 = cs.cs_ch_invariants(plan, stream)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            mass, energy = cs.cs_ch_step(plan, steps, invariants=True, stream=stream)
            dt_s = time.perf_counter() - t0
            cs.cs_destroy(plan)
            scale = h * h * float(c0.double().abs().sum().item())
            e = np.concatenate([[e0], energy])
            de = np.diff(e)
            key = f"n{n}_{'f64' if storage == cs.CS_F64 else 'f32'}"
            out[key] = {"steps": steps, "steps_per_s_with_invariants": round(steps / dt_s, 1),
                        "mass_drift_max": float(f"{np.abs(mass - m0).max() / scale:.3e}"),
                        "energy_start": round(float(e0), 6), "energy_end": round(float(e[-1]), 6),
                        "energy_rises": int((de > 0).sum()),
                        "first_rise_step": int(np.argmax(de > 0)) + 1 if (de > 0).any() else None,
                        "largest_rise_rel": float(f"{(de / np.abs(e[:-1])).max():.3e}")}
            del c0, f
    return out


def bench_group(cs, torch, stream, reps=50):
    """Small 2D grids in one persistent launch against one launch per grid: 64 grids drawn from
    {32, 64, 128, 256, 512}^2 (seeded), periodic xy 9-point Laplacian, FP32 and FP64 storage.
    Arms: a plain cs_compute per grid, each grid's own CUDA graph, one grouped launch
    (cs_compute_group), and that grouped launch captured in a CUDA graph.  Time per batch of
    all 64 sweeps: mean over `reps` back-to-back batches between CUDA events (the grids, 83 MB
    in FP64, sit in L2: this is the launch- and latency-bound regime that batching targets)."""
    rng = np.random.Generator(np.random.PCG64(64))
    ns = [int(v) for v in rng.choice([32, 64, 128, 256, 512], size=64)]
    pts = sum(n * n for n in ns)
    out = {"grids": len(ns), "sizes": "n in {32, 64, 128, 256, 512}", "points": pts}
    for dtype in (cs.CS_F32, cs.CS_F64):
        tdt = torch.float64 if dtype == cs.CS_F64 else torch.float32
        plans, keep = [], []
        for k, n in enumerate(ns):
            h = 2 * np.pi / n
            x = torch.from_numpy(W.sines_field(n, seed=900 + k)).to("cuda", tdt)
            y = torch.zeros_like(x)
            keep += [x, y]
            w = np.array([1, 4, 1, 4, -20, 4, 1, 4, 1.0]) / (6 * h * h)
            desc = cs.StencilDesc(nx=n, ny=n, dir=cs.CS_DIR_XY, bc=cs.CS_BC_PERIODIC, dtype=dtype,
                                  left=1, right=1, top=1, bottom=1, weights=w)
            p = cs.cs_plan_create_2d(desc, x, y)
            cs.cs_plan_set_tile_choice(p, 1)
            plans.append(p)

        def timed(fn):
            for _ in range(5):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) * 1e3 / reps

        def per_call():
            for p in plans:
                cs.cs_compute(p, stream)

        res = {"per_call_us": timed(per_call)}
        for p in plans:
            cs.cs_plan_use_graph(p, True)
        res["per_call_graph_us"] = timed(per_call)
        for p in plans:
            cs.cs_plan_use_graph(p, False)
        res["grouped_us"] = timed(lambda: cs.cs_compute_group(plans, stream))
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            cs.cs_compute_group(plans, torch.cuda.current_stream())
        torch.cuda.synchronize()
        res["grouped_graph_us"] = timed(g.replay)
        del g
        for p in plans:
            cs.cs_destroy(p)
        res = {k: round(v, 2) for k, v in res.items()}
        res["grouped_graph_gpts"] = round(pts / (res["grouped_graph_us"] * 1e-6) / 1e9, 2)
        res["speedup_vs_per_call"] = round(res["per_call_us"] / res["grouped_graph_us"], 2)
        out["f64" if dtype == cs.CS_F64 else "f32"] = res
    return out


def bench_streamed(cs, torch, stream, budget_mib=256, reps=5):
    """Host-resident (out-of-core) plans: the grid in pinned host memory streams through a
    256 MiB ring of device band slots.  Time per sweep (wall clock around cs_compute_host,
    which synchronises), grid points per second and host-link bytes per second (copy in plus
    copy out) for a periodic 9-point Laplacian; 8192^2 FP64 and 16384^2 FP32 (1 GiB grids)."""
    out = {}
    for n, dtype in ((8192, cs.CS_F64), (16384, cs.CS_F32)):
        h = 2 * np.pi / n
        tdt = torch.float64 if dtype == cs.CS_F64 else torch.float32
        eb = 8 if dtype == cs.CS_F64 else 4
        w = np.array([1, 4, 1, 4, -20, 4, 1, 4, 1.0]) / (6 * h * h)
        desc = cs.StencilDesc(nx=n, ny=n, dir=cs.CS_DIR_XY, bc=cs.CS_BC_PERIODIC, dtype=dtype,
                              left=1, right=1, top=1, bottom=1, weights=w)
        plan = cs.cs_plan_create_2d_host(desc, budget_mib << 20)
        rows, held = cs.cs_plan_host_info(plan)
        h_in = torch.from_numpy(W.sines_field(n, seed=61)).to(tdt).pin_memory()
        h_out = torch.empty(n, n, dtype=tdt).pin_memory()
        cs.cs_compute_host(plan, h_in, h_out, stream)  # warm-up: streams and events
        times = []
        for _ in range(reps):
            t0 = time.perf_counter()
            cs.cs_compute_host(plan, h_in, h_out, stream)
            times.append(time.perf_counter() - t0)
        cs.cs_destroy(plan)
        t = statistics.median(times)
        key = f"n{n}_{'f64' if dtype == cs.CS_F64 else 'f32'}"
        out[key] = {"ms": round(t * 1e3, 3), "gpts_per_s": round(n * n / t / 1e9, 2),
                    "link_gbs": round(2 * n * n * eb / t / 1e9, 1), "band_rows": rows,
                    "bands": -(-n // rows), "device_mib": round(held / 2 ** 20, 1)}
        del h_in, h_out
    return out


def bench_weno(cs, torch, stream, hbm_peak, reps=20):
    """Periodic XY WENO advection (Sec. 4.2) at 8192^2, FP64 and FP32: one launch per sweep on
    inputs larger than L2 (three 512 MB / 256 MB fields), timed with CUDA events; HBM bytes per
    point = C, u, v read + the term written."""
    out = {}
    n = 8192
    h = 2 * np.pi / n
    x = torch.arange(n, dtype=torch.float64, device="cuda") * h
    for dtype in (cs.CS_F64, cs.CS_F32):
        tdt = torch.float64 if dtype == cs.CS_F64 else torch.float32
        eb = 8 if dtype == cs.CS_F64 else 4
        c = (torch.sin(3 * x)[None, :] * torch.cos(5 * x)[:, None]).to(tdt)
        u = (torch.cos(x)[:, None] + 0.0 * x[None, :]).to(tdt)
        v = (torch.sin(x)[None, :] - 0.2 + 0.0 * x[:, None]).to(tdt)
        o = torch.empty_like(c)
        plan = cs.cs_plan_create_weno_adv(n, n, dtype, h, h, c, u, v, o)
        for _ in range(3):
            cs.cs_compute(plan, stream)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        ev[0].record(stream)
        for _ in range(reps):
            cs.cs_compute(plan, stream)
        ev[1].record(stream)
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1]) / reps
        cs.cs_destroy(plan)
        gbs = 4 * eb * n * n / (ms * 1e-3) / 1e9
        out["f64" if dtype == cs.CS_F64 else "f32"] = {
            "ms": round(ms, 4), "gpts_per_s": round(n * n / (ms * 1e-3) / 1e9, 2),
            "hbm_gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm_peak, 3)}
        del c, u, v, o
    return out


def bench_coarsening(cs, torch, stream, n=512, T=100.0, samples=25, window=(2.0, 30.0)):
    """The long run of Sec. 5.1: deep quench (U[-0.1, 0.1]) on 512^2, dt = 0.1 dx, D = 1,
    gamma = 0.01, to t = T, FP64 storage.  s(t) and k_1(t) are measured on the device at
    log-spaced times; the exponents of s and 1 / k_1 are least-squares slopes in log-log over
    the window (t^(1/3) is the expected law; finite-size effects bend it late in the run)."""
    h = 2 * np.pi / n
    dt = 0.1 * h
    total = int(round(T / dt))
    c0 = torch.from_numpy(W.ch_initial(n, seed=2019)).to("cuda", torch.float64)
    f = [c0.clone(), c0.clone(), torch.zeros_like(c0)]
    plan = cs.cs_ch_create(cs.CHDesc(n=n, storage=cs.CS_F64, D=1.0, gamma=0.01, dt=dt), *f)
    cs.cs_autotune(plan, stream)
    torch.cuda.synchronize()
    marks = sorted(set(int(round(v)) for v in np.geomspace(0.25 / dt, total, samples)))
    ev = lambda: torch.cuda.Event(enable_timing=True)
    step_ms = diag_ms = 0.0
    series, done = [], 0
    for m in marks:
        e0, e1, e2 = ev(), ev(), ev()
        e0.record(stream)
        cs.cs_ch_step(plan, m - done, stream=stream)
        e1.record(stream)
        s, k1 = cs.cs_ch_coarsening(plan, stream)
        e2.record(stream)
        torch.cuda.synchronize()
        step_ms += e0.elapsed_time(e1)
        diag_ms += e1.elapsed_time(e2)
        done = m
        series.append((m * dt, s, k1))
    cs.cs_destroy(plan)
    t = np.array([v[0] for v in series])
    sel = (t >= window[0]) & (t <= window[1])
    slope = lambda y: float(np.polyfit(np.log(t[sel]), np.log(y[sel]), 1)[0])
    s_arr = np.array([v[1] for v in series])
    inv_k1 = 1.0 / np.array([v[2] for v in series])
    return {"n": n, "T": T, "dt": dt, "steps": total, "steps_per_s": round(total / (step_ms * 1e-3), 1),
            "run_s": round(step_ms * 1e-3, 3), "diag_ms": round(diag_ms / len(series), 3),
            "fit_window": list(window), "s_exponent": round(slope(s_arr), 3),
            "inv_k1_exponent": round(slope(inv_k1), 3),
            "series": [[round(a, 4), round(b, 6), round(c, 5)] for a, b, c in series]}


def bench_serve(cs, torch, factors=(0.5, 0.9, 1.5), count=120, seed=2026):
    """Poisson stream of mixed jobs (2D sweeps and 10-step FP32 Cahn-Hilliard advances, grids
    128^2..4096^2), continuous batching vs sequential plain calls at arrival rates that are
    fractions of the sequential capacity (1 / mean service time, measured back to back)."""
    from paper_1902_09931_gb300 import serving as S
    be = S.GpuBackend(cs, torch, streams=8, keep_outputs=False)
    be.warmup(S.SIZES, copies=3)
    calib = S.poisson_jobs(count, rate=0.0, seed=seed)  # all at t = 0: back to back
    S.run_sequential(be, calib[:20])  # warm-up
    seq0 = S.run_sequential(be, calib)
    capacity = seq0["jobs"] / seq0["span_s"]
    out = {"capacity_jobs_per_s": round(capacity, 1), "jobs_per_run": count,
           "mix": "50% sweeps (lap9/biharm13/ddx4/ddy4), 50% 10-step CH advances, FP32, n in 128..4096"}
    for f in factors:
        rate = f * capacity
        a = S.poisson_jobs(count, rate=rate, seed=seed + 1)
        b = S.poisson_jobs(count, rate=rate, seed=seed + 1)
        srv = S.Server(be, max_inflight=12).run(a)
        seq = S.run_sequential(be, b)
        keep = ("p50_ms", "p99_ms", "jobs_per_s", "gpts_per_s")
        out[f"load_{f}"] = {"server": {k: round(srv[k], 3) for k in keep} | {"launches": srv["launches"]},
                            "sequential": {k: round(seq[k], 3) for k in keep}}
    return out


def ch_fp64_ops_per_point(chunks: int, m: int, fp32_storage: bool = False) -> float:
    """FP64-pipe operations per grid point of one ADI step as the kernels perform them (ncu's
    DFMA + DADD + DMUL counts of the 4096^2 FP64 step: 5.45 + 5 + 5 + 5 + 6 = 26.4 at 16 chunks
    of 256).  The right-hand side, per CTA of 64 x 32 points: Cbar = 2 C^n - C^{n-1} on the 68 x 36
    halo-2 tile (one FMA; FP32 storage forms it in FP32), Z's one digit-combination FMA on the
    66 x 34 halo-1 tile (the cubic term joins the integer digit sum), then per point the second
    combination, C^n - C^{n-1} and the final FMA, and one multiply per thread for the combination's
    constant.  Each sweep: local LU 4 FMAs and 1 multiply, the spike correction 4 FMAs and the
    chunk-end system 16 chunks / m.  The update: one add (Cbar comes from the right-hand side kernel
    through the C^{n+1} buffer; FP32 storage narrows on the integer pipe)."""
    tile = 64 * 32
    rhs = (0 if fp32_storage else 68 * 36 / tile) + 66 * 34 / tile + 3 + 256 / tile
    per_sweep = 5 + 4 + 16.0 * chunks / m
    return rhs + 2 * per_sweep + 1


def _median_event_ms(torch, stream, launch, flush, reps=12, skip=2):
    times = []
    for _ in range(reps):
        flush_l2(flush)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        launch()
        e1.record(stream)
        times.append((e0, e1))
    torch.cuda.synchronize()
    return statistics.median([a.elapsed_time(b) for a, b in times[skip:]])


def bench_batch1d(cs, torch, stream, hbm_peak):
    """The ragged batch (65,536 lines, lengths log-uniform in 64..4096, 4th-order second
    derivative, periodic per line), L2 evicted before every launch, CUDA events:
      * persistent: FP32 storage, one persistent launch replayed from a CUDA graph, launch shape
        from the autotuner (the configuration's form);
      * fp64_plain: the same lines in FP64 storage, one plain launch per call, default shape;
      * per_length_class: FP32, one plain launch per length class [2^k, 2^(k+1)) over that
        class's lines packed contiguously (7 launches; the naive batching baseline)."""
    off = W.ragged_offsets(65536, seed=2019)
    x64 = W.sines_lines(off, seed=2020)
    x = x64.astype(np.float32)
    d_off = torch.from_numpy(off).cuda()
    w = np.array([-1, 16, -30, 16, -1.0]) / 12.0
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    total = int(off[-1])
    nbytes32 = 8 * total + 8 * off.size
    out = {"lines": off.size - 1, "points": total}

    def arm(ms, eb):
        nb = 2 * eb * total + 8 * off.size
        return {"ms": round(ms, 4), "gpts_per_s": round(total / (ms * 1e-3) / 1e9, 2),
                "hbm_gbs": round(nb / (ms * 1e-3) / 1e9, 1), "hbm_frac": round(nb / (ms * 1e-3) / 1e9 / hbm_peak, 3)}

    d_in = torch.from_numpy(x).cuda()
    d_out = torch.zeros_like(d_in)
    desc = cs.StencilDesc(dir=cs.CS_DIR_X, bc=cs.CS_BC_PERIODIC, dtype=cs.CS_F32, left=2, right=2, weights=w)
    plan = cs.cs_plan_create_1d_batch(desc, off.size - 1, d_off, total, d_in, d_out)
    cs.cs_autotune(plan, stream)
    cs.cs_plan_use_graph(plan, True)
    ms = _median_event_ms(torch, stream, lambda: cs.cs_compute(plan, stream), flush)
    cs.cs_destroy(plan)
    out.update({"ms": round(ms, 4), "gpts_per_s": round(total / (ms * 1e-3) / 1e9, 2),
                "hbm_gbs": round(nbytes32 / (ms * 1e-3) / 1e9, 1),
                "hbm_frac": round(nbytes32 / (ms * 1e-3) / 1e9 / hbm_peak, 3)})
    out["persistent"] = arm(ms, 4)

    d_in64 = torch.from_numpy(x64).cuda()
    d_out64 = torch.zeros_like(d_in64)
    desc64 = cs.StencilDesc(dir=cs.CS_DIR_X, bc=cs.CS_BC_PERIODIC, dtype=cs.CS_F64, left=2, right=2, weights=w)
    plan64 = cs.cs_plan_create_1d_batch(desc64, off.size - 1, d_off, total, d_in64, d_out64)
    ms64 = _median_event_ms(torch, stream, lambda: cs.cs_compute(plan64, stream), flush)
    cs.cs_destroy(plan64)
    out["fp64_plain"] = arm(ms64, 8)
    del d_in64, d_out64

    lens = np.diff(off)
    cls = np.floor(np.log2(lens)).astype(int)
    plans, keep = [], []
    for k in sorted(set(cls.tolist())):
        sel = np.nonzero(cls == k)[0]
        o = np.concatenate([[0], np.cumsum(lens[sel])]).astype(np.int64)
        xs = np.concatenate([x[off[m]:off[m + 1]] for m in sel])
        ci, co, cof = torch.from_numpy(xs).cuda(), torch.zeros(xs.size, dtype=torch.float32, device="cuda"), \
            torch.from_numpy(o).cuda()
        keep += [ci, co, cof]
        plans.append(cs.cs_plan_create_1d_batch(desc, sel.size, cof, int(o[-1]), ci, co))

    def per_class():
        for p in plans:
            cs.cs_compute(p, stream)

    msc = _median_event_ms(torch, stream, per_class, flush)
    for p in plans:
        cs.cs_destroy(p)
    out["per_length_class"] = arm(msc, 4) | {"launches": len(plans)}
    return out


# --------------------------------------------------------------------------------------------
def cpu_sample(seconds: float):
    """The oracle (single-threaded C) on row bands of the suite's grids: the same stencils,
    periodic and non-periodic, FP64 arithmetic.  Returns (points, seconds, description)."""
    import oracle
    oracle.build()
    rows = 16
    pts = 0
    t_total = 0.0
    done = 0
    deadline = time.perf_counter() + seconds
    while time.perf_counter() < deadline:
        for n in SIZES:
            h = 2 * np.pi / n
            band = W.sines_field(n, seed=1902 + n, ny=rows)
            for name, d, L, R, T, B, w, fn, coe, taps in stencil_suite(h):
                for bc in (1, 0):
                    t0 = time.perf_counter()
                    if fn:
                        oracle.stencil2d_fn(band, fn, coe, bc)
                    else:
                        oracle.stencil2d(band, w, d, bc, L, R, T, B)
                    t_total += time.perf_counter() - t0
                    pts += band.size
            done += 1
    desc = (f"oracle (C, 1 thread) on {rows}-row bands of the 4096^2 and 8192^2 grids, all 10 "
            f"stencil/bc combinations, {done} passes")
    return pts, t_total, desc


def cpu_rows(seconds_each: float = 2.0):
    """The oracle on bounded samples of the other rows' workloads (the same code the parity tests
    trust, as it stands): units per second on the host, 1 thread for the C parts, numpy/scipy's
    defaults for the rest.  Each sample repeats until `seconds_each` have passed."""
    import oracle
    oracle.build()

    def timed(fn):
        reps, t = 0, 0.0
        while t < seconds_each:
            t0 = time.perf_counter()
            fn()
            t += time.perf_counter() - t0
            reps += 1
        return reps, t

    out = {}
    n = 512
    h = 2 * np.pi / n
    c0 = W.ch_initial(n, seed=5)
    reps, t = timed(lambda: oracle.ch_step(c0, c0, 1.0, 0.01, 0.1 * h))
    out["ch_adi_f64"] = {"steps_per_s_at_512": round(reps / t, 2),
                         "steps_per_s_at_4096_scaled": round(reps / t * (n / 4096) ** 2, 4)}
    reps, t = timed(lambda: oracle.ch_step_noflux(c0, c0, 1.0, 0.01, 0.1 * h))
    out["ch_noflux_f64"] = {"steps_per_s_at_512": round(reps / t, 2),
                            "steps_per_s_at_4096_scaled": round(reps / t * (n / 4096) ** 2, 4)}
    reps, t = timed(lambda: (oracle.ch_coarsening_s(c0), oracle.ch_coarsening_k1(c0)))
    out["coarsening_measure_at_512"] = {"ms": round(t / reps * 1e3, 3)}
    m = 1024
    hw = 2 * np.pi / m
    cw = W.sines_field(m, seed=61)
    uw, vw = np.cos(cw), np.sin(cw)
    reps, t = timed(lambda: oracle.weno_advection(cw, uw, vw, hw, hw))
    out["weno_f64"] = {"gpts_per_s": round(reps * m * m / t / 1e9, 6), "sample": "1024^2"}
    offs = W.ragged_offsets(2048, seed=7)
    packed = W.sines_lines(offs, seed=8)
    wts = np.array([-1, 16, -30, 16, -1.0]) / 12.0
    reps, t = timed(lambda: oracle.stencil1d_batch(packed, offs, wts, 1, 2, 2))
    out["batch1d_f64"] = {"gpts_per_s": round(reps * int(offs[-1]) / t / 1e9, 6), "sample": "2048 ragged lines"}
    out["threads"] = "C parts 1; numpy / scipy default"
    return out


def cpu_parallel(seconds: float):
    """The same oracle sample on every host core at once: one thread per core, each calling the
    C oracle (ctypes releases the interpreter lock during the call) on its own row bands for
    `seconds`; throughput = all points / wall time.  The second form of the CPU baseline."""
    import concurrent.futures as cf
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    rows = 16
    bands = []
    for n in SIZES:
        h = 2 * np.pi / n
        bands.append((W.sines_field(n, seed=1902 + n, ny=rows), stencil_suite(h)))

    def worker(_):
        pts = 0
        deadline = time.perf_counter() + seconds
        while time.perf_counter() < deadline:
            for band, suite in bands:
                for name, d, L, R, T, B, w, fn, coe, taps in suite:
                    for bc in (1, 0):
                        if fn:
                            oracle.stencil2d_fn(band, fn, coe, bc)
                        else:
                            oracle.stencil2d(band, w, d, bc, L, R, T, B)
                        pts += band.size
        return pts

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        pts = sum(ex.map(worker, range(cores)))
    wall = time.perf_counter() - t0
    return {"value": round(pts / wall / 1e9, 6), "unit": "Gpts/s", "cores": cores, "kind": "oracle",
            "sample": f"oracle (C) on {rows}-row bands of the 4096^2 and 8192^2 grids, all 10 stencil/bc "
                      f"combinations, one thread per host core for {seconds:.0f} s",
            "seconds": round(wall, 2)}


def cpu_baseline(seconds: float):
    pts, t, desc = cpu_sample(seconds)
    return {"value": round(pts / t / 1e9, 6), "unit": "Gpts/s", "cores": 1, "kind": "oracle",
            "sample": desc, "seconds": round(t, 2), "host_cores_available": os.cpu_count(),
            "all_cores": cpu_parallel(max(2.0, seconds / 3))}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    per_step = max(1.0, args.cpu_seconds / max(1, args.steps))
    for _ in range(args.warmup):
        cpu_sample(min(1.0, per_step / 4))
    tot_pts, tot_t, desc = 0, 0.0, ""
    for _ in range(args.steps):
        p, t, desc = cpu_sample(per_step)
        tot_pts += p
        tot_t += t
    value = tot_pts / tot_t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "Gpts/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * tot_t / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": desc},
            "cpu_baseline": {"value": round(value, 6), "unit": "Gpts/s", "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": round(value, 6), "unit": "Gpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_sharded(args):
    """--sharded: one periodic CH grid (n = 4096 by default, FP64) split into row bands over the
    ranks (one GPU each; NCCL, or a single gloo rank on one GPU), stepped with the library's band
    entry points: halo exchange, band right-hand side, x solves, the y solves by chunks with the
    chunks' end values all-gathered (or, when the chunks do not split evenly over the ranks,
    through all-to-all transposes), update (strong scaling: the grid is fixed).  Prints one JSON
    line."""
    import torch
    import torch.distributed as dist
    import paper_1902_09931_gb300 as cs
    from paper_1902_09931_gb300 import distributed as DD
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    else:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        os.environ.setdefault("MASTER_PORT", "29533")
        dist.init_process_group("gloo", rank=0, world_size=1)
    cs.load()
    n = args.sharded_n
    h = 2 * np.pi / n
    r0, r1 = DD.band(n, world, rank)
    c0 = torch.from_numpy(W.ch_initial(n, seed=1902)[r0:r1].copy()).cuda()
    b = DD.DeviceCHBand(n, cs.CS_F64, 1.0, 0.01, 0.1 * h, c0)
    b.step(args.warmup)
    torch.cuda.synchronize()
    dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    b.step(args.steps)
    e1.record()
    torch.cuda.synchronize()
    dist.barrier()
    ms = max_over_ranks(world, e0.elapsed_time(e1) / args.steps) if world > 1 else e0.elapsed_time(e1) / args.steps
    mass, energy = b.invariants()
    b.close()
    if rank == 0:
        print(json.dumps({"metric": "CH-ADI steps/s, one periodic grid in row bands", "value": round(1e3 / ms, 1),
                          "unit": "steps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "strong",
                          "dtype": "f64", "data": "synthetic",
                          "config": {"workload": f"CH-ADI periodic {n}^2, FP64, row bands of {r1 - r0} rows",
                                     "parallelism": f"row bands x{world}", "y_lines": b.mode},
                          "mass": mass, "energy": energy}), flush=True)
    dist.destroy_process_group()


def run_part(args):
    """One part of the metric on its own (used to profile it): --part ch:<n>:<f64|f32>:<steps>[:noflux],
    batch1d, serve, coarsening, streamed or weno."""
    import torch
    import paper_1902_09931_gb300 as cs
    torch.cuda.set_device(0)
    cs.load()
    stream = torch.cuda.current_stream()
    hbm_peak, _ = peaks()
    kind = args.part.split(":")
    if kind[0] == "ch":
        n, dt, steps = int(kind[1]), kind[2], int(kind[3])
        bnd = cs.CS_CH_NOFLUX if len(kind) > 4 and kind[4] == "noflux" else cs.CS_CH_PERIODIC
        res = bench_ch(cs, torch, stream, [(n, cs.CS_F64 if dt == "f64" else cs.CS_F32, steps, bnd)],
                       autotune=not args.no_autotune)
    elif kind[0] == "serve":
        res = bench_serve(cs, torch)
    elif kind[0] == "single_call":
        res = bench_single_call(cs, torch, stream)
    elif kind[0] == "group":
        res = bench_group(cs, torch, stream)
    elif kind[0] == "ch_runs":
        res = bench_ch_runs(cs, torch, stream)
    elif kind[0] == "coarsening":
        res = bench_coarsening(cs, torch, stream)
    elif kind[0] == "streamed":
        res = bench_streamed(cs, torch, stream)
    elif kind[0] == "weno":
        res = bench_weno(cs, torch, stream, hbm_peak)
    else:
        res = bench_batch1d(cs, torch, stream, hbm_peak)
    print(json.dumps({"part": args.part, "result": res}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-parts", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tile-choice", type=int, default=-1, help="force a tile choice (0, 1, 2) instead of autotuning")
    ap.add_argument("--only", default="", help="profile one sweep: name,n,f64|f32,p|np")
    ap.add_argument("--tune-file", default="", help="stencil suite: load the tile choices from this autotuner "
                    "cache if it exists (no autotuning), else autotune and save them there")
    ap.add_argument("--sharded", action="store_true", help="one CH grid split into row bands over the ranks")
    ap.add_argument("--sharded-n", type=int, default=4096)
    ap.add_argument("--part", default="", help="run one part alone: ch:<n>:<f64|f32>:<steps>[:noflux], ch_runs, single_call, group, batch1d, serve, coarsening, streamed or weno")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.sharded:
        run_sharded(args)
    elif args.part:
        run_part(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
