"""Continuous-batching serving loop for stencil sweeps and Cahn-Hilliard advances.

Jobs arrive over time (Poisson).  The server admits them in arrival order as long as an
in-flight slot is free and their fields fit the device-memory budget, keeps every job's fields
resident on the device, launches every admitted 2D sweep of the same stencil shape in one
grouped kernel launch (cs_compute_group), runs each Cahn-Hilliard advance on its own stream so
independent jobs overlap on the GPU, and retires jobs as their completion events fire, which
frees their slot and memory for the next arrivals.  Heavy jobs (those of at least
HEAVY_WORK point-steps: the Cahn-Hilliard advances of 2048^2 and 4096^2, each of which fills the
GPU alone) run at most `max_heavy` at a time in arrival order, and lighter jobs may pass a heavy
job that waits for that limit; two heavy advances sharing the GPU would each take about twice as
long, which is what sets the tail latency at light load.  The backend runs light jobs on
higher-priority streams, so a heavy advance in flight does not hold their kernels back.  The
sequential baseline runs the same jobs one at a time with plain calls.  All GPU work goes
through the C ABI; this module only schedules.

The scheduler talks to a backend (prepare / launch_sweeps / launch_ch / query / release) so
that its admission and slot logic can be exercised without a GPU.
"""
from __future__ import annotations

import collections
import math
import statistics
import time
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional

import numpy as np

SWEEP_STENCILS = ("lap9", "biharm13", "ddx4", "ddy4")
SIZES = (128, 256, 512, 1024, 2048, 4096)
HEAVY_WORK = 2048 * 2048 * 10  # point-steps from which a job counts as heavy


@dataclass
class Job:
    jid: int
    kind: str  # "sweep" or "ch"
    n: int
    arrival: float  # seconds after the start of the run
    stencil: str = "lap9"
    steps: int = 10
    seed: int = 0
    start: float = math.nan  # admission time
    done: float = math.nan  # completion time
    output: object = None  # device tensor holding the result
    res: dict = field(default_factory=dict)
    heavy: bool = False  # set by the server: runs under the heavy-job limit, lower stream priority

    @property
    def latency(self) -> float:
        return self.done - self.arrival

    @property
    def work(self) -> int:
        """Point-steps: n^2 for a sweep, n^2 times the steps for a Cahn-Hilliard advance."""
        return self.n * self.n * (self.steps if self.kind == "ch" else 1)


def footprint(job: Job, elem_bytes: int = 4) -> int:
    """Device bytes a job keeps resident while in flight: in + out for a sweep; three fields
    plus the line-solve scratch (two n^2 FP64 arrays) for a Cahn-Hilliard advance."""
    nn = job.n * job.n
    if job.kind == "sweep":
        return 2 * nn * elem_bytes
    return 3 * nn * elem_bytes + 2 * nn * 8


def poisson_jobs(count: int, rate: float, seed: int, sizes=SIZES, sweep_fraction: float = 0.5,
                 steps: int = 10) -> List[Job]:
    """`count` jobs with exponential inter-arrival times of mean 1/rate, half sweeps (stencil
    drawn from SWEEP_STENCILS) and half Cahn-Hilliard advances of `steps` steps, square sizes
    drawn uniformly from `sizes`."""
    g = np.random.Generator(np.random.PCG64(seed))
    t = np.cumsum(g.exponential(1.0 / rate, size=count)) if rate > 0 else np.zeros(count)
    jobs = []
    for i in range(count):
        kind = "sweep" if g.uniform() < sweep_fraction else "ch"
        n = int(sizes[g.integers(0, len(sizes))])
        st = SWEEP_STENCILS[g.integers(0, len(SWEEP_STENCILS))]
        jobs.append(Job(jid=i, kind=kind, n=n, arrival=float(t[i]), stencil=st, steps=steps,
                        seed=10_000 + i))
    return jobs


class Server:
    """Continuous batching: admit while slots and memory allow, group sweeps per launch,
    overlap independent jobs on streams, retire on completion."""

    def __init__(self, backend, max_inflight: int = 8, hbm_budget: Optional[int] = None,
                 group: bool = True, clock: Callable[[], float] = time.perf_counter,
                 max_heavy: Optional[int] = 1, heavy_work: int = HEAVY_WORK):
        self.backend = backend
        self.max_inflight = max_inflight
        self.budget = hbm_budget if hbm_budget is not None else backend.default_budget()
        self.group = group
        self.clock = clock
        if max_inflight < 1:
            raise ValueError("max_inflight must be at least 1")
        if max_heavy is not None and max_heavy < 1:
            raise ValueError("max_heavy must be at least 1, or None for no limit")
        self.max_heavy = max_heavy  # None: no limit
        self.heavy_work = heavy_work
        self.launches = 0

    def run(self, jobs: List[Job]) -> Dict:
        jobs = sorted(jobs, key=lambda j: j.arrival)
        for j in jobs:
            if footprint(j) > self.budget:
                raise ValueError(f"job {j.jid} needs {footprint(j)} bytes, above the budget {self.budget}")
            j.heavy = self.max_heavy is not None and j.work >= self.heavy_work
        waiting = collections.deque()
        inflight = []  # (handle, [jobs])
        used = 0
        busy = 0
        heavy = 0  # heavy jobs in flight
        nxt = 0
        finished = 0
        peak_inflight = 0
        t0 = self.clock()
        while finished < len(jobs):
            now = self.clock() - t0
            while nxt < len(jobs) and jobs[nxt].arrival <= now:
                waiting.append(jobs[nxt])
                nxt += 1
            # admission in arrival order (a job that does not fit the memory budget waits, and no
            # job passes it); a heavy job that waits for the heavy-job limit lets lighter ones pass
            admitted = []
            i = 0
            while i < len(waiting) and busy + len(admitted) < self.max_inflight:
                j = waiting[i]
                if used + footprint(j) > self.budget:
                    break
                if j.heavy and heavy >= self.max_heavy:
                    i += 1
                    continue
                del waiting[i]
                self.backend.prepare(j)
                j.start = self.clock() - t0
                used += footprint(j)
                heavy += j.heavy
                admitted.append(j)
            # dispatch: sweeps of one stencil shape share a launch; each CH job has its stream
            if admitted:
                groups: Dict[str, List[Job]] = collections.OrderedDict()
                for j in admitted:
                    if j.kind == "sweep":
                        key = j.stencil if self.group else f"{j.stencil}#{j.jid}"
                        groups.setdefault(key, []).append(j)
                    else:
                        inflight.append((self.backend.launch_ch(j), [j]))
                        self.launches += 1
                for js in groups.values():
                    inflight.append((self.backend.launch_sweeps(js), js))
                    self.launches += 1
                busy += len(admitted)
                peak_inflight = max(peak_inflight, busy)
            # retire completed work
            still = []
            for h, js in inflight:
                if self.backend.query(h):
                    t = self.clock() - t0
                    for j in js:
                        j.done = t
                        used -= footprint(j)
                        heavy -= j.heavy
                        self.backend.release(j)
                        finished += 1
                    busy -= len(js)
                    self.backend.release_handle(h)
                else:
                    still.append((h, js))
            inflight = still
            if not admitted and not inflight and not waiting and nxt < len(jobs):
                self.backend.idle_until(t0 + jobs[nxt].arrival, self.clock)
        return summarize(jobs, peak_inflight=peak_inflight, launches=self.launches)


def run_sequential(backend, jobs: List[Job], clock: Callable[[], float] = time.perf_counter) -> Dict:
    """The plain baseline: jobs in arrival order, one at a time, each call waited for."""
    jobs = sorted(jobs, key=lambda j: j.arrival)
    t0 = clock()
    for j in jobs:
        if clock() - t0 < j.arrival:
            backend.idle_until(t0 + j.arrival, clock)
        backend.prepare(j)
        j.start = clock() - t0
        h = backend.launch_ch(j) if j.kind == "ch" else backend.launch_sweeps([j])
        backend.wait(h)
        j.done = clock() - t0
        backend.release(j)
        backend.release_handle(h)
    return summarize(jobs, peak_inflight=1, launches=len(jobs))


def summarize(jobs: List[Job], **extra) -> Dict:
    lat = np.array([j.latency for j in jobs]) * 1e3
    span = max(j.done for j in jobs) - min(j.arrival for j in jobs)
    pts = sum(j.n * j.n * (j.steps if j.kind == "ch" else 1) for j in jobs)
    out = {"jobs": len(jobs), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
           "mean_ms": float(lat.mean()), "jobs_per_s": len(jobs) / span if span > 0 else math.inf,
           "gpts_per_s": pts / span / 1e9 if span > 0 else math.inf, "span_s": span}
    out.update(extra)
    return out


class GpuBackend:
    """Runs jobs through the C ABI on the current CUDA device (FP32 storage)."""

    def __init__(self, cs, torch, streams: int = 8, ch_dt_factor: float = 0.1, D: float = 1.0,
                 gamma: float = 0.01, keep_outputs: bool = True):
        self.cs, self.torch = cs, torch
        self.keep_outputs = keep_outputs
        self.dev = torch.device("cuda", torch.cuda.current_device())
        # light jobs on streams of the highest priority, heavy ones on default-priority streams
        self.pool_streams = {False: [torch.cuda.Stream(priority=-1) for _ in range(streams)],
                             True: [torch.cuda.Stream() for _ in range(max(1, streams // 4))]}
        self.free_streams = {k: list(v) for k, v in self.pool_streams.items()}
        self.ch_plans: Dict[int, list] = collections.defaultdict(list)
        # sweep plans are reused (rebound to each job's buffers): creating and destroying a plan
        # per job allocates and frees device memory, and a free synchronises the device
        self.sweep_plans: Dict[tuple, list] = collections.defaultdict(list)
        self.ch_dt_factor, self.D, self.gamma = ch_dt_factor, D, gamma

    # -- resources -------------------------------------------------------------------------
    def default_budget(self) -> int:
        free, _total = self.torch.cuda.mem_get_info()
        return int(0.5 * free)

    def warmup(self, sizes, copies: int = 2):
        """Creates Cahn-Hilliard plans (and their device workspace) and sweep plans of every
        stencil of the mix ahead of the run."""
        made = []
        for n in sizes:
            for _ in range(copies):
                made.append((n, self._new_ch_plan(n)))
        for n, p in made:
            self.ch_plans[n].append(p)
        t = self.torch
        for n in sizes:
            x = t.zeros(n, n, dtype=t.float32, device=self.dev)
            y = t.zeros_like(x)
            for st in SWEEP_STENCILS:
                for _ in range(copies):
                    self.sweep_plans[(n, st)].append(self._new_sweep_plan(n, st, x, y))

    def _new_sweep_plan(self, n, stencil, x, y):
        cs = self.cs
        name, d, L, R, T, B, w = sweep_stencil(stencil, 2 * np.pi / n)
        return cs.cs_plan_create_2d(cs.StencilDesc(nx=n, ny=n, dir=d, bc=cs.CS_BC_PERIODIC, dtype=cs.CS_F32,
                                                   left=L, right=R, top=T, bottom=B, weights=w), x, y)

    def _new_ch_plan(self, n):
        t = self.torch
        f = [t.zeros(n, n, dtype=t.float32, device=self.dev) for _ in range(3)]
        h = 2 * np.pi / n
        plan = self.cs.cs_ch_create(self.cs.CHDesc(n=n, storage=self.cs.CS_F32, D=self.D, gamma=self.gamma,
                                                   dt=self.ch_dt_factor * h), *f)
        return plan

    def prepare(self, job: Job):
        import workloads as W
        t, cs = self.torch, self.cs
        n = job.n
        if job.kind == "sweep":
            x = W.device_uniform((n, n), job.seed, -1.0, 1.0, self.dev, t.float32)
            y = t.zeros_like(x)
            pool = self.sweep_plans[(n, job.stencil)]
            if pool:
                plan = pool.pop()
                cs.cs_set_buffers(plan, x, y)
            else:
                plan = self._new_sweep_plan(n, job.stencil, x, y)
            job.res = {"plan": plan, "x": x}
            job.output = y
        else:
            c0 = W.device_uniform((n, n), job.seed, -0.1, 0.1, self.dev, t.float32)
            c0 -= c0.mean()
            f = [c0, c0.clone(), t.zeros_like(c0)]
            plan = self.ch_plans[n].pop() if self.ch_plans[n] else self._new_ch_plan(n)
            cs.cs_ch_set_fields(plan, *f)
            job.res = {"plan": plan, "fields": f}

    def _stream(self, heavy: bool):
        free = self.free_streams[heavy]
        s = free.pop() if free else self.pool_streams[heavy][0]
        # the job's inputs were produced on the current stream at admission
        s.wait_stream(self.torch.cuda.current_stream())
        return s

    def launch_sweeps(self, jobs: List[Job]):
        s = self._stream(any(j.heavy for j in jobs))
        plans = [j.res["plan"] for j in jobs]
        with self.torch.cuda.stream(s):
            if len(plans) == 1:
                self.cs.cs_compute(plans[0], s)
            else:
                try:
                    self.cs.cs_compute_group(plans, s)
                except self.cs.CSError:
                    for p in plans:
                        self.cs.cs_compute(p, s)
            ev = self.torch.cuda.Event()
            ev.record(s)
        return (ev, s)

    def launch_ch(self, job: Job):
        s = self._stream(job.heavy)
        with self.torch.cuda.stream(s):
            self.cs.cs_ch_step(job.res["plan"], job.steps, stream=s)
            ev = self.torch.cuda.Event()
            ev.record(s)
        return (ev, s)

    def query(self, handle) -> bool:
        return handle[0].query()

    def wait(self, handle):
        handle[0].synchronize()

    def release_handle(self, handle):
        s = handle[1]
        for heavy, pool in self.pool_streams.items():
            if any(s is q for q in pool) and not any(s is q for q in self.free_streams[heavy]):
                self.free_streams[heavy].append(s)

    def release(self, job: Job):
        if job.kind == "sweep":
            self.sweep_plans[(job.n, job.stencil)].append(job.res["plan"])
        else:
            plan = job.res["plan"]
            _, cur, _ = self.cs.cs_ch_fields(plan)
            job.output = [f for f in job.res["fields"] if f.data_ptr() == cur][0]
            self.ch_plans[job.n].append(plan)
        if not self.keep_outputs:
            job.output = None
        job.res = {}

    def idle_until(self, t_abs: float, clock):
        """Waits for the next arrival: sleeps while more than 0.2 ms remain, then spins (a sleep
        alone overshoots by tens of microseconds)."""
        while True:
            left = t_abs - clock()
            if left <= 0:
                return
            if left > 2e-4:
                time.sleep(left - 1.5e-4)


def sweep_stencil(name: str, h: float):
    """The serving mix's weighted stencils (those of the benchmark suite), scaled for spacing h."""
    if name == "lap9":
        return name, 2, 1, 1, 1, 1, np.array([1, 4, 1, 4, -20, 4, 1, 4, 1.0]) / (6 * h * h)
    if name == "biharm13":
        b = np.zeros((5, 5))
        b[2, 2] = 20
        b[1, 2] = b[3, 2] = b[2, 1] = b[2, 3] = -8
        b[1, 1] = b[1, 3] = b[3, 1] = b[3, 3] = 2
        b[0, 2] = b[4, 2] = b[2, 0] = b[2, 4] = 1
        return name, 2, 2, 2, 2, 2, b.ravel() / h ** 4
    d1 = np.array([1, -8, 0, 8, -1.0]) / (12 * h)
    if name == "ddx4":
        return name, 0, 2, 2, 0, 0, d1
    if name == "ddy4":
        return name, 1, 0, 0, 2, 2, d1
    raise ValueError(name)


def percentiles(values) -> Dict[str, float]:
    v = list(values)
    return {"p50": statistics.median(v), "p99": float(np.percentile(v, 99))}
