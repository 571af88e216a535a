"""Host logic of the serving loop (no GPU): admission by slots and memory, arrival order,
grouping of sweeps per launch, overlap, retirement, and the sequential baseline, driven by a
fake backend on a simulated clock."""
import math

import pytest

from paper_1902_09931_gb300 import serving as S


class FakeClock:
    def __init__(self, dt=1e-5):
        self.t = 0.0
        self.dt = dt

    def __call__(self):
        self.t += self.dt
        return self.t


class FakeBackend:
    """Service time proportional to grid points; several launches run concurrently."""

    def __init__(self, clock, budget):
        self.clock = clock
        self.budget = budget
        self.resident = 0
        self.peak_resident = 0
        self.inflight_jobs = 0
        self.peak_inflight = 0
        self.launches = []
        self.prepared = []

    def default_budget(self):
        return self.budget

    def prepare(self, job):
        self.resident += S.footprint(job)
        self.peak_resident = max(self.peak_resident, self.resident)
        self.prepared.append(job.jid)

    def _service(self, jobs):
        return sum(j.n * j.n * (j.steps if j.kind == "ch" else 1) for j in jobs) * 1e-9

    def launch_sweeps(self, jobs):
        self.launches.append(("sweep", [j.jid for j in jobs], {j.stencil for j in jobs}))
        return self._launch(jobs)

    def launch_ch(self, job):
        self.launches.append(("ch", [job.jid], None))
        return self._launch([job])

    def _launch(self, jobs):
        self.inflight_jobs += len(jobs)
        self.peak_inflight = max(self.peak_inflight, self.inflight_jobs)
        return {"end": self.clock.t + self._service(jobs), "n": len(jobs)}

    def query(self, h):
        return self.clock.t >= h["end"]

    def wait(self, h):
        while self.clock() < h["end"]:
            pass

    def release_handle(self, h):
        self.inflight_jobs -= h["n"]

    def release(self, job):
        self.resident -= S.footprint(job)

    def idle_until(self, t_abs, clock):
        while clock() < t_abs:
            pass


def test_poisson_jobs_recipe():
    jobs = S.poisson_jobs(400, rate=100.0, seed=3)
    gaps = [b.arrival - a.arrival for a, b in zip(jobs, jobs[1:])]
    assert all(g >= 0 for g in gaps)
    assert abs(sum(gaps) / len(gaps) - 0.01) < 0.003
    kinds = [j.kind for j in jobs]
    assert 0.4 < kinds.count("sweep") / len(kinds) < 0.6
    assert {j.n for j in jobs} <= set(S.SIZES)
    assert all(j.steps == 10 for j in jobs)


@pytest.mark.parametrize("max_inflight", [1, 3, 8])
def test_server_respects_slots_and_memory(max_inflight):
    clock = FakeClock()
    jobs = S.poisson_jobs(60, rate=2000.0, seed=11, sizes=(128, 256, 512, 1024))
    budget = 3 * S.footprint(S.Job(0, "ch", 1024, 0.0))
    be = FakeBackend(clock, budget)
    srv = S.Server(be, max_inflight=max_inflight, clock=clock)
    stats = srv.run(jobs)
    assert stats["jobs"] == 60
    assert all(not math.isnan(j.done) and j.done >= j.start >= j.arrival for j in jobs)
    assert be.peak_inflight <= max_inflight
    assert be.peak_resident <= budget
    assert be.resident == 0 and be.inflight_jobs == 0
    # admission in arrival order
    assert be.prepared == sorted(be.prepared, key=lambda i: jobs[i].arrival)


def test_sweeps_share_launches_and_jobs_overlap():
    clock = FakeClock()
    # a burst of sweeps arriving together: one launch per stencil shape
    jobs = [S.Job(i, "sweep", 256, 0.0, stencil=S.SWEEP_STENCILS[i % 2], seed=i) for i in range(8)]
    be = FakeBackend(clock, 1 << 40)
    S.Server(be, max_inflight=16, clock=clock).run(jobs)
    sweeps = [l for l in be.launches if l[0] == "sweep"]
    assert len(sweeps) == 2 and all(len(l[2]) == 1 for l in sweeps)
    assert sorted(sum((l[1] for l in sweeps), [])) == list(range(8))
    # without grouping every sweep is its own launch
    be2 = FakeBackend(FakeClock(), 1 << 40)
    S.Server(be2, max_inflight=16, group=False, clock=be2.clock).run(
        [S.Job(i, "sweep", 256, 0.0, stencil="lap9", seed=i) for i in range(8)])
    assert len(be2.launches) == 8
    assert be.peak_inflight == 8


def test_continuous_batching_beats_sequential_under_load():
    jobs_a = S.poisson_jobs(80, rate=3000.0, seed=5, sizes=(128, 256, 512))
    jobs_b = S.poisson_jobs(80, rate=3000.0, seed=5, sizes=(128, 256, 512))
    c1 = FakeClock()
    seq = S.run_sequential(FakeBackend(c1, 1 << 40), jobs_a, clock=c1)
    c2 = FakeClock()
    srv = S.Server(FakeBackend(c2, 1 << 40), max_inflight=8, clock=c2).run(jobs_b)
    assert srv["p99_ms"] < seq["p99_ms"]
    assert srv["jobs_per_s"] > seq["jobs_per_s"]


def test_oversized_job_rejected():
    clock = FakeClock()
    be = FakeBackend(clock, 1000)
    with pytest.raises(ValueError):
        S.Server(be, clock=clock).run([S.Job(0, "ch", 4096, 0.0)])


def test_sequential_runs_one_at_a_time():
    clock = FakeClock()
    jobs = S.poisson_jobs(20, rate=5000.0, seed=2, sizes=(128, 256))
    be = FakeBackend(clock, 1 << 40)
    S.run_sequential(be, jobs, clock=clock)
    order = sorted(jobs, key=lambda j: j.arrival)
    for a, b in zip(order, order[1:]):
        assert b.start >= a.done
    assert be.peak_inflight == 1


def test_heavy_jobs_run_one_at_a_time_and_light_jobs_pass():
    """Heavy jobs (Cahn-Hilliard advances of 2048^2 and up) run one at a time in arrival order;
    lighter jobs that arrive behind a waiting heavy job go ahead of it."""
    clock = FakeClock()
    jobs = [S.Job(0, "ch", 4096, 0.0, seed=1), S.Job(1, "ch", 2048, 0.0, seed=2),
            S.Job(2, "sweep", 256, 0.0, seed=3), S.Job(3, "ch", 128, 0.0, seed=4),
            S.Job(4, "sweep", 4096, 0.0, seed=5)]
    be = FakeBackend(clock, 1 << 40)
    S.Server(be, max_inflight=8, clock=clock).run(jobs)
    h0, h1, l2, l3, l4 = jobs
    assert h0.heavy and h1.heavy and not (l2.heavy or l3.heavy or l4.heavy)
    assert h1.start >= h0.done
    assert max(l2.start, l3.start, l4.start) < h0.done
    # without the limit both heavy jobs are in flight together
    jobs2 = [S.Job(0, "ch", 4096, 0.0), S.Job(1, "ch", 2048, 0.0)]
    be2 = FakeBackend(FakeClock(), 1 << 40)
    S.Server(be2, max_inflight=8, clock=be2.clock, max_heavy=None).run(jobs2)
    assert jobs2[1].start < jobs2[0].done and be2.peak_inflight == 2


def test_heavy_limit_keeps_memory_order():
    """A job that does not fit the memory budget still blocks the jobs behind it (no job passes
    it), whether or not a heavy job waits ahead of it."""
    clock = FakeClock()
    big = S.Job(0, "ch", 4096, 0.0)
    budget = S.footprint(big) + S.footprint(S.Job(0, "sweep", 256, 0.0))
    jobs = [big, S.Job(1, "ch", 2048, 0.0), S.Job(2, "sweep", 256, 0.0), S.Job(3, "sweep", 2048, 0.0),
            S.Job(4, "sweep", 128, 0.0)]
    be = FakeBackend(clock, budget)
    S.Server(be, max_inflight=8, clock=clock).run(jobs)
    assert all(not math.isnan(j.done) for j in jobs)
    assert be.peak_resident <= budget
    # job 3 (2048^2 sweep) does not fit beside job 0: job 4 waits behind it
    assert jobs[4].start >= jobs[3].start


@pytest.mark.parametrize("kw", [dict(max_heavy=0), dict(max_inflight=0)])
def test_limits_that_would_stall_the_loop_are_refused(kw):
    with pytest.raises(ValueError):
        S.Server(FakeBackend(FakeClock(), 1 << 40), **kw)
