"""GPU parity of the Cahn-Hilliard ADI step with no-flux boundaries (reflected ghost cells,
non-cyclic line solves; cs_ch_desc.boundary = CS_CH_NOFLUX) against the oracle, through the C ABI.
Per-step tolerances as for the periodic step (gpu_helpers.ch_step_bound: 8 eps (S + kappa (max|w|
+ max|v|)) with S the size of the right-hand side's terms, plus the FP32 roundings for FP32
storage, which must also stay within 1e-5 max|C^{n+1}|)."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import check_ch_step

pytestmark = pytest.mark.gpu

D, GAMMA = 1.0, 0.01


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    pytest.importorskip("scipy")
    import oracle
    import paper_1902_09931_gb300 as cs
    cs.load()
    return cs, torch, oracle


class Run:
    def __init__(self, cs, torch, prev, cur, storage, dt):
        self.cs, self.torch = cs, torch
        tdt = torch.float64 if storage == 0 else torch.float32
        n = cur.shape[0]
        self.f = [torch.from_numpy(np.ascontiguousarray(prev)).to("cuda", tdt),
                  torch.from_numpy(np.ascontiguousarray(cur)).to("cuda", tdt),
                  torch.zeros(n, n, dtype=tdt, device="cuda")]
        desc = cs.CHDesc(n=n, storage=storage, D=D, gamma=GAMMA, dt=dt, boundary=cs.CS_CH_NOFLUX)
        self.plan = cs.cs_ch_create(desc, *self.f)

    def step(self, k, invariants=False):
        r = self.cs.cs_ch_step(self.plan, k, invariants=invariants)
        self.torch.cuda.synchronize()
        return r

    def state(self):
        p, c, s = self.cs.cs_ch_fields(self.plan)
        get = lambda ptr: [t for t in self.f if t.data_ptr() == ptr][0].cpu().numpy().astype(np.float64)
        return get(p), get(c), s

    def close(self):
        self.cs.cs_destroy(self.plan)


@pytest.mark.parametrize("storage", [0, 1])
@pytest.mark.parametrize("n", [64, 128, 256, 512])
def test_single_step_from_identical_state(env, storage, n):
    cs, torch, orc = env
    h = 2 * np.pi / n
    dt = 0.1 * h
    prev = W.ch_initial(n, seed=n + 7)
    cur = prev + 0.01 * W.ch_initial(n, seed=n + 8)
    if storage == 1:
        prev = prev.astype(np.float32).astype(np.float64)
        cur = cur.astype(np.float32).astype(np.float64)
    r = Run(cs, torch, prev, cur, storage, dt)
    r.step(1)
    _, got, steps = r.state()
    r.close()
    assert steps == 1
    check_ch_step(orc, prev, cur, got, n, dt, storage, "two-level state", noflux=True)


@pytest.mark.parametrize("n", [1024, 4096])
def test_full_size_single_step(env, n):
    cs, torch, orc = env
    h = 2 * np.pi / n
    dt = 0.1 * h
    c0 = W.ch_initial(n, seed=1903)
    r = Run(cs, torch, c0, c0, 0, dt)
    r.step(1)
    p1, c1, _ = r.state()
    check_ch_step(orc, c0, c0, c1, n, dt, 0, "first step", noflux=True)
    r.step(1)
    _, c2, _ = r.state()
    r.close()
    check_ch_step(orc, p1, c1, c2, n, dt, 0, "second step", noflux=True)


def test_full_size_single_step_fp32_storage(env):
    """4096^2 with FP32 fields (the bench's FP32 configuration), against the FP64 oracle fed the
    same FP32-rounded state."""
    cs, torch, orc = env
    n = 4096
    h = 2 * np.pi / n
    dt = 0.1 * h
    prev = W.ch_initial(n, seed=1904).astype(np.float32).astype(np.float64)
    cur = (prev + 0.01 * W.ch_initial(n, seed=1905)).astype(np.float32).astype(np.float64)
    r = Run(cs, torch, prev, cur, 1, dt)
    r.step(1)
    _, got, _ = r.state()
    r.close()
    check_ch_step(orc, prev, cur, got, n, dt, 1, "two-level state", noflux=True)


@pytest.mark.parametrize("k,l", [(1, 0), (3, 2), (20, 1), (63, 63)])
def test_linear_limit_cosine_modes_on_gpu(env, k, l):
    """cos(k pi (i + 1/2) / n) cos(l pi (j + 1/2) / n), amplitude 1e-8: the amplitude follows the
    two-term recurrence with the reflected symbols."""
    cs, torch, orc = env
    n = 64
    h = 2 * np.pi / n
    dt = 0.1 * h
    A = 1e-8
    x = (np.arange(n) + 0.5) * np.pi / n
    c0 = A * np.cos(l * x)[:, None] * np.cos(k * x)[None, :]
    a = orc.ch_coefficient_a(n, D, GAMMA, dt)
    sx, sy = np.sin(k * np.pi / (2 * n)) ** 2, np.sin(l * np.pi / (2 * n)) ** 2
    mu = 4 / h ** 2 * (sx + sy)
    lam = (1 + 16 * a * sx ** 2) * (1 + 16 * a * sy ** 2)
    a1 = 2 + (-2 / 3 - (4 / 3) * D * GAMMA * dt * mu ** 2 + (2 / 3) * D * dt * mu) / lam
    a0 = -1 + (2 / 3 + (2 / 3) * D * GAMMA * dt * mu ** 2) / lam
    r = Run(cs, torch, c0, c0, 0, dt)
    ap, ac = 1.0, 1.0
    for _ in range(5):
        r.step(1)
        ap, ac = ac, a1 * ac + a0 * ap
        _, got, _ = r.state()
        assert np.abs(got - ac * c0).max() <= 1e-9 * A
    r.close()


@pytest.mark.parametrize("storage", [0, 1])
def test_mass_conserved_and_invariants_match_oracle(env, storage):
    cs, torch, orc = env
    n = 128
    h = 2 * np.pi / n
    dt = 0.1 * h
    c0 = W.ch_initial(n, seed=31) + 0.2  # off-critical: a non-zero mean must stay put
    if storage == 1:
        c0 = c0.astype(np.float32).astype(np.float64)
    r = Run(cs, torch, c0, c0, storage, dt)
    m0, e0 = cs.cs_ch_invariants(r.plan)
    assert m0 == pytest.approx(h * h * c0.sum(), rel=1e-13)
    assert e0 == pytest.approx(orc.ch_energy_noflux(c0, GAMMA), rel=1e-12)
    mass, energy = r.step(60, invariants=True)
    _, cur, _ = r.state()
    r.close()
    scale = h * h * np.abs(c0).sum()
    drift = 1e-12 if storage == 0 else 1e-5
    assert np.abs(mass - m0).max() <= drift * scale
    assert energy[-1] == pytest.approx(orc.ch_energy_noflux(cur, GAMMA), rel=1e-12 if storage == 0 else 1e-5)


def test_trajectory_matches_oracle(env):
    """40 FP64 steps at n = 128 from the deep quench, with the growth-aware bound of the
    periodic trajectory test."""
    cs, torch, orc = env
    n = 128
    h = 2 * np.pi / n
    dt = 0.1 * h
    c0 = W.ch_initial(n, seed=12)
    steps = 40
    r = Run(cs, torch, c0, c0, 0, dt)
    r.step(steps)
    _, got, _ = r.state()
    r.close()
    ref, _, _ = orc.ch_run_noflux(c0, D, GAMMA, dt, steps)
    growth = np.exp(D / (4 * GAMMA) * steps * dt)
    assert np.abs(got - ref).max() <= 1e-12 * growth * steps * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("storage", [0, 1])
def test_autotune_every_partition_keeps_parity(env, storage):
    """cs_autotune runs one step with every chunk count (1, 2, 4, 8, 16 at n = 256: the single-chunk
    tables, and first / interior / last chunks) and restores the state; the tuned plan matches."""
    cs, torch, orc = env
    n = 256
    h = 2 * np.pi / n
    dt = 0.1 * h
    prev = W.ch_initial(n, seed=15)
    cur = prev + 0.01 * W.ch_initial(n, seed=16)
    if storage == 1:
        prev = prev.astype(np.float32).astype(np.float64)
        cur = cur.astype(np.float32).astype(np.float64)
    r = Run(cs, torch, prev, cur, storage, dt)
    cs.cs_autotune(r.plan)
    torch.cuda.synchronize()
    p0, c0, s0 = r.state()
    assert s0 == 0 and np.array_equal(p0, prev) and np.array_equal(c0, cur)
    r.step(1)
    _, got, _ = r.state()
    r.close()
    check_ch_step(orc, prev, cur, got, n, dt, storage, "after autotune", noflux=True)


def test_coarsening_measures_refused(env):
    cs, torch, _ = env
    n = 64
    c0 = W.ch_initial(n, seed=1)
    r = Run(cs, torch, c0, c0, 0, 0.01)
    try:
        with pytest.raises(Exception) as e:
            cs.cs_ch_coarsening(r.plan)
        assert getattr(e.value, "code", None) == cs.CS_EUNSUPPORTED
    finally:
        r.close()
