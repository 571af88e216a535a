"""GPU parity of the Cahn-Hilliard ADI step (Sec. 5.1) against the CPU oracle, through the C ABI.

Per-step tolerance.  From an identical state (C^{n-1}, C^n) both implementations evaluate the same
FP64 arithmetic, so they differ by rounding alone.  Its size follows from the step's terms:
  * the right-hand side sums terms of size S = max|C^n| + max|C^{n-1}| + 64 a max|Cbar|
    + 8 alpha max|N| (the 13-point biharmonic's weights sum to 64 in units of a = (2/3) D gamma
    dt / h^4, the 5-point Laplacian's to 8 in units of alpha = (2/3) D dt / h^2), each rounded at
    eps = 2^-52 relative; L^-1 has norm <= 1 (its eigenvalues are >= 1), so these errors reach
    C^{n+1} undamped at the low wavenumbers;
  * the y line solve is backward stable, so it adds at most kappa eps |v| (kappa = 1 + 16 a,
    v = L_y^-1 w); the x-solve's rounding lies in high wavenumbers that L_y^-1 damps.
The bound is B = eps (S + kappa max|v|) (gpu_helpers.ch_step_bound); the tests allow 8 B and
print the measured error as a multiple of B.  FP32 storage
adds two roundings to FP32 (Cbar in the update and the stored result), 2^-24 (max|Cbar| +
max|C^{n+1}|), and must stay within 1e-5 max|C^{n+1}|.  Whole trajectories are compared on the
invariants and on fields with a growth-aware tolerance.
"""
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
        self.plan = cs.cs_ch_create(cs.CHDesc(n=n, storage=storage, D=D, gamma=GAMMA, dt=dt), *self.f)

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
    prev = W.ch_initial(n, seed=n)
    cur = prev + 0.01 * W.ch_initial(n, seed=n + 1)  # a genuine two-level state
    if storage == 1:
        prev = prev.astype(np.float32).astype(np.float64)
        cur = cur.astype(np.float32).astype(np.float64)
    r = Run(cs, torch, prev, cur, storage, dt)
    r.step(1)
    _, got, steps = r.state()
    r.close()
    assert steps == 1
    check_ch_step(orc, prev, cur, got, n, dt, storage, "two-level state")


@pytest.mark.parametrize("storage", [0, 1])
@pytest.mark.parametrize("n", [1024, 4096])
def test_full_size_single_step(env, n, storage):
    """The benchmark grids (N = 1024, 4096; dt = 0.1 h), FP64 and FP32 storage, with the line-solve
    partition the autotuner picks (as the benchmark runs it): one step from the deep-quench
    initial condition (C^{-1} = C^0) and a second step from the resulting two-level state."""
    cs, torch, orc = env
    h = 2 * np.pi / n
    dt = 0.1 * h
    c0 = W.ch_initial(n, seed=1902)
    if storage == 1:
        c0 = c0.astype(np.float32).astype(np.float64)
    r = Run(cs, torch, c0, c0, storage, dt)
    cs.cs_autotune(r.plan)
    torch.cuda.synchronize()
    r.step(1)
    p1, c1, _ = r.state()
    check_ch_step(orc, c0, c0, c1, n, dt, storage, "first step")
    r.step(1)
    _, c2, _ = r.state()
    r.close()
    check_ch_step(orc, p1, c1, c2, n, dt, storage, "second step")


@pytest.mark.parametrize("k,l", [(1, 0), (3, 2), (20, 1)])
def test_linear_limit_closed_form_on_gpu(env, k, l):
    """A mode of amplitude 1e-8 follows c_{n+1} = alpha c_n + beta c_{n-1} (discrete symbols)."""
    cs, torch, orc = env
    n = 64
    h = 2 * np.pi / n
    dt = 0.1 * h
    A = 1e-8
    c0 = W.single_mode(n, k, l, A, phase=0.3)
    a = (2 / 3) * D * GAMMA * dt / h ** 4
    mu = (4 / h ** 2) * (np.sin(k * h / 2) ** 2 + np.sin(l * h / 2) ** 2)
    lam = (1 + 16 * a * np.sin(k * h / 2) ** 4) * (1 + 16 * a * np.sin(l * h / 2) ** 4)
    alpha = 2 + (-2 / 3 - (4 / 3) * D * GAMMA * dt * mu ** 2 + (2 / 3) * D * dt * mu) / lam
    beta = -1 + (2 / 3 + (2 / 3) * D * GAMMA * dt * mu ** 2) / lam
    r = Run(cs, torch, c0, c0, 0, dt)
    amp_p, amp_c = 1.0, 1.0
    for _ in range(5):
        r.step(1)
        amp_p, amp_c = amp_c, alpha * amp_c + beta * amp_p
        _, got, _ = r.state()
        assert np.abs(got - amp_c * c0).max() <= 1e-9 * A
    r.close()


@pytest.mark.parametrize("storage", [0, 1])
def test_mass_conserved_and_invariants_match_oracle(env, storage):
    """Mass is conserved to rounding over 300 steps (deep quench, n = 128); the device FP64
    mass and energy equal the oracle's definitions on the device's own fields."""
    cs, torch, orc = env
    n = 128
    h = 2 * np.pi / n
    c0 = W.ch_initial(n, seed=77)
    if storage == 1:
        c0 = c0.astype(np.float32).astype(np.float64)
    r = Run(cs, torch, c0, c0, storage, 0.1 * h)
    m0, e0 = cs.cs_ch_invariants(r.plan)
    assert abs(m0 - orc.ch_mass(c0)) <= 1e-14
    assert abs(e0 - orc.ch_energy(c0, GAMMA)) <= 1e-12 * abs(e0)
    mass, energy = r.step(300, invariants=True)
    _, cur, steps = r.state()
    r.close()
    assert steps == 300
    scale = h * h * np.abs(c0).sum()
    # FP32 storage rounds C to FP32 each step: drift bounded by steps * n^2 * ulp-level terms
    mtol = 1e-12 * scale if storage == 0 else 300 * 6e-8 * scale
    assert np.abs(mass - m0).max() <= mtol
    assert abs(mass[-1] - orc.ch_mass(cur)) <= 1e-13 * scale + 1e-15
    assert abs(energy[-1] - orc.ch_energy(cur, GAMMA)) <= 1e-12 * abs(energy[-1])


def test_energy_nonincreasing_resolved_data(env):
    cs, torch, orc = env
    n = 128
    h = 2 * np.pi / n
    c0 = W.low_mode_field(n, seed=3)
    r = Run(cs, torch, c0, c0, 0, 0.1 * h)
    e0 = cs.cs_ch_invariants(r.plan)[1]
    mass, energy = r.step(int(2.0 / (0.1 * h)), invariants=True)
    r.close()
    e = np.concatenate([[e0], energy])
    assert np.all(np.diff(e) <= 1e-12 * np.abs(e[:-1]))


def test_trajectory_matches_oracle(env):
    """40 FP64 steps at n = 128 from the deep quench: the field stays within a growth-aware bound
    (rounding differences grow at most like exp(sigma_max t), sigma_max = D / (4 gamma))."""
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
    ref, _, _ = orc.ch_run(c0, D, GAMMA, dt, steps)
    growth = np.exp(D / (4 * GAMMA) * steps * dt)
    assert np.abs(got - ref).max() <= 1e-12 * growth * steps * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("storage", [0, 1])
def test_autotune_restores_state_and_keeps_parity(env, storage):
    """cs_autotune on a Cahn-Hilliard plan times the line-solve partitions, restores the fields
    and the step count, and the tuned plan still matches the oracle step."""
    cs, torch, orc = env
    n = 256
    h = 2 * np.pi / n
    dt = 0.1 * h
    prev = W.ch_initial(n, seed=5)
    cur = prev + 0.01 * W.ch_initial(n, seed=6)
    if storage == 1:
        prev = prev.astype(np.float32).astype(np.float64)
        cur = cur.astype(np.float32).astype(np.float64)
    r = Run(cs, torch, prev, cur, storage, dt)
    cs.cs_autotune(r.plan)
    torch.cuda.synchronize()
    p0, c0, steps0 = r.state()
    assert steps0 == 0 and np.array_equal(p0, prev) and np.array_equal(c0, cur)
    chunks, m = cs.cs_ch_config(r.plan)
    assert chunks * m == n
    r.step(1)
    _, got, _ = r.state()
    r.close()
    check_ch_step(orc, prev, cur, got, n, dt, storage, "after autotune")


@pytest.mark.parametrize("storage", [0, 1])
@pytest.mark.parametrize("boundary", [0, 1])
@pytest.mark.parametrize("via", ["create", "set_fields"])
def test_resume_from_checkpoint_is_bit_identical(env, storage, boundary, via):
    """Checkpoint and resume: a run stopped after 7 steps (C^{n-1} and C^n copied to the host, the
    plan destroyed or rebound) and resumed from those two fields, on a new plan or on another
    plan through cs_ch_set_fields, ends bit for bit where the run straight through ends after 20
    steps, with the same per-step mass and energy; the step count restarts at 0."""
    cs, torch, orc = env
    n = 128
    tdt = torch.float64 if storage == 0 else torch.float32
    c0 = W.ch_initial(n, seed=31 + boundary)
    desc = cs.CHDesc(n=n, storage=storage, D=D, gamma=GAMMA, dt=0.1 * 2 * np.pi / n, boundary=boundary)

    def fields(prev, cur):
        return [torch.from_numpy(np.ascontiguousarray(prev)).to("cuda", tdt),
                torch.from_numpy(np.ascontiguousarray(cur)).to("cuda", tdt), torch.zeros(n, n, dtype=tdt, device="cuda")]

    def current(plan, f):
        p, c, s = cs.cs_ch_fields(plan)
        pick = lambda ptr: [t for t in f if t.data_ptr() == ptr][0].cpu()
        return pick(p), pick(c), s

    f = fields(c0, c0)
    straight = cs.cs_ch_create(desc, *f)
    m_all, e_all = cs.cs_ch_step(straight, 20, invariants=True)
    _, end_straight, steps = current(straight, f)
    cs.cs_destroy(straight)
    assert steps == 20

    g = fields(c0, c0)
    first = cs.cs_ch_create(desc, *g)
    m1, e1 = cs.cs_ch_step(first, 7, invariants=True)
    ck_prev, ck_cur, steps = current(first, g)
    assert steps == 7
    h = fields(ck_prev.numpy(), ck_cur.numpy())
    if via == "create":
        cs.cs_destroy(first)
        second = cs.cs_ch_create(desc, *h)
    else:
        second = first
        cs.cs_ch_set_fields(second, *h)
    assert cs.cs_ch_fields(second)[2] == 0
    m2, e2 = cs.cs_ch_step(second, 13, invariants=True)
    _, end_resumed, steps = current(second, h)
    cs.cs_destroy(second)
    assert steps == 13
    assert torch.equal(end_straight, end_resumed)
    assert np.array_equal(np.concatenate([m1, m2]), m_all) and np.array_equal(np.concatenate([e1, e2]), e_all)
