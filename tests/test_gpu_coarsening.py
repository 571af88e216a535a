"""GPU parity of the coarsening measures s(t) and k_1(t) (Sec. 5.1, "Numerical Results") against
the CPU oracle, through the C ABI.

Both sides work in FP64 on the same field (FP32-storage fields are widened exactly), so they
differ only in summation order: the Simpson sum and the power sums are sums of positive terms,
and a radix-2 FFT's error is O(log2(n) eps) of the field's L2 norm, so 1e-12 relative holds with
a wide margin for mean-free fields (k = 0 is left out of both spectral sums)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

D, GAMMA = 1.0, 0.01
REL = 1e-12


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import oracle
    import paper_1902_09931_gb300 as cs
    cs.load()
    return cs, torch, oracle


def make_plan(cs, torch, c, storage, dt=None):
    n = c.shape[0]
    tdt = torch.float64 if storage == 0 else torch.float32
    f = [torch.from_numpy(np.ascontiguousarray(c)).to("cuda", tdt) for _ in range(2)]
    f.append(torch.zeros(n, n, dtype=tdt, device="cuda"))
    dt = 0.1 * (2 * np.pi / n) if dt is None else dt
    return cs.cs_ch_create(cs.CHDesc(n=n, storage=storage, D=D, gamma=GAMMA, dt=dt), *f), f


def current(cs, plan, f):
    _, c, _ = cs.cs_ch_fields(plan)
    return [t for t in f if t.data_ptr() == c][0].cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("storage", [0, 1])
@pytest.mark.parametrize("n", [64, 512, 2048])
def test_measures_match_oracle(env, storage, n):
    cs, torch, orc = env
    c = W.ch_initial(n, seed=40 + n)
    if storage == 1:
        c = c.astype(np.float32).astype(np.float64)
    plan, f = make_plan(cs, torch, c, storage)
    s, k1 = cs.cs_ch_coarsening(plan)
    cs.cs_destroy(plan)
    assert s == pytest.approx(orc.ch_coarsening_s(c), rel=REL)
    assert k1 == pytest.approx(orc.ch_coarsening_k1(c), rel=REL)


@pytest.mark.parametrize("storage", [0, 1])
def test_measures_after_steps_match_oracle(env, storage):
    """On an evolved (phase-separating) field, read back from the plan's current buffer."""
    cs, torch, orc = env
    n = 256
    plan, f = make_plan(cs, torch, W.ch_initial(n, seed=7), storage)
    cs.cs_ch_step(plan, 400)
    torch.cuda.synchronize()
    s, k1 = cs.cs_ch_coarsening(plan)
    c = current(cs, plan, f)
    cs.cs_destroy(plan)
    assert s == pytest.approx(orc.ch_coarsening_s(c), rel=REL)
    assert k1 == pytest.approx(orc.ch_coarsening_k1(c), rel=REL)
    assert s > 1.0 + 1e-3  # phase separation has raised <C^2>


@pytest.mark.parametrize("n,k,l", [(64, 3, 4), (256, 12, 5), (1024, 0, 7)])
def test_single_mode_closed_form(env, n, k, l):
    """A sin(k x + l y + phase): Simpson's rule on the periodic grid averages C^2 exactly to
    A^2 / 2 (2k, 2l below n / 2), and the spectrum sits at +-(k, l), so k_1 = |(k, l)|."""
    cs, torch, _ = env
    amp = 0.8
    c = W.single_mode(n, k, l, amp)
    plan, _ = make_plan(cs, torch, c, 0)
    s, k1 = cs.cs_ch_coarsening(plan)
    cs.cs_destroy(plan)
    assert s == pytest.approx(1.0 / (1.0 - amp * amp / 2), rel=1e-13)
    assert k1 == pytest.approx(np.hypot(k, l), rel=1e-12)


def test_full_size_matches_oracle(env):
    """The largest grid the shared-memory FFT takes (8192^2), FP32 storage."""
    cs, torch, orc = env
    n = 8192
    c = W.ch_initial(n, seed=9).astype(np.float32).astype(np.float64)
    plan, _ = make_plan(cs, torch, c, 1)
    s, k1 = cs.cs_ch_coarsening(plan)
    cs.cs_destroy(plan)
    assert s == pytest.approx(orc.ch_coarsening_s(c), rel=REL)
    assert k1 == pytest.approx(orc.ch_coarsening_k1(c), rel=REL)


def test_measuring_between_steps_leaves_the_trajectory(env):
    """The measures use the plan's scratch between steps: a run that measures halfway ends
    bit-identical to one that does not."""
    cs, torch, _ = env
    n = 128
    c0 = W.ch_initial(n, seed=3)
    a, fa = make_plan(cs, torch, c0, 0)
    b, fb = make_plan(cs, torch, c0, 0)
    cs.cs_ch_step(a, 10)
    cs.cs_ch_coarsening(a)
    cs.cs_ch_step(a, 10)
    cs.cs_ch_step(b, 20)
    torch.cuda.synchronize()
    ca, cb = current(cs, a, fa), current(cs, b, fb)
    cs.cs_destroy(a)
    cs.cs_destroy(b)
    assert np.array_equal(ca, cb)


def test_not_a_power_of_two_rejected(env):
    cs, torch, _ = env
    plan, _ = make_plan(cs, torch, W.ch_initial(192, seed=1), 0)
    try:
        with pytest.raises(Exception) as e:
            cs.cs_ch_coarsening(plan)
        assert getattr(e.value, "code", None) == cs.CS_EUNSUPPORTED
    finally:
        cs.cs_destroy(plan)


def test_measures_grow_during_coarsening(env):
    """Deep quench at n = 128 to t = 10: after spinodal decomposition both length scales, s and
    1 / k_1, grow (Sec. 5.1)."""
    cs, torch, _ = env
    n = 128
    dt = 0.1 * (2 * np.pi / n)
    plan, _ = make_plan(cs, torch, W.ch_initial(n, seed=21), 0, dt)
    marks = [1.0, 3.0, 10.0]
    done, vals = 0, []
    for t in marks:
        k = int(round(t / dt)) - done
        cs.cs_ch_step(plan, k)
        done += k
        vals.append(cs.cs_ch_coarsening(plan))
    cs.cs_destroy(plan)
    s = [v[0] for v in vals]
    inv_k1 = [1.0 / v[1] for v in vals]
    assert s[0] < s[1] < s[2]
    assert inv_k1[0] < inv_k1[1] < inv_k1[2]
