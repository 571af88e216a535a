"""Serving loop on the GPU: every job's result is the same alone and in the continuous-batching
mix (grouped sweep launches, overlapping Cahn-Hilliard advances on several streams), and the
results are right against the oracle."""
import copy

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import oracle
    import paper_1902_09931_gb300 as cs
    from paper_1902_09931_gb300 import serving as S
    cs.load()
    return cs, torch, oracle, S


def test_results_identical_alone_and_in_the_mix(env):
    cs, torch, orc, S = env
    jobs = S.poisson_jobs(32, rate=20000.0, seed=9, sizes=(128, 256, 512))
    be = S.GpuBackend(cs, torch, streams=8)
    be.warmup((128, 256, 512), copies=4)
    mix = copy.deepcopy(jobs)
    stats = S.Server(be, max_inflight=12).run(mix)
    torch.cuda.synchronize()
    assert stats["jobs"] == 32 and stats["peak_inflight"] > 1
    assert stats["launches"] < 32  # sweeps were batched into shared launches
    for j in jobs:
        alone = copy.deepcopy(j)
        alone.arrival = 0.0
        S.run_sequential(be, [alone])
        torch.cuda.synchronize()
        got = [m for m in mix if m.jid == j.jid][0]
        assert torch.equal(got.output, alone.output), (j.jid, j.kind, j.n)


def test_served_results_match_oracle(env):
    cs, torch, orc, S = env
    be = S.GpuBackend(cs, torch, streams=4)
    sweep = S.Job(0, "sweep", 256, 0.0, stencil="biharm13", seed=77)
    ch = S.Job(1, "ch", 128, 0.0, steps=10, seed=78)
    S.Server(be, max_inflight=4).run([sweep, ch])
    torch.cuda.synchronize()
    import workloads as W
    x = W.device_uniform((256, 256), 77, -1.0, 1.0, torch.device("cuda"), torch.float32).cpu().numpy().astype(np.float64)
    h = 2 * np.pi / 256
    _, d, L, R, T, B, w = S.sweep_stencil("biharm13", h)
    ref = orc.stencil2d(x, w, d, 1, L, R, T, B)
    err = np.abs(sweep.output.cpu().numpy() - ref).max() / (np.abs(w).sum() * np.abs(x).max())
    assert err <= 1e-5
    c0 = W.device_uniform((128, 128), 78, -0.1, 0.1, torch.device("cuda"), torch.float32)
    c0 = (c0 - c0.mean()).cpu().numpy().astype(np.float64)
    hc = 2 * np.pi / 128
    ref_c, ref_m, ref_e = orc.ch_run(c0, 1.0, 0.01, 0.1 * hc, 10)
    got = ch.output.cpu().numpy().astype(np.float64)
    # an FP32-storage trajectory is compared on its invariants and on s(t), not pointwise: mass is
    # conserved up to two FP32 roundings per point and step (Cbar in the update, the stored
    # result); energy and s follow the FP64 run to the FP32 rounding, grown over t = 10 dt
    scale = hc * hc * np.abs(c0).sum()
    assert abs(orc.ch_mass(got) - orc.ch_mass(c0)) <= 10 * 2 * 2.0 ** -24 * 3 * scale
    assert abs(orc.ch_energy(got, 0.01) - ref_e[-1]) <= 1e-5 * abs(ref_e[-1])
    s_ref = orc.ch_coarsening_s(ref_c)
    assert abs(orc.ch_coarsening_s(got) - s_ref) <= 1e-5 * s_ref


def test_heavy_jobs_in_the_mix_match_alone(env):
    """Two heavy jobs (10-step CH advances of 2048^2, run one at a time on default-priority streams)
    among light ones (on high-priority streams, passing the waiting heavy job): every result is the
    same as the job's run alone, bit for bit, and the heavy jobs did not overlap."""
    cs, torch, orc, S = env
    jobs = [S.Job(0, "ch", 2048, 0.0, seed=501), S.Job(1, "ch", 2048, 0.0, seed=502),
            S.Job(2, "sweep", 512, 0.0, stencil="lap9", seed=503), S.Job(3, "ch", 256, 0.0, seed=504),
            S.Job(4, "sweep", 1024, 0.0, stencil="biharm13", seed=505)]
    be = S.GpuBackend(cs, torch, streams=8)
    mix = copy.deepcopy(jobs)
    S.Server(be, max_inflight=8).run(mix)
    torch.cuda.synchronize()
    h0, h1 = [m for m in mix if m.jid in (0, 1)]
    assert h0.heavy and h1.heavy and h1.start >= h0.done
    for j in jobs:
        alone = copy.deepcopy(j)
        S.run_sequential(be, [alone])
        torch.cuda.synchronize()
        got = [m for m in mix if m.jid == j.jid][0]
        assert torch.equal(got.output, alone.output), (j.jid, j.kind, j.n)
