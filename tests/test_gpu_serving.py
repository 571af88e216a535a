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
    ref_c, _, _ = orc.ch_run(c0, 1.0, 0.01, 0.1 * 2 * np.pi / 128, 10)
    got = ch.output.cpu().numpy().astype(np.float64)
    assert np.abs(got - ref_c).max() <= 1e-4 * max(1.0, np.abs(ref_c).max())
