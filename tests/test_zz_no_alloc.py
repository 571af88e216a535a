"""The allocation-free batched 1D entry point (cs_batch1d_compute_noalloc), through the C ABI.

It serves callers that cannot let a library allocate device memory; its scratch lives in a
fixed device array inside the library.  Its results must equal the plan-based entry point's
(cs_plan_create_1d_batch + cs_compute) on two calls in a row -- the shared array keeps the
previous call's contents -- and it must refuse sizes beyond its fixed maximum and invalid
offsets.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_1902_09931_gb300 as cs
    cs.load()
    return cs, torch


def plan_result(cs, torch, desc, off_d, total, x_d):
    out = torch.zeros_like(x_d)
    plan = cs.cs_plan_create_1d_batch(desc, off_d.numel() - 1, off_d, total, x_d, out)
    cs.cs_compute(plan)
    torch.cuda.synchronize()
    cs.cs_destroy(plan)
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("dtype", [1, 0])
def test_noalloc_matches_plan_two_calls(env, dtype):
    cs, torch = env
    ndt = np.float32 if dtype == 1 else np.float64
    w = np.array([-1.0, 16.0, -30.0, 16.0, -1.0]) / 12.0
    desc = cs.StencilDesc(dir=cs.CS_DIR_X, bc=cs.CS_BC_PERIODIC, dtype=dtype, left=2, right=2, weights=w)
    # two different batches in a row: the second call must not see the first call's table
    for seed, nlines in [(31, 20000), (32, 3000)]:
        off = W.ragged_offsets(nlines, seed=seed)
        x = W.sines_lines(off, seed=seed + 1).astype(ndt)
        off_d = torch.from_numpy(off).cuda()
        x_d = torch.from_numpy(x).cuda()
        total = int(off[-1])
        ref = plan_result(cs, torch, desc, off_d, total, x_d)
        out = torch.zeros_like(x_d)
        cs.cs_batch1d_compute_noalloc(desc, nlines, off_d, total, x_d, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        err = np.abs(got - ref).max() / (np.abs(w).sum() * np.abs(x).max())
        assert err <= TOL[dtype], (seed, err)


def test_noalloc_allocates_no_device_memory(env):
    """The device's free memory is the same before and after a run of calls on a batch shape
    the entry point has not seen (inputs created and the first call made beforehand)."""
    cs, torch = env
    w = np.array([-1.0, 16.0, -30.0, 16.0, -1.0]) / 12.0
    desc = cs.StencilDesc(dir=cs.CS_DIR_X, bc=cs.CS_BC_PERIODIC, dtype=cs.CS_F32, left=2, right=2, weights=w)
    warm = W.ragged_offsets(100, seed=40)
    warm_x = torch.from_numpy(W.sines_lines(warm, seed=41).astype(np.float32)).cuda()
    cs.cs_batch1d_compute_noalloc(desc, 100, torch.from_numpy(warm).cuda(), int(warm[-1]), warm_x,
                                  torch.empty_like(warm_x))
    off = W.ragged_offsets(40000, seed=42)
    off_d = torch.from_numpy(off).cuda()
    x_d = torch.from_numpy(W.sines_lines(off, seed=43).astype(np.float32)).cuda()
    out = torch.empty_like(x_d)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        cs.cs_batch1d_compute_noalloc(desc, 40000, off_d, int(off[-1]), x_d, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_oversize_and_bad_offsets(env):
    cs, torch = env
    w = np.array([1.0, -2.0, 1.0])
    desc = cs.StencilDesc(dir=cs.CS_DIR_X, bc=cs.CS_BC_PERIODIC, dtype=cs.CS_F32, left=1, right=1, weights=w)
    x = torch.ones(64, dtype=torch.float32, device="cuda")
    out = torch.full_like(x, 5.0)
    big = (1 << 26) + 1
    off = torch.tensor([0, big], dtype=torch.int64, device="cuda")
    with pytest.raises(cs.CSError) as e:
        cs.cs_batch1d_compute_noalloc(desc, 1, off, big, x, out)
    assert e.value.code == cs.CS_EINVAL and "maximum" in str(e.value)
    bad = torch.tensor([0, 40, 30, 64], dtype=torch.int64, device="cuda")  # decreasing
    with pytest.raises(cs.CSError) as e:
        cs.cs_batch1d_compute_noalloc(desc, 3, bad, 64, x, out)
    assert e.value.code == cs.CS_EINVAL
    torch.cuda.synchronize()
    assert torch.all(out == 5.0)
    good = torch.tensor([0, 40, 64], dtype=torch.int64, device="cuda")
    cs.cs_batch1d_compute_noalloc(desc, 2, good, 64, x, out)  # the flag was cleared
    torch.cuda.synchronize()
    assert torch.all(out == 0.0)  # second difference of a constant
