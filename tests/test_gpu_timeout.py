"""Failure detection of the TMA-pipelined sweep: a bounded mbarrier wait that runs out is
reported by cs_plan_check as CS_ETIMEOUT (per plan), the output cells it could not write keep
their contents, and the plan works again once the stall is lifted.

The wait is made to run out the safe way (cs_plan_debug_stall): from a given CTA-local tile on,
the sweep issues no copies, so each CTA waits on a barrier nothing will complete, with no copy in
flight, and returns after its short bounded wait.  Nothing faults or hangs."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import lap9

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_1902_09931_gb300 as cs
    cs.load()
    return cs, torch


def make(cs, torch, n, dtype, seed):
    tdt = torch.float64 if dtype == cs.CS_F64 else torch.float32
    x = torch.from_numpy(W.sines_field(n, seed=seed)).to("cuda", tdt)
    y = torch.full_like(x, float("nan"))
    h = 2 * np.pi / n
    desc = cs.StencilDesc(nx=n, ny=n, dir=cs.CS_DIR_XY, bc=cs.CS_BC_PERIODIC, dtype=dtype,
                          left=1, right=1, top=1, bottom=1, weights=lap9(h))
    plan = cs.cs_plan_create_2d(desc, x, y)
    cs.cs_plan_set_tile_choice(plan, 2)
    return plan, x, y


@pytest.mark.parametrize("dtype", [0, 1])
def test_timeout_reported_per_plan_and_recovered(env, dtype):
    cs, torch = env
    n = 4096
    ref_plan, x, y_ref = make(cs, torch, n, dtype, seed=31)
    cs.cs_compute(ref_plan)
    cs.cs_plan_check(ref_plan)  # a full sweep: no wait ran out
    assert not torch.isnan(y_ref).any()

    plan, x2, y = make(cs, torch, n, dtype, seed=31)
    other, _, y_other = make(cs, torch, 512, dtype, seed=32)
    cs.cs_plan_debug_stall(plan, 1)  # every CTA computes its first tile, then its wait runs out
    cs.cs_compute(plan)
    cs.cs_compute(other)
    cs.cs_plan_check(other)  # the other plan's count is its own
    with pytest.raises(cs.CSError) as e:
        cs.cs_plan_check(plan)
    assert e.value.code == cs.CS_ETIMEOUT
    cs.cs_plan_check(plan)  # the count was consumed by the check
    written = ~torch.isnan(y)
    frac = written.double().mean().item()
    assert 0.0 < frac < 1.0, frac  # the first tile of each CTA only
    assert torch.equal(y[written], y_ref[written])  # what was written is right

    cs.cs_plan_debug_stall(plan, -1)
    cs.cs_compute(plan)
    cs.cs_plan_check(plan)
    assert torch.equal(y, y_ref)
    for p in (ref_plan, plan, other):
        cs.cs_destroy(p)


def test_compute_host_reports_timeout(env):
    cs, torch = env
    n = 2048
    plan, x, y = make(cs, torch, n, 1, seed=33)
    h_in = x.cpu().pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    cs.cs_plan_debug_stall(plan, 0)  # no tile is copied at all
    with pytest.raises(cs.CSError) as e:
        cs.cs_compute_host(plan, h_in, h_out)
    assert e.value.code == cs.CS_ETIMEOUT
    cs.cs_plan_debug_stall(plan, -1)
    cs.cs_compute_host(plan, h_in, h_out)
    ref = torch.empty_like(y)
    cs.cs_set_buffers(plan, x, ref)
    cs.cs_compute(plan)
    cs.cs_plan_check(plan)
    assert torch.equal(h_out, ref.cpu())
    cs.cs_destroy(plan)
