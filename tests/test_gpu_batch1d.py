"""GPU parity of the ragged batched 1D stencil against the CPU oracle, through the C ABI.

Integer data is bit-exact (index maps: per-line periodic wrap, non-periodic clipping, short and
empty lines, warp segments straddling line ends); sine data meets 1e-12 (FP64) / 1e-5 (FP32)
scaled by sum |w| * max |in|.  The full 65536-line workload is compared element by element.
"""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import D2_4

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import oracle
    import paper_1902_09931_gb300 as cs
    cs.load()
    return cs, torch, oracle


def run_batch(cs, torch, packed, offsets, dtype, bc, L, R, w, out_init=None, graph=False, reps=1,
              autotune=False):
    ndt = np.float64 if dtype == 0 else np.float32
    d_in = torch.from_numpy(np.ascontiguousarray(packed, dtype=ndt)).cuda()
    d_out = torch.zeros_like(d_in) if out_init is None else torch.from_numpy(np.ascontiguousarray(out_init, dtype=ndt)).cuda()
    d_off = torch.from_numpy(np.ascontiguousarray(offsets, dtype=np.int64)).cuda()
    desc = cs.StencilDesc(dir=cs.CS_DIR_X, bc=bc, dtype=dtype, left=L, right=R, weights=w)
    plan = cs.cs_plan_create_1d_batch(desc, offsets.size - 1, d_off, int(offsets[-1]), d_in, d_out)
    try:
        if autotune:
            cs.cs_autotune(plan)
        if graph:
            cs.cs_plan_use_graph(plan, True)
        for _ in range(reps):
            cs.cs_compute(plan)
        torch.cuda.synchronize()
    finally:
        cs.cs_destroy(plan)
    return d_out.cpu().numpy().astype(np.float64)


def mixed_offsets(seed):
    """Short, empty and long lines mixed, so warp segments straddle many line ends."""
    g = np.random.Generator(np.random.PCG64(seed))
    lengths = np.concatenate([g.integers(0, 9, 120), g.integers(60, 700, 40), [1, 2, 3, 4, 5, 0, 0, 4096]])
    g.shuffle(lengths)
    return np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("ext", [(2, 2), (1, 1), (2, 1), (0, 2), (0, 0), (3, 1), (0, 4), (6, 5)])
def test_integer_bit_exact(env, dtype, bc, ext):
    cs, torch, orc = env
    L, R = ext
    off = mixed_offsets(L * 10 + R)
    u = W.integer_field(1, int(off[-1]), seed=3).ravel()
    w = W.integer_weights(L + R + 1, seed=L + R)
    sentinel = np.full(u.shape, 777.0)
    got = run_batch(cs, torch, u, off, dtype, bc, L, R, w, out_init=sentinel)
    ref = orc.stencil1d_batch(u, off, w, bc, L, R, out=sentinel)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("bc", [0, 1])
def test_sines_match_oracle(env, dtype, bc):
    cs, torch, orc = env
    off = W.ragged_offsets(3000, seed=5)
    u = W.sines_lines(off, seed=6)
    if dtype == 1:
        u = u.astype(np.float32).astype(np.float64)
    got = run_batch(cs, torch, u, off, dtype, bc, 2, 2, D2_4)
    ref = orc.stencil1d_batch(u, off, D2_4, bc, 2, 2)
    assert np.abs(got - ref).max() / (np.abs(D2_4).sum() * np.abs(u).max()) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [1, 0])
def test_full_workload_persistent_graph_autotuned(env, dtype):
    """65536 lines, lengths log-uniform in [64, 4096], radius-2 4th-order second derivative,
    periodic, one persistent launch replayed from a CUDA graph after autotuning."""
    cs, torch, orc = env
    off = W.ragged_offsets(65536, seed=2019)
    u = W.sines_lines(off, seed=2020)
    if dtype == 1:
        u = u.astype(np.float32).astype(np.float64)
    got = run_batch(cs, torch, u, off, dtype, 1, 2, 2, D2_4, graph=True, reps=2, autotune=True)
    ref = orc.stencil1d_batch(u, off, D2_4, 1, 2, 2)
    assert np.abs(got - ref).max() / (np.abs(D2_4).sum() * np.abs(u).max()) <= TOL[dtype]


def test_empty_batch_and_single_line(env):
    cs, torch, orc = env
    off = np.array([0, 5], dtype=np.int64)
    u = np.arange(5, dtype=float)
    w = np.array([1.0, 10.0, 100.0])
    got = run_batch(cs, torch, u, off, 0, 1, 1, 1, w)
    assert np.array_equal(got, orc.stencil1d_batch(u, off, w, 1, 1, 1))
