"""Host-resident 2D plans (Sec. 2's y-tiles, streamed through a bounded ring of device band
slots): results equal the device-resident sweep bit for bit -- every tile of a band stages the
same values, halo rows included -- for every kernel family, both boundary kinds, both storage
types, every tile choice and ragged band counts; non-periodic boundary cells of the host output
stay untouched; device memory stays within the budget whatever the grid's size."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import run2d, stencil_cases

pytestmark = pytest.mark.gpu

MIB = 1 << 20


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import oracle
    import paper_1902_09931_gb300 as cs
    cs.load()
    return cs, torch, oracle


def streamed(cs, torch, u, kw, dtype, budget, out_init=5.0, tile_choice=None, fp64_mode=None, pinned=True):
    ny, nx = u.shape
    tdt = torch.float64 if dtype == cs.CS_F64 else torch.float32
    ndt = np.float64 if dtype == cs.CS_F64 else np.float32
    plan = cs.cs_plan_create_2d_host(cs.StencilDesc(nx=nx, ny=ny, dtype=dtype, **kw), budget)
    try:
        if tile_choice is not None:
            cs.cs_plan_set_tile_choice(plan, tile_choice)
        if fp64_mode is not None:
            cs.cs_plan_set_fp64_mode(plan, fp64_mode)
        rows, held = cs.cs_plan_host_info(plan)
        if pinned:
            h_in = torch.from_numpy(np.ascontiguousarray(u, dtype=ndt)).pin_memory()
            h_out = torch.full((ny, nx), out_init, dtype=tdt).pin_memory()
            cs.cs_compute_host(plan, h_in, h_out)
            out = h_out.numpy().astype(np.float64)
        else:
            h_in = np.ascontiguousarray(u, dtype=ndt)
            h_out = np.full((ny, nx), out_init, dtype=ndt)
            cs.cs_compute_host(plan, h_in.ctypes.data, h_out.ctypes.data)
            out = h_out.astype(np.float64)
    finally:
        cs.cs_destroy(plan)
    return out, rows, held


FAMILIES = ("lap9", "biharm13", "ddx4", "d2y8", "asym3102", "generic5", "box5x5")


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("nx", [300, 301])
def test_streamed_equals_device_sweep(env, dtype, bc, nx):
    """1000 x 300 grid (neither a multiple of the tile), bands of 64 rows: 16 bands through 3
    slots, a ragged last band, wrapped or zero halos at both grid ends; 301 columns make rows that
    are not a multiple of 16 bytes (the element-wise loader)."""
    cs, torch, _ = env
    ny = 1000
    h = 2 * np.pi / nx
    u = W.sines_field(nx, seed=51, ny=ny)
    eb = 8 if dtype == 0 else 4
    budget = 2 * 3 * nx * eb * (64 + 64 + 80)  # exactly one 64-row band per slot
    for name, L, R, T, B, d, w in [c for c in stencil_cases(h) if c[0] in FAMILIES]:
        kw = dict(dir=d, bc=bc, left=L, right=R, top=T, bottom=B, weights=w)
        ref = run2d(cs, torch, u, kw, dtype, out_init=np.full((ny, nx), 5.0))
        got, rows, held = streamed(cs, torch, u, kw, dtype, budget)
        assert rows == 64 and held <= budget
        assert np.array_equal(got, ref), name


@pytest.mark.parametrize("tile_choice", [0, 1, 2])
@pytest.mark.parametrize("dtype", [0, 1])
def test_streamed_every_tile_choice(env, tile_choice, dtype):
    cs, torch, _ = env
    ny, nx = 777, 1024
    h = 2 * np.pi / nx
    u = W.sines_field(nx, seed=52, ny=ny)
    for bc in (0, 1):
        for name, L, R, T, B, d, w in [c for c in stencil_cases(h) if c[0] in ("biharm13", "ddy4", "d2x8")]:
            kw = dict(dir=d, bc=bc, left=L, right=R, top=T, bottom=B, weights=w)
            ref = run2d(cs, torch, u, kw, dtype, out_init=np.full((ny, nx), 5.0), tile_choice=tile_choice)
            got, rows, _ = streamed(cs, torch, u, kw, dtype, 16 * MIB, tile_choice=tile_choice)
            assert np.array_equal(got, ref), (name, bc)


@pytest.mark.parametrize("fn", [2, 3])
def test_streamed_user_functions(env, fn):
    """The compiled-in functions (Laplacian of C^3 - C; C^3 - C - Laplacian C) through the ring,
    FP64 (double-float arithmetic) and FP32."""
    cs, torch, _ = env
    ny, nx = 600, 520
    h = 2 * np.pi / nx
    u = W.sines_field(nx, seed=53, ny=ny)
    coe = [1.0 / h ** 2]
    for dtype in (0, 1):
        for bc in (0, 1):
            kw = dict(dir=2, bc=bc, left=1, right=1, top=1, bottom=1, fn=fn, coe=coe)
            ref = run2d(cs, torch, u, kw, dtype, out_init=np.full((ny, nx), 5.0))
            got, _, _ = streamed(cs, torch, u, kw, dtype, 8 * MIB)
            assert np.array_equal(got, ref), (dtype, bc)


def test_streamed_native_fp64_and_pageable(env):
    cs, torch, _ = env
    ny, nx = 500, 256
    u = W.sines_field(nx, seed=54, ny=ny)
    h = 2 * np.pi / nx
    name, L, R, T, B, d, w = [c for c in stencil_cases(h) if c[0] == "lap9"][0]
    kw = dict(dir=d, bc=1, left=L, right=R, top=T, bottom=B, weights=w)
    ref = run2d(cs, torch, u, kw, 0, fp64_mode=1)
    got, _, _ = streamed(cs, torch, u, kw, 0, 4 * MIB, out_init=0.0, fp64_mode=1, pinned=False)
    assert np.array_equal(got, ref)


def test_streamed_matches_oracle(env):
    cs, torch, orc = env
    ny, nx = 300, 200
    u = W.sines_field(nx, seed=55, ny=ny)
    h = 2 * np.pi / nx
    name, L, R, T, B, d, w = [c for c in stencil_cases(h) if c[0] == "biharm13"][0]
    for bc in (0, 1):
        kw = dict(dir=d, bc=bc, left=L, right=R, top=T, bottom=B, weights=w)
        got, _, _ = streamed(cs, torch, u, kw, 0, 2 * MIB, out_init=0.0)
        ref = orc.stencil2d(u, w, d, bc, L, R, T, B)
        scale = np.abs(w).sum() * np.abs(u).max()
        if bc == 0:  # untouched cells: the output's initial zeros, as the oracle leaves them
            assert np.all(got[:T] == 0) and np.all(got[ny - B:] == 0)
            assert np.all(got[:, :L] == 0) and np.all(got[:, nx - R:] == 0)
        assert np.abs(got - ref).max() <= 1e-12 * scale


def test_full_size_streamed_equals_device_sweep(env):
    """8192^2 FP64, 13-point biharmonic (the suite's heaviest digit kernel), 128 MiB of slots
    (43 bands of 192 rows)."""
    cs, torch, _ = env
    n = 8192
    h = 2 * np.pi / n
    u = W.sines_field(n, seed=56)
    name, L, R, T, B, d, w = [c for c in stencil_cases(h) if c[0] == "biharm13"][0]
    kw = dict(dir=d, bc=1, left=L, right=R, top=T, bottom=B, weights=w)
    ref = run2d(cs, torch, u, kw, 0)
    got, rows, held = streamed(cs, torch, u, kw, 0, 128 * MIB)
    assert held <= 128 * MIB and rows < n
    assert np.array_equal(got, ref)


def test_grid_larger_than_device_memory_plans_within_budget(env):
    """A 2^23 x 8192 FP64 grid (512 GiB per field, more than the GPU holds) gets a plan whose
    device memory is the budget alone."""
    cs, torch, _ = env
    free0, total = torch.cuda.mem_get_info()
    ny, nx = 1 << 23, 8192
    assert ny * nx * 8 > total
    kw = dict(dir=2, bc=1, left=1, right=1, top=1, bottom=1, weights=[0, 1, 0, 1, -4, 1, 0, 1, 0.0])
    plan = cs.cs_plan_create_2d_host(cs.StencilDesc(nx=nx, ny=ny, dtype=0, **kw), 256 * MIB)
    try:
        rows, held = cs.cs_plan_host_info(plan)
        assert held <= 256 * MIB and rows % 64 == 0 and rows >= 64
        with pytest.raises(Exception) as e:  # no device buffers to compute on
            cs.cs_compute(plan)
        assert getattr(e.value, "code", None) == cs.CS_EINVAL
    finally:
        cs.cs_destroy(plan)
