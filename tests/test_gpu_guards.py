"""Out-of-bounds write checks for every kernel family, through the C ABI.

Every device buffer a kernel receives sits between two guard regions filled with a NaN bit
pattern (and inputs are compared with their own copies afterwards): after the launches the
guards must hold that pattern bit for bit and the inputs must be unchanged.  A write past either
end of an output, or into an input, fails.  The buffers start at an offset of 0 or 1 element
past a 32-byte boundary, so both the aligned (vector, TMA, 32-byte) paths and the element-wise
fallbacks are covered.  Shapes are ragged: partial tiles on both axes, grids smaller than the
stencil, single rows.
"""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import stencil_cases

pytestmark = pytest.mark.gpu

GUARD = 4096  # elements on each side
SENT = {8: 0x7FF4DEADBEEFCAFE, 4: 0x7FA5CAFE}  # quiet NaNs with a payload, by element size


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_1902_09931_gb300 as cs
    cs.load()
    return cs, torch


class Guarded:
    """A device buffer of n elements at element offset `off` inside guard regions."""

    def __init__(self, torch, n, dtype, off=0, init=None):
        self.torch, self.n, self.off = torch, n, off
        self.buf = torch.empty(n + off + 2 * GUARD, dtype=dtype, device="cuda")
        self.es = self.buf.element_size()
        self.ibuf = self.buf.view(torch.int64 if self.es == 8 else torch.int32)
        self.ibuf.fill_(SENT[self.es])
        self.t = self.buf[GUARD + off:GUARD + off + n]
        if init is not None:
            self.t.copy_(torch.as_tensor(np.ascontiguousarray(init).ravel()).to(dtype))
        self.before = self.t.clone()

    def view(self, *shape):
        return self.t.view(*shape)

    def guards_ok(self) -> bool:
        s = SENT[self.es]
        head = self.ibuf[:GUARD + self.off]
        tail = self.ibuf[GUARD + self.off + self.n:]
        return bool((head == s).all().item()) and bool((tail == s).all().item())

    def unchanged(self) -> bool:
        return bool(self.torch.equal(self.t.view(self.ibuf.dtype), self.before.view(self.ibuf.dtype)))


def run_stencil(cs, torch, field, kw, dtype, off, tile_choice):
    ny, nx = field.shape
    tdt = torch.float64 if dtype == cs.CS_F64 else torch.float32
    gin = Guarded(torch, nx * ny, tdt, off, field)
    gout = Guarded(torch, nx * ny, tdt, off, np.full(field.shape, 3.0))
    plan = cs.cs_plan_create_2d(cs.StencilDesc(nx=nx, ny=ny, dtype=dtype, **kw), gin.view(ny, nx), gout.view(ny, nx))
    try:
        cs.cs_plan_set_tile_choice(plan, tile_choice)
        cs.cs_compute(plan)
        torch.cuda.synchronize()
        cs.cs_plan_check(plan)
    finally:
        cs.cs_destroy(plan)
    return gin, gout


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("shape", [(130, 300), (67, 517), (45, 7), (1, 200), (256, 384), (3, 2)])
@pytest.mark.parametrize("off", [0, 1])
def test_stencil_writes_stay_inside_the_output(env, dtype, bc, shape, off):
    cs, torch = env
    ny, nx = shape
    h = 2 * np.pi / max(nx, 8)
    field = W.sines_field(nx, seed=nx + 3 * ny, ny=ny)
    cases = list(stencil_cases(h)) + [("fn1", 1, 1, 0, 0, 0, None), ("fn2", 1, 1, 1, 1, 2, None),
                                     ("fn3", 1, 1, 1, 1, 2, None)]
    for name, L, R, T, B, d, w in cases:
        if d == 0 and (T or B):
            continue
        if w is None:
            kw = dict(dir=d, bc=bc, left=L, right=R, top=T, bottom=B, fn=int(name[-1]), coe=[1 / h ** 2])
        else:
            kw = dict(dir=d, bc=bc, left=L, right=R, top=T, bottom=B, weights=w)
        for choice in (0, 1, 2):
            gin, gout = run_stencil(cs, torch, field, kw, dtype, off, choice)
            assert gout.guards_ok(), (name, choice)
            assert gin.guards_ok() and gin.unchanged(), (name, choice)


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("off", [0, 1])
def test_grouped_launch_writes_stay_inside_the_outputs(env, dtype, off):
    cs, torch = env
    tdt = torch.float64 if dtype == cs.CS_F64 else torch.float32
    h = 2 * np.pi / 64
    w = np.array([1, 4, 1, 4, -20, 4, 1, 4, 1.0]) / (6 * h * h)
    shapes = [(33, 70), (64, 64), (5, 200), (130, 67), (1, 9)]
    bufs, plans = [], []
    for i, (ny, nx) in enumerate(shapes):
        gin = Guarded(torch, nx * ny, tdt, off, W.sines_field(nx, seed=i, ny=ny))
        gout = Guarded(torch, nx * ny, tdt, off)
        desc = cs.StencilDesc(nx=nx, ny=ny, dtype=dtype, dir=cs.CS_DIR_XY, bc=i % 2, left=1, right=1, top=1,
                              bottom=1, weights=w)
        plans.append(cs.cs_plan_create_2d(desc, gin.view(ny, nx), gout.view(ny, nx)))
        bufs.append((gin, gout))
    try:
        cs.cs_compute_group(plans)
        torch.cuda.synchronize()
    finally:
        for p in plans:
            cs.cs_destroy(p)
    for gin, gout in bufs:
        assert gout.guards_ok() and gin.guards_ok() and gin.unchanged()


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("off", [0, 1])
def test_batch1d_writes_stay_inside_the_output(env, dtype, bc, off):
    cs, torch = env
    tdt = torch.float64 if dtype == cs.CS_F64 else torch.float32
    rng = np.random.default_rng(5 + off)
    lengths = np.concatenate([rng.integers(1, 300, size=200), [1, 2, 3, 4, 5, 4096, 63, 65]])
    offsets = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    total = int(offsets[-1])
    gin = Guarded(torch, total, tdt, off, rng.uniform(-1, 1, total))
    gout = Guarded(torch, total, tdt, off)
    goff = Guarded(torch, offsets.size, torch.int64, 0, offsets)
    h = 0.01
    for L, R, w in [(2, 2, np.array([-1, 16, -30, 16, -1.0]) / (12 * h * h)), (1, 1, np.array([1, -2, 1.0])),
                    (4, 4, rng.uniform(-1, 1, 9))]:
        desc = cs.StencilDesc(dir=cs.CS_DIR_X, bc=bc, dtype=dtype, left=L, right=R, weights=w)
        plan = cs.cs_plan_create_1d_batch(desc, offsets.size - 1, goff.t, total, gin.t, gout.t)
        try:
            cs.cs_compute(plan)
            torch.cuda.synchronize()
        finally:
            cs.cs_destroy(plan)
        assert gout.guards_ok(), (L, R)
        assert gin.guards_ok() and gin.unchanged() and goff.guards_ok() and goff.unchanged()


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("shape", [(32, 64), (100, 77), (5, 3), (67, 1030), (256, 384)])
@pytest.mark.parametrize("off", [0, 1])
def test_weno_writes_stay_inside_the_output(env, dtype, shape, off):
    cs, torch = env
    tdt = torch.float64 if dtype == cs.CS_F64 else torch.float32
    ny, nx = shape
    rng = np.random.default_rng(nx * ny + off)
    g = [Guarded(torch, nx * ny, tdt, off, rng.uniform(-1, 1, nx * ny)) for _ in range(3)]
    gout = Guarded(torch, nx * ny, tdt, off)
    plan = cs.cs_plan_create_weno_adv(nx, ny, dtype, 2 * np.pi / nx, 2 * np.pi / ny, g[0].t, g[1].t, g[2].t, gout.t)
    try:
        cs.cs_compute(plan)
        torch.cuda.synchronize()
    finally:
        cs.cs_destroy(plan)
    assert gout.guards_ok()
    assert all(x.guards_ok() and x.unchanged() for x in g)


@pytest.mark.parametrize("storage", [0, 1])
@pytest.mark.parametrize("boundary", [0, 1])
@pytest.mark.parametrize("n", [64, 128, 256])
def test_ch_step_writes_stay_inside_its_fields(env, storage, boundary, n):
    """Seven steps (one more than two 3-step graphs), with the invariants read back every step,
    then the coarsening measures of a periodic grid: only the three fields are written."""
    cs, torch = env
    tdt = torch.float64 if storage == cs.CS_F64 else torch.float32
    c0 = W.ch_initial(n, seed=n + boundary)
    f = [Guarded(torch, n * n, tdt, 0, c0), Guarded(torch, n * n, tdt, 0, c0), Guarded(torch, n * n, tdt, 0)]
    h = 2 * np.pi / n
    plan = cs.cs_ch_create(cs.CHDesc(n=n, storage=storage, D=1.0, gamma=0.01, dt=0.1 * h, boundary=boundary),
                           *[g.view(n, n) for g in f])
    try:
        cs.cs_ch_step(plan, 7, invariants=True)
        cs.cs_ch_step(plan, 5)
        if boundary == cs.CS_CH_PERIODIC:
            cs.cs_ch_coarsening(plan)
        torch.cuda.synchronize()
    finally:
        cs.cs_destroy(plan)
    assert all(g.guards_ok() for g in f)
