"""GPU parity of the periodic XY WENO advection (Sec. 4.2 "Advection") against the oracle,
through the C ABI.

Tolerance: the output is a sum of u times a convex combination of candidates that are O(1)
combinations of the one-sided differences, so both sides are held to
    |a_gpu - a_oracle| <= tol * (max|u| max|D C|_x + max|v| max|D C|_y),
D C the one-sided differences over h, tol = 1e-12 (FP64) or 1e-5 (FP32, FP32 arithmetic on the
same FP32 inputs the oracle widens)."""
import numpy as np
import pytest

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


def scale_of(c, u, v, hx, hy):
    dx = np.abs(np.roll(c, -1, axis=1) - c).max() / hx
    dy = np.abs(np.roll(c, -1, axis=0) - c).max() / hy
    return np.abs(u).max() * dx + np.abs(v).max() * dy


def run(cs, torch, c, u, v, hx, hy, dtype, offset=0, graph=False):
    tdt = torch.float64 if dtype == 0 else torch.float32
    ny, nx = c.shape
    n = nx * ny

    def dev(a):
        buf = torch.zeros(n + offset, dtype=tdt, device="cuda")
        buf[offset:] = torch.from_numpy(np.ascontiguousarray(a).ravel()).to(tdt)
        return buf

    bc, bu, bv, bo = dev(c), dev(u), dev(v), torch.full((n + offset,), 7.0, dtype=tdt, device="cuda")
    es = bc.element_size()
    ptr = lambda t: t.data_ptr() + offset * es
    plan = cs.cs_plan_create_weno_adv(nx, ny, dtype, hx, hy, ptr(bc), ptr(bu), ptr(bv), ptr(bo))
    try:
        if graph:
            cs.cs_plan_use_graph(plan, True)
            cs.cs_compute(plan)
        cs.cs_compute(plan)
        torch.cuda.synchronize()
    finally:
        cs.cs_destroy(plan)
    return bo[offset:].cpu().numpy().astype(np.float64).reshape(ny, nx)


def fields(ny, nx, seed, kind):
    rng = np.random.default_rng(seed)
    hx, hy = 2 * np.pi / nx, 2 * np.pi / ny
    x = np.arange(nx) * hx
    y = np.arange(ny) * hy
    X, Y = np.meshgrid(x, y)
    if kind == "smooth":
        c = np.sin(X + 0.3) * np.cos(2 * Y) + 0.5 * np.cos(3 * X - Y)
    elif kind == "random":
        c = rng.uniform(-1, 1, (ny, nx))
    else:  # a disc of 1 in 0 plus noise: weights far from optimal along its edge
        c = ((X - np.pi) ** 2 + (Y - np.pi) ** 2 < 2.0).astype(np.float64) + 1e-3 * rng.uniform(-1, 1, (ny, nx))
    u = np.cos(Y) + 0.3 * rng.uniform(-1, 1, (ny, nx))
    v = np.sin(X) - 0.1 + 0.3 * rng.uniform(-1, 1, (ny, nx))
    u[:, nx // 3] = 0.0  # zero velocity: the term vanishes either way
    v[ny // 2, :] = 0.0
    return c, u, v, hx, hy


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("shape", [(32, 64), (100, 77), (5, 3), (300, 520), (67, 1030)])
@pytest.mark.parametrize("kind", ["smooth", "random", "disc"])
def test_matches_oracle(env, dtype, shape, kind):
    cs, torch, orc = env
    c, u, v, hx, hy = fields(*shape, seed=sum(shape), kind=kind)
    if dtype == 1:
        c, u, v = (a.astype(np.float32).astype(np.float64) for a in (c, u, v))
    got = run(cs, torch, c, u, v, hx, hy, dtype)
    ref = orc.weno_advection(c, u, v, hx, hy)
    assert np.abs(got - ref).max() <= TOL[dtype] * scale_of(c, u, v, hx, hy)


@pytest.mark.parametrize("mag", [1e-170, 1e-40, 1e40, 1e60])
def test_extreme_magnitudes_fp64(env, mag):
    """Tiny fields reach the branch where eps's floor outweighs every indicator (weights equal
    the optimal ones); large ones exercise the power-of-two scaling (the oracle's plain formula,
    which squares the indicators, stays finite up to differences of about 1e75)."""
    cs, torch, orc = env
    c, u, v, hx, hy = fields(64, 96, seed=3, kind="disc")
    c = c * mag
    got = run(cs, torch, c, u, v, hx, hy, 0)
    ref = orc.weno_advection(c, u, v, hx, hy)
    assert np.abs(got - ref).max() <= 1e-12 * scale_of(c, u, v, hx, hy)


@pytest.mark.parametrize("dtype", [0, 1])
def test_unaligned_buffers_and_graph_replay(env, dtype):
    """Buffers one element off 16-byte alignment (u and v then read per row from global memory)
    give the same bits as aligned ones (whole 128 x 32 tiles staged in shared memory, the last
    tile column read per row), plain and graph-replayed."""
    cs, torch, orc = env
    c, u, v, hx, hy = fields(70, 260, seed=9, kind="random")
    if dtype == 1:
        c, u, v = (a.astype(np.float32).astype(np.float64) for a in (c, u, v))
    ref = orc.weno_advection(c, u, v, hx, hy)
    a = run(cs, torch, c, u, v, hx, hy, dtype, offset=1)
    b = run(cs, torch, c, u, v, hx, hy, dtype, graph=True)
    d = run(cs, torch, c, u, v, hx, hy, dtype)
    assert np.array_equal(a, d) and np.array_equal(b, d)
    assert np.abs(d - ref).max() <= TOL[dtype] * scale_of(c, u, v, hx, hy)


def test_constant_field_and_zero_velocity(env):
    cs, torch, _ = env
    c = np.full((40, 72), 0.37)
    _, u, v, hx, hy = fields(40, 72, seed=1, kind="random")
    assert np.all(run(cs, torch, c, u, v, hx, hy, 0) == 0.0)
    c2, _, _, _, _ = fields(40, 72, seed=2, kind="random")
    assert np.all(run(cs, torch, c2, 0 * u, 0 * v, hx, hy, 0) == 0.0)


@pytest.mark.parametrize("dtype", [0, 1])
def test_full_size_sampled_rows(env, dtype):
    """8192^2, sampled 16-row blocks at both periodic ends and in the middle: the oracle runs on
    each block with a 3-row wrapped halo and the block's interior rows are compared."""
    cs, torch, orc = env
    n = 8192
    rng = np.random.default_rng(81)
    h = 2 * np.pi / n
    x = np.arange(n) * h
    c = (np.sin(3 * x)[None, :] * np.cos(5 * x)[:, None] + 0.01 * rng.uniform(-1, 1, (n, n)))
    c[4000:4200, 3000:3300] += 1.0  # an edge
    u = np.cos(x)[:, None] + 0.1 * rng.uniform(-1, 1, (n, n))
    v = np.sin(x)[None, :] - 0.2 + 0.1 * rng.uniform(-1, 1, (n, n))
    if dtype == 1:
        c, u, v = (a.astype(np.float32).astype(np.float64) for a in (c, u, v))
    got = run(cs, torch, c, u, v, h, h, dtype)
    sc = scale_of(c, u, v, h, h)
    for j0 in (0, 4090, n - 16):
        rows = np.arange(j0 - 3, j0 + 16 + 3) % n
        blk = lambda a: a[rows]
        ref = orc.weno_advection(blk(c), blk(u), blk(v), h, h)[3:-3]
        assert np.abs(got[j0:j0 + 16] - ref).max() <= TOL[dtype] * sc, j0


def test_homogeneous_beyond_the_oracles_range(env):
    """Scaling C by 2^498 (differences near 1e150, where the plain formula overflows) scales the
    term by 2^498: the kernel's weights see the same scaled differences, up to eps's floor."""
    cs, torch, _ = env
    c, u, v, hx, hy = fields(64, 96, seed=4, kind="disc")
    a = run(cs, torch, c, u, v, hx, hy, 0)
    b = run(cs, torch, c * 2.0 ** 498, u, v, hx, hy, 0)
    assert np.all(np.isfinite(b))
    assert np.abs(b * 2.0 ** -498 - a).max() <= 1e-12 * scale_of(c, u, v, hx, hy)


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("h", [1e-30, 1e30])
def test_extreme_grid_spacings(env, dtype, h):
    """eps's floor is 1e-99 in units of the differences over h: scaled by h^2 where the kernel
    works on differences, so very fine and very coarse spacings keep their weights."""
    cs, torch, orc = env
    c, u, v, _, _ = fields(64, 96, seed=12, kind="disc")
    if dtype == 1:
        c, u, v = (a.astype(np.float32).astype(np.float64) for a in (c, u, v))
    got = run(cs, torch, c, u, v, h, 2 * h, dtype)
    ref = orc.weno_advection(c, u, v, h, 2 * h)
    assert np.abs(got - ref).max() <= TOL[dtype] * scale_of(c, u, v, h, 2 * h)
