"""GPU parity of the 2D stencil sweep against the CPU oracle, through the C ABI.

Tolerances: max |gpu - oracle| / (sum |w| * max |in|) <= 1e-12 for
FP64 storage and <= 1e-5 for FP32 storage (the oracle reads the same FP32 inputs widened to
FP64).  Integer-valued data with small-integer weights makes every sum exact in both precisions,
so the index and halo maps must then match bit for bit.  Non-periodic runs pre-fill the output
with a sentinel that must survive bit for bit outside the written interior.
"""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import run2d, scaled_err, stencil_cases, biharm13, lap5, lap9, D1_4

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


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("shape", [(130, 300), (67, 517), (1, 200), (45, 7)])
def test_all_stencil_variants_match_oracle(env, dtype, bc, shape):
    cs, torch, orc = env
    ny, nx = shape
    h = 2 * np.pi / nx
    field = W.sines_field(nx, seed=nx + ny, ny=ny)
    if dtype == 1:
        field = field.astype(np.float32).astype(np.float64)
    sentinel = np.full(shape, -2.0 ** 120)  # exactly representable in FP32 and FP64
    for name, L, R, T, B, d, w in stencil_cases(h):
        if d == 0 and (T or B):
            continue
        kw = dict(dir=d, bc=bc, left=L, right=R, top=T, bottom=B, weights=w)
        got = run2d(cs, torch, field, kw, dtype, out_init=sentinel)
        ref = orc.stencil2d(field, w, d, bc, L, R, T, B, out=sentinel)
        written = np.ones(shape, bool)
        if bc == 0:
            written[:] = False
            written[T:ny - B, L:nx - R] = True
            assert np.array_equal(got[~written], ref[~written]), name  # untouched cells
        if written.any():
            err = scaled_err(got[written], ref[written], w, field)
            assert err <= TOL[dtype], (name, err)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("bc", [0, 1])
def test_fp64_double_float_and_native_match_oracle(env, mode, bc):
    """FP64 storage in both arithmetic modes (double-float on the FP32 pipes, native FP64) on
    every specialised stencil, against the oracle at the FP64 tolerance."""
    cs, torch, orc = env
    ny, nx = 150, 260
    h = 2 * np.pi / nx
    field = W.sines_field(nx, seed=17, ny=ny)
    for name, L, R, T, B, d, w in stencil_cases(h):
        kw = dict(dir=d, bc=bc, left=L, right=R, top=T, bottom=B, weights=w)
        got = run2d(cs, torch, field, kw, 0, fp64_mode=mode)
        ref = orc.stencil2d(field, w, d, bc, L, R, T, B)
        written = np.zeros(field.shape, bool)
        written[T:ny - B, L:nx - R] = True
        if bc == 1:
            written[:] = True
        assert scaled_err(got[written], ref[written], w, field) <= 1e-12, (name, mode)


@pytest.mark.parametrize("case", ["huge", "tiny", "subnormal", "tiny_tile", "weights"])
def test_double_float_falls_back_outside_its_range(env, case):
    """Tiles holding values outside the double-float range, tiles whose values are all tiny,
    and weights outside the range are computed exactly as in native FP64."""
    cs, torch, orc = env
    ny, nx = 140, 200
    h = 2 * np.pi / nx
    field = W.sines_field(nx, seed=23, ny=ny)
    w = biharm13(h)
    if case == "huge":
        field[70, 100] = 3.0e25
    elif case == "tiny":
        field[10:20, 10:20] *= 1e-30
    elif case == "subnormal":
        field[5, 5] = 4.9e-320
    elif case == "tiny_tile":
        field[:64, :64] = W.uniform_field(64, 64, seed=2) * 1e-12
    else:
        w = w * 1e-25
    kw = dict(dir=2, bc=1, left=2, right=2, top=2, bottom=2, weights=w)
    got = run2d(cs, torch, field, kw, 0)
    ref = orc.stencil2d(field, w, 2, 1, 2, 2, 2, 2)
    assert scaled_err(got, ref, w, field) <= 1e-12
    if case == "tiny_tile":
        # native FP64 keeps every output accurate on its own neighbourhood's scale; the fast
        # paths are bounded by the largest value a tile (with its halo) holds
        nat = run2d(cs, torch, field, kw, 0, fp64_mode=1)
        blk = (slice(2, 62), slice(2, 62))
        assert scaled_err(nat[blk], ref[blk], w, field[:64, :64]) <= 1e-12


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 16, 17, 64, 255])
@pytest.mark.parametrize("ext", [(0, 0, 0, 0), (1, 1, 1, 1), (3, 0, 1, 2), (2, 3, 3, 2), (2, 2, 0, 0), (0, 0, 2, 2)])
def test_integer_data_bit_exact(env, dtype, bc, n, ext):
    """Index and halo maps (periodic wrap of any multiplicity, non-periodic clipping) are exact."""
    cs, torch, orc = env
    L, R, T, B = ext
    field = W.integer_field(n, n + 3, seed=n)
    w = W.integer_weights((L + R + 1) * (T + B + 1), seed=L + 7 * R + 49 * T + 343 * B)
    d = 2 if (T or B) and (L or R) else (1 if (T or B) else 0)
    sentinel = np.full(field.shape, 12345.0)
    got = run2d(cs, torch, field, dict(dir=d, bc=bc, left=L, right=R, top=T, bottom=B, weights=w),
                dtype, out_init=sentinel)
    ref = orc.stencil2d(field, w, d, bc, L, R, T, B, out=sentinel)
    assert np.array_equal(got, ref)


BIHARM_N = np.array([0, 0, 1, 0, 0, 0, 2, -8, 2, 0, 1, -8, 20, -8, 1, 0, 2, -8, 2, 0, 0, 0, 1, 0, 0], float)


@pytest.mark.parametrize("sign", [1.0, -1.0])
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("tile_choice", [0, 1])
@pytest.mark.parametrize("shape", [(1, 1), (3, 5), (17, 64), (67, 130), (130, 67), (256, 384)])
def test_biharmonic_digits_bit_exact(env, sign, bc, tile_choice, shape):
    """FP64 weights c (1, 2, -8, 20) and their negatives on the 13-point footprint (the digit
    path's integer ratios n_k); on integer data every sum is exact, so the output equals the
    oracle's bit for bit in both tile heights: edge tiles, periodic wrap of grids smaller than the
    footprint, and the cells a non-periodic sweep leaves untouched."""
    cs, torch, orc = env
    ny, nx = shape
    field = W.integer_field(ny, nx, seed=ny * 1000 + nx)
    w = sign * 0.25 * BIHARM_N
    sentinel = np.full(shape, 12345.0)
    kw = dict(dir=2, bc=bc, left=2, right=2, top=2, bottom=2, weights=w)
    got = run2d(cs, torch, field, kw, 0, out_init=sentinel, tile_choice=tile_choice)
    ref = orc.stencil2d(field, w, 2, bc, 2, 2, 2, 2, out=sentinel)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("dtype", [0, 1])
def test_impulse_gives_flipped_stencil(env, dtype):
    cs, torch, orc = env
    L, R, T, B = 2, 1, 0, 3
    w = np.arange(1, (L + R + 1) * (T + B + 1) + 1, dtype=float)
    u = np.zeros((20, 30))
    u[9, 12] = 1.0
    got = run2d(cs, torch, u, dict(dir=2, bc=1, left=L, right=R, top=T, bottom=B, weights=w), dtype)
    expect = np.zeros_like(u)
    for q in range(T + B + 1):
        for p in range(L + R + 1):
            expect[9 + T - q, 12 + L - p] = w[q * (L + R + 1) + p]
    assert np.array_equal(got, expect)


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("fn", [1, 2, 3])
@pytest.mark.parametrize("bc", [0, 1])
def test_user_functions_match_oracle(env, dtype, fn, bc):
    """Sec. 4.2 / Sec. 5.2 user functions (compiled in) against the oracle's per-point functions."""
    cs, torch, orc = env
    ny, nx = 97, 258
    h = 2 * np.pi / nx
    field = W.sines_field(nx, seed=5, ny=ny)
    if dtype == 1:
        field = field.astype(np.float32).astype(np.float64)
    coe = [1.0 / h ** 2]
    if fn == 1:
        kw = dict(dir=0, bc=bc, left=1, right=1, fn=fn, coe=coe)
        scale_w = 4 / h ** 2
    else:
        kw = dict(dir=2, bc=bc, left=1, right=1, top=1, bottom=1, fn=fn, coe=coe)
        scale_w = 8 / h ** 2 + 2
    sentinel = np.full(field.shape, 9.0)
    got = run2d(cs, torch, field, kw, dtype, out_init=sentinel)
    ref = orc.stencil2d_fn(field, fn, coe, bc, out=sentinel)
    scale = scale_w * max(1.0, np.abs(field).max() ** 3)
    assert np.abs(got - ref).max() / scale <= TOL[dtype]
    if bc == 0:
        assert np.all(got[:, 0] == 9.0) and np.all(got[:, -1] == 9.0)
        if fn != 1:  # the x-only function writes every row
            assert np.all(got[0] == 9.0) and np.all(got[-1] == 9.0)


def test_paper_example_sec41_on_gpu(env):
    """Sec. 4.1: 8th-order d2/dx2 of sin(x), 1024 x 512, 4 points each side, non-periodic;
    interior ~ -sin(x); the 4 cells at each x end stay 0."""
    cs, torch, orc = env
    nx, ny = 1024, 512
    dx = 2 * np.pi / nx
    x = np.arange(nx) * dx
    u = np.tile(np.sin(x), (ny, 1))
    w = np.array([-1 / 560, 8 / 315, -1 / 5, 8 / 5, -205 / 72, 8 / 5, -1 / 5, 8 / 315, -1 / 560]) / dx ** 2
    got = run2d(cs, torch, u, dict(dir=0, bc=0, left=4, right=4, weights=w), 0)
    assert np.abs(got[:, 4:-4] + np.sin(x)[None, 4:-4]).max() < 1e-9
    assert np.all(got[:, :4] == 0) and np.all(got[:, -4:] == 0)


def test_swap_applies_stencil_again(env):
    cs, torch, orc = env
    u = W.uniform_field(70, 140, seed=3)
    w = lap5()
    kw = dict(dir=2, bc=1, left=1, right=1, top=1, bottom=1, weights=w)
    got = run2d(cs, torch, u, kw, 0, reps=3)
    ref = u
    for _ in range(3):
        ref = orc.stencil2d(ref, w, 2, 1, 1, 1, 1, 1)
    assert np.abs(got - ref).max() <= 1e-12 * 8 ** 3


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("dtype", [0, 1])
def test_graph_replay_matches_direct(env, dtype, bc):
    """Graph replay equals direct compute; for the non-periodic FP64 grid (4 x 4 whole tiles) the
    captured sweep includes the fork to the plan's second stream (border ring) and the join."""
    cs, torch, orc = env
    u = W.sines_field(256, seed=8)
    kw = dict(dir=2, bc=bc, left=2, right=2, top=2, bottom=2, weights=biharm13())
    a = run2d(cs, torch, u, kw, dtype, reps=4)
    b = run2d(cs, torch, u, kw, dtype, reps=4, graph=True)
    assert np.array_equal(a, b)


def test_compute_host_buffers(env):
    """Host-buffer form of Compute: pinned host input in, host output back."""
    cs, torch, orc = env
    n = 256
    u = W.uniform_field(n, n, seed=21)
    d_in = torch.zeros(n, n, dtype=torch.float64, device="cuda")
    d_out = torch.zeros_like(d_in)
    h_in = torch.from_numpy(u).pin_memory()
    h_out = torch.zeros(n, n, dtype=torch.float64).pin_memory()
    desc = cs.StencilDesc(nx=n, ny=n, dir=2, bc=1, dtype=0, left=1, right=1, top=1, bottom=1, weights=lap9())
    plan = cs.cs_plan_create_2d(desc, d_in, d_out)
    cs.cs_compute_host(plan, h_in, h_out)
    cs.cs_destroy(plan)
    ref = orc.stencil2d(u, lap9(), 2, 1, 1, 1, 1, 1)
    assert scaled_err(h_out.numpy(), ref, lap9(), u) <= 1e-12


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("tile_choice", [0, 2])
def test_compute_host_banded_equals_device_sweep(env, dtype, bc, tile_choice):
    """Grids of 16 MB or more go through the banded host path (row bands copied in, swept and
    copied out on overlapping streams, the halo of each band waiting for its neighbours, the
    periodic wrap for the last band copied first).  Results equal the device-resident sweep bit
    for bit, for xy, x-only and y-only stencils and a row count that is not a multiple of the
    band height; untouched non-periodic cells keep the output buffer's contents."""
    cs, torch, orc = env
    ny, nx = 1100, 2048 if dtype == 0 else 4096
    h = 2 * np.pi / nx
    tdt = torch.float64 if dtype == 0 else torch.float32
    ndt = np.float64 if dtype == 0 else np.float32
    u = W.sines_field(nx, seed=31, ny=ny).astype(ndt)
    for name, L, R, T, B, d, w in [c for c in stencil_cases(h) if c[0] in ("biharm13", "ddx4", "d2y8", "lap9")]:
        kw = dict(dir=d, bc=bc, left=L, right=R, top=T, bottom=B, weights=w)
        ref = run2d(cs, torch, u.astype(np.float64), kw, dtype, out_init=np.full((ny, nx), 5.0), tile_choice=tile_choice)
        d_in = torch.zeros(ny, nx, dtype=tdt, device="cuda")
        d_out = torch.full((ny, nx), 5.0, dtype=tdt, device="cuda")
        h_in = torch.from_numpy(u).pin_memory()
        h_out = torch.zeros(ny, nx, dtype=tdt).pin_memory()
        plan = cs.cs_plan_create_2d(cs.StencilDesc(nx=nx, ny=ny, dtype=dtype, **kw), d_in, d_out)
        cs.cs_plan_set_tile_choice(plan, tile_choice)
        cs.cs_compute_host(plan, h_in, h_out)
        cs.cs_destroy(plan)
        assert np.array_equal(h_out.numpy().astype(np.float64), ref), name


def test_autotune_keeps_results(env, tmp_path):
    cs, torch, orc = env
    n = 512
    u = W.sines_field(n, seed=2)
    d_in = torch.from_numpy(u).cuda()
    d_out = torch.zeros_like(d_in)
    desc = cs.StencilDesc(nx=n, ny=n, dir=2, bc=1, dtype=0, left=2, right=2, top=2, bottom=2, weights=biharm13())
    plan = cs.cs_plan_create_2d(desc, d_in, d_out)
    cs.cs_autotune(plan)
    d_out.zero_()
    cs.cs_compute(plan)
    torch.cuda.synchronize()
    cs.cs_destroy(plan)
    ref = orc.stencil2d(u, biharm13(), 2, 1, 2, 2, 2, 2)
    assert scaled_err(d_out.cpu().numpy(), ref, biharm13(), u) <= 1e-12
    path = str(tmp_path / "tune.json")
    cs.cs_tune_save(path)
    cs.cs_tune_load(path)
    assert "stencil2d|f64" in open(path).read()


@pytest.mark.parametrize("n", [4096, 8192])
@pytest.mark.parametrize("dtype", [0, 1])
def test_full_size_configs(env, n, dtype):
    """The benchmark's full sizes and launch configuration (A9 sine fields), every config
    stencil, periodic and non-periodic: rows sampled across the grid, compared element by
    element with the oracle evaluated on exactly those rows."""
    cs, torch, orc = env
    h = 2 * np.pi / n
    field = W.sines_field(n, seed=11)
    if dtype == 1:
        field = field.astype(np.float32).astype(np.float64)
    rows = np.unique(np.concatenate([[0, 1, 2, n // 2, n - 3, n - 2, n - 1],
                                     np.random.Generator(np.random.PCG64(n)).integers(0, n, 9)]))
    cases = [("lap9", 1, 1, 1, 1, 2, lap9(h)), ("biharm13", 2, 2, 2, 2, 2, biharm13(h)),
             ("ddx4", 2, 2, 0, 0, 0, D1_4 / h), ("ddy4", 0, 0, 2, 2, 1, D1_4 / h)]
    for bc in (1, 0):
        for name, L, R, T, B, d, w in cases:
            got = run2d(cs, torch, field, dict(dir=d, bc=bc, left=L, right=R, top=T, bottom=B, weights=w), dtype)
            for j in rows:
                if bc == 0 and (j < T or j >= n - B):
                    assert np.all(got[j] == 0.0)
                    continue
                band_rows = [(j - T + q) % n for q in range(T + B + 1)]
                band = field[band_rows]
                # the band holds exactly the rows row j reads; apply the stencil in x only
                ref = orc.stencil2d(band, w, 2, bc, L, R, T, B) if bc == 1 else \
                    orc.stencil2d(band, w, 2, 0, L, R, T, B)
                ref_row = ref[T] if T + B + 1 > 1 else ref[0]
                if bc == 0:
                    assert np.all(got[j, :L] == 0) and np.all(got[j, n - R:] == 0)
                    sl = slice(L, n - R)
                    err = scaled_err(got[j, sl], ref_row[sl], w, field)
                else:
                    err = scaled_err(got[j], ref_row, w, field)
                assert err <= TOL[dtype], (name, bc, j, err)
    # the functor of the config: c^3 - c - Laplacian(c)
    got = run2d(cs, torch, field, dict(dir=2, bc=1, left=1, right=1, top=1, bottom=1, fn=3, coe=[1 / h ** 2]), dtype)
    ref = orc.stencil2d_fn(field, 3, [1 / h ** 2], 1)
    assert np.abs(got - ref).max() / (8 / h ** 2 + 2) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [0, 1])
def test_grouped_launch_equals_individual_plans(env, dtype):
    """cs_compute_group over grids of different sizes (one persistent launch) gives bit-for-bit
    the results of computing each plan alone: storage-type arithmetic for FP32, the exact digit
    path for FP64 (integer weight ratios), on the same 64-row tiles."""
    cs, torch, orc = env
    tdt = torch.float64 if dtype == 0 else torch.float32
    sizes = [(64, 64), (100, 260), (257, 129), (31, 517), (128, 128)]
    ins, outs, refs, plans = [], [], [], []
    for k, (ny, nx) in enumerate(sizes):
        h = 2 * np.pi / nx
        x = torch.from_numpy(W.sines_field(nx, seed=k, ny=ny)).to("cuda", tdt)
        y = torch.zeros_like(x)
        r = torch.zeros_like(x)
        w = biharm13(h)
        desc = cs.StencilDesc(nx=nx, ny=ny, dir=2, bc=k % 2, dtype=dtype, left=2, right=2, top=2, bottom=2, weights=w)
        p_alone = cs.cs_plan_create_2d(desc, x, r)
        cs.cs_plan_set_tile_choice(p_alone, 1)
        cs.cs_compute(p_alone)
        cs.cs_destroy(p_alone)
        plans.append(cs.cs_plan_create_2d(desc, x, y))
        ins.append(x); outs.append(y); refs.append(r)
    cs.cs_compute_group(plans)
    torch.cuda.synchronize()
    for p in plans:
        cs.cs_destroy(p)
    for y, r in zip(outs, refs):
        assert torch.equal(y, r)


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("fn", [None, 3])
def test_grouped_launch_many_grids_and_graph(env, dtype, fn):
    """150 grids of the serving size mix (more than one launch's job table), weighted 9-point
    Laplacian or the cubic user function: grouped results equal the plans computed alone bit
    for bit, and a CUDA graph captured around cs_compute_group replays to the same bits on new
    inputs written into the same buffers."""
    cs, torch, orc = env
    tdt = torch.float64 if dtype == 0 else torch.float32
    rng = np.random.Generator(np.random.PCG64(5))
    ns = rng.choice([16, 32, 64, 128, 200, 256], size=150)
    xs, ys, refs, plans = [], [], [], []
    for k, n in enumerate(ns):
        h = 2 * np.pi / n
        x = torch.from_numpy(W.sines_field(int(n), seed=300 + k)).to("cuda", tdt)
        y = torch.full_like(x, 7.0)
        r = torch.full_like(x, 7.0)
        if fn is None:
            kw = dict(dir=2, left=1, right=1, top=1, bottom=1, weights=lap9(h))
        else:
            kw = dict(dir=2, left=1, right=1, top=1, bottom=1, fn=fn, coe=[1 / h ** 2])
        desc = cs.StencilDesc(nx=int(n), ny=int(n), bc=k % 2, dtype=dtype, **kw)
        p_alone = cs.cs_plan_create_2d(desc, x, r)
        cs.cs_plan_set_tile_choice(p_alone, 1)
        cs.cs_compute(p_alone)
        cs.cs_destroy(p_alone)
        plans.append(cs.cs_plan_create_2d(desc, x, y))
        xs.append(x); ys.append(y); refs.append(r)
    before = cs.cs_launch_count()
    cs.cs_compute_group(plans)
    torch.cuda.synchronize()
    assert cs.cs_launch_count() - before == 3  # 150 plans, 64 per launch
    for y, r in zip(ys, refs):
        assert torch.equal(y, r)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        cs.cs_compute_group(plans, torch.cuda.current_stream())
    for x in xs:
        x.mul_(-0.5)
    for y in ys:
        y.fill_(7.0)
    g.replay()
    torch.cuda.synchronize()
    for k, (x, y) in enumerate(zip(xs, ys)):
        r = torch.full_like(x, 7.0)
        p = cs.cs_plan_create_2d(cs.StencilDesc(nx=x.shape[1], ny=x.shape[0], bc=k % 2, dtype=dtype,
                                                **(dict(dir=2, left=1, right=1, top=1, bottom=1,
                                                        weights=lap9(2 * np.pi / x.shape[1])) if fn is None else
                                                   dict(dir=2, left=1, right=1, top=1, bottom=1, fn=fn,
                                                        coe=[1 / (2 * np.pi / x.shape[1]) ** 2]))), x, r)
        cs.cs_plan_set_tile_choice(p, 1)
        cs.cs_compute(p)
        cs.cs_destroy(p)
        assert torch.equal(y, r), k
    for p in plans:
        cs.cs_destroy(p)


@pytest.mark.parametrize("case", ["plain", "wide_range", "nan_inf", "huge_tile", "zeros"])
def test_exact_digit_path_matches_oracle(env, case):
    """FP64 stencils whose weights are c * small integers take the exact digit path: against the
    oracle at the FP64 tolerance; tiles with inf / nan or values beyond 2^900 fall back to native
    FP64 (non-finite outputs exactly where the oracle has them)."""
    cs, torch, orc = env
    ny, nx = 130, 200
    h = 2 * np.pi / nx
    field = W.sines_field(nx, seed=29, ny=ny)
    if case == "wide_range":
        field[:, :64] *= 1e-20  # tiles of very different scales
        field[40:50, 100:110] *= 1e12
    elif case == "nan_inf":
        field[3, 7] = np.nan
        field[100, 150] = np.inf
    elif case == "huge_tile":
        field[60:70, 60:70] = 1e280
    elif case == "zeros":
        field[:64, :] = 0.0
    bad = (~np.isfinite(field)).astype(float)
    for name, L, R, T, B, d, w in stencil_cases(h)[:10]:
        kw = dict(dir=d, bc=1, left=L, right=R, top=T, bottom=B, weights=w)
        got = run2d(cs, torch, field, kw, 0)
        ref = orc.stencil2d(field, w, d, 1, L, R, T, B)
        # zero weights are not part of the stencil: a non-finite input reaches exactly the
        # outputs whose non-zero taps touch it
        hit = orc.stencil2d(bad, (np.asarray(w) != 0).astype(float), d, 1, L, R, T, B) > 0
        assert np.array_equal(hit, ~np.isfinite(got)), name
        fin = np.isfinite(ref) & ~hit
        scale = np.abs(w).sum() * np.abs(field[np.isfinite(field)]).max()
        assert np.abs(got[fin] - ref[fin]).max() <= 1e-12 * scale, name


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("shape", [(200, 384), (70, 136), (130, 520), (5, 8), (256, 384)])
def test_tma_pipeline_equals_cp_async_tiles(env, dtype, bc, shape):
    """The TMA-pipelined persistent sweep (tile choice 2) gives bit for bit the results of the
    cp.async tiles of the same height (choice 1) for every specialised stencil, including edge
    tiles whose periodic halo is patched after the copy and grids smaller than a tile; at
    256 x 384 the cp.async sweep of a non-periodic FP64 grid runs its inner tiles in the FULL form
    and its border ring on a second stream."""
    cs, torch, orc = env
    ny, nx = shape
    h = 2 * np.pi / nx
    field = W.sines_field(nx, seed=nx * ny, ny=ny)
    cases = stencil_cases(h)[:12] + [("fn2", 1, 1, 1, 1, 2, None), ("fn3", 1, 1, 1, 1, 2, None)]
    for name, L, R, T, B, d, w in cases:
        if w is None:
            kw = dict(dir=2, bc=bc, left=1, right=1, top=1, bottom=1, fn=int(name[-1]), coe=[1 / h ** 2])
        else:
            kw = dict(dir=d, bc=bc, left=L, right=R, top=T, bottom=B, weights=w)
        a = run2d(cs, torch, field, kw, dtype, tile_choice=1, out_init=np.full(shape, 3.0))
        b = run2d(cs, torch, field, kw, dtype, tile_choice=2, out_init=np.full(shape, 3.0))
        assert np.array_equal(a, b), name


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("offsets", [(0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("bc", [0, 1])
def test_unaligned_buffers_match_oracle(env, dtype, offsets, bc):
    """Input and output buffers that start one element past a 16-byte boundary take the
    element-wise copies and stores; results equal the oracle's, untouched cells keep the
    sentinel."""
    cs, torch, orc = env
    ny, nx = 130, 300
    h = 2 * np.pi / nx
    field = W.sines_field(nx, seed=77, ny=ny)
    tdt = torch.float64 if dtype == 0 else torch.float32
    ndt = np.float64 if dtype == 0 else np.float32
    if dtype == 1:
        field = field.astype(np.float32).astype(np.float64)
    sentinel = -2.0 ** 120
    in_off, out_off = offsets
    for name, L, R, T, B, d, w in [c for c in stencil_cases(h) if c[0] in ("lap9", "biharm13", "ddx4", "d2y8")]:
        buf_in = torch.zeros(ny * nx + 1, dtype=tdt, device="cuda")
        buf_out = torch.full((ny * nx + 1,), sentinel, dtype=tdt, device="cuda")
        x = buf_in[in_off:in_off + ny * nx].view(ny, nx)
        y = buf_out[out_off:out_off + ny * nx].view(ny, nx)
        x.copy_(torch.from_numpy(field.astype(ndt)))
        plan = cs.cs_plan_create_2d(cs.StencilDesc(nx=nx, ny=ny, dir=d, bc=bc, dtype=dtype, left=L, right=R,
                                                   top=T, bottom=B, weights=w), x, y)
        cs.cs_compute(plan)
        torch.cuda.synchronize()
        cs.cs_destroy(plan)
        got = y.cpu().numpy().astype(np.float64)
        ref = orc.stencil2d(field, w, d, bc, L, R, T, B, out=np.full((ny, nx), sentinel))
        written = np.ones((ny, nx), bool)
        if bc == 0:
            written[:] = False
            written[T:ny - B, L:nx - R] = True
            assert np.array_equal(got[~written], ref[~written]), name
        assert scaled_err(got[written], ref[written], w, field) <= TOL[dtype], name
        spare = buf_out[0] if out_off == 1 else buf_out[-1]
        assert spare.item() == sentinel, name  # nothing written outside the view


@pytest.mark.parametrize("wscale,uscale", [(2.0 ** -55, 2.0 ** -895), (2.0 ** 45, 2.0 ** 885),
                                           (2.0 ** -50, 2.0 ** 800), (1e200, 1e100)])
def test_exact_digit_path_extreme_scales(env, wscale, uscale):
    """Integer-ratio weights near the ends of the fast-path weight range [2^-60, 2^50) on values
    near the ends of the digit range [2^-900, 2^900]: tiles whose scale c * 2^(G - 50) leaves the
    range of the one-FMA conversion take native FP64, the others the digit path (with constants
    up to 2^56 scale); weights outside the range take native FP64 throughout.  Every output meets
    the FP64 tolerance against the oracle."""
    cs, torch, orc = env
    ny, nx = 130, 200
    field = W.sines_field(nx, seed=41, ny=ny) * uscale
    for name, L, R, T, B, d, w in [c for c in stencil_cases(1.0) if c[0] in ("lap5", "biharm13", "x1", "ddy4")]:
        w = np.asarray(w) * wscale
        kw = dict(dir=d, bc=1, left=L, right=R, top=T, bottom=B, weights=w)
        got = run2d(cs, torch, field, kw, 0)
        ref = orc.stencil2d(field, w, d, 1, L, R, T, B)
        assert np.all(np.isfinite(got)), name
        assert scaled_err(got, ref, w, field) <= 1e-12, name
