"""The sharded sweep's device path on one GPU (a single gloo rank: the halo exchange is the
periodic wrap of the only band), with this library's plan over the padded band, against the
oracle."""
import os
import socket

import numpy as np
import pytest

import workloads as W
from gpu_helpers import stencil_cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import torch.distributed as dist
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import oracle
    import paper_1902_09931_gb300 as cs
    from paper_1902_09931_gb300 import distributed as D
    cs.load()
    if not dist.is_initialized():
        with socket.socket() as s:
            s.bind(("127.0.0.1", 0))
            port = s.getsockname()[1]
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        dist.init_process_group("gloo", rank=0, world_size=1)
    yield cs, torch, oracle, D
    dist.destroy_process_group()


@pytest.mark.parametrize("bc", [0, 1])
def test_device_band_sweep_matches_oracle(env, bc):
    cs, torch, orc, D = env
    ny, nx = 300, 256
    h = 2 * np.pi / nx
    u = W.sines_field(nx, seed=71, ny=ny)
    for name, L, R, T, B, d, w in [c for c in stencil_cases(h) if c[0] in ("lap9", "biharm13", "ddy4")]:
        sweep = D.DeviceBandSweep(dict(dir=d, bc=bc, left=L, right=R, top=T, bottom=B, weights=w, dtype=0))
        got = D.sharded_sweep(torch.from_numpy(u).cuda(), sweep, T, B, bc == 1).cpu().numpy()
        sweep.close()
        ref = orc.stencil2d(u, w, d, bc, L, R, T, B)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(w).sum() * np.abs(u).max(), name


def _full_grid_run(cs, torch, c0, storage, dt, steps, boundary=0):
    tdt = torch.float64 if storage == 0 else torch.float32
    f = [torch.from_numpy(c0).to("cuda", tdt), torch.from_numpy(c0).to("cuda", tdt),
         torch.zeros(c0.shape, dtype=tdt, device="cuda")]
    plan = cs.cs_ch_create(cs.CHDesc(n=c0.shape[0], storage=storage, D=1.0, gamma=0.01, dt=dt, boundary=boundary), *f)
    mass, energy = cs.cs_ch_step(plan, steps, invariants=True)
    _, cur, _ = cs.cs_ch_fields(plan)
    out = [t for t in f if t.data_ptr() == cur][0].clone()
    cs.cs_destroy(plan)
    return out, mass[-1], energy[-1]


@pytest.mark.parametrize("mode", ["chunks", "transposes"])
@pytest.mark.parametrize("boundary", [0, 1])
@pytest.mark.parametrize("storage", [0, 1])
def test_device_band_ch_step_equals_full_grid_step(env, storage, boundary, mode):
    """The decomposed Cahn-Hilliard step (cs_ch_band_* with the halo exchange of the distributed
    module; the y lines by chunks with their end values gathered, or through transposes) on one
    rank gives the full-grid cs_ch_step's fields bit for bit (the same kernels on the same values)
    and the same invariants, periodic and with no-flux boundaries (mirrored halos, non-cyclic line
    solves)."""
    cs, torch, orc, D = env
    n = 320  # a size no other test autotunes: every process uses the default partition
    dt = 0.1 * 2 * np.pi / n
    c0 = W.ch_initial(n, seed=44)
    if storage == 1:
        c0 = c0.astype(np.float32).astype(np.float64)
    ref, m_ref, e_ref = _full_grid_run(cs, torch, c0, storage, dt, 3, boundary)
    tdt = torch.float64 if storage == 0 else torch.float32
    b = D.DeviceCHBand(n, storage, 1.0, 0.01, dt, torch.from_numpy(c0).to("cuda", tdt), boundary=boundary,
                       mode=mode)
    assert b.mode == mode
    b.step(3)
    mass, energy = b.invariants()
    got = b.field().clone()
    b.close()
    torch.cuda.synchronize()
    assert torch.equal(got, ref)
    assert mass == m_ref and energy == e_ref


def _band_worker(rank, world, port, storage, boundary, mode, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    import workloads as W
    import paper_1902_09931_gb300 as cs
    from paper_1902_09931_gb300 import distributed as D
    torch.cuda.set_device(0)
    cs.load()
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n = 320  # a size no other test autotunes: every process uses the default partition
    dt = 0.1 * 2 * np.pi / n
    c0 = W.ch_initial(n, seed=45)
    tdt = torch.float64 if storage == 0 else torch.float32
    r0, r1 = D.band(n, world, rank)
    b = D.DeviceCHBand(n, storage, 1.0, 0.01, dt, torch.from_numpy(c0[r0:r1].copy()).to("cuda", tdt),
                       boundary=boundary, mode=mode)
    assert b.mode == mode
    b.step(3)
    mass, energy = b.invariants()
    q.put((rank, b.field().cpu().numpy().astype(np.float64), mass, energy))
    b.close()
    dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["chunks", "transposes"])
@pytest.mark.parametrize("boundary", [0, 1])
@pytest.mark.parametrize("storage", [0, 1])
def test_device_band_ch_step_two_ranks(env, storage, boundary, mode):
    """Two ranks (two processes sharing this GPU, gloo through host memory; nothing on the device
    waits for the other rank) each step their 160-row band (4 of the 8 chunks of every column)
    three times, the y lines by chunks with the end values all-gathered, or through transposes;
    the bands put together equal the full-grid step bit for bit, and the allreduced invariants
    agree to rounding."""
    cs, torch, orc, D = env
    import multiprocessing as mp
    n = 320  # a size no other test autotunes: every process uses the default partition
    dt = 0.1 * 2 * np.pi / n
    c0 = W.ch_initial(n, seed=45)
    if storage == 1:
        c0 = c0.astype(np.float32).astype(np.float64)
    ref, m_ref, e_ref = _full_grid_run(cs, torch, c0, storage, dt, 3, boundary)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    procs = [ctx.Process(target=_band_worker, args=(r, 2, port, storage, boundary, mode, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=300) for _ in procs], key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got = np.concatenate([r[1] for r in res])
    assert np.array_equal(got, ref.cpu().numpy().astype(np.float64))
    scale = (2 * np.pi / n) ** 2 * np.abs(c0).sum()
    for r in res:
        assert abs(r[2] - m_ref) <= 1e-14 * scale and abs(r[3] - e_ref) <= 1e-13 * abs(e_ref)


BAND_STENCILS = [("lap9", 1, 1, 1, 1, 2), ("biharm13", 2, 2, 2, 2, 2), ("ddy4", 0, 0, 2, 2, 1),
                 ("asym", 3, 1, 0, 2, 2)]


def _band_stencil_run(cs, torch, D, u, rows_of, dtype, bc, name, L, R, T, B, d, sweeps):
    """This rank's band after `sweeps` sweeps of DeviceBandStencil (swapping between sweeps)."""
    w = W.integer_weights((L + R + 1) * (T + B + 1), seed=len(name) + 7 * T + L, bound=3)
    r0, r1 = rows_of
    s = D.DeviceBandStencil(r1 - r0, u.shape[1], dict(dir=d, bc=bc, left=L, right=R, top=T, bottom=B,
                                                       weights=w, dtype=dtype))
    tdt = torch.float64 if dtype == 0 else torch.float32
    s.band().copy_(torch.from_numpy(u[r0:r1].copy()).to(tdt))
    for k in range(sweeps):
        out = s()
        if k + 1 < sweeps:
            s.swap()
    got = out.cpu().numpy().astype(np.float64)
    s.close()
    return got, w


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("bc", [0, 1])
def test_device_band_stencil_one_rank_bit_exact(env, dtype, bc):
    """DeviceBandStencil on one rank (the band is the grid, its halo the periodic wrap or nothing):
    on integer data every sum is exact, so one sweep and two sweeps with swap equal the oracle's bit
    for bit (non-periodic: cells the sweep leaves untouched read 0 in a first sweep and keep the
    first sweep's values in the second, as the band's own buffers do)."""
    cs, torch, orc, D = env
    ny, nx = 75, 130
    u = W.integer_field(ny, nx, seed=13, bound=64)
    for name, L, R, T, B, d in BAND_STENCILS:
        got1, w = _band_stencil_run(cs, torch, D, u, (0, ny), dtype, bc, name, L, R, T, B, d, 1)
        ref1 = orc.stencil2d(u, w, d, bc, L, R, T, B)
        assert np.array_equal(got1, ref1), name
        got2, _ = _band_stencil_run(cs, torch, D, u, (0, ny), dtype, bc, name, L, R, T, B, d, 2)
        ref2 = orc.stencil2d(ref1, w, d, bc, L, R, T, B, out=np.zeros_like(u) if bc == 1 else u.copy())
        assert np.array_equal(got2, ref2), name


def _band_stencil_worker(rank, world, port, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    sys.path.insert(0, os.path.join(root, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    import workloads as W
    import paper_1902_09931_gb300 as cs
    from paper_1902_09931_gb300 import distributed as D
    torch.cuda.set_device(0)
    cs.load()
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ny, nx = 75, 130
    u = W.integer_field(ny, nx, seed=13, bound=64)
    res = {}
    for dtype in (0, 1):
        for bc in (0, 1):
            for name, L, R, T, B, d in BAND_STENCILS:
                got, _ = _band_stencil_run(cs, torch, D, u, D.band(ny, world, rank), dtype, bc, name, L, R, T, B, d, 1)
                res[(dtype, bc, name)] = got
    q.put((rank, res))
    dist.destroy_process_group()


def test_device_band_stencil_two_ranks_bit_exact(env):
    """Two ranks (two processes sharing this GPU, gloo through host memory) each sweep their band
    with DeviceBandStencil; on integer data the bands put together equal the oracle's full-grid
    sweep bit for bit, for every stencil, both boundary conditions and both storage types."""
    cs, torch, orc, D = env
    import multiprocessing as mp
    ny, nx = 75, 130
    u = W.integer_field(ny, nx, seed=13, bound=64)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    procs = [ctx.Process(target=_band_stencil_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=300) for _ in procs], key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for key in res[0][1]:
        dtype, bc, name = key
        L, R, T, B, d = [c for c in BAND_STENCILS if c[0] == name][0][1:]
        w = W.integer_weights((L + R + 1) * (T + B + 1), seed=len(name) + 7 * T + L, bound=3)
        ref = orc.stencil2d(u, w, d, bc, L, R, T, B)
        got = np.concatenate([res[0][1][key], res[1][1][key]])
        assert np.array_equal(got, ref), key
