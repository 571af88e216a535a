"""The multi-GPU decomposition (row bands with halo exchange; the CH step's all-to-all
transposes and allreduced invariants) on CPU ranks over gloo: a sharded oracle must equal the
unsharded one.  World sizes 2 and 3, band heights that differ by one row, periodic and
non-periodic stencils, and the transpose on its own."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    return dist


STENCILS = [  # (name, L, R, T, B, dir)
    ("lap9", 1, 1, 1, 1, 2), ("biharm13", 2, 2, 2, 2, 2), ("ddy4", 0, 0, 2, 2, 1),
    ("asym", 3, 1, 0, 2, 2), ("generic", 2, 3, 4, 1, 2),
]


def _stencil_worker(rank, world, port, q):
    dist = _init(rank, world, port)
    import torch
    import oracle
    import workloads as W
    from paper_1902_09931_gb300 import distributed as D
    ny, nx = 47, 36
    u = W.sines_field(nx, seed=3, ny=ny)
    rng = np.random.default_rng(5)
    r0, r1 = D.band(ny, world, rank)
    ok = []
    for name, L, R, T, B, d in STENCILS:
        w = rng.uniform(-1, 1, (L + R + 1) * (T + B + 1))
        for bc in (0, 1):
            full = oracle.stencil2d(u, w, d, bc, L, R, T, B)
            compute = lambda padded: torch.from_numpy(oracle.stencil2d(padded.numpy(), w, d, bc, L, R, T, B))
            got = D.sharded_sweep(torch.from_numpy(u[r0:r1].copy()), compute, T, B, bc == 1)
            ok.append((name, bc, bool(np.array_equal(got.numpy(), full[r0:r1]))))
    q.put((rank, ok))
    dist.destroy_process_group()


def _ch_worker(rank, world, port, q):
    dist = _init(rank, world, port)
    import torch
    import oracle
    import workloads as W
    from paper_1902_09931_gb300 import distributed as D
    n, Dm, G = 48, 1.0, 0.01
    h = 2 * np.pi / n
    dt = 0.1 * h
    a = oracle.ch_coefficient_a(n, Dm, G, dt)
    prev = W.ch_initial(n, seed=8)
    cur = prev + 0.01 * W.ch_initial(n, seed=9)
    r0, r1 = D.band(n, world, rank)
    lap5 = np.array([0, 1, 0, 1, -4, 1, 0, 1, 0.0]) / h ** 2
    bih = np.zeros((5, 5))
    bih[2, 2] = 20
    bih[1, 2] = bih[3, 2] = bih[2, 1] = bih[2, 3] = -8
    bih[1, 1] = bih[1, 3] = bih[3, 1] = bih[3, 3] = 2
    bih[0, 2] = bih[4, 2] = bih[2, 0] = bih[2, 4] = 1
    bih = bih.ravel() / h ** 4

    def rhs(pp, cp):  # the right-hand side of Sec. 5.1 on a band padded by 2 rows
        p, c = pp.numpy(), cp.numpy()
        cbar = 2 * c - p
        b4 = oracle.stencil2d(cbar, bih, 2, 1, 2, 2, 2, 2)[2:-2]
        l2 = oracle.stencil2d(c ** 3 - c, lap5, 2, 1, 1, 1, 1, 1)[2:-2]
        r = -(2 / 3) * (c[2:-2] - p[2:-2]) - (2 / 3) * Dm * G * dt * b4 + (2 / 3) * Dm * dt * l2
        return torch.from_numpy(r)

    solve = lambda b: torch.from_numpy(oracle.cyclic_penta_solve(b.numpy(), a))
    got = D.sharded_ch_step(torch.from_numpy(prev[r0:r1].copy()), torch.from_numpy(cur[r0:r1].copy()), n, rhs, solve)
    ref = oracle.ch_step(prev, cur, Dm, G, dt)
    err = float(np.abs(got.numpy() - ref[r0:r1]).max())
    v = ref - (2 * cur - prev)  # the per-step bound of the CH parity tests
    tol = 1e-12 * (np.abs(cur).max() + np.abs(oracle.ch_rhs(prev, cur, Dm, G, dt)).max() + (1 + 16 * a) * np.abs(v).max())
    # invariants of the new field from per-rank partials
    g = got.numpy()
    e_loc = np.vstack([g, D.exchange_halo(got, 0, 1, True)[0].numpy()[-1:]])  # one row below for D+y
    gx = (np.roll(g, -1, axis=1) - g) / h
    gy = (e_loc[1:] - e_loc[:-1]) / h
    part = torch.tensor([h * h * g.sum(), h * h * np.sum(0.25 * (g * g - 1) ** 2 + 0.5 * G * (gx ** 2 + gy ** 2))])
    tot = D.allreduce_sum(part).numpy()
    q.put((rank, err, tol, tot.tolist(), oracle.ch_mass(ref), oracle.ch_energy(ref, G)))
    dist.destroy_process_group()


def _transpose_worker(rank, world, port, q):
    dist = _init(rank, world, port)
    import torch
    from paper_1902_09931_gb300 import distributed as D
    n = 23
    A = np.arange(n * n, dtype=np.float64).reshape(n, n)
    r0, r1 = D.band(n, world, rank)
    t = D.transpose_bands(torch.from_numpy(A[r0:r1].copy()), n)
    q.put((rank, bool(np.array_equal(t.numpy(), A.T[r0:r1]))))
    dist.destroy_process_group()


def _run(target, world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=target, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(out)


def test_band_partition():
    sys.path.insert(0, ROOT)
    from paper_1902_09931_gb300 import distributed as D
    for n in (1, 7, 47, 64):
        for world in (1, 2, 3, 8):
            bands = [D.band(n, world, r) for r in range(world)]
            assert bands[0][0] == 0 and bands[-1][1] == n
            assert all(bands[i][1] == bands[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in bands]
            assert max(sizes) - min(sizes) <= 1


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_stencil_equals_unsharded_oracle(world):
    for rank, ok in _run(_stencil_worker, world):
        bad = [x for x in ok if not x[2]]
        assert not bad, (rank, bad)


@pytest.mark.parametrize("world", [2, 3])
def test_transpose_bands(world):
    assert all(ok for _, ok in _run(_transpose_worker, world))


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_ch_step_equals_unsharded_oracle(world):
    """x-solves on row bands, an all-to-all transpose, y-solves, the transpose back; mass and
    energy of the result from allreduced per-rank partials."""
    for rank, err, tol, tot, mass, energy in _run(_ch_worker, world):
        assert err <= tol, (rank, err, tol)
        assert tot[0] == pytest.approx(mass, rel=1e-12, abs=1e-13)
        assert tot[1] == pytest.approx(energy, rel=1e-12)


def _errors_worker(rank, world, port, q):
    dist = _init(rank, world, port)
    import torch
    from paper_1902_09931_gb300 import distributed as D
    out = {}
    try:
        D.exchange_halo(torch.zeros(1, 8, dtype=torch.float64), 2, 2, True)
        out["thin"] = False
    except ValueError:
        out["thin"] = True
    try:
        D.transpose_bands(torch.zeros(3, 8, dtype=torch.float64), 8)
        out["shape"] = False
    except ValueError:
        out["shape"] = True
    # one rank: the halo of a periodic band is its own wrap; a non-periodic band gets none
    x = torch.arange(20, dtype=torch.float64).reshape(5, 4)
    p, t, b = D.exchange_halo(x, 2, 1, True)
    out["wrap"] = bool(t == 2 and b == 1 and torch.equal(p, torch.cat([x[3:], x, x[:1]])))
    p, t, b = D.exchange_halo(x, 2, 1, False)
    out["nowrap"] = bool(t == 0 and b == 0 and torch.equal(p, x))
    q.put((rank, out))
    dist.destroy_process_group()


def test_single_rank_halo_and_errors():
    (rank, out), = _run(_errors_worker, 1)
    assert out == {"thin": True, "shape": True, "wrap": True, "nowrap": True}


def _halo_worker(rank, world, port, q):
    dist = _init(rank, world, port)
    import torch
    from paper_1902_09931_gb300 import distributed as D
    n, halo = 29, 2
    A = np.arange(n * 5, dtype=np.float64).reshape(n, 5)
    r0, r1 = D.band(n, world, rank)
    ok = {}
    for periodic in (True, False):
        padded = torch.full((r1 - r0 + 2 * halo, 5), -1.0, dtype=torch.float64)
        padded[halo:-halo] = torch.from_numpy(A[r0:r1])
        D.exchange_halo_inplace(padded, halo, periodic=periodic)
        rows = []
        for j in range(-halo, r1 - r0 + halo):
            g = r0 + j
            if periodic:
                g %= n
            else:  # even reflection about the grid's edges: -1 -> 0, -2 -> 1, n -> n-1, n+1 -> n-2
                g = -1 - g if g < 0 else (2 * n - 1 - g if g >= n else g)
            rows.append(A[g])
        ok[periodic] = bool(np.array_equal(padded.numpy(), np.array(rows)))
    q.put((rank, ok))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [1, 2, 3])
def test_halo_exchange_in_place_periodic_and_mirrored(world):
    """exchange_halo_inplace fills the 2 rows above and below each rank's band with the global
    rows the full-grid step reads there: wrapped rows (periodic) or the even reflection about the
    grid's first and last rows (no-flux), with neighbours' rows between bands."""
    for rank, ok in _run(_halo_worker, world):
        assert ok == {True: True, False: True}, (rank, ok)


def _rows_worker(rank, world, port, q):
    dist = _init(rank, world, port)
    import torch
    import oracle
    from paper_1902_09931_gb300 import distributed as D
    n, nx = 31, 6
    A = np.arange(n * nx, dtype=np.float64).reshape(n, nx)
    r0, r1 = D.band(n, world, rank)
    ok = []
    for top, bottom in [(1, 1), (2, 2), (0, 2), (3, 1), (4, 0)]:
        for periodic in (True, False):
            t = top if top > 0 and (periodic or rank > 0) else 0
            b = bottom if bottom > 0 and (periodic or rank < world - 1) else 0
            padded = torch.full((r1 - r0 + t + b, nx), -1.0, dtype=torch.float64)
            padded[t:t + r1 - r0] = torch.from_numpy(A[r0:r1])
            D.exchange_rows_inplace(padded, top, bottom, periodic=periodic)
            want = A[[(g % n) for g in range(r0 - t, r1 + b)]]
            good = bool(np.array_equal(padded.numpy(), want))
            # the sweep of the padded band, restricted to the band, is the full grid's sweep
            w = np.arange(1, 4 * (top + bottom + 1) + 1, dtype=np.float64)
            full = oracle.stencil2d(A, w, 2, int(periodic), 1, 2, top, bottom)
            part = oracle.stencil2d(padded.numpy(), w, 2, int(periodic), 1, 2, top, bottom)
            good = good and bool(np.array_equal(part[t:t + r1 - r0], full[r0:r1]))
            ok.append(((top, bottom, periodic), good))
    q.put((rank, ok))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [1, 2, 3])
def test_row_exchange_in_place_for_stencil_bands(world):
    """exchange_rows_inplace fills the `top` rows above and `bottom` rows below each rank's band
    (asymmetric reaches, none at a non-periodic grid's first and last rows) with the global rows,
    and the stencil of the padded band restricted to the band equals the full grid's, periodic and
    non-periodic (whose untouched edge rows then match too)."""
    for rank, ok in _run(_rows_worker, world):
        assert all(g for _, g in ok), (rank, [k for k, g in ok if not g])


def _gather_worker(rank, world, port, q):
    dist = _init(rank, world, port)
    import torch
    from paper_1902_09931_gb300 import distributed as D
    chunks, chunk_len, n = 8, 16, 5
    rows = D.band(chunks * chunk_len, world, rank)
    c0, c1 = rows[0] // chunk_len, rows[1] // chunk_len
    # each value names its place in the whole line's chunk-major array: (chunk, end value k, column)
    mine = torch.tensor([[[c * 100 + k * 10 + j for j in range(n)] for k in range(4)] for c in range(c0, c1)],
                        dtype=torch.float64).reshape(-1)
    got = D._all_gather_rows(mine, None)
    want = torch.tensor([[[c * 100 + k * 10 + j for j in range(n)] for k in range(4)] for c in range(chunks)],
                        dtype=torch.float64).reshape(-1)
    q.put((rank, [(rows, bool(torch.equal(got, want)))]))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [1, 2, 4])
def test_chunk_ends_gather_in_chunk_order(world):
    """The band CH step's y-line exchange: when the chunks of a line split evenly over the ranks,
    each rank's band starts at a chunk boundary, and the ranks' chunk-major end values gathered in
    rank order are the whole line's end values in chunk order."""
    for rank, ok in _run(_gather_worker, world):
        assert all(g for _, g in ok), (rank, ok)
