"""Decomposition of one grid over several GPUs (one process per GPU, torch.distributed).

The paper sketches the multi-GPU extension as non-periodic stencils plus halo swaps between
ranks (Sec. 6.2, MPI).  Here:

* 2D stencils: the grid is cut into contiguous row bands along y (the layout of the paper's
  y-tiles, Sec. 2).  Before a sweep each rank receives the ``top`` rows above its band and the
  ``bottom`` rows below it from its neighbours; with periodic rows the last and first ranks are
  neighbours.  The sweep then runs on the padded band; the halo rows' own outputs are dropped.
* Cahn-Hilliard ADI (Sec. 5.1): the right-hand side needs a 2-row halo of C^n and C^{n-1}; the
  x-line solves are local to a row band.  The y lines are cut into the partitioned solver's
  chunks; when the bands are whole numbers of chunks each rank solves its own chunks and the ranks
  all-gather only the chunks' end values (4 per column and chunk) for the spike correction;
  otherwise the y-line solves run after an all-to-all transpose that gives every rank a band of
  columns, and a second transpose brings the result back.  Mass and energy are sums of per-rank
  FP64 partials (an allreduce).

Everything here is communication and index bookkeeping: the arithmetic of a band is a callable
the caller supplies (a device plan of this library on the GPU path).  Point-to-point exchanges use
``isend`` / ``irecv``, so any backend works (gloo for CPU tensors, NCCL for CUDA tensors).  On the
device the bands stay in place: DeviceBandStencil and DeviceCHBand keep each band inside a
persistent padded buffer and receive the neighbours' rows into its halo rows.
"""
from __future__ import annotations

from typing import Callable

import torch
import torch.distributed as dist

_TAG_TOP, _TAG_BOTTOM, _TAG_T = 11, 12, 13


def band(n: int, world: int, rank: int) -> tuple[int, int]:
    """Rows [r0, r1) of rank `rank` when n rows are cut into `world` contiguous bands whose sizes
    differ by at most one (the first n % world bands take the extra row)."""
    base, extra = divmod(n, world)
    r0 = rank * base + min(rank, extra)
    return r0, r0 + base + (1 if rank < extra else 0)


def exchange_halo(local: torch.Tensor, top: int, bottom: int, periodic: bool, group=None):
    """The band `local` (rows x nx) with the `top` rows of the band above and the `bottom` rows of
    the band below stacked on.  Non-periodic grids have no neighbour beyond their first and last
    bands, and those bands get no halo on that side.  Returns (padded, top_rows, bottom_rows): the
    halo rows actually added on each side."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    rows, nx = local.shape
    if rows < max(top, bottom):
        raise ValueError(f"band of {rows} rows is thinner than the stencil's reach ({top}, {bottom})")
    has_top = top > 0 and (periodic or rank > 0)
    has_bottom = bottom > 0 and (periodic or rank < world - 1)
    up, down = (rank - 1) % world, (rank + 1) % world
    if world == 1:  # the only band is its own neighbour
        t = local[rows - top:] if has_top else local[:0]
        b = local[:bottom] if has_bottom else local[:0]
        return torch.cat([t, local, b]), (top if has_top else 0), (bottom if has_bottom else 0)
    recv_top = torch.empty((top, nx), dtype=local.dtype, device=local.device) if has_top else None
    recv_bottom = torch.empty((bottom, nx), dtype=local.dtype, device=local.device) if has_bottom else None
    reqs = []
    if has_top:
        reqs.append(dist.irecv(recv_top, src=up, group=group, tag=_TAG_TOP))
    if has_bottom:
        reqs.append(dist.irecv(recv_bottom, src=down, group=group, tag=_TAG_BOTTOM))
    # my last `top` rows are the top halo of the band below; my first `bottom` rows the bottom
    # halo of the band above
    if top > 0 and (periodic or rank < world - 1):
        reqs.append(dist.isend(local[rows - top:].contiguous(), dst=down, group=group, tag=_TAG_TOP))
    if bottom > 0 and (periodic or rank > 0):
        reqs.append(dist.isend(local[:bottom].contiguous(), dst=up, group=group, tag=_TAG_BOTTOM))
    for r in reqs:
        r.wait()
    parts = ([recv_top] if has_top else []) + [local] + ([recv_bottom] if has_bottom else [])
    return torch.cat(parts), (top if has_top else 0), (bottom if has_bottom else 0)


def sharded_sweep(local: torch.Tensor, compute: Callable[[torch.Tensor], torch.Tensor], top: int,
                  bottom: int, periodic: bool, group=None) -> torch.Tensor:
    """One stencil sweep of a row band: halo exchange, then `compute` on the padded band (a
    stencil with the grid's x boundary; its rows' wrap or untouched edges only reach halo rows),
    then the band's own rows of the result."""
    padded, t, _ = exchange_halo(local, top, bottom, periodic, group)
    out = compute(padded)
    return out[t:t + local.shape[0]]


def transpose_bands(local: torch.Tensor, n: int, group=None) -> torch.Tensor:
    """Row band -> column band of an n x n field: rank q holds rows band(n, world, q) of A and
    receives rows band(n, world, q) of A^T (the columns of its band, as rows)."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    r0, r1 = band(n, world, rank)
    if local.shape != (r1 - r0, n):
        raise ValueError(f"band of shape {tuple(local.shape)}, expected {(r1 - r0, n)}")
    out = torch.empty((r1 - r0, n), dtype=local.dtype, device=local.device)
    out[:, r0:r1] = local[:, r0:r1].t()  # my rows x my columns
    # from every other rank q: its rows x my columns, transposed into my rows of A^T
    reqs = []
    recv = {}
    for q in range(world):
        if q == rank:
            continue
        q0, q1 = band(n, world, q)
        recv[q] = torch.empty((q1 - q0, r1 - r0), dtype=local.dtype, device=local.device)
        reqs.append(dist.irecv(recv[q], src=q, group=group, tag=_TAG_T))
    for q in range(world):
        if q == rank:
            continue
        c0, c1 = band(n, world, q)
        reqs.append(dist.isend(local[:, c0:c1].contiguous(), dst=q, group=group, tag=_TAG_T))
    for r in reqs:
        r.wait()
    for q, blk in recv.items():
        q0, q1 = band(n, world, q)
        out[:, q0:q1] = blk.t()
    return out


def allreduce_sum(values: torch.Tensor, group=None) -> torch.Tensor:
    """Sum over ranks of per-rank FP64 partial sums (mass, energy)."""
    t = values.to(torch.float64).clone()
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def sharded_ch_step(prev: torch.Tensor, cur: torch.Tensor, n: int,
                    rhs: Callable[[torch.Tensor, torch.Tensor], torch.Tensor],
                    line_solve: Callable[[torch.Tensor], torch.Tensor], group=None) -> torch.Tensor:
    """One ADI step (Sec. 5.1) of row bands of C^{n-1}, C^n of an n x n periodic grid.
    `rhs(prev_padded, cur_padded)` returns the right-hand side of the band from the bands padded
    with 2 rows each side; `line_solve(b)` solves (I + a P) x = b along the last axis of b."""
    pp, _, _ = exchange_halo(prev, 2, 2, True, group)
    cp, _, _ = exchange_halo(cur, 2, 2, True, group)
    w = line_solve(rhs(pp, cp))                       # x-lines: rows of the band
    v = line_solve(transpose_bands(w, n, group))      # y-lines: columns, as rows
    return 2 * cur - prev + transpose_bands(v, n, group)


class DeviceBandSweep:
    """`compute` for sharded_sweep on the GPU: a 2D plan of this library over the padded band
    (created on first use and kept while the padded shape stays the same; its output buffer starts
    at zero, so cells a non-periodic sweep leaves untouched come back as zeros).  `desc_kw` are the
    StencilDesc fields other than nx, ny."""

    def __init__(self, desc_kw: dict, stream=None):
        from . import StencilDesc, cs_plan_create_2d
        self._desc_kw = dict(desc_kw)
        self._make = lambda nx, ny, i, o: cs_plan_create_2d(StencilDesc(nx=nx, ny=ny, **self._desc_kw), i, o)
        self._stream = stream
        self._plan = None
        self._bufs = None

    def __call__(self, padded: torch.Tensor) -> torch.Tensor:
        from . import cs_compute
        ny, nx = padded.shape
        if self._bufs is None or self._bufs[0].shape != padded.shape or self._bufs[0].dtype != padded.dtype:
            self.close()
            self._bufs = (torch.empty_like(padded), torch.zeros_like(padded))
            self._plan = self._make(nx, ny, self._bufs[0], self._bufs[1])
        self._bufs[0].copy_(padded)
        cur = torch.cuda.current_stream()
        if self._stream is not None:  # the copy above ran on the current stream
            self._stream.wait_stream(cur)
        cs_compute(self._plan, self._stream)
        if self._stream is not None:  # the clone below runs on the current stream
            cur.wait_stream(self._stream)
        return self._bufs[1].clone()

    def close(self):
        if self._plan is not None:
            from . import cs_destroy
            cs_destroy(self._plan)
        self._plan = None
        self._bufs = None


def _stage(t: torch.Tensor, group) -> torch.Tensor:
    """gloo moves CPU tensors only: a device tensor travels through host memory there."""
    return t.cpu() if t.is_cuda and dist.get_backend(group) == "gloo" else t


def exchange_halo_inplace(padded: torch.Tensor, halo: int, group=None, periodic: bool = True) -> None:
    """Fills the `halo` rows above and below the band held in padded[halo:-halo] with the
    neighbours' rows, in place, so the band never moves.  Periodic rows: the first band's
    neighbour above is the last band.  Otherwise (no-flux boundaries) the first band's rows above
    and the last band's rows below are its own rows mirrored about the grid's edge (ghost row -1
    holds row 0, -2 holds row 1, and likewise below), the reflection the full-grid step uses."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    rows = padded.shape[0] - 2 * halo
    if rows < halo:
        raise ValueError(f"band of {rows} rows is thinner than the halo ({halo})")
    up = rank - 1 if rank > 0 else (world - 1 if periodic else None)
    down = rank + 1 if rank < world - 1 else (0 if periodic else None)
    if up is None:
        padded[:halo] = padded[halo:2 * halo].flip(0)
    if down is None:
        padded[rows + halo:] = padded[rows:rows + halo].flip(0)
    if world == 1:
        if periodic:
            padded[:halo] = padded[rows:rows + halo]
            padded[rows + halo:] = padded[halo:2 * halo]
        return
    top = _stage(torch.empty_like(padded[:halo]), group)
    bottom = _stage(torch.empty_like(padded[:halo]), group)
    reqs = []
    if up is not None:
        reqs.append(dist.irecv(top, src=up, group=group, tag=_TAG_TOP))
        reqs.append(dist.isend(_stage(padded[halo:2 * halo].contiguous(), group), dst=up, group=group, tag=_TAG_BOTTOM))
    if down is not None:
        reqs.append(dist.irecv(bottom, src=down, group=group, tag=_TAG_BOTTOM))
        reqs.append(dist.isend(_stage(padded[rows:rows + halo].contiguous(), group), dst=down, group=group, tag=_TAG_TOP))
    for r in reqs:
        r.wait()
    if up is not None:
        padded[:halo].copy_(top)
    if down is not None:
        padded[rows + halo:].copy_(bottom)


def exchange_rows_inplace(padded: torch.Tensor, top: int, bottom: int, group=None, periodic: bool = True) -> None:
    """The stencil sweep's halo exchange, in place: `padded` holds this rank's band with room for
    the `top` rows of the band above and the `bottom` rows of the band below (a stencil's reach
    upwards and downwards).  A non-periodic grid's first band has no room above and its last band
    none below (its sweep leaves those rows untouched, as the full grid's does); with periodic
    rows the first band's neighbour above is the last band.  The received rows land in the
    padded buffer's halo rows, so the band never moves."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    has_top = top > 0 and (periodic or rank > 0)
    has_bottom = bottom > 0 and (periodic or rank < world - 1)
    t = top if has_top else 0
    b = bottom if has_bottom else 0
    rows = padded.shape[0] - t - b
    if rows < max(top, bottom):
        raise ValueError(f"band of {rows} rows is thinner than the stencil's reach ({top}, {bottom})")
    if world == 1:
        if has_top:
            padded[:t] = padded[rows:rows + t]
        if has_bottom:
            padded[t + rows:] = padded[t:t + b]
        return
    up, down = (rank - 1) % world, (rank + 1) % world
    recv_top = _stage(torch.empty_like(padded[:t]), group) if has_top else None
    recv_bottom = _stage(torch.empty_like(padded[t + rows:]), group) if has_bottom else None
    reqs = []
    if has_top:
        reqs.append(dist.irecv(recv_top, src=up, group=group, tag=_TAG_TOP))
    if has_bottom:
        reqs.append(dist.irecv(recv_bottom, src=down, group=group, tag=_TAG_BOTTOM))
    # my last `top` rows are the top halo of the band below; my first `bottom` rows the bottom
    # halo of the band above
    if top > 0 and (periodic or rank < world - 1):
        reqs.append(dist.isend(_stage(padded[t + rows - top:t + rows].contiguous(), group), dst=down, group=group,
                               tag=_TAG_TOP))
    if bottom > 0 and (periodic or rank > 0):
        reqs.append(dist.isend(_stage(padded[t:t + bottom].contiguous(), group), dst=up, group=group,
                               tag=_TAG_BOTTOM))
    for r in reqs:
        r.wait()
    if has_top:
        padded[:t].copy_(recv_top)
    if has_bottom:
        padded[t + rows:].copy_(recv_bottom)


class DeviceBandStencil:
    """A stencil sweep of this rank's row band of an nx-wide grid with no copy of the band: the
    band lives in the middle of a persistent padded input buffer (`band()` is a view of it: write
    the band there), the neighbours' rows are received in place into its halo rows
    (exchange_rows_inplace), one plan of this library is bound to the padded input and output
    buffers for the object's life, and `__call__` returns the band's rows of the output as a view.
    `swap()` makes the output the next sweep's input (cs_swap), for repeated sweeps.  `desc_kw` are
    the StencilDesc fields other than nx and ny (the grid's boundary condition, extents, weights or
    function, dtype).  The output buffer starts at zero, so cells a non-periodic sweep leaves
    untouched read 0 until written."""

    def __init__(self, rows: int, nx: int, desc_kw: dict, group=None):
        from . import StencilDesc, cs_plan_create_2d, CS_BC_PERIODIC, CS_F64
        self.group = group
        self._kw = dict(desc_kw)
        self.T, self.B = int(self._kw.get("top", 0)), int(self._kw.get("bottom", 0))
        self.periodic = self._kw.get("bc", CS_BC_PERIODIC) == CS_BC_PERIODIC
        world = dist.get_world_size(group)
        rank = dist.get_rank(group)
        self.t = self.T if self.T > 0 and (self.periodic or rank > 0) else 0
        self.b = self.B if self.B > 0 and (self.periodic or rank < world - 1) else 0
        self.rows = rows
        tdt = torch.float64 if self._kw.get("dtype", CS_F64) == CS_F64 else torch.float32
        self._in = torch.zeros(rows + self.t + self.b, nx, dtype=tdt, device="cuda")
        self._out = torch.zeros_like(self._in)
        self.plan = cs_plan_create_2d(StencilDesc(nx=nx, ny=rows + self.t + self.b, **self._kw), self._in, self._out)

    def band(self) -> torch.Tensor:
        """This rank's band of the input (a view of the padded input buffer)."""
        return self._in[self.t:self.t + self.rows]

    def __call__(self) -> torch.Tensor:
        from . import cs_compute
        exchange_rows_inplace(self._in, self.T, self.B, self.group, self.periodic)
        cs_compute(self.plan)
        return self._out[self.t:self.t + self.rows]

    def swap(self) -> None:
        from . import cs_swap
        cs_swap(self.plan)
        self._in, self._out = self._out, self._in

    def close(self) -> None:
        from . import cs_destroy
        if self.plan is not None:
            cs_destroy(self.plan)
        self.plan = None


def transpose_bands_device(local: torch.Tensor, n: int, group=None) -> torch.Tensor:
    """transpose_bands for device tensors on any backend: a single rank transposes in device memory;
    gloo ranks exchange through host memory, NCCL ranks device to device."""
    if dist.get_world_size(group) == 1:
        return local.t().contiguous()
    if local.is_cuda and dist.get_backend(group) == "gloo":
        return transpose_bands(local.cpu(), n, group).to(local.device)
    return transpose_bands(local, n, group)


def _all_gather_rows(t: torch.Tensor, group=None) -> torch.Tensor:
    """The ranks' equal-sized tensors `t` concatenated in rank order (through host memory on gloo)."""
    world = dist.get_world_size(group)
    if world == 1:
        return t
    src = _stage(t.contiguous(), group)
    parts = [torch.empty_like(src) for _ in range(world)]
    dist.all_gather(parts, src, group=group)
    return torch.cat(parts).to(t.device)


class DeviceCHBand:
    """The Cahn-Hilliard ADI step (Sec. 5.1) of an n x n grid split into row bands over the ranks
    of `group`, one band per rank, computed by this library's band entry points (cs_ch_band_*):
    halo exchange of C^n and C^{n-1} (2 rows, in place in padded buffers), the band's right-hand
    side, the x line solves, the y line solves and the update.  The y lines run in one of two ways:
      * "chunks" (whenever the spike method's chunks of a line, cs_ch_partition, split evenly over
        the ranks: then every band is a whole number of chunks of every column): each rank solves
        its chunks locally (cs_ch_band_ycols_local), the ranks all-gather the chunks' end values (4
        per column and chunk: 4 * chunks * n values in all), and each applies the spike correction
        to its own chunks (cs_ch_band_ycols_correct); the field never moves between ranks;
      * "transposes" (otherwise): an all-to-all transpose gives each rank a band of columns, solved
        as rows, and a second transpose brings the result back.
    Both give the full-grid step's values bit for bit.  `c0` is this rank's band of the initial
    field (rows band(n, world, rank), on the GPU; C^{-1} = C^0).  `boundary` is CS_CH_PERIODIC or
    CS_CH_NOFLUX (mirrored halos at the grid's first and last rows, non-cyclic line solves).  The
    three padded fields rotate as in cs_ch_step."""

    HALO = 2

    def __init__(self, n: int, storage: int, D: float, gamma: float, dt: float, c0: torch.Tensor, group=None,
                 boundary: int = 0, mode: str = "auto"):
        from . import CHDesc, CS_F64, CS_CH_PERIODIC, cs_ch_band_create, cs_ch_partition
        self.group = group
        self.periodic = boundary == CS_CH_PERIODIC
        self.n = n
        world = dist.get_world_size(group)
        rank = dist.get_rank(group)
        r0, r1 = band(n, world, rank)
        self.rows = r1 - r0
        desc = CHDesc(n=n, storage=storage, D=D, gamma=gamma, dt=dt, boundary=boundary)
        chunks, chunk_len = cs_ch_partition(desc)
        even = chunks % world == 0  # then band(n, world, rank) is a whole number of chunks
        if mode == "auto":
            mode = "chunks" if even else "transposes"
        if mode not in ("chunks", "transposes") or (mode == "chunks" and not even):
            raise ValueError(f"mode {mode!r}: the {chunks} chunks of a line do not split over {world} ranks"
                             if mode == "chunks" else f"unknown mode {mode!r}")
        self.mode = mode
        self.chunk0 = r0 // chunk_len
        if tuple(c0.shape) != (self.rows, n):
            raise ValueError(f"band of shape {tuple(c0.shape)}, expected {(self.rows, n)}")
        tdt = torch.float64 if storage == CS_F64 else torch.float32
        self.f = [torch.zeros(self.rows + 2 * self.HALO, n, dtype=tdt, device=c0.device) for _ in range(3)]
        for k in (0, 1):
            self.f[k][self.HALO:self.HALO + self.rows] = c0.to(tdt)
        self.ip, self.ic, self.inext = 0, 1, 2
        self.rhs = torch.empty(self.rows, n, dtype=torch.float64, device=c0.device)
        self.sums = torch.zeros(2, dtype=torch.float64, device=c0.device)
        self.ends = torch.empty(4 * (self.rows // chunk_len) * n, dtype=torch.float64, device=c0.device) \
            if mode == "chunks" else None
        self.plan = cs_ch_band_create(desc, self.rows)
        self.steps = 0

    def _halos(self):
        exchange_halo_inplace(self.f[self.ip], self.HALO, self.group, self.periodic)
        exchange_halo_inplace(self.f[self.ic], self.HALO, self.group, self.periodic)

    def invariants(self):
        """(mass, energy) of the current field: the bands' FP64 sums, allreduced."""
        from . import cs_ch_band_rhs
        self._halos()
        cs_ch_band_rhs(self.plan, self.f[self.ip], self.f[self.ic], None, self.sums)
        return tuple(float(v) for v in allreduce_sum(_stage(self.sums, self.group), self.group))

    def step(self, nsteps: int = 1) -> None:
        from . import (cs_ch_band_rhs, cs_ch_band_solve, cs_ch_band_update, cs_ch_band_ycols_correct,
                       cs_ch_band_ycols_local)
        for _ in range(nsteps):
            self._halos()
            cs_ch_band_rhs(self.plan, self.f[self.ip], self.f[self.ic], self.rhs)
            cs_ch_band_solve(self.plan, self.rhs, self.rhs)                   # x lines: the band's rows
            if self.mode == "chunks":
                # y lines: the band's chunks of every column, then their end values from all bands
                cs_ch_band_ycols_local(self.plan, self.chunk0, self.rhs, self.ends)
                ends_all = _all_gather_rows(self.ends, self.group)
                cs_ch_band_ycols_correct(self.plan, self.chunk0, ends_all, self.rhs)
                v = self.rhs
            else:
                wt = transpose_bands_device(self.rhs, self.n, self.group)     # a band of columns, as rows
                cs_ch_band_solve(self.plan, wt, wt)                           # y lines
                v = transpose_bands_device(wt, self.n, self.group)
            cs_ch_band_update(self.plan, self.f[self.ip], self.f[self.ic], v, self.f[self.inext])
            self.ip, self.ic, self.inext = self.ic, self.inext, self.ip
            self.steps += 1

    def field(self) -> torch.Tensor:
        """This rank's band of the current field C^n (a view of its padded buffer)."""
        return self.f[self.ic][self.HALO:self.HALO + self.rows]

    def close(self) -> None:
        from . import cs_destroy
        if self.plan is not None:
            cs_destroy(self.plan)
        self.plan = None
