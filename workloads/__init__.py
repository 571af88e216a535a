"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module only draws input data (numpy PCG64, seed recorded by the caller); it contains none
of the stencil or Cahn-Hilliard arithmetic, so it can feed both the GPU library and the CPU
oracle without coupling them.  The recipes follow the workloads of the paper's examples and
benchmark (Sec. 4: derivatives of trigonometric fields; Sec. 5.3-5.4: Cahn-Hilliard deep quench
C0 ~ U[-0.1, 0.1], N x N periodic grids on (0, 2 pi)^2).
"""
from __future__ import annotations

import numpy as np

TWO_PI = 2.0 * np.pi


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_field(ny: int, nx: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """U[lo, hi) values, FP64, shape (ny, nx)."""
    return rng(seed).uniform(lo, hi, size=(ny, nx))


def integer_field(ny: int, nx: int, seed: int, bound: int = 1024) -> np.ndarray:
    """Integers in [-bound, bound] stored as FP64: with small-integer weights every stencil sum
    is exact in FP64 and FP32, so index and halo maps can be compared bit for bit."""
    return rng(seed).integers(-bound, bound + 1, size=(ny, nx)).astype(np.float64)


def integer_weights(count: int, seed: int, bound: int = 8) -> np.ndarray:
    return rng(seed).integers(-bound, bound + 1, size=count).astype(np.float64)


def sines_field(n: int, seed: int, modes: int = 8, kmax: int = 32, noise: float = 1e-3,
                ny: int | None = None) -> np.ndarray:
    """Sum of ``modes`` random-phase plane waves on the periodic (0, 2 pi)^2 grid,
    u = sum_m (1/modes) sin(kx_m x + ky_m y + phi_m) + U[-noise, noise],
    kx, ky integers in [1, kmax], phi ~ U[0, 2 pi).  x = i h, y = j h, h = 2 pi / n."""
    ny = n if ny is None else ny
    g = rng(seed)
    kx = g.integers(1, kmax + 1, size=modes)
    ky = g.integers(1, kmax + 1, size=modes)
    phi = g.uniform(0.0, TWO_PI, size=modes)
    x = np.arange(n) * (TWO_PI / n)
    y = np.arange(ny) * (TWO_PI / ny)
    u = np.zeros((ny, n))
    for m in range(modes):
        # sin(a + b) = sin a cos b + cos a sin b, evaluated as two outer products
        ax = kx[m] * x
        by = ky[m] * y + phi[m]
        u += (np.outer(np.cos(by), np.sin(ax)) + np.outer(np.sin(by), np.cos(ax))) / modes
    u += g.uniform(-noise, noise, size=(ny, n))
    return u


def ragged_offsets(num_lines: int, seed: int, lmin: int = 64, lmax: int = 4096) -> np.ndarray:
    """Line lengths log-uniform in [lmin, lmax]: l = min(lmax, floor(exp(U[ln lmin, ln(lmax+1))))).
    Lines are packed back to back; returns offsets[num_lines + 1] (int64)."""
    g = rng(seed)
    u = g.uniform(np.log(lmin), np.log(lmax + 1), size=num_lines)
    lengths = np.minimum(lmax, np.floor(np.exp(u))).astype(np.int64)
    lengths = np.maximum(lengths, lmin)
    off = np.zeros(num_lines + 1, dtype=np.int64)
    np.cumsum(lengths, out=off[1:])
    return off


def sines_lines(offsets: np.ndarray, seed: int, modes: int = 8, kmax: int = 32,
                noise: float = 1e-3) -> np.ndarray:
    """A periodic random-phase sine sum on each line of a ragged batch (wavenumbers capped at
    length/4 so every mode is resolved), plus U[-noise, noise]."""
    g = rng(seed)
    nl = offsets.size - 1
    total = int(offsets[-1])
    out = np.empty(total)
    lengths = np.diff(offsets)
    k = g.integers(1, kmax + 1, size=(nl, modes))
    phi = g.uniform(0.0, TWO_PI, size=(nl, modes))
    for L in np.unique(lengths):
        rows = np.nonzero(lengths == L)[0]
        kk = np.minimum(k[rows], max(1, L // 4))
        x = np.arange(L) * (TWO_PI / L)
        vals = np.sin(kk[:, :, None] * x[None, None, :] + phi[rows][:, :, None]).sum(axis=1) / modes
        idx = offsets[rows][:, None] + np.arange(L)[None, :]
        out[idx] = vals
    out += g.uniform(-noise, noise, size=total)
    return out


def ch_initial(n: int, seed: int, amplitude: float = 0.1) -> np.ndarray:
    """Deep-quench initial condition of Sec. 5.3: U[-amplitude, amplitude], sample mean removed."""
    c = rng(seed).uniform(-amplitude, amplitude, size=(n, n))
    return c - c.mean()


def low_mode_field(n: int, seed: int, modes: int = 6, kmax: int = 6, amplitude: float = 0.1) -> np.ndarray:
    """A resolved field: ``modes`` plane waves with wavenumbers in [1, kmax], total amplitude
    ``amplitude``, sample mean removed."""
    g = rng(seed)
    x = np.arange(n) * (TWO_PI / n)
    c = np.zeros((n, n))
    for _ in range(modes):
        k, l = g.integers(1, kmax + 1, size=2)
        ph = g.uniform(0.0, TWO_PI)
        c += amplitude / modes * np.sin(k * x[None, :] + l * x[:, None] + ph)
    return c - c.mean()


def single_mode(n: int, k: int, l: int, amplitude: float, phase: float = 0.3) -> np.ndarray:
    """amplitude * sin(k x + l y + phase) on the n x n periodic grid."""
    x = np.arange(n) * (TWO_PI / n)
    return amplitude * np.sin(k * x[None, :] + l * x[:, None] + phase)


def device_uniform(shape, seed: int, lo: float, hi: float, device, dtype):
    """U[lo, hi) values drawn directly on the device (torch Philox generator, seeded); used for
    the serving workload, whose many resident fields are too large to stage through the host."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return torch.empty(shape, dtype=dtype, device=device).uniform_(lo, hi, generator=g)
