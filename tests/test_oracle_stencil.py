"""Pins for the oracle's stencil routines (CPU only).

Each check ties the oracle to something other than itself: exact discrete symbols of Fourier
modes, exactness on polynomials, the paper's worked example (Sec. 4.1), impulse responses that
fix the weight ordering of Sec. 5.2, translation invariance, and a library correlation
(scipy.signal.correlate2d) on integer data where every sum is exact.
"""
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.signal

import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def load_fd8():
    rows = []
    with open(os.path.join(GOLD, "fd8_second_derivative.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            off, num, den = line.split()
            rows.append((int(off), Fraction(int(num), int(den))))
    return rows


def load_example_config():
    cfg = {}
    with open(os.path.join(GOLD, "paper_example_config.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split()[:2]
            cfg[k] = float(v)
    return cfg


def test_fd8_golden_weights_are_taylor_exact():
    """The golden 8th-order weights satisfy the Taylor conditions exactly:
    sum_k w_k k^m = 2 (m = 2), 0 for every other m < 10."""
    rows = load_fd8()
    assert [o for o, _ in rows] == list(range(-4, 5))
    for m in range(10):
        s = sum(w * Fraction(o) ** m for o, w in rows)
        assert s == (2 if m == 2 else 0), m


def test_paper_example_sec41_second_derivative_of_sin(orc):
    """Sec. 4.1: 8th-order d^2/dx^2 of sin(x), nx=1024, ny=512, lx=2 pi, 4 points left/right,
    non-periodic.  Interior = -sin(x) to O(h^8) + rounding; the 4 cells at each x end stay 0."""
    cfg = load_example_config()
    nx, ny = int(cfg["example_nx"]), int(cfg["example_ny"])
    L = int(cfg["example_numStenLeft"])
    R = int(cfg["example_numStenRight"])
    dx = cfg["example_lx"] / nx
    x = np.arange(nx) * dx
    data_old = np.tile(np.sin(x), (ny, 1))
    w = np.array([float(f) for _, f in load_fd8()]) / dx ** 2
    assert w.size == int(cfg["example_numSten"])
    out = orc.stencil2d(data_old, w, orc.DIR_X, orc.BC_NONPERIODIC, left=L, right=R)
    interior = out[:, L:nx - R]
    err = np.abs(interior + np.sin(x)[None, L:nx - R]).max()
    # truncation ~ h^8 |f^(10)| / 1260 ~ 1e-21; rounding ~ eps * sum|w| = eps * 6.7/dx^2 ~ 4e-11
    assert err < 1e-9
    assert np.all(out[:, :L] == cfg["example_untouched_value"])
    assert np.all(out[:, nx - R:] == cfg["example_untouched_value"])


def lap5(h):
    return np.array([0, 1, 0, 1, -4, 1, 0, 1, 0], dtype=float) / h ** 2


def lap9(h):
    return np.array([1, 4, 1, 4, -20, 4, 1, 4, 1], dtype=float) / (6 * h ** 2)


def biharm13(h):
    w = np.zeros((5, 5))
    w[2, 2] = 20
    for d in [(1, 2), (3, 2), (2, 1), (2, 3)]:
        w[d] = -8
    for d in [(1, 1), (1, 3), (3, 1), (3, 3)]:
        w[d] = 2
    for d in [(0, 2), (4, 2), (2, 0), (2, 4)]:
        w[d] = 1
    return w.ravel() / h ** 4


D1X4 = np.array([1, -8, 0, 8, -1], dtype=float) / 12.0  # 4th-order d/dx, per unit h


@pytest.mark.parametrize("n,k,l", [(64, 3, 5), (96, 17, 2), (128, 40, 63)])
def test_periodic_symbols_of_fourier_modes(orc, n, k, l):
    """On u = sin(kx + ly + phi) a periodic stencil returns its exact discrete symbol times u
    (or times the quadrature mode for odd stencils)."""
    h = 2 * np.pi / n
    u = W.single_mode(n, k, l, 1.0, phase=0.7)
    x = np.arange(n) * h
    theta = k * x[None, :] + l * x[:, None] + 0.7
    sk2, sl2 = np.sin(k * h / 2) ** 2, np.sin(l * h / 2) ** 2
    ck, cl = np.cos(k * h), np.cos(l * h)
    cases = [
        (lap5(h), 1, 1, 1, 1, -(4 / h ** 2) * (sk2 + sl2) * u),
        (lap9(h), 1, 1, 1, 1, (-20 + 8 * ck + 8 * cl + 4 * ck * cl) / (6 * h ** 2) * u),
        (biharm13(h), 2, 2, 2, 2, (16 / h ** 4) * (sk2 + sl2) ** 2 * u),
    ]
    for w, L, R, T, B, expect in cases:
        out = orc.stencil2d(u, w, orc.DIR_XY, orc.BC_PERIODIC, L, R, T, B)
        scale = np.abs(w).sum()
        # the inputs sin(theta) carry ~|theta| eps rounding (|theta| <= ~200 here)
        assert np.abs(out - expect).max() <= 1e-13 * scale, (L, T)
    # odd first-derivative stencils: x direction and y direction
    out = orc.stencil2d(u, D1X4 / h, orc.DIR_X, orc.BC_PERIODIC, 2, 2)
    expect = (8 * np.sin(k * h) - np.sin(2 * k * h)) / (6 * h) * np.cos(theta)
    assert np.abs(out - expect).max() <= 1e-13 * np.abs(D1X4 / h).sum()
    out = orc.stencil2d(u, D1X4 / h, orc.DIR_Y, orc.BC_PERIODIC, 0, 0, 2, 2)
    expect = (8 * np.sin(l * h) - np.sin(2 * l * h)) / (6 * h) * np.cos(theta)
    assert np.abs(out - expect).max() <= 1e-13 * np.abs(D1X4 / h).sum()


def test_polynomial_exactness_nonperiodic(orc):
    """Interior values are exact (to rounding) on polynomials of the stencil's order:
    5-point Laplacian on cubics, 4th-order d/dx on quartics, 13-point biharmonic on quintics."""
    n = 40
    h = 1.0 / 16
    x = (np.arange(n) - n / 2) * h
    X, Y = np.meshgrid(x, x)  # X varies along axis 1 (i), Y along axis 0 (j)
    u3 = 1 + 2 * X - Y + X * Y + 0.5 * X ** 3 - 0.25 * X * Y ** 2 + Y ** 3
    lap_u3 = 3 * X - 0.5 * X + 6 * Y
    out = orc.stencil2d(u3, lap5(h), orc.DIR_XY, orc.BC_NONPERIODIC, 1, 1, 1, 1)
    assert np.abs(out[1:-1, 1:-1] - lap_u3[1:-1, 1:-1]).max() < 1e-10
    u4 = X ** 4 - 2 * X ** 3 * Y + X + Y ** 2
    dx_u4 = 4 * X ** 3 - 6 * X ** 2 * Y + 1
    out = orc.stencil2d(u4, D1X4 / h, orc.DIR_X, orc.BC_NONPERIODIC, 2, 2)
    assert np.abs(out[:, 2:-2] - dx_u4[:, 2:-2]).max() < 1e-11
    u5 = X ** 5 / 120 + X ** 2 * Y ** 2 / 4 + Y ** 4 / 24 - X * Y ** 3
    bih_u5 = X + 2 * 1.0 + 1.0  # d4x: X; 2 d2x d2y: 2*(1); d4y: 1
    out = orc.stencil2d(u5, biharm13(h), orc.DIR_XY, orc.BC_NONPERIODIC, 2, 2, 2, 2)
    assert np.abs(out[2:-2, 2:-2] - bih_u5[2:-2, 2:-2]).max() < 1e-7


def test_constant_field_gives_zero_for_zero_sum_weights(orc):
    u = np.full((33, 47), 3.25)
    for w, L, R, T, B, d in [(np.array([1, 4, 1, 4, -20, 4, 1, 4, 1.0]), 1, 1, 1, 1, orc.DIR_XY),
                             (np.array([-1, 16, -30, 16, -1.0]), 2, 2, 0, 0, orc.DIR_X),
                             (np.array([1, -8, 0, 8, -1.0]), 0, 0, 2, 2, orc.DIR_Y)]:
        for bc in (orc.BC_PERIODIC, orc.BC_NONPERIODIC):
            out = orc.stencil2d(u, w, d, bc, L, R, T, B)
            assert np.all(out == 0.0)


@pytest.mark.parametrize("L,R,T,B", [(0, 2, 1, 0), (3, 1, 0, 2), (1, 0, 2, 3), (2, 3, 3, 1)])
def test_impulse_response_fixes_weight_order(orc, L, R, T, B):
    """A unit impulse at (j0, i0) returns the flipped stencil: out[j0 + T - q, i0 + L - p] = w[q, p]
    with row q = 0 the top row (j - T), as Sec. 5.2 orders the weights."""
    ny, nx = 13, 17
    width, height = L + R + 1, T + B + 1
    w = np.arange(1, width * height + 1, dtype=float)
    j0, i0 = 6, 8
    u = np.zeros((ny, nx))
    u[j0, i0] = 1.0
    out = orc.stencil2d(u, w, orc.DIR_XY, orc.BC_PERIODIC, L, R, T, B)
    expect = np.zeros((ny, nx))
    for q in range(height):
        for p in range(width):
            expect[(j0 + T - q) % ny, (i0 + L - p) % nx] = w[q * width + p]
    assert np.array_equal(out, expect)


@pytest.mark.parametrize("shape", [(1, 1), (2, 3), (5, 4), (7, 16), (17, 9)])
@pytest.mark.parametrize("L,R,T,B", [(0, 0, 0, 0), (1, 1, 1, 1), (3, 0, 1, 2), (2, 3, 3, 2)])
def test_integer_fields_match_library_correlation(orc, shape, L, R, T, B):
    """Periodic: the oracle equals scipy.signal.correlate2d of the wrap-padded field, bit for bit
    on integer data (all sums exact), including grids smaller than the stencil."""
    ny, nx = shape
    u = W.integer_field(ny, nx, seed=ny * 100 + nx)
    w = W.integer_weights((L + R + 1) * (T + B + 1), seed=L + 10 * R + 100 * T + 1000 * B)
    out = orc.stencil2d(u, w, orc.DIR_XY, orc.BC_PERIODIC, L, R, T, B)
    padded = np.pad(u, ((T, B), (L, R)), mode="wrap")  # repeats periodically when wider
    lib = scipy.signal.correlate2d(padded, w.reshape(T + B + 1, L + R + 1), mode="valid")
    assert np.array_equal(out, lib)


@pytest.mark.parametrize("L,R,T,B", [(1, 2, 0, 3), (3, 3, 2, 1)])
def test_nonperiodic_writes_exactly_the_interior(orc, L, R, T, B):
    """np: cells within the stencil extent of the boundary keep their prior contents bit for bit;
    interior cells equal the (unwrapped) library correlation."""
    ny, nx = 15, 21
    u = W.integer_field(ny, nx, seed=5)
    w = W.integer_weights((L + R + 1) * (T + B + 1), seed=9)
    sentinel = np.full((ny, nx), np.float64(-7.123456789e300))
    out = orc.stencil2d(u, w, orc.DIR_XY, orc.BC_NONPERIODIC, L, R, T, B, out=sentinel)
    lib = scipy.signal.correlate2d(u, w.reshape(T + B + 1, L + R + 1), mode="valid")
    assert np.array_equal(out[T:ny - B, L:nx - R], lib)
    mask = np.ones((ny, nx), bool)
    mask[T:ny - B, L:nx - R] = False
    assert np.array_equal(out[mask], sentinel[mask])


def test_translation_invariance_and_linearity(orc):
    n = 48
    u = W.uniform_field(n, n, seed=3)
    v = W.uniform_field(n, n, seed=4)
    w = W.uniform_field(5, 5, seed=6).ravel()
    S = lambda f: orc.stencil2d(f, w, orc.DIR_XY, orc.BC_PERIODIC, 2, 2, 2, 2)
    su = S(u)
    for dy, dx in [(1, 0), (0, 5), (7, 3)]:
        assert np.array_equal(np.roll(su, (dy, dx), axis=(0, 1)), S(np.roll(u, (dy, dx), axis=(0, 1))))
    lin = S(2.5 * u - 0.75 * v)
    assert np.abs(lin - (2.5 * su - 0.75 * S(v))).max() < 1e-13 * np.abs(w).sum() * 4


def test_x_and_y_directions_are_transposes(orc):
    u = W.uniform_field(20, 31, seed=8)
    w = np.array([0.5, -1.25, 3.0, 2.0])
    ox = orc.stencil2d(u, w, orc.DIR_X, orc.BC_PERIODIC, 1, 2)
    oy = orc.stencil2d(u.T, w, orc.DIR_Y, orc.BC_PERIODIC, 0, 0, 1, 2)
    assert np.array_equal(ox, oy.T)


def test_invalid_arguments_are_rejected(orc):
    u = np.zeros((4, 4))
    with pytest.raises(ValueError):
        orc.stencil2d(u, np.ones(3), orc.DIR_X, orc.BC_PERIODIC, 1, 1, 1, 0)
    with pytest.raises(ValueError):
        orc.stencil2d(u, np.ones(2), orc.DIR_X, orc.BC_PERIODIC, 1, 1)


# ---- user-function stencils (Sec. 4.2, Sec. 5.2) ----------------------------------------------

def test_fn_central_d2x_matches_sec42_example(orc):
    """Sec. 4.2: the function-pointer version of the second derivative of sin(x) with
    coe = {1/dx^2}; interior equals the discrete symbol -(4/dx^2) sin^2(dx/2) sin(x) exactly."""
    nx, ny = 1024, 8
    dx = 2 * np.pi / nx
    x = np.arange(nx) * dx
    u = np.tile(np.sin(x), (ny, 1))
    out = orc.stencil2d_fn(u, orc.FN_CENTRAL_D2X, [1.0 / dx ** 2], orc.BC_NONPERIODIC)
    sym = -(4 / dx ** 2) * np.sin(dx / 2) ** 2
    assert np.abs(out[:, 1:-1] - sym * np.sin(x)[None, 1:-1]).max() < 1e-14 * 4 / dx ** 2
    assert np.abs(out[:, 1:-1] + np.sin(x)[None, 1:-1]).max() < 1e-5  # O(dx^2) truncation
    assert np.all(out[:, 0] == 0) and np.all(out[:, -1] == 0)


@pytest.mark.parametrize("n,k,l,A", [(64, 2, 3, 0.9), (128, 5, 1, 0.4)])
def test_fn_nonlinear_closed_forms(orc, n, k, l, A):
    """For c = A sin(theta): c^3 - c = (3A^3/4 - A) sin(theta) - (A^3/4) sin(3 theta), and the
    5-point Laplacian has symbol -mu(k, l) = -(4/h^2)(sin^2(kh/2) + sin^2(lh/2)), so
    Lap(c^3 - c) and c^3 - c - Lap(c) have exact closed forms."""
    h = 2 * np.pi / n
    x = np.arange(n) * h
    th = k * x[None, :] + l * x[:, None] + 0.2
    c = A * np.sin(th)
    mu = lambda kk, ll: (4 / h ** 2) * (np.sin(kk * h / 2) ** 2 + np.sin(ll * h / 2) ** 2)
    lap_n = -mu(k, l) * (3 * A ** 3 / 4 - A) * np.sin(th) + mu(3 * k, 3 * l) * (A ** 3 / 4) * np.sin(3 * th)
    out = orc.stencil2d_fn(c, orc.FN_CH_NONLIN_LAP, [1 / h ** 2], orc.BC_PERIODIC)
    assert np.abs(out - lap_n).max() < 1e-13 * 8 / h ** 2
    cml = (3 * A ** 3 / 4 - A) * np.sin(th) - (A ** 3 / 4) * np.sin(3 * th) + mu(k, l) * c
    out = orc.stencil2d_fn(c, orc.FN_CUBIC_MINUS_LAP, [1 / h ** 2], orc.BC_PERIODIC)
    assert np.abs(out - cml).max() < 1e-13 * 8 / h ** 2


def test_fn_nonperiodic_leaves_boundary(orc):
    u = W.uniform_field(9, 11, seed=2)
    sentinel = np.full(u.shape, 5.5)
    out = orc.stencil2d_fn(u, orc.FN_CUBIC_MINUS_LAP, [2.0], orc.BC_NONPERIODIC, out=sentinel)
    assert np.all(out[0] == 5.5) and np.all(out[-1] == 5.5)
    assert np.all(out[:, 0] == 5.5) and np.all(out[:, -1] == 5.5)
    assert not np.any(out[1:-1, 1:-1] == 5.5)


# ---- batched 1D lines -------------------------------------------------------------------------

def test_batch1d_matches_per_line_library_correlation(orc):
    """Integer data: each periodic line equals numpy.correlate of the wrap-padded line."""
    off = W.ragged_offsets(40, seed=11, lmin=3, lmax=50)
    u = W.integer_field(1, int(off[-1]), seed=12).ravel()
    w = np.array([-1.0, 16.0, -30.0, 16.0, -1.0])
    out = orc.stencil1d_batch(u, off, w, orc.BC_PERIODIC, 2, 2)
    for m in range(off.size - 1):
        line = u[off[m]:off[m + 1]]
        padded = np.pad(line, (2, 2), mode="wrap")
        assert np.array_equal(out[off[m]:off[m + 1]], np.correlate(padded, w, mode="valid"))


def test_batch1d_symbol_and_polynomial(orc):
    """Periodic lines of different lengths: the 4th-order second derivative
    (-1, 16, -30, 16, -1) / (12 h^2) has symbol (-30 + 32 cos kh - 2 cos 2kh) / (12 h^2), each line
    with its own h = 2 pi / length; non-periodic interiors are exact on quintics."""
    lengths = [64, 100, 257, 4096]
    off = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    u = np.empty(off[-1])
    expect = np.empty_like(u)
    k = 5
    for m, L in enumerate(lengths):
        h = 2 * np.pi / L
        x = np.arange(L) * h
        u[off[m]:off[m + 1]] = np.sin(k * x + 0.4)
        expect[off[m]:off[m + 1]] = (-30 + 32 * np.cos(k * h) - 2 * np.cos(2 * k * h)) / (12 * h ** 2) * np.sin(k * x + 0.4)
    # the per-line h enters through a per-line weight scale; check each line separately
    for m, L in enumerate(lengths):
        h = 2 * np.pi / L
        w = np.array([-1.0, 16, -30, 16, -1]) / (12 * h ** 2)
        out = orc.stencil1d_batch(u, off, w, orc.BC_PERIODIC, 2, 2)
        seg = slice(off[m], off[m + 1])
        assert np.abs(out[seg] - expect[seg]).max() < 1e-14 * 64 / (12 * h ** 2)
    h = 0.05
    x = (np.arange(30) - 15) * h
    p = x ** 5 - 3 * x ** 4 + x
    d2p = 20 * x ** 3 - 36 * x ** 2
    out = orc.stencil1d_batch(p, np.array([0, 30]), np.array([-1.0, 16, -30, 16, -1]) / (12 * h * h),
                              orc.BC_NONPERIODIC, 2, 2)
    assert np.abs(out[2:-2] - d2p[2:-2]).max() < 1e-9
    assert np.all(out[:2] == 0) and np.all(out[-2:] == 0)
