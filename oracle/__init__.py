"""Plain FP64 CPU oracle for the cuSten hot path (arXiv:1902.09931).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.  It wraps ``cs_oracle.c`` (plain C loops over the
paper's definitions, binary64) through ctypes and builds it with gcc on first use.  It shares
no code with the GPU library in ``paper_1902_09931_gb300``.

What each routine computes, with the passage it follows:

* ``stencil2d``        -- weighted stencil, x / y / xy, periodic or non-periodic (Sec. 2, 3, 5.2)
* ``stencil2d_fn``     -- user-function stencils of Sec. 4.2 and Sec. 5.2
* ``stencil1d_batch``  -- the x stencil on each line of a ragged batch (Abstract, Sec. 5.4)
* ``cyclic_penta_solve`` -- (I + a circ(1,-4,6,-4,1)) x = b by banded LU + Woodbury (Sec. 5.1)
* ``ch_rhs``, ``ch_step``, ``ch_run`` -- the Cahn-Hilliard ADI scheme, Eq. (ch_adi) (Sec. 5.1)
* ``ch_mass``, ``ch_energy`` -- the integral of C and the free energy F[C] of Eq. (1)
* ``ch_coarsening_s``, ``ch_coarsening_k1`` -- the coarsening measures s(t) and k_1(t) of
  Sec. 5.1 "Numerical Results" (numpy; the FFT is numpy's)
* ``ch_rhs_noflux``, ``noflux_penta_solve``, ``ch_step_noflux``, ``ch_run_noflux``,
  ``ch_energy_noflux`` -- the same ADI scheme with no-flux boundaries (reflected ghost cells,
  non-cyclic line solves; numpy, scipy's banded solve)
* ``weno5_hj``, ``weno5_derivatives``, ``weno_advection`` -- the periodic XY WENO advection variant
  of Sec. 4.2 "Advection" (numpy), with the fifth-order Hamilton-Jacobi WENO derivatives of the
  reference it cites (Osher & Fedkiw, Sec. 3.4)

Fields are 2D numpy arrays of shape (ny, nx), row-major, x fastest.  FP32 inputs are widened to
FP64 before the oracle sees them, so the oracle works on exactly the values the GPU read.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

DIR_X, DIR_Y, DIR_XY = 0, 1, 2
BC_NONPERIODIC, BC_PERIODIC = 0, 1
FN_CENTRAL_D2X, FN_CH_NONLIN_LAP, FN_CUBIC_MINUS_LAP = 1, 2, 3

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles cs_oracle.c into a shared library (plain -O2, no fast-math) and returns its path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
            lib.orc_stencil2d.argtypes = [i64, i64, i32, i32, i32, i32, i32, i32, vp, vp, vp]
            lib.orc_stencil2d_fn.argtypes = [i64, i64, i32, i32, vp, i32, vp, vp]
            lib.orc_stencil1d_batch.argtypes = [i64, vp, i32, i32, i32, vp, vp, vp]
            lib.orc_cyclic_penta_solve.argtypes = [i64, dbl, i64, vp, vp]
            lib.orc_ch_rhs.argtypes = [i64, dbl, dbl, dbl, vp, vp, vp]
            lib.orc_ch_step.argtypes = [i64, dbl, dbl, dbl, vp, vp, vp]
            lib.orc_ch_run.argtypes = [i64, dbl, dbl, dbl, i64, vp, vp, vp, vp]
            lib.orc_ch_mass.argtypes = [i64, vp]
            lib.orc_ch_mass.restype = dbl
            lib.orc_ch_energy.argtypes = [i64, dbl, vp]
            lib.orc_ch_energy.restype = dbl
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ValueError(f"oracle {what} rejected its arguments (code {rc})")


def stencil2d(field, weights, direction: int, bc: int, left: int = 0, right: int = 0,
              top: int = 0, bottom: int = 0, out=None) -> np.ndarray:
    """Weighted stencil of Sec. 3.  ``out`` (if given) supplies the untouched cells for np."""
    f = _f64(field)
    ny, nx = f.shape
    w = _f64(weights).ravel()
    if w.size != (left + right + 1) * (top + bottom + 1):
        raise ValueError("weight count must be (left+right+1)*(top+bottom+1)")
    o = np.zeros_like(f) if out is None else _f64(out).copy()
    _check(_load().orc_stencil2d(nx, ny, direction, bc, left, right, top, bottom,
                                 _ptr(w), _ptr(f), _ptr(o)), "stencil2d")
    return o


def stencil2d_fn(field, fn: int, coe, bc: int, out=None) -> np.ndarray:
    """User-function stencil of Sec. 4.2 / Sec. 5.2 (``fn`` is one of the FN_* codes)."""
    f = _f64(field)
    ny, nx = f.shape
    c = _f64(coe).ravel()
    o = np.zeros_like(f) if out is None else _f64(out).copy()
    _check(_load().orc_stencil2d_fn(nx, ny, bc, fn, _ptr(c), c.size, _ptr(f), _ptr(o)),
           "stencil2d_fn")
    return o


def stencil1d_batch(packed, offsets, weights, bc: int, left: int, right: int,
                    out=None) -> np.ndarray:
    """The x stencil on every line [offsets[m], offsets[m+1]) of a packed ragged buffer."""
    f = _f64(packed).ravel()
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    w = _f64(weights).ravel()
    if w.size != left + right + 1:
        raise ValueError("weight count must be left+right+1")
    o = np.zeros_like(f) if out is None else _f64(out).ravel().copy()
    _check(_load().orc_stencil1d_batch(off.size - 1, _ptr(off), bc, left, right, _ptr(w),
                                       _ptr(f), _ptr(o)), "stencil1d_batch")
    return o


def cyclic_penta_solve(b, a: float) -> np.ndarray:
    """Solves (I + a circ(1,-4,6,-4,1)) x = b for each row of ``b`` (shape (n,) or (m, n))."""
    bb = _f64(b)
    n = bb.shape[-1]
    m = bb.size // n
    x = np.empty_like(bb)
    _check(_load().orc_cyclic_penta_solve(n, float(a), m, _ptr(bb), _ptr(x)), "cyclic_penta_solve")
    return x


def ch_coefficient_a(n: int, D: float, gamma: float, dt: float) -> float:
    """a = (2/3) D gamma dt / h^4 of L = I + a d^4 (Sec. 5.1), h = 2 pi / n."""
    h = 2.0 * np.pi / n
    return (2.0 / 3.0) * D * gamma * dt / h ** 4


def ch_rhs(c_prev, c_cur, D: float, gamma: float, dt: float) -> np.ndarray:
    p, c = _f64(c_prev), _f64(c_cur)
    n = c.shape[0]
    r = np.empty_like(c)
    _check(_load().orc_ch_rhs(n, D, gamma, dt, _ptr(p), _ptr(c), _ptr(r)), "ch_rhs")
    return r


def ch_step(c_prev, c_cur, D: float, gamma: float, dt: float) -> np.ndarray:
    """One ADI step, Eq. (ch_adi): returns C^{n+1} from C^{n-1}, C^n."""
    p, c = _f64(c_prev), _f64(c_cur)
    n = c.shape[0]
    if c.shape != (n, n) or p.shape != (n, n):
        raise ValueError("Cahn-Hilliard fields must be square n x n")
    o = np.empty_like(c)
    _check(_load().orc_ch_step(n, D, gamma, dt, _ptr(p), _ptr(c), _ptr(o)), "ch_step")
    return o


def ch_run(c0, D: float, gamma: float, dt: float, nsteps: int):
    """The time loop of Sec. 5.1 (C^{-1} := C^0).  Returns (C_final, mass[nsteps], energy[nsteps])."""
    c = _f64(c0)
    n = c.shape[0]
    out = np.empty_like(c)
    mass = np.empty(nsteps)
    energy = np.empty(nsteps)
    _check(_load().orc_ch_run(n, D, gamma, dt, nsteps, _ptr(c), _ptr(out), _ptr(mass),
                              _ptr(energy)), "ch_run")
    return out, mass, energy


def ch_mass(c) -> float:
    c = _f64(c)
    return _load().orc_ch_mass(c.shape[0], _ptr(c))


def ch_energy(c, gamma: float) -> float:
    c = _f64(c)
    return _load().orc_ch_energy(c.shape[0], gamma, _ptr(c))


def simpson_weights(n: int) -> np.ndarray:
    """Composite Simpson weights (without the h/3 factor) for the n grid points of one periodic
    direction: Simpson's rule over [0, 2 pi] with n intervals (n even) on x_i = i h, where the
    end point x_n = 2 pi carries the value at x_0, so x_0 takes the weights of both ends."""
    if n % 2:
        raise ValueError("Simpson's rule needs an even number of intervals")
    w = np.where(np.arange(n) % 2 == 1, 4.0, 2.0)
    w[0] = 2.0  # 1 (x_0) + 1 (x_n, the same periodic point)
    return w


def simpson_mean(f) -> float:
    """Spatial average of f over the periodic domain [0, 2 pi)^2 by Simpson's rule in x and y:
    (1 / (2 pi)^2) * (h / 3)^2 * sum_ij w_i w_j f_ij with h = 2 pi / n."""
    f = _f64(f)
    ny, nx = f.shape
    wy, wx = simpson_weights(ny), simpson_weights(nx)
    return float(wy @ f @ wx) / (9.0 * nx * ny)


def ch_coarsening_s(c) -> float:
    """s(t) = 1 / (1 - <C^2>), <.> the spatial average by Simpson's rule (Sec. 5.1)."""
    return 1.0 / (1.0 - simpson_mean(_f64(c) ** 2))


def ch_coarsening_k1(c) -> float:
    """k_1(t) = sum |C^(k)|^2 / sum |k|^-1 |C^(k)|^2 over the discrete wavenumbers of the periodic
    grid (the k-space integrals of Sec. 5.1 with their common measure cancelled; numpy's FFT).
    The k = 0 mode, where |k|^-1 is undefined, is left out of both sums."""
    c = _f64(c)
    ny, nx = c.shape
    p = np.abs(np.fft.fft2(c)) ** 2
    ky = np.fft.fftfreq(ny, d=1.0 / ny)[:, None]
    kx = np.fft.fftfreq(nx, d=1.0 / nx)[None, :]
    k = np.sqrt(kx ** 2 + ky ** 2)
    p[0, 0] = 0.0
    k[0, 0] = 1.0
    return float(p.sum() / (p / k).sum())



# ---- WENO advection (Sec. 4.2 "Advection": the 2D periodic XY variant with inputs C, u, v) -------
# The derivative approximations are the fifth-order WENO scheme for Hamilton-Jacobi equations of
# Osher & Fedkiw, "Level Set Methods and Dynamic Implicit Surfaces" (the reference the paper
# gives for its solver), Sec. 3.4, written out from its definitions in numpy, FP64.

WENO_EPS_SCALE = 1e-6   # epsilon = 1e-6 * max(v_k^2) + 1e-99
WENO_EPS_FLOOR = 1e-99


def weno5_hj(v1, v2, v3, v4, v5, eps_scale: float = WENO_EPS_SCALE, eps_floor: float = WENO_EPS_FLOOR):
    """The WENO5 derivative from the five one-sided differences v1..v5 (arrays or scalars): the
    three third-order candidates, their smoothness indicators and the nonlinear weights built on
    the optimal weights 0.1, 0.6, 0.3."""
    v1, v2, v3, v4, v5 = (np.asarray(v, dtype=np.float64) for v in (v1, v2, v3, v4, v5))
    phi1 = v1 / 3.0 - 7.0 * v2 / 6.0 + 11.0 * v3 / 6.0
    phi2 = -v2 / 6.0 + 5.0 * v3 / 6.0 + v4 / 3.0
    phi3 = v3 / 3.0 + 5.0 * v4 / 6.0 - v5 / 6.0
    s1 = 13.0 / 12.0 * (v1 - 2.0 * v2 + v3) ** 2 + 0.25 * (v1 - 4.0 * v2 + 3.0 * v3) ** 2
    s2 = 13.0 / 12.0 * (v2 - 2.0 * v3 + v4) ** 2 + 0.25 * (v2 - v4) ** 2
    s3 = 13.0 / 12.0 * (v3 - 2.0 * v4 + v5) ** 2 + 0.25 * (3.0 * v3 - 4.0 * v4 + v5) ** 2
    eps = eps_scale * np.maximum.reduce([v1 * v1, v2 * v2, v3 * v3, v4 * v4, v5 * v5]) + eps_floor
    a1 = 0.1 / (s1 + eps) ** 2
    a2 = 0.6 / (s2 + eps) ** 2
    a3 = 0.3 / (s3 + eps) ** 2
    return (a1 * phi1 + a2 * phi2 + a3 * phi3) / (a1 + a2 + a3)


def _at(a, k: int, axis: int):
    """a at index i + k along `axis`, periodic."""
    return np.roll(a, -k, axis=axis)


def weno5_derivatives(c, h: float, axis: int, **eps):
    """(left-biased, right-biased) WENO5 approximations of dC/dx along `axis` (1: x, 0: y) on the
    periodic grid: the first from the backward differences D-C at i-2 .. i+2, the second from the
    forward differences D+C at i+2 .. i-2."""
    c = _f64(c)
    d = (_at(c, 1, axis) - c) / h  # d[i] = D+C at i = D-C at i+1
    minus = weno5_hj(_at(d, -3, axis), _at(d, -2, axis), _at(d, -1, axis), d, _at(d, 1, axis), **eps)
    plus = weno5_hj(_at(d, 2, axis), _at(d, 1, axis), d, _at(d, -1, axis), _at(d, -2, axis), **eps)
    return minus, plus


def weno_advection(c, u, v, hx: float, hy: float, **eps):
    """The advection term u C_x + v C_y on the periodic grid, each derivative upwinded: the
    left-biased WENO5 value where the velocity component is positive, the right-biased one where
    it is negative (where it is zero the term is zero either way).  Rows are y, columns x."""
    u, v = _f64(u), _f64(v)
    cx_m, cx_p = weno5_derivatives(c, hx, 1, **eps)
    cy_m, cy_p = weno5_derivatives(c, hy, 0, **eps)
    return u * np.where(u > 0, cx_m, cx_p) + v * np.where(v > 0, cy_m, cy_p)


# ---- Cahn-Hilliard with no-flux boundaries (the ADI scheme of Sec. 5.1 on a bounded domain) -------
# Cell-centred grid x_i = (i + 1/2) h, h = 2 pi / n, on [0, 2 pi]^2; every stencil reads ghost cells
# by even reflection about the boundary (C_{-1-k} = C_k, C_{n+k} = C_{n-1-k}), which imposes
# dC/dn = 0 and d(lap C)/dn = 0, so no mass crosses the boundary.  The line operator becomes
# L = I + a D4 with D4 the reflected 5-point fourth difference (numpy and scipy, FP64).

def _reflect(f, width: int) -> np.ndarray:
    return np.pad(_f64(f), width, mode="symmetric")  # [b a | a b c | c b]: even reflection


def ch_rhs_noflux(c_prev, c_cur, D: float, gamma: float, dt: float) -> np.ndarray:
    """-(2/3)(C^n - C^{n-1}) - (2/3) D gamma dt lap4(Cbar) + (2/3) D dt lap2(C^3 - C)^n with
    Cbar = 2 C^n - C^{n-1}, lap4 the 13-point dxxxx + 2 dxxyy + dyyyy and lap2 the 5-point
    Laplacian (Eq. 5), ghost cells by reflection."""
    p, c = _f64(c_prev), _f64(c_cur)
    n = c.shape[0]
    h = 2.0 * np.pi / n
    cb = _reflect(2.0 * c - p, 2)
    s = lambda dj, di: cb[2 + dj:2 + dj + n, 2 + di:2 + di + n]  # Cbar at (j + dj, i + di)
    dxxxx = s(0, -2) - 4 * s(0, -1) + 6 * s(0, 0) - 4 * s(0, 1) + s(0, 2)
    dyyyy = s(-2, 0) - 4 * s(-1, 0) + 6 * s(0, 0) - 4 * s(1, 0) + s(2, 0)
    dxxyy = (s(-1, -1) - 2 * s(-1, 0) + s(-1, 1)) - 2 * (s(0, -1) - 2 * s(0, 0) + s(0, 1)) \
        + (s(1, -1) - 2 * s(1, 0) + s(1, 1))
    lap4 = (dxxxx + 2 * dxxyy + dyyyy) / h ** 4
    nl = _reflect(c ** 3 - c, 1)
    t = lambda dj, di: nl[1 + dj:1 + dj + n, 1 + di:1 + di + n]
    lap2 = (t(0, -1) + t(0, 1) + t(-1, 0) + t(1, 0) - 4 * t(0, 0)) / h ** 2
    return -(2.0 / 3.0) * (c - p) - (2.0 / 3.0) * D * gamma * dt * lap4 + (2.0 / 3.0) * D * dt * lap2


def noflux_line_matrix(n: int, a: float) -> np.ndarray:
    """L = I + a D2 D2 (dense), D2 the reflected second difference (rows (1, -2, 1), first and
    last rows (-1, 1) and (1, -1)); D2 D2 is the reflected fourth difference."""
    d2 = np.diag(np.full(n, -2.0)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)
    d2[0, 0] = d2[-1, -1] = -1.0
    return np.eye(n) + a * (d2 @ d2)


def _two_sum(a, b):
    """Error-free sum (Knuth's TwoSum): a + b = s + e exactly."""
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def _two_prod(a, b):
    """Error-free product by Veltkamp splitting (Dekker 1971): a * b = p + e exactly."""
    def split(x):
        c = 134217729.0 * x  # 2^27 + 1
        hi = c - (c - x)
        return hi, x - hi
    p = a * b
    ah, al = split(a)
    bh, bl = split(b)
    return p, ((ah * bh - p) + ah * bl + al * bh) + al * bl


def _noflux_residual(b, x, a: float):
    """r = b - L x along the last axis (L = noflux_line_matrix) with every sum and the product by
    a carried as an unevaluated pair (error-free transformations): r is exact up to ~2^-100 of
    the terms it cancels, far below the rounding of a plain FP64 evaluation."""
    def d2(y):  # reflected second difference: y_{-1} = y_0, y_n = y_{n-1}
        yp = np.concatenate([y[..., :1], y, y[..., -1:]], axis=-1)
        return yp[..., :-2], yp[..., 1:-1], yp[..., 2:]
    xm, x0, xp = d2(x)
    s, e1 = _two_sum(xm, xp)
    q, e2 = _two_sum(s, -2.0 * x0)          # D2 x = q + (e1 + e2)
    qm, q0, qp = d2(q)
    s, e3 = _two_sum(qm, qp)
    r4, e4 = _two_sum(s, -2.0 * q0)         # D2 D2 x = r4 + low
    lm, l0, lp = d2(e1 + e2)
    low = e3 + e4 + ((lm + lp) - 2.0 * l0)
    p, pe = _two_prod(r4, np.full_like(r4, a))
    pe = pe + low * a                       # a D2 D2 x = p + pe
    t, te = _two_sum(b, -x)
    t2, te2 = _two_sum(t, -p)
    return t2 + ((te + te2) - pe)


def noflux_penta_solve(b, a: float) -> np.ndarray:
    """Solves L x = b along the last axis of b (every line), L = noflux_line_matrix: a banded
    solve of its five diagonals (LAPACK, partial pivoting), then one step of iterative refinement
    with the residual evaluated exactly to rounding (_noflux_residual).  Without the refinement
    the banded solve's forward error reaches kappa eps |x| (kappa = 1 + 16 a, 3e6 at n = 4096),
    above the rounding of the step's other terms; with it the solve is exact to FP64 rounding."""
    from scipy.linalg import solve_banded
    b = _f64(b)
    n = b.shape[-1]
    L = noflux_line_matrix(n, a)
    ab = np.zeros((5, n))
    for k in range(-2, 3):  # ab[2 + i - j, j] = L[i, j]
        diag = np.diagonal(L, k)
        if k >= 0:
            ab[2 - k, k:] = diag
        else:
            ab[2 - k, :n + k] = diag
    flat = b.reshape(-1, n)
    x = solve_banded((2, 2), ab, flat.T).T
    r = _noflux_residual(flat, x, a)
    x = x + solve_banded((2, 2), ab, r.T).T
    return x.reshape(b.shape)


def ch_step_noflux(c_prev, c_cur, D: float, gamma: float, dt: float) -> np.ndarray:
    """One ADI step (Eq. ch_adi) with no-flux boundaries: L_x w = RHS, L_y v = w, C^{n+1} = Cbar + v."""
    p, c = _f64(c_prev), _f64(c_cur)
    n = c.shape[0]
    if c.shape != (n, n) or p.shape != (n, n):
        raise ValueError("Cahn-Hilliard fields must be square n x n")
    a = ch_coefficient_a(n, D, gamma, dt)
    rhs = ch_rhs_noflux(p, c, D, gamma, dt)
    w = noflux_penta_solve(rhs, a)          # lines along x (rows)
    v = noflux_penta_solve(w.T, a).T        # lines along y (columns)
    return 2.0 * c - p + v


def ch_energy_noflux(c, gamma: float) -> float:
    """Free energy of Eq. (1) by the rectangle rule with forward differences, the difference
    across the boundary being zero (reflected ghost)."""
    c = _f64(c)
    n = c.shape[0]
    h = 2.0 * np.pi / n
    e = _reflect(c, 1)[1:n + 2, 1:n + 2]
    gx = (e[:n, 1:n + 1] - c) / h
    gy = (e[1:n + 1, :n] - c) / h
    return float(h * h * np.sum(0.25 * (c * c - 1.0) ** 2 + 0.5 * gamma * (gx * gx + gy * gy)))


def ch_run_noflux(c0, D: float, gamma: float, dt: float, nsteps: int):
    """The time loop (C^{-1} := C^0) with no-flux boundaries: (C_final, mass[], energy[])."""
    prev = cur = _f64(c0)
    n = cur.shape[0]
    h = 2.0 * np.pi / n
    mass, energy = np.empty(nsteps), np.empty(nsteps)
    for s in range(nsteps):
        prev, cur = cur, ch_step_noflux(prev, cur, D, gamma, dt)
        mass[s] = h * h * cur.sum()
        energy[s] = ch_energy_noflux(cur, gamma)
    return cur, mass, energy
