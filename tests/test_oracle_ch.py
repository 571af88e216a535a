"""Pins for the oracle's cyclic pentadiagonal solve and Cahn-Hilliard ADI step (CPU only).

The solve is pinned by a dense LAPACK solve (numpy.linalg.solve) on small systems, by the FFT
solve of the circulant system at every size (eigenvalues 1 + 16 a sin^4(pi k / n)) within the
conditioning bound, and by its residual.  The ADI step is pinned by the closed-form linear limit
(a single Fourier mode of amplitude 1e-8 obeys c_{n+1} = alpha c_n + beta c_{n-1} with alpha,
beta from the discrete symbols; the first step, with C^{-1} = C^0, multiplies it by alpha + beta),
by exact mass conservation, a non-increasing free energy, the stationarity of constant fields,
and the x <-> y symmetry of the scheme.
"""
import numpy as np
import pytest
import scipy.linalg

import workloads as W

EPS = np.finfo(np.float64).eps
D, GAMMA = 1.0, 0.01


def circulant_matrix(n, a):
    col = np.zeros(n)
    for off, c in [(0, 6.0), (1, -4.0), (-1, -4.0), (2, 1.0), (-2, 1.0)]:
        col[off % n] += c
    return np.eye(n) + a * scipy.linalg.circulant(col)


def fft_solve(b, a):
    n = b.shape[-1]
    lam = 1 + 16 * a * np.sin(np.pi * np.arange(n) / n) ** 4
    return np.real(np.fft.ifft(np.fft.fft(b, axis=-1) / lam, axis=-1))


@pytest.mark.parametrize("n", [5, 6, 7, 8, 13, 32, 64])
@pytest.mark.parametrize("a", [0.0, 0.3, 17.0, 2.5e3])
def test_solve_matches_dense_lapack(orc, n, a):
    b = W.uniform_field(3, n, seed=n + int(a))
    x = orc.cyclic_penta_solve(b, a)
    M = circulant_matrix(n, a)
    ref = np.linalg.solve(M, b.T).T
    kappa = 1 + 16 * a
    assert np.abs(x - ref).max() <= 4 * kappa * EPS * np.abs(ref).max() + 1e-15


@pytest.mark.parametrize("n", [64, 256, 1024, 4096])
def test_solve_matches_fft_within_conditioning(orc, n):
    """The CH operator L = I + a P at the paper's parameters (dt = 0.1 h, D = 1, gamma = 0.01):
    forward error vs the (well-conditioned) FFT solve bounded by kappa * eps; residual (backward
    error) at the rounding level."""
    h = 2 * np.pi / n
    a = orc.ch_coefficient_a(n, D, GAMMA, 0.1 * h)
    kappa = 1 + 16 * a
    b = W.uniform_field(4, n, seed=n)
    x = orc.cyclic_penta_solve(b, a)
    ref = fft_solve(b, a)
    assert np.abs(x - ref).max() <= kappa * EPS * np.abs(ref).max() + 4 * EPS * np.abs(b).max()
    Px = np.roll(x, 2, 1) - 4 * np.roll(x, 1, 1) + 6 * x - 4 * np.roll(x, -1, 1) + np.roll(x, -2, 1)
    res = np.abs(x + a * Px - b).max()
    assert res <= 64 * EPS * kappa * np.abs(x).max()


def test_solve_identity_when_a_is_zero(orc):
    b = W.uniform_field(2, 37, seed=1)
    assert np.array_equal(orc.cyclic_penta_solve(b, 0.0), b)


def test_solve_rejects_short_lines(orc):
    with pytest.raises(ValueError):
        orc.cyclic_penta_solve(np.ones(4), 1.0)


def linear_factors(n, k, l, dt):
    """alpha, beta of the linearised scheme for the mode (k, l) (see module docstring)."""
    h = 2 * np.pi / n
    a = (2 / 3) * D * GAMMA * dt / h ** 4
    mu = (4 / h ** 2) * (np.sin(k * h / 2) ** 2 + np.sin(l * h / 2) ** 2)
    lam = (1 + 16 * a * np.sin(k * h / 2) ** 4) * (1 + 16 * a * np.sin(l * h / 2) ** 4)
    alpha = 2 + (-2 / 3 - (4 / 3) * D * GAMMA * dt * mu ** 2 + (2 / 3) * D * dt * mu) / lam
    beta = -1 + (2 / 3 + (2 / 3) * D * GAMMA * dt * mu ** 2) / lam
    return alpha, beta


@pytest.mark.parametrize("n,k,l", [(32, 1, 0), (32, 3, 2), (64, 5, 7), (64, 20, 1), (48, 12, 12)])
def test_linear_limit_closed_form(orc, n, k, l):
    """A mode of amplitude 1e-8 (cubic term ~1e-24, negligible) follows the two-term recurrence;
    this fixes the D gamma coefficient of the biharmonic term, the extrapolation
    Cbar = 2 C^n - C^{n-1} and the explicit level-n nonlinearity together."""
    h = 2 * np.pi / n
    dt = 0.1 * h
    A = 1e-8
    c0 = W.single_mode(n, k, l, A, phase=0.3)
    alpha, beta = linear_factors(n, k, l, dt)
    prev, cur = c0, c0
    amp_prev, amp_cur = 1.0, 1.0
    for step in range(6):
        nxt = orc.ch_step(prev, cur, D, GAMMA, dt)
        amp_next = alpha * amp_cur + beta * amp_prev
        if step == 0:
            assert abs(amp_next - (alpha + beta)) < 1e-15
        assert np.abs(nxt - amp_next * c0).max() <= 1e-9 * A, step
        prev, cur = cur, nxt
        amp_prev, amp_cur = amp_cur, amp_next


def test_linear_limit_rejects_printed_coefficient(orc):
    """With the coefficient printed in Eq. (ch_adi) (no D gamma on the biharmonic term) the mode
    factor would differ; the oracle follows the D gamma reading."""
    n, k, l = 32, 4, 3
    h = 2 * np.pi / n
    dt = 0.1 * h
    c0 = W.single_mode(n, k, l, 1e-8)
    nxt = orc.ch_step(c0, c0, D, GAMMA, dt)
    alpha, beta = linear_factors(n, k, l, dt)
    mu = (4 / h ** 2) * (np.sin(k * h / 2) ** 2 + np.sin(l * h / 2) ** 2)
    a = (2 / 3) * D * GAMMA * dt / h ** 4
    lam = (1 + 16 * a * np.sin(k * h / 2) ** 4) * (1 + 16 * a * np.sin(l * h / 2) ** 4)
    printed = 1 + (2 / 3) * dt * (D * mu - mu ** 2) / lam
    ratio = (nxt * c0).sum() / (c0 * c0).sum()
    assert abs(ratio - (alpha + beta)) < 1e-12
    assert abs(ratio - printed) > 1e-3


def test_constant_field_is_stationary(orc):
    c = np.full((16, 16), 0.37)
    nxt = orc.ch_step(c, c, D, GAMMA, 0.1 * 2 * np.pi / 16)
    assert np.abs(nxt - c).max() < 1e-15


def test_mass_conserved_exactly(orc):
    """Row sums of L are 1 and the discrete lap2, lap4 sum to zero on the periodic grid, so with
    C^{-1} = C^0 the sum of C is conserved to rounding (deep-quench data, 300 steps)."""
    n = 64
    h = 2 * np.pi / n
    c0 = W.ch_initial(n, seed=7)
    c, mass, energy = orc.ch_run(c0, D, GAMMA, 0.1 * h, 300)
    m0 = orc.ch_mass(c0)
    scale = h * h * np.abs(c0).sum()
    assert np.abs(mass - m0).max() <= 1e-12 * scale
    assert np.abs(c).max() < 1.3


@pytest.mark.parametrize("n", [64, 128])
def test_energy_nonincreasing_for_resolved_data(orc, n):
    """The free energy decreases every step for resolved initial data (t = 0 .. 2).  (With
    grid-scale random data the weakly damped stiff modes of the ADI factorisation let the energy
    rise in the first steps; that is a property of the scheme, reported by the benchmark.)"""
    h = 2 * np.pi / n
    c0 = W.low_mode_field(n, seed=3)
    c, mass, energy = orc.ch_run(c0, D, GAMMA, 0.1 * h, int(2.0 / (0.1 * h)))
    e = np.concatenate([[orc.ch_energy(c0, GAMMA)], energy])
    assert np.all(np.diff(e) <= 1e-12 * np.abs(e[:-1]))
    assert e[-1] < 0.6 * e[0]  # phase separation lowers F substantially
    assert np.abs(mass - orc.ch_mass(c0)).max() < 1e-12


def test_xy_symmetry(orc):
    """L_x and L_y commute, so the scheme commutes with transposition up to rounding."""
    n = 24
    h = 2 * np.pi / n
    p = W.ch_initial(n, seed=1)
    c = W.ch_initial(n, seed=2)
    a = orc.ch_step(p, c, D, GAMMA, 0.1 * h)
    b = orc.ch_step(p.T, c.T, D, GAMMA, 0.1 * h)
    assert np.abs(a - b.T).max() < 1e-13


def test_mass_and_energy_definitions(orc):
    """Mass and energy of closed-form fields: C = s constant gives M = 4 pi^2 s and
    F = 4 pi^2 (s^2-1)^2/4; C = A sin(kx) adds gamma/2 * A^2 (2 sin(kh/2)/h)^2 * 2 pi^2."""
    n = 32
    h = 2 * np.pi / n
    s = 0.3
    c = np.full((n, n), s)
    assert abs(orc.ch_mass(c) - 4 * np.pi ** 2 * s) < 1e-12
    assert abs(orc.ch_energy(c, GAMMA) - np.pi ** 2 * (s * s - 1) ** 2) < 1e-12
    A, k = 0.5, 3
    c = W.single_mode(n, k, 0, A, phase=0.0)
    x = np.arange(n) * h
    bulk = h * h * n * np.sum(0.25 * ((A * np.sin(k * x)) ** 2 - 1) ** 2)
    grad = 0.5 * GAMMA * A ** 2 * (2 * np.sin(k * h / 2) / h) ** 2 * 2 * np.pi ** 2
    assert abs(orc.ch_energy(c, GAMMA) - (bulk + grad)) < 1e-12
    assert abs(orc.ch_mass(c)) < 1e-12
