"""Pins of the coarsening measures s(t) and k_1(t) of Sec. 5.1 ("Numerical Results") in the
oracle: Simpson's rule on the periodic grid, and the spectral length scale, checked against
closed forms, a direct DFT on a tiny grid, and invariances."""
import numpy as np
import pytest

import oracle


def grid(n):
    x = np.arange(n) * 2 * np.pi / n
    return np.meshgrid(x, x)  # X varies along axis 1 (x), Y along axis 0 (y)


def test_simpson_weights_and_constant():
    for n in (2, 4, 16, 512):
        w = oracle.simpson_weights(n)
        assert w.sum() == 3 * n  # (h / 3) * sum w = 2 pi
        assert oracle.simpson_mean(np.full((n, n), 2.5)) == pytest.approx(2.5, rel=1e-15)
    with pytest.raises(ValueError):
        oracle.simpson_weights(5)


@pytest.mark.parametrize("k", [0, 1, 3, 7])
def test_simpson_mean_of_low_modes_is_exact(k):
    """On a periodic grid the weights (2, 4, 2, 4, ...) sum e^{i m x} to 2 n [m = 0 mod n] plus
    a term that vanishes unless m = 0 mod n / 2, so Simpson's mean is exact for every mode except
    the Nyquist ones; the squares here hold modes up to 14 on n = 32."""
    n = 32
    X, Y = grid(n)
    assert oracle.simpson_mean(np.sin(k * X + 2 * Y + 0.3) ** 2) == pytest.approx(0.5, abs=1e-15)
    assert oracle.simpson_mean(np.cos(k * X)) == pytest.approx(1.0 if k == 0 else 0.0, abs=1e-15)


def test_simpson_is_not_the_trapezoid_rule_at_the_nyquist_mode():
    """f_i = (-1)^i: the trapezoid mean is 0, Simpson's weights (2, 4, 2, 4, ...) give
    (-n)(3n) / (9 n^2) = -1/3."""
    n = 16
    f = np.tile((-1.0) ** np.arange(n), (n, 1))
    assert f.mean() == 0.0
    assert oracle.simpson_mean(f) == pytest.approx(-1.0 / 3.0, rel=1e-15)


@pytest.mark.parametrize("amp", [0.1, 0.5, 1.2])
def test_s_of_a_single_mode(amp):
    n = 64
    X, Y = grid(n)
    c = amp * np.sin(3 * X - 5 * Y)
    assert oracle.ch_coarsening_s(c) == pytest.approx(1.0 / (1.0 - amp * amp / 2.0), rel=1e-14)


@pytest.mark.parametrize("kx,ky", [(1, 0), (3, 4), (0, 7), (5, 12)])
def test_k1_of_a_single_mode_is_its_wavenumber(kx, ky):
    n = 64
    X, Y = grid(n)
    assert oracle.ch_coarsening_k1(np.sin(kx * X + ky * Y + 0.7)) == pytest.approx(np.hypot(kx, ky), rel=1e-13)


def test_k1_of_two_modes_weights_by_power():
    """k_1 = (A^2 + B^2) / (A^2 / |k| + B^2 / |q|) for two modes of amplitudes A, B."""
    n = 64
    X, Y = grid(n)
    c = 2.0 * np.sin(3 * X) + np.cos(5 * Y + 1.0)
    assert oracle.ch_coarsening_k1(c) == pytest.approx((4.0 + 1.0) / (4.0 / 3.0 + 1.0 / 5.0), rel=1e-13)


def test_k1_invariances():
    g = np.random.Generator(np.random.PCG64(11))
    c = g.uniform(-1, 1, (32, 32))
    k = oracle.ch_coarsening_k1(c)
    assert oracle.ch_coarsening_k1(np.roll(c, (5, -3), axis=(0, 1))) == pytest.approx(k, rel=1e-13)
    assert oracle.ch_coarsening_k1(3.0 * c) == pytest.approx(k, rel=1e-13)
    assert oracle.ch_coarsening_k1(c + 0.25) == pytest.approx(k, rel=1e-13)  # only k = 0 changes


def test_k1_matches_a_direct_dft_on_a_tiny_grid():
    n = 8
    g = np.random.Generator(np.random.PCG64(5))
    c = g.uniform(-1, 1, (n, n))
    num = den = 0.0
    for ky in range(n):
        for kx in range(n):
            if kx == 0 and ky == 0:
                continue
            z = 0j
            for j in range(n):
                for i in range(n):
                    z += c[j, i] * np.exp(-2j * np.pi * (kx * i + ky * j) / n)
            fx = kx if kx <= n // 2 else kx - n
            fy = ky if ky <= n // 2 else ky - n
            p = abs(z) ** 2
            num += p
            den += p / np.hypot(fx, fy)
    assert oracle.ch_coarsening_k1(c) == pytest.approx(num / den, rel=1e-13)
