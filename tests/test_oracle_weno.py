"""Pins of the WENO advection oracle (Sec. 4.2 "Advection"; the fifth-order Hamilton-Jacobi
WENO derivatives of Osher & Fedkiw, Sec. 3.4) against what the mathematics fixes:

* fifth-order convergence to the exact advection term on smooth periodic data (a dropped or
  mis-signed term in a candidate, an indicator or a weight, or a shifted stencil, lowers it);
* with epsilon forced huge the weights become the optimal ones and the scheme must equal the
  unique 6-point upwind-biased stencil exact for degree-5 polynomials, solved for here from the
  Taylor (Vandermonde) conditions;
* every candidate is exact for cubics, so the WENO value is exact for cubic data whatever the
  weights;
* on a step the nonlinear weights drop the candidates that cross the jump (no oscillation) where
  the linear scheme does not;
* reflection x -> -x with u -> -u, transposition, translation and constants."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def smooth_case(n):
    h = 2 * np.pi / n
    x = np.arange(n) * h
    X, Y = np.meshgrid(x, x)
    c = np.sin(X + 0.3) * np.cos(2 * Y) + 0.5 * np.cos(3 * X - Y)
    cx = np.cos(X + 0.3) * np.cos(2 * Y) - 1.5 * np.sin(3 * X - Y)
    cy = -2 * np.sin(X + 0.3) * np.sin(2 * Y) + 0.5 * np.sin(3 * X - Y)
    u = np.cos(Y) + 0.2
    v = np.sin(X) - 0.1
    return c, u, v, h, u * cx + v * cy


def test_fifth_order_convergence():
    errs = []
    for n in (128, 256):
        c, u, v, h, exact = smooth_case(n)
        errs.append(np.abs(oracle.weno_advection(c, u, v, h, h) - exact).max())
    assert errs[1] <= 1e-6
    assert errs[0] / errs[1] >= 28.0  # 2^5 = 32


def upwind_biased_weights():
    """Weights a_k, k = -3..2, with sum_k a_k f(x + k h) = h f'(x) for every polynomial of
    degree <= 5 (exact rational solve of the Taylor conditions)."""
    from fractions import Fraction
    ks = list(range(-3, 3))
    m = [[Fraction(k) ** p for k in ks] for p in range(6)]
    rhs = [Fraction(1 if p == 1 else 0) for p in range(6)]
    # Gaussian elimination on the 6x6 rational system
    a = [row[:] + [r] for row, r in zip(m, rhs)]
    for col in range(6):
        piv = next(r for r in range(col, 6) if a[r][col] != 0)
        a[col], a[piv] = a[piv], a[col]
        for r in range(6):
            if r != col and a[r][col] != 0:
                f = a[r][col] / a[col][col]
                a[r] = [x - f * y for x, y in zip(a[r], a[col])]
    return {k: float(a[i][6] / a[i][i]) for i, k in enumerate(ks)}


def test_linear_limit_is_the_fifth_order_upwind_stencil():
    w = upwind_biased_weights()
    rng = np.random.default_rng(5)
    n = 64
    h = 2 * np.pi / n
    c = rng.uniform(-1, 1, (n, n))
    minus, plus = oracle.weno5_derivatives(c, h, 1, eps_scale=1e30)
    lin_m = sum(wk * np.roll(c, -k, axis=1) for k, wk in w.items()) / h
    lin_p = -sum(wk * np.roll(c, k, axis=1) for k, wk in w.items()) / h  # mirror image
    scale = np.abs(c).max() / h
    assert np.abs(minus - lin_m).max() <= 1e-13 * scale
    assert np.abs(plus - lin_p).max() <= 1e-13 * scale


@pytest.mark.parametrize("seed", range(5))
def test_exact_for_cubics(seed):
    rng = np.random.default_rng(seed)
    p = rng.uniform(-1, 1, 4)
    h = 0.1
    x0 = rng.uniform(-1, 1)
    xs = x0 + h * np.arange(-3, 4)
    f = np.polyval(p, xs)
    d = np.diff(f) / h  # d[k] = D+ f at x0 + (k - 3) h, k = 0..5
    exact = np.polyval(np.polyder(p), x0)
    minus = oracle.weno5_hj(d[0], d[1], d[2], d[3], d[4])
    plus = oracle.weno5_hj(d[5], d[4], d[3], d[2], d[1])
    assert abs(minus - exact) <= 1e-12 * (1 + abs(exact))
    assert abs(plus - exact) <= 1e-12 * (1 + abs(exact))


def test_step_is_not_oscillatory():
    """C = 1 on columns >= J, 0 before (one periodic jump back far away): two cells either side
    of the jump only the candidates crossing it see a non-zero difference, and WENO gives them a
    weight near zero; the linear scheme does not."""
    n, J = 64, 32
    h = 2 * np.pi / n
    c = np.zeros((4, n))
    c[:, J:] = 1.0
    minus, plus = oracle.weno5_derivatives(c, h, 1)
    lin_m, lin_p = oracle.weno5_derivatives(c, h, 1, eps_scale=1e30)
    for i in (J - 2, J + 2):
        assert abs(minus[0, i]) <= 1e-10 / h and abs(plus[0, i]) <= 1e-10 / h
    assert abs(lin_m[0, J + 2]) >= 1e-2 / h and abs(lin_p[0, J - 2]) >= 1e-2 / h
    # far from the jumps every difference is zero
    assert minus[0, J + 8] == 0.0 and plus[0, J - 8] == 0.0


def random_case(n, seed):
    rng = np.random.default_rng(seed)
    c = rng.uniform(-1, 1, (n, n))
    u = rng.uniform(-1, 1, (n, n))
    v = rng.uniform(-1, 1, (n, n))
    return c, u, v


def test_reflection_swaps_the_upwind_sides_exactly():
    n = 32
    h = 2 * np.pi / n
    c, u, v = random_case(n, 7)
    a = oracle.weno_advection(c, u, v, h, h)
    refl = lambda f: np.roll(f[:, ::-1], 1, axis=1)  # column i -> (n - i) mod n
    b = oracle.weno_advection(refl(c), -refl(u), refl(v), h, h)
    assert np.array_equal(b, refl(a))


def test_transpose_translation_constant():
    n = 32
    hx, hy = 2 * np.pi / n, 2 * np.pi / n * 1.5
    c, u, v = random_case(n, 8)
    a = oracle.weno_advection(c, u, v, hx, hy)
    assert np.array_equal(oracle.weno_advection(c.T, v.T, u.T, hy, hx), a.T)
    sh = lambda f: np.roll(np.roll(f, 5, axis=0), -3, axis=1)
    assert np.array_equal(oracle.weno_advection(sh(c), sh(u), sh(v), hx, hy), sh(a))
    assert np.array_equal(oracle.weno_advection(np.full((n, n), 0.7), u, v, hx, hy), np.zeros((n, n)))
