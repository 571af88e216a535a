"""Pins of the no-flux Cahn-Hilliard oracle (the Sec. 5.1 ADI scheme with reflected ghost cells
and non-cyclic line solves) against what the mathematics fixes:

* mirror doubling: a field reflected evenly across both edges of a 2n x 2n periodic grid stays
  reflected under the periodic scheme, and its n x n quarter evolves by the no-flux scheme; with
  the periodic grid's spacing h/2, the same a and alpha need D/4 and gamma/4.  So one no-flux step
  (numpy + scipy banded solve) must equal the restriction of one periodic step of the separately
  pinned C oracle (cyclic LU + Woodbury), and the energies and masses must agree too;
* the linear limit on the cosine modes of the reflected grid (the eigenvectors of the reflected
  second difference), which fixes the corner rows of the line operator;
* mass conservation, energy decay on resolved data, constant fields and x <-> y symmetry."""
import numpy as np
import pytest

import workloads as W

D, GAMMA = 1.0, 0.01


@pytest.fixture(scope="module")
def orc():
    pytest.importorskip("scipy")
    import oracle
    return oracle


def extend(f):
    n = f.shape[0]
    idx = np.r_[0:n, n - 1:-1:-1]
    return f[idx][:, idx]


@pytest.mark.parametrize("n", [16, 32, 64])
def test_mirror_doubling_equals_periodic_oracle(orc, n):
    h = 2 * np.pi / n
    dt = 0.1 * h
    prev = W.ch_initial(n, seed=n) * 5
    cur = prev + 0.05 * W.ch_initial(n, seed=n + 1)
    got = orc.ch_step_noflux(prev, cur, D, GAMMA, dt)
    ref = orc.ch_step(extend(prev), extend(cur), D / 4, GAMMA / 4, dt)
    assert np.abs(ref - extend(ref[:n, :n])).max() <= 1e-13  # the periodic step kept the reflection
    assert np.abs(got - ref[:n, :n]).max() <= 1e-12 * np.abs(ref).max()
    assert orc.ch_energy_noflux(cur, GAMMA) == pytest.approx(orc.ch_energy(extend(cur), GAMMA / 4), rel=1e-13)
    assert h * h * cur.sum() == pytest.approx(orc.ch_mass(extend(cur)), rel=1e-12, abs=1e-14)


def cos_mode(n, k, l, amp):
    x = (np.arange(n) + 0.5) * np.pi / n  # cos(k pi (i + 1/2) / n): eigenvectors of the reflected D2
    return amp * np.cos(l * x)[:, None] * np.cos(k * x)[None, :]


@pytest.mark.parametrize("n,k,l", [(16, 3, 5), (32, 1, 0), (32, 7, 12), (64, 31, 2)])
def test_linear_limit_cosine_modes(orc, n, k, l):
    """Amplitude 1e-8 (cubic ~1e-24): the mode amplitude follows A+ = a1 A - a0 A- with the
    reflected symbols mu = (4/h^2)(sin^2(k pi/2n) + sin^2(l pi/2n)) and line factors
    1 + 16 a sin^4(k pi/2n)."""
    h = 2 * np.pi / n
    dt = 0.1 * h
    a = orc.ch_coefficient_a(n, D, GAMMA, dt)
    sx, sy = np.sin(k * np.pi / (2 * n)) ** 2, np.sin(l * np.pi / (2 * n)) ** 2
    mu = 4 / h ** 2 * (sx + sy)
    lam = (1 + 16 * a * sx ** 2) * (1 + 16 * a * sy ** 2)
    a1 = 2 + (-2 / 3 - (4 / 3) * D * GAMMA * dt * mu ** 2 + (2 / 3) * D * dt * mu) / lam
    a0 = -1 + (2 / 3 + (2 / 3) * D * GAMMA * dt * mu ** 2) / lam
    c0 = cos_mode(n, k, l, 1e-8)
    prev, cur, ap, ac = c0, c0, 1.0, 1.0
    for step in range(6):
        nxt = orc.ch_step_noflux(prev, cur, D, GAMMA, dt)
        an = a1 * ac + a0 * ap
        assert np.abs(nxt - an * c0).max() <= 1e-9 * 1e-8, step
        prev, cur, ap, ac = cur, nxt, ac, an


def test_line_operator_corners(orc):
    """The reflected fourth difference is (1,-4,6,-4,1) inside and (2,-3,1), (-3,6,-4,1) in the
    first two rows (mirrored at the end): ghost values C_{-1} = C_0, C_{-2} = C_1 folded in."""
    L = orc.noflux_line_matrix(8, 1.0) - np.eye(8)
    assert list(L[0, :3]) == [2, -3, 1] and list(L[1, :4]) == [-3, 6, -4, 1]
    assert list(L[4, 2:7]) == [1, -4, 6, -4, 1]
    assert np.array_equal(L, L[::-1, ::-1]) and np.array_equal(L, L.T)
    assert np.array_equal(L.sum(axis=0), np.zeros(8))  # columns sum to zero: no flux


def test_mass_conserved_and_energy(orc):
    n = 32
    h = 2 * np.pi / n
    c0 = W.ch_initial(n, seed=4)
    _, mass, _ = orc.ch_run_noflux(c0, D, GAMMA, 0.1 * h, 20)
    m0 = h * h * c0.sum()
    assert np.abs(mass - m0).max() <= 1e-13 * h * h * np.abs(c0).sum() + 1e-15
    c1 = cos_mode(n, 2, 1, 0.3) + cos_mode(n, 0, 3, 0.2)  # resolved data
    _, _, energy = orc.ch_run_noflux(c1, D, GAMMA, 0.1 * h, 30)
    e = np.concatenate([[orc.ch_energy_noflux(c1, GAMMA)], energy])
    assert np.all(np.diff(e) <= 1e-12 * np.abs(e[:-1]))


def test_constant_and_transpose(orc):
    n = 16
    h = 2 * np.pi / n
    c = np.full((n, n), 0.4)
    assert np.array_equal(orc.ch_step_noflux(c, c, D, GAMMA, 0.1 * h), c)
    p = W.ch_initial(n, seed=9)
    q = p + 0.01 * W.ch_initial(n, seed=10)
    a = orc.ch_step_noflux(p, q, D, GAMMA, 0.1 * h)
    b = orc.ch_step_noflux(p.T, q.T, D, GAMMA, 0.1 * h)
    assert np.abs(a - b.T).max() <= 1e-14 * np.abs(a).max()
