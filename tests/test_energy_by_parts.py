"""The free energy of Eq. (1) as the device's invariant reduction forms it: the gradient part summed
by parts, sum(|D+x C|^2 + |D+y C|^2) = -sum C Lap5(C), with Lap5 the unscaled 5-point Laplacian
reading the periodic wrap, or with no-flux boundaries the even reflection (ghost -1 = 0,
n = n - 1).  On the CPU, against the oracle's forward-difference energy (rectangle rule), for
random and smooth fields: the two forms agree to rounding."""
import numpy as np
import pytest

import oracle
import workloads as W


def energy_by_parts(c: np.ndarray, gamma: float, noflux: bool) -> float:
    n = c.shape[0]
    h = 2 * np.pi / n
    if noflux:
        p = np.pad(c, 1, mode="symmetric")  # even reflection: ghost -1 holds row 0, n holds n - 1
    else:
        p = np.pad(c, 1, mode="wrap")
    lap = p[:-2, 1:-1] + p[2:, 1:-1] + p[1:-1, :-2] + p[1:-1, 2:] - 4 * c
    w = c * c - 1
    return h * h * float(np.sum(0.25 * w * w) - 0.5 * gamma / (h * h) * np.sum(c * lap))


@pytest.mark.parametrize("noflux", [False, True])
@pytest.mark.parametrize("n", [16, 64, 256])
@pytest.mark.parametrize("kind", ["random", "quench", "smooth"])
def test_energy_summed_by_parts_equals_forward_differences(noflux, n, kind):
    rng = np.random.default_rng(n + 7 * noflux)
    if kind == "random":
        c = rng.uniform(-1, 1, (n, n))
    elif kind == "quench":
        c = W.ch_initial(n, seed=n)
    else:
        x = np.arange(n) * 2 * np.pi / n
        c = np.tanh(4 * np.sin(x)[None, :] * np.cos(2 * x)[:, None])
    gamma = 0.01
    ref = oracle.ch_energy_noflux(c, gamma) if noflux else oracle.ch_energy(c, gamma)
    got = energy_by_parts(c, gamma, noflux)
    assert abs(got - ref) <= 1e-12 * abs(ref), (got, ref)
