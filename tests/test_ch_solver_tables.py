"""The device line solver's tables, replayed on the host (cs_ch_solver_check; no GPU needed).

The Cahn-Hilliard step solves (I + a D4) x = b along every row and column with a partitioned
spike method: per chunk an LU solve, then the chunk-end values from the inverse of the chunk
coupling system, then a correction by precomputed spikes (Sec. 5.1's cyclic pentadiagonal solves,
and the non-cyclic ones of the no-flux boundary).  cs_ch_solver_check builds the tables
cs_ch_create builds and runs both phases on the host in the kernels' order of operations; the
backward error of the result against the operator itself must be at rounding level (64 eps) for every
partition and every coefficient a up to the n = 4096 benchmark's 1.8e5 and beyond.
"""
import numpy as np
import pytest

PARTS = [1, 2, 4, 8, 16, 32, 64]


@pytest.fixture(scope="module")
def cs():
    import paper_1902_09931_gb300 as cs
    cs.load()
    return cs


@pytest.mark.parametrize("boundary", [0, 1])
@pytest.mark.parametrize("n", [64, 256, 1024, 4096])
def test_backward_error_at_rounding_level(cs, boundary, n):
    worst = 0.0
    for P in PARTS:
        if n % P or n // P < 16 or (n // P) % 8:
            continue
        for a in (0.0, 0.7, 45.0, 2885.8, 1.85e5, 3.0e5):
            r = cs.cs_ch_solver_check(n, P, a, boundary)
            worst = max(worst, r)
            assert r <= 64 * 2.0 ** -52, (n, P, a, r)
    print(f"[solver tables] boundary={boundary} n={n}: worst backward error {worst:.2e} of (1 + 16 a) |x|")


def test_rejects_invalid_partitions(cs):
    for n, P in [(64, 3), (100, 4), (64, 8), (1024, 128)]:
        with pytest.raises(cs.CSError) as e:
            cs.cs_ch_solver_check(n, P, 1.0, 0)
        assert e.value.code == cs.CS_EINVAL
    with pytest.raises(cs.CSError):
        cs.cs_ch_solver_check(64, 2, -1.0, 0)
    with pytest.raises(cs.CSError):
        cs.cs_ch_solver_check(64, 2, 1.0, 7)
