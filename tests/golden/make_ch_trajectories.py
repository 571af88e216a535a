"""Writes the oracle's Cahn-Hilliard trajectories used by the GPU tests of the 1000-step runs.

The workload is the scheme of Sec. 5.1 (periodic ADI, BDF2 with the explicit nonlinearity) on
the deep-quench initial field of Sec. 5.3 -- C0 ~ U[-0.1, 0.1] with the sample mean removed,
D = 1, gamma = 0.01, dt = 0.1 h, h = 2 pi / n -- for 1000 steps at n = 1024 and 4096, in FP64.
Every value below comes from ``oracle.ch_run`` (plain C, binary64); nothing else is called.

Output ``ch_trajectory_n<n>.txt``:
  * ``m0 e0``: mass and free energy of C0;
  * one line ``k mass energy`` per step k = 1..1000 (the invariants after step k);
  * 64 lines ``j i C[j, i]`` of the final field at fixed points (rows and columns 8 k n/64 + 5).

Usage: ``python tests/golden/make_ch_trajectories.py 1024 4096`` (about 4 minutes at 1024 and
2 hours at 4096 on one core).
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import workloads as W  # noqa: E402

D, GAMMA, SEED, STEPS = 1.0, 0.01, 1902, 1000


def sample_points(n):
    idx = [8 * k * n // 64 + 5 for k in range(8)]
    return [(j, i) for j in idx for i in idx]


def main(sizes):
    oracle.build()
    for n in sizes:
        h = 2 * np.pi / n
        dt = 0.1 * h
        c0 = W.ch_initial(n, seed=SEED)
        t0 = time.time()
        c, mass, energy = oracle.ch_run(c0, D, GAMMA, dt, STEPS)
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"ch_trajectory_n{n}.txt")
        with open(path, "w") as f:
            f.write(f"# oracle.ch_run: periodic CH-ADI (Sec. 5.1), n={n}, D={D}, gamma={GAMMA}, dt=0.1h, "
                    f"C0 = workloads.ch_initial(n, seed={SEED}) (Sec. 5.3), {STEPS} steps, FP64\n")
            f.write(f"# written by tests/golden/make_ch_trajectories.py in {time.time() - t0:.0f} s\n")
            f.write(f"m0e0 {float(oracle.ch_mass(c0))!r} {float(oracle.ch_energy(c0, GAMMA))!r}\n")
            for k in range(STEPS):
                f.write(f"{k + 1} {float(mass[k])!r} {float(energy[k])!r}\n")
            for j, i in sample_points(n):
                f.write(f"C {j} {i} {float(c[j, i])!r}\n")
        print(path, f"{time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main([int(a) for a in sys.argv[1:]] or [1024, 4096])
