"""The 1000-step Cahn-Hilliard runs of the benchmark configuration (Sec. 5.1 scheme, Sec. 5.3
set-up: C0 ~ U[-0.1, 0.1] with the mean removed, D = 1, gamma = 0.01, dt = 0.1 h) at n = 1024
and 4096, FP64 and FP32 storage, with the mass and the free energy read back after every step
(cs_ch_step's h_mass / h_energy), against the oracle's own 1000-step FP64 runs of the same
initial field (tests/golden/ch_trajectory_n<n>.txt, written by make_ch_trajectories.py).

* Mass.  The scheme conserves mass exactly; in floating point it drifts by the rounding of the
  right-hand side's large terms (~64 a |Cbar|, a = 2.9e3 at n = 1024 and 1.8e5 at 4096), which
  the line solves pass on to the sum undamped.  The oracle itself drifts by up to 2.1e-12 (n =
  1024) of h^2 sum|C0| over the run, more than a flat 1e-12.  So FP64 storage is held to 32 times
  the oracle's drift envelope (max over the steps so far), and FP32 storage in addition to the
  random walk of its two roundings to FP32 per point and step: 4 sqrt(k) n h^2 2^-24 max|C|.
* Energy.  The free energy is compared with the oracle's at every step (FP64: 1e-9 relative
  growing as exp(25 t), 25 = D / (4 gamma) being the largest growth rate of the linearised
  equation; FP32 storage starts from C0 rounded to FP32 and rounds every step: 1e-5 with the same
  growth), and every step where the oracle's energy rises
  by more than that tolerance must rise on the device too (and vice versa): the rises are the
  scheme's (the stiffest modes under the ADI factorisation are barely damped), reported, not
  clamped.
* The final field is compared with the oracle's at 64 fixed points with the same growth-aware
  tolerance (FP64 only; FP32 trajectories are compared on invariants).
"""
import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

D, GAMMA, SEED, STEPS = 1.0, 0.01, 1902, 1000
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_golden(n):
    m0 = e0 = None
    mass, energy, pts = [], [], []
    for line in open(os.path.join(GOLDEN, f"ch_trajectory_n{n}.txt")):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        if f[0] == "m0e0":
            m0, e0 = float(f[1]), float(f[2])
        elif f[0] == "C":
            pts.append((int(f[1]), int(f[2]), float(f[3])))
        else:
            mass.append(float(f[1]))
            energy.append(float(f[2]))
    return m0, e0, np.array(mass), np.array(energy), pts


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_1902_09931_gb300 as cs
    cs.load()
    return cs, torch


@pytest.mark.parametrize("storage", [0, 1])
@pytest.mark.parametrize("n", [1024, 4096])
def test_thousand_steps_invariants_every_step(env, n, storage):
    cs, torch = env
    h = 2 * np.pi / n
    dt = 0.1 * h
    m0_o, e0_o, mass_o, energy_o, pts = load_golden(n)
    c0 = W.ch_initial(n, seed=SEED)
    if storage == 1:
        c0 = c0.astype(np.float32).astype(np.float64)
    tdt = torch.float64 if storage == 0 else torch.float32
    f = [torch.from_numpy(c0).to("cuda", tdt), torch.from_numpy(c0).to("cuda", tdt),
         torch.zeros(n, n, dtype=tdt, device="cuda")]
    plan = cs.cs_ch_create(cs.CHDesc(n=n, storage=storage, D=D, gamma=GAMMA, dt=dt), *f)
    cs.cs_autotune(plan)
    torch.cuda.synchronize()
    m0, e0 = cs.cs_ch_invariants(plan)
    mass, energy = cs.cs_ch_step(plan, STEPS, invariants=True)
    _, cur, steps = cs.cs_ch_fields(plan)
    c_end = [t for t in f if t.data_ptr() == cur][0].cpu().numpy().astype(np.float64)
    cs.cs_destroy(plan)
    assert steps == STEPS

    k = np.arange(1, STEPS + 1)
    t = k * dt
    scale = h * h * np.abs(c0).sum()
    # mass
    drift = np.abs(mass - m0) / scale
    envelope = np.maximum.accumulate(np.abs(mass_o - m0_o) / scale)
    bound = 32 * np.maximum(envelope, 1e-14)
    if storage == 1:
        cmax = max(np.abs(c0).max(), np.abs(c_end).max())
        bound = bound + 4 * np.sqrt(k) * n * h * h * 2.0 ** -24 * cmax / scale
    # energy
    growth = np.exp(D / (4 * GAMMA) * t)
    etol = (1e-9 if storage == 0 else 1e-5) * growth * np.abs(energy_o)
    de, de_o = np.diff(np.concatenate([[e0], energy])), np.diff(np.concatenate([[e0_o], energy_o]))
    resolved = np.abs(de_o) > 2 * etol
    rises, rises_o = int((de > 0).sum()), int((de_o > 0).sum())
    print(f"[ch run] n={n} storage={'f32' if storage else 'f64'}: mass drift max {drift.max():.3e} of h^2 sum|C0| "
          f"(oracle {envelope[-1]:.3e}); energy {e0:.6f} -> {energy[-1]:.6f}, max |dE| vs oracle "
          f"{(np.abs(energy - energy_o) / np.abs(energy_o)).max():.3e} relative ({(np.abs(energy - energy_o) / etol).max():.3f} "
          f"of the tolerance); energy rose in {rises} steps "
          f"(oracle {rises_o}), first at step {int(np.argmax(de > 0)) + 1 if rises else 0}, largest rise "
          f"{(de / np.abs(energy - de)).max():.3e} relative")
    if storage == 0:
        assert abs(m0 - m0_o) <= 1e-14 * scale + 1e-15
        assert abs(e0 - e0_o) <= 1e-12 * abs(e0_o)
    else:  # C0 rounded to FP32
        assert abs(m0 - m0_o) <= 2.0 ** -24 * scale
        assert abs(e0 - e0_o) <= 2.0 ** -20 * abs(e0_o)
    assert np.all(drift <= bound), (drift.max(), int(np.argmax(drift > bound)))
    assert np.all(np.abs(energy - energy_o) <= etol), int(np.argmax(np.abs(energy - energy_o) > etol))
    assert np.array_equal(np.sign(de[resolved]), np.sign(de_o[resolved]))
    if storage == 0:
        tol_c = 1e-9 * growth[-1] * max(1.0, np.abs(c_end).max())
        for j, i, v in pts:
            assert abs(c_end[j, i] - v) <= tol_c, (j, i, c_end[j, i], v)
