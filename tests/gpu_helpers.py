"""Helpers for the GPU parity tests: run the library through its C ABI on torch buffers."""
import numpy as np

STENCILS = {}


def _register(name, L, R, T, B, direction, weights):
    STENCILS[name] = dict(L=L, R=R, T=T, B=B, dir=direction, w=np.asarray(weights, dtype=np.float64).ravel())


def lap5(h=1.0):
    return np.array([0, 1, 0, 1, -4, 1, 0, 1, 0.0]) / h ** 2


def lap9(h=1.0):
    return np.array([1, 4, 1, 4, -20, 4, 1, 4, 1.0]) / (6 * h ** 2)


def biharm13(h=1.0):
    w = np.zeros((5, 5))
    w[2, 2] = 20
    w[1, 2] = w[3, 2] = w[2, 1] = w[2, 3] = -8
    w[1, 1] = w[1, 3] = w[3, 1] = w[3, 3] = 2
    w[0, 2] = w[4, 2] = w[2, 0] = w[2, 4] = 1
    return w.ravel() / h ** 4


D1_4 = np.array([1, -8, 0, 8, -1.0]) / 12.0
D2_4 = np.array([-1, 16, -30, 16, -1.0]) / 12.0
FD8_D2 = np.array([-1 / 560, 8 / 315, -1 / 5, 8 / 5, -205 / 72, 8 / 5, -1 / 5, 8 / 315, -1 / 560])


def stencil_cases(h):
    """(name, L, R, T, B, dir, weights): the workload stencils plus shapes that exercise every
    specialised kernel and the generic one."""
    rng = np.random.Generator(np.random.PCG64(99))
    return [
        ("lap5", 1, 1, 1, 1, 2, lap5(h)),
        ("lap9", 1, 1, 1, 1, 2, lap9(h)),
        ("biharm13", 2, 2, 2, 2, 2, biharm13(h)),
        ("box5x5", 2, 2, 2, 2, 2, rng.uniform(-1, 1, 25)),
        ("ddx4", 2, 2, 0, 0, 0, D1_4 / h),
        ("ddy4", 0, 0, 2, 2, 1, D1_4 / h),
        ("d2x4", 2, 2, 0, 0, 0, D2_4 / h ** 2),
        ("d2y4", 0, 0, 2, 2, 1, D2_4 / h ** 2),
        ("d2x8", 4, 4, 0, 0, 0, FD8_D2 / h ** 2),
        ("d2y8", 0, 0, 4, 4, 1, FD8_D2 / h ** 2),
        ("x1", 1, 1, 0, 0, 0, [1.0, -2.0, 1.0]),
        ("y1", 0, 0, 1, 1, 1, [0.5, -1.0, 0.25]),
        ("asym3102", 3, 1, 0, 2, 2, rng.uniform(-1, 1, 15)),
        ("generic5", 5, 4, 3, 5, 2, rng.uniform(-1, 1, 90)),
    ]


def run2d(cs, torch, field, desc_kw, dtype, out_init=None, graph=False, reps=1, fp64_mode=None,
          tile_choice=None):
    """Applies a plan once (or `reps` times, swapping) on the GPU; returns the output as FP64."""
    tdt = torch.float64 if dtype == cs.CS_F64 else torch.float32
    ndt = np.float64 if dtype == cs.CS_F64 else np.float32
    ny, nx = field.shape
    d_in = torch.from_numpy(np.ascontiguousarray(field, dtype=ndt)).cuda()
    if out_init is None:
        d_out = torch.zeros_like(d_in)
    else:
        d_out = torch.from_numpy(np.ascontiguousarray(out_init, dtype=ndt)).cuda()
    desc = cs.StencilDesc(nx=nx, ny=ny, dtype=dtype, **desc_kw)
    plan = cs.cs_plan_create_2d(desc, d_in, d_out)
    try:
        if fp64_mode is not None:
            cs.cs_plan_set_fp64_mode(plan, fp64_mode)
        if tile_choice is not None:
            cs.cs_plan_set_tile_choice(plan, tile_choice)
        if graph:
            cs.cs_plan_use_graph(plan, True)
        for r in range(reps):
            cs.cs_compute(plan)
            if r + 1 < reps:
                cs.cs_swap(plan)
                d_in, d_out = d_out, d_in
        torch.cuda.synchronize()
    finally:
        cs.cs_destroy(plan)
    return d_out.cpu().numpy().astype(np.float64)


def scaled_err(got, ref, weights, field):
    """Error normalised by the size of the terms the stencil sums (sum |w| * max |in|)."""
    scale = np.abs(np.asarray(weights)).sum() * max(np.abs(field).max(), 1e-300)
    return np.abs(got - ref).max() / scale


CH_D, CH_GAMMA = 1.0, 0.01
EPS64 = 2.0 ** -52


def ch_step_bound(orc, prev, cur, nxt_ref, n, dt, storage, noflux=False):
    """Rounding bound for one Cahn-Hilliard ADI step (Sec. 5.1) taken by two FP64 implementations
    from the same state (C^{n-1}, C^n): (tolerance, B).

    B = eps (S + kappa max|v|), eps = 2^-52: S = max|C^n| + max|C^{n-1}| + 64 a max|Cbar| +
    8 alpha max|N| is the size of the right-hand side's terms (the 13-point biharmonic's weights
    sum to 64 in units of a = (2/3) D gamma dt / h^4, the 5-point Laplacian's to 8 in units of
    alpha = (2/3) D dt / h^2), whose roundings reach C^{n+1} undamped at low wavenumbers since
    ||L^-1|| <= 1; the backward-stable y-solve adds at most kappa eps |v|, kappa = 1 + 16 a,
    v = C^{n+1} - Cbar.  (The x-solve's own rounding, of size kappa eps |w| before L_y^-1, lies
    in the rows' high wavenumbers that L_y^-1 damps; measured, the total stays near B.)  The
    tolerance is 8 B, plus 2^-24 (max|Cbar| + max|C^{n+1}|) for FP32 storage (Cbar in the update
    and the stored result are rounded to FP32)."""
    h = 2 * np.pi / n
    a = orc.ch_coefficient_a(n, CH_D, CH_GAMMA, dt)
    alpha = (2.0 / 3.0) * CH_D * dt / h ** 2
    cbar = 2 * cur - prev
    S = (np.abs(cur).max() + np.abs(prev).max() + 64 * a * np.abs(cbar).max()
         + 8 * alpha * np.abs(cur ** 3 - cur).max())
    v = nxt_ref - cbar
    B = EPS64 * (S + (1 + 16 * a) * np.abs(v).max())
    tol = 8 * B
    if storage == 1:
        tol += 2.0 ** -24 * (np.abs(cbar).max() + np.abs(nxt_ref).max())
    return tol, B


def check_ch_step(orc, prev, cur, got, n, dt, storage, what, noflux=False):
    """Compares one device step with the oracle's from the same state; prints err / B."""
    step = orc.ch_step_noflux if noflux else orc.ch_step
    ref = step(prev, cur, CH_D, CH_GAMMA, dt)
    tol, B = ch_step_bound(orc, prev, cur, ref, n, dt, storage, noflux)
    err = np.abs(got - ref).max()
    print(f"[ch step{' noflux' if noflux else ''}] {what} n={n} storage={'f32' if storage else 'f64'}: "
          f"err {err:.3e} = {err / tol:.3f} of the tolerance {tol:.3e} (the FP64 rounding bound B = {B:.3e}"
          f"{'; FP32 storage adds the roundings to FP32' if storage else ''}), {err / np.abs(ref).max():.3e} of max|C|")
    assert err <= tol, (what, err, tol, err / B)
    if storage == 1:
        assert err <= 1e-5 * np.abs(ref).max(), (what, err / np.abs(ref).max())
    return ref
