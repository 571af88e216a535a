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
