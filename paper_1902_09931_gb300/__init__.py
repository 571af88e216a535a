"""GB300-native cuSten hot path (arXiv:1902.09931): stencils and Cahn-Hilliard ADI.

A thin ctypes binding over the C ABI declared in ``include/custen_gb.h``; every function keeps
the C name and only marshals arguments (tensors become device pointers, streams become
``cudaStream_t`` handles).  All computation runs in the CUDA kernels of ``libcusten_gb.so``;
there is no CPU path.  If the library is missing or fails to load, every call raises.

Quick use (PyTorch supplies the memory and the stream)::

    import torch, paper_1902_09931_gb300 as cs
    u = torch.rand(4096, 4096, device="cuda", dtype=torch.float64)
    out = torch.empty_like(u)
    desc = cs.StencilDesc(nx=4096, ny=4096, dir=cs.CS_DIR_XY, bc=cs.CS_BC_PERIODIC,
                          dtype=cs.CS_F64, left=1, right=1, top=1, bottom=1,
                          weights=[0, 1, 0, 1, -4, 1, 0, 1, 0])
    plan = cs.cs_plan_create_2d(desc, u, out)
    cs.cs_compute(plan)          # on torch's current stream
    cs.cs_destroy(plan)
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence

from . import _build

CS_OK, CS_EINVAL, CS_EALIAS, CS_ENOMEM, CS_ECUDA, CS_EUNSUPPORTED, CS_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
CS_DIR_X, CS_DIR_Y, CS_DIR_XY = 0, 1, 2
CS_BC_NONPERIODIC, CS_BC_PERIODIC = 0, 1
CS_F64, CS_F32 = 0, 1
CS_FN_NONE, CS_FN_CENTRAL_D2X, CS_FN_CH_NONLIN_LAP, CS_FN_CUBIC_MINUS_LAP = 0, 1, 2, 3
CS_CH_PERIODIC, CS_CH_NOFLUX = 0, 1
CS_FP64_AUTO, CS_FP64_NATIVE = 0, 1
CS_MAX_EXTENT = 16

LIB_PATH = _build.LIB


class CSError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"[{code}] {message}")
        self.code = code


class _CStencilDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("dir", ctypes.c_int32),
                ("bc", ctypes.c_int32), ("dtype", ctypes.c_int32), ("left", ctypes.c_int32),
                ("right", ctypes.c_int32), ("top", ctypes.c_int32), ("bottom", ctypes.c_int32),
                ("weights", ctypes.POINTER(ctypes.c_double)), ("fn", ctypes.c_int32),
                ("num_coe", ctypes.c_int32), ("coe", ctypes.POINTER(ctypes.c_double))]


class _CCHDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("storage", ctypes.c_int32), ("boundary", ctypes.c_int32),
                ("D", ctypes.c_double), ("gamma", ctypes.c_double), ("dt", ctypes.c_double)]


class _CWenoDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("dtype", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("hx", ctypes.c_double), ("hy", ctypes.c_double)]


@dataclass
class StencilDesc:
    """Python mirror of ``cs_stencil_desc`` (Sec. 3 / Sec. 4.1 parameters)."""
    nx: int = 0
    ny: int = 1
    dir: int = CS_DIR_X
    bc: int = CS_BC_PERIODIC
    dtype: int = CS_F64
    left: int = 0
    right: int = 0
    top: int = 0
    bottom: int = 0
    weights: Optional[Sequence[float]] = None
    fn: int = CS_FN_NONE
    coe: Optional[Sequence[float]] = None


@dataclass
class CHDesc:
    """Python mirror of ``cs_ch_desc`` (Sec. 5.1 / 5.3 parameters)."""
    n: int
    storage: int = CS_F64
    D: float = 1.0
    gamma: float = 0.01
    dt: float = 0.0
    boundary: int = 0  # CS_CH_PERIODIC, or CS_CH_NOFLUX (reflected ghost cells)


_lib = None
_SYMBOLS = {
    # name: (restype, argtypes)
    "cs_plan_create_2d": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(_CStencilDesc), ctypes.c_void_p, ctypes.c_void_p]),
    "cs_plan_create_2d_host": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(_CStencilDesc), ctypes.c_int64]),
    "cs_plan_host_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "cs_plan_create_weno_adv": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(_CWenoDesc), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "cs_plan_create_1d_batch": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(_CStencilDesc), ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]),
    "cs_compute": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "cs_compute_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "cs_compute_group": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32, ctypes.c_void_p]),
    "cs_swap": (ctypes.c_int, [ctypes.c_void_p]),
    "cs_set_buffers": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "cs_plan_use_graph": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "cs_plan_set_fp64_mode": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "cs_plan_set_tile_choice": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "cs_plan_get_tile_choice": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)]),
    "cs_plan_check": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "cs_plan_debug_stall": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "cs_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "cs_tune_save": (ctypes.c_int, [ctypes.c_char_p]),
    "cs_tune_load": (ctypes.c_int, [ctypes.c_char_p]),
    "cs_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "cs_ch_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(_CCHDesc), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "cs_ch_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "cs_ch_invariants": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "cs_ch_coarsening": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "cs_ch_fields": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int64)]),
    "cs_ch_set_fields": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "cs_ch_config": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "cs_ch_band_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(_CCHDesc), ctypes.c_int64]),
    "cs_ch_band_rhs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "cs_ch_band_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "cs_ch_band_update": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "cs_ch_partition": (ctypes.c_int, [ctypes.POINTER(_CCHDesc), ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "cs_ch_band_ycols_local": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "cs_ch_band_ycols_correct": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "cs_ch_solver_check": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]),
    "cs_batch1d_compute_noalloc": (ctypes.c_int, [ctypes.POINTER(_CStencilDesc), ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "cs_last_error": (ctypes.c_char_p, []),
    "cs_launch_count": (ctypes.c_int64, []),
    "cs_version": (ctypes.c_char_p, []),
}


def load(path: Optional[str] = None):
    """Loads libcusten_gb.so (building it first if this checkout has no build).  Raises when the
    library cannot be built or loaded: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        _build.build_library()
    lib = ctypes.CDLL(p)
    for name, (res, args) in _SYMBOLS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(x) -> int:
    """Device (or host) address of a tensor / array / int."""
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if hasattr(x, "ctypes"):
        return int(x.ctypes.data)
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(s) -> int:
    if s is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(s, int):
        return s
    if hasattr(s, "cuda_stream"):
        return int(s.cuda_stream)
    raise TypeError(f"not a stream: {type(s)}")


def _check(rc: int) -> None:
    if rc != CS_OK:
        raise CSError(rc, load().cs_last_error().decode())


def _desc(d: StencilDesc):
    c = _CStencilDesc()
    c.nx, c.ny, c.dir, c.bc, c.dtype = d.nx, d.ny, d.dir, d.bc, d.dtype
    c.left, c.right, c.top, c.bottom = d.left, d.right, d.top, d.bottom
    keep = []
    if d.weights is not None:
        w = (ctypes.c_double * len(d.weights))(*[float(v) for v in d.weights])
        c.weights = ctypes.cast(w, ctypes.POINTER(ctypes.c_double))
        keep.append(w)
    c.fn = d.fn
    if d.coe is not None:
        co = (ctypes.c_double * len(d.coe))(*[float(v) for v in d.coe])
        c.coe = ctypes.cast(co, ctypes.POINTER(ctypes.c_double))
        c.num_coe = len(d.coe)
        keep.append(co)
    return c, keep


def cs_plan_create_2d(desc: StencilDesc, d_in, d_out) -> ctypes.c_void_p:
    c, _keep = _desc(desc)
    plan = ctypes.c_void_p()
    _check(load().cs_plan_create_2d(ctypes.byref(plan), ctypes.byref(c), _ptr(d_in), _ptr(d_out)))
    return plan


def cs_plan_create_2d_host(desc: StencilDesc, device_bytes: int = 0) -> ctypes.c_void_p:
    """A 2D plan for a grid in host memory, streamed through device band slots of at most
    ``device_bytes`` (0: the library default); compute with cs_compute_host."""
    c, _keep = _desc(desc)
    plan = ctypes.c_void_p()
    _check(load().cs_plan_create_2d_host(ctypes.byref(plan), ctypes.byref(c), int(device_bytes)))
    return plan


def cs_plan_host_info(plan):
    """(band rows, device bytes held) of a host-resident plan."""
    r, b = ctypes.c_int64(), ctypes.c_int64()
    _check(load().cs_plan_host_info(plan, ctypes.byref(r), ctypes.byref(b)))
    return r.value, b.value


def cs_plan_create_weno_adv(nx: int, ny: int, dtype: int, hx: float, hy: float, d_c, d_u, d_v, d_out):
    """Periodic XY WENO advection plan: cs_compute writes u C_x + v C_y into d_out."""
    c = _CWenoDesc(nx=int(nx), ny=int(ny), dtype=int(dtype), reserved=0, hx=float(hx), hy=float(hy))
    plan = ctypes.c_void_p()
    _check(load().cs_plan_create_weno_adv(ctypes.byref(plan), ctypes.byref(c), _ptr(d_c), _ptr(d_u),
                                          _ptr(d_v), _ptr(d_out)))
    return plan


def cs_plan_create_1d_batch(desc: StencilDesc, num_lines: int, d_offsets, total_len: int, d_in,
                            d_out) -> ctypes.c_void_p:
    c, _keep = _desc(desc)
    plan = ctypes.c_void_p()
    _check(load().cs_plan_create_1d_batch(ctypes.byref(plan), ctypes.byref(c), int(num_lines),
                                          _ptr(d_offsets), int(total_len), _ptr(d_in), _ptr(d_out)))
    return plan


def cs_compute(plan, stream=None) -> None:
    _check(load().cs_compute(plan, _stream(stream)))


def cs_compute_group(plans, stream=None) -> None:
    """One grouped launch (per 16 plans) over several 2D stencil plans of the same shape."""
    arr = (ctypes.c_void_p * len(plans))(*[p.value if hasattr(p, "value") else p for p in plans])
    _check(load().cs_compute_group(arr, len(plans), _stream(stream)))


def cs_compute_host(plan, h_in, h_out, stream=None) -> None:
    _check(load().cs_compute_host(plan, _ptr(h_in), _ptr(h_out), _stream(stream)))


def cs_swap(plan) -> None:
    _check(load().cs_swap(plan))


def cs_set_buffers(plan, d_in, d_out) -> None:
    _check(load().cs_set_buffers(plan, _ptr(d_in), _ptr(d_out)))


def cs_plan_set_fp64_mode(plan, mode: int) -> None:
    _check(load().cs_plan_set_fp64_mode(plan, int(mode)))


def cs_plan_set_tile_choice(plan, choice: int) -> None:
    _check(load().cs_plan_set_tile_choice(plan, int(choice)))


def cs_plan_get_tile_choice(plan) -> int:
    c = ctypes.c_int32()
    _check(load().cs_plan_get_tile_choice(plan, ctypes.byref(c)))
    return c.value


def cs_plan_check(plan, stream=None) -> None:
    """Waits for the stream; raises CSError(CS_ETIMEOUT) if a TMA sweep of the plan had a bounded
    wait run out since the last check."""
    _check(load().cs_plan_check(plan, _stream(stream)))


def cs_plan_debug_stall(plan, tile: int) -> None:
    """Test hook: the plan's TMA sweep issues no copies from CTA-local tile `tile` on (< 0: off)."""
    _check(load().cs_plan_debug_stall(plan, int(tile)))


def cs_plan_use_graph(plan, enable: bool = True) -> None:
    _check(load().cs_plan_use_graph(plan, 1 if enable else 0))


def cs_autotune(plan, stream=None) -> None:
    _check(load().cs_autotune(plan, _stream(stream)))


def cs_tune_save(path: str) -> None:
    _check(load().cs_tune_save(path.encode()))


def cs_tune_load(path: str) -> None:
    _check(load().cs_tune_load(path.encode()))


def cs_destroy(plan) -> None:
    if plan is not None:
        _check(load().cs_destroy(plan))


def cs_ch_create(desc: CHDesc, d_c_prev, d_c_cur, d_c_next) -> ctypes.c_void_p:
    c = _CCHDesc()
    c.n, c.storage, c.boundary, c.D, c.gamma, c.dt = desc.n, desc.storage, desc.boundary, desc.D, desc.gamma, desc.dt
    plan = ctypes.c_void_p()
    _check(load().cs_ch_create(ctypes.byref(plan), ctypes.byref(c), _ptr(d_c_prev), _ptr(d_c_cur),
                               _ptr(d_c_next)))
    return plan


def cs_ch_step(plan, nsteps: int, invariants: bool = False, stream=None):
    """Advances nsteps; with invariants=True returns (mass[nsteps], energy[nsteps]) as numpy."""
    if not invariants:
        _check(load().cs_ch_step(plan, int(nsteps), None, None, _stream(stream)))
        return None
    import numpy as np
    mass = np.empty(int(nsteps))
    energy = np.empty(int(nsteps))
    _check(load().cs_ch_step(plan, int(nsteps), mass.ctypes.data, energy.ctypes.data, _stream(stream)))
    return mass, energy


def cs_ch_invariants(plan, stream=None):
    m, e = ctypes.c_double(), ctypes.c_double()
    _check(load().cs_ch_invariants(plan, ctypes.byref(m), ctypes.byref(e), _stream(stream)))
    return m.value, e.value


def cs_ch_coarsening(plan, stream=None):
    """(s, k_1) of the current field: the coarsening measures of Sec. 5.1, in FP64."""
    s, k1 = ctypes.c_double(), ctypes.c_double()
    _check(load().cs_ch_coarsening(plan, ctypes.byref(s), ctypes.byref(k1), _stream(stream)))
    return s.value, k1.value


def cs_ch_fields(plan):
    """(device pointer of C^{n-1}, device pointer of C^n, steps taken)."""
    p, c, s = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_int64()
    _check(load().cs_ch_fields(plan, ctypes.byref(p), ctypes.byref(c), ctypes.byref(s)))
    return p.value, c.value, s.value


def cs_ch_set_fields(plan, d_c_prev, d_c_cur, d_c_next) -> None:
    _check(load().cs_ch_set_fields(plan, _ptr(d_c_prev), _ptr(d_c_cur), _ptr(d_c_next)))


def cs_ch_config(plan):
    """(chunks per line, chunk length) of the plan's partitioned line solve."""
    c, m = ctypes.c_int32(), ctypes.c_int32()
    _check(load().cs_ch_config(plan, ctypes.byref(c), ctypes.byref(m)))
    return c.value, m.value


def cs_ch_band_create(desc: CHDesc, rows: int) -> ctypes.c_void_p:
    plan = ctypes.c_void_p()
    c = _CCHDesc()
    c.n, c.storage, c.D, c.gamma, c.dt = desc.n, desc.storage, desc.D, desc.gamma, desc.dt
    c.boundary = desc.boundary
    _check(load().cs_ch_band_create(ctypes.byref(plan), ctypes.byref(c), int(rows)))
    return plan


def cs_ch_band_rhs(plan, d_prev, d_cur, d_rhs, d_sums=None, stream=None) -> None:
    _check(load().cs_ch_band_rhs(plan, _ptr(d_prev), _ptr(d_cur), _ptr(d_rhs), _ptr(d_sums), _stream(stream)))


def cs_ch_band_solve(plan, d_in, d_out, stream=None) -> None:
    _check(load().cs_ch_band_solve(plan, _ptr(d_in), _ptr(d_out), _stream(stream)))


def cs_ch_band_update(plan, d_prev, d_cur, d_v, d_next, stream=None) -> None:
    _check(load().cs_ch_band_update(plan, _ptr(d_prev), _ptr(d_cur), _ptr(d_v), _ptr(d_next), _stream(stream)))


def cs_ch_partition(desc: CHDesc):
    """(chunks per line, chunk length) that cs_ch_create / cs_ch_band_create pick for desc."""
    c = _CCHDesc()
    c.n, c.storage, c.D, c.gamma, c.dt = desc.n, desc.storage, desc.D, desc.gamma, desc.dt
    c.boundary = desc.boundary
    k, m = ctypes.c_int32(), ctypes.c_int32()
    _check(load().cs_ch_partition(ctypes.byref(c), ctypes.byref(k), ctypes.byref(m)))
    return k.value, m.value


def cs_ch_band_ycols_local(plan, chunk0: int, d_in, d_ends, stream=None) -> None:
    _check(load().cs_ch_band_ycols_local(plan, int(chunk0), _ptr(d_in), _ptr(d_ends), _stream(stream)))


def cs_ch_band_ycols_correct(plan, chunk0: int, d_ends_all, d_v, stream=None) -> None:
    _check(load().cs_ch_band_ycols_correct(plan, int(chunk0), _ptr(d_ends_all), _ptr(d_v), _stream(stream)))


def cs_ch_solver_check(n: int, chunks: int, a: float, boundary: int) -> float:
    """Backward error of the line solver's host replay on its own tables (no GPU needed)."""
    r = ctypes.c_double()
    _check(load().cs_ch_solver_check(int(n), int(chunks), float(a), int(boundary), ctypes.byref(r)))
    return r.value


def cs_batch1d_compute_noalloc(desc: StencilDesc, num_lines: int, d_offsets, total_len: int, d_in,
                               d_out, stream=None) -> None:
    """Batched 1D sweep without a plan and without any device allocation (see the header)."""
    c, _keep = _desc(desc)
    _check(load().cs_batch1d_compute_noalloc(ctypes.byref(c), int(num_lines), _ptr(d_offsets),
                                             int(total_len), _ptr(d_in), _ptr(d_out), _stream(stream)))


def cs_last_error() -> str:
    return load().cs_last_error().decode()


def cs_launch_count() -> int:
    return int(load().cs_launch_count())


def cs_version() -> str:
    return load().cs_version().decode()


def exported_symbols():
    return sorted(_SYMBOLS)
