"""The sharded sweep's device path on one GPU (a single gloo rank: the halo exchange is the
periodic wrap of the only band), with this library's plan over the padded band, against the
oracle."""
import os
import socket

import numpy as np
import pytest

import workloads as W
from gpu_helpers import stencil_cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import torch.distributed as dist
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import oracle
    import paper_1902_09931_gb300 as cs
    from paper_1902_09931_gb300 import distributed as D
    cs.load()
    if not dist.is_initialized():
        with socket.socket() as s:
            s.bind(("127.0.0.1", 0))
            port = s.getsockname()[1]
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        dist.init_process_group("gloo", rank=0, world_size=1)
    yield cs, torch, oracle, D
    dist.destroy_process_group()


@pytest.mark.parametrize("bc", [0, 1])
def test_device_band_sweep_matches_oracle(env, bc):
    cs, torch, orc, D = env
    ny, nx = 300, 256
    h = 2 * np.pi / nx
    u = W.sines_field(nx, seed=71, ny=ny)
    for name, L, R, T, B, d, w in [c for c in stencil_cases(h) if c[0] in ("lap9", "biharm13", "ddy4")]:
        sweep = D.DeviceBandSweep(dict(dir=d, bc=bc, left=L, right=R, top=T, bottom=B, weights=w, dtype=0))
        got = D.sharded_sweep(torch.from_numpy(u).cuda(), sweep, T, B, bc == 1).cpu().numpy()
        sweep.close()
        ref = orc.stencil2d(u, w, d, bc, L, R, T, B)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(w).sum() * np.abs(u).max(), name
